"""Autotuner of the launch tiling: prisms per thread block (the tile of whole
columns each block owns: 128, 256 or 512) and the register budget of the heavy
split-step kernels (2, 3 or 4 resident blocks of 256 threads per SM in the mixed
form; the FP64 form has one budget), and, in the mixed split scheme, whether the 2D
run is one cooperative launch per split stage or one launch per RK stage.

Every candidate is a separate mesh tiling and state; each runs a few warm-up
steps and is timed over a few steps with CUDA events on the current stream.  The
fastest configuration is cached in a JSON file keyed by the GPU name, the mesh
signature (triangles, prisms, layer histogram), the precision and the scheme.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import slim

TILES = (128, 256, 512)
OCCS = (2, 3, 4)
CACHE = os.path.join(os.path.expanduser("~"), ".cache", "slim_gb300_autotune.json")


def mesh_signature(mesh) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(mesh.n_layers, np.int32).tobytes())
    h.update(np.ascontiguousarray(mesh.tri, np.int32)[:: max(1, mesh.tri.shape[0] // 4096)].tobytes())
    return f"{mesh.tri.shape[0]}-{int(mesh.n_layers.sum())}-{h.hexdigest()[:16]}"


def _key(mesh, precision: int, params) -> str:
    import torch
    return "|".join([torch.cuda.get_device_name(), mesh_signature(mesh), str(precision),
                     str(params.scheme), str(params.n_sub)])


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(d):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as fh:
            json.dump(d, fh, indent=1)
    except Exception:
        pass


def time_config(mesh, precision: int, params, fields: dict, dt: float, tile: int, occ: int,
                warmup: int = 2, steps: int = 3, persistent: int | None = None) -> float:
    """Milliseconds per step of one configuration."""
    import torch
    p = slim.SlimParams.from_buffer_copy(params)
    p.tile_prisms = tile
    p.blocks_per_sm = occ
    if persistent is not None:
        p.persistent_2d = persistent
    stream = torch.cuda.current_stream()
    with slim.Model(mesh, precision, p, tile_prisms=tile) as mod:
        for k, v in fields.items():
            mod.upload(k, v)
        t = 0.0
        for _ in range(warmup):
            slim.slim_step(mod.state, t, dt, stream.cuda_stream)
            t += dt
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            slim.slim_step(mod.state, t, dt, stream.cuda_stream)
            t += dt
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps


def autotune(mesh, precision: int, params, fields: dict, dt: float, use_cache: bool = True,
             verbose: bool = False) -> dict:
    """Best {tile_prisms, blocks_per_sm, ms_per_step} and all timings."""
    key = _key(mesh, precision, params)
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]
    if params.scheme != slim.SLIM_SCHEME_SPLIT:
        occs = (4,)
    elif precision == slim.SLIM_FP64:
        occs = (2,)                      # one register budget in the FP64 form
    else:
        occs = OCCS
    results = {}
    for tile in TILES:
        for occ in occs:
            if occ == 3 and tile == 512:
                continue
            ms = time_config(mesh, precision, params, fields, dt, tile, occ)
            results[f"{tile}/{occ}"] = ms
            if verbose:
                print(f"autotune tile={tile} blocks_per_sm={occ}: {ms:.3f} ms/step", flush=True)
    best = min(results, key=results.get)
    tile, occ = (int(x) for x in best.split("/"))
    out = dict(tile_prisms=tile, blocks_per_sm=occ, ms_per_step=results[best], all=results,
               persistent_2d=int(params.persistent_2d))
    if params.scheme == slim.SLIM_SCHEME_SPLIT and precision == slim.SLIM_MIXED:
        # the mixed 2D run as one cooperative launch per split stage or one launch per
        # RK stage: the grid barrier pays on large meshes, the launches on small ones
        other = 0 if params.persistent_2d else 1
        ms = time_config(mesh, precision, params, fields, dt, tile, occ, persistent=other)
        results[f"{tile}/{occ}/persistent{other}"] = ms
        if verbose:
            print(f"autotune tile={tile} blocks_per_sm={occ} persistent_2d={other}: {ms:.3f} ms/step", flush=True)
        if ms < out["ms_per_step"]:
            out.update(persistent_2d=other, ms_per_step=ms)
    cache[key] = out
    if use_cache:
        _store(cache)
    return out
