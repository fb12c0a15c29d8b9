"""Python binding of libslim (ctypes): the C ABI of include/slim.h with the same
names, argument marshalling only.  Every operation runs in the library's CUDA
kernels; there is no fallback.  A missing library raises immediately.

Device buffers are passed as integer addresses (e.g. ``tensor.data_ptr()``) and
streams as integer handles (e.g. ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libslim.so")

SLIM_FP64, SLIM_MIXED = 0, 1
SLIM_SCHEME_TRACER, SLIM_SCHEME_SPLIT = 0, 1
SLIM_VERTICAL_LUMPED, SLIM_VERTICAL_COUPLED = 0, 1
FIELD = dict(T=0, S=1, U=2, V=3, W=4, R_X=5, R_Y=6, T_EXT=7, S_EXT=8, ETA=16, QX=17, QY=18, ETA_NEXT=19,
             QBAR_X=20, QBAR_Y=21, S3_X=22, S3_Y=23, F2D_X=24, F2D_Y=25, U_EXT=26, V_EXT=27,
             U_EXT_B=28, V_EXT_B=29, T_EXT_B=30, S_EXT_B=31)
FIELD_IS_3D = {f: (v < 16 or v >= 26) for f, v in FIELD.items()}   # 16..25: 2D

# every symbol declared in include/slim.h
EXPORTED = ["slim_params_default", "slim_status_string", "slim_last_error", "slim_mesh_create",
            "slim_mesh_destroy", "slim_mesh_info", "slim_state_alloc", "slim_state_free",
            "slim_state_set_params", "slim_state_upload", "slim_state_download",
            "slim_state_field_ptr", "slim_state_check", "slim_rhs3d", "slim_continuity",
            "slim_rhs2d", "slim_vertical_solve", "slim_hpg", "slim_step", "slim_tracer_mass",
            "slim_step_kernel_count", "slim_profile_begin", "slim_profile_end",
            "slim_phase_name", "slim_tracer_mass_noalloc", "slim_selftest_conversions",
            "slim_selftest_barrier", "slim_selftest_neighbour_wait", "slim_selftest_fma_peak", "slim_mesh_create_part",
            "slim_halo_create", "slim_halo_destroy", "slim_halo_exchange", "slim_halo_step"]
PHASES = ["continuity", "tracer_stage", "hpg", "mom_pred", "ext2d", "momentum", "tracers", "misc"]


class SlimParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "g", "rho0", "coriolis_f", "eos_alpha", "eos_beta", "eos_T0", "eos_S0", "kappa_v",
        "nu_v", "kappa_h", "nu_h", "drag_cd", "flux_top", "flux_bot", "penalty_v", "penalty_h",
        "tide_amp", "tide_period")] + [(n, C.c_int) for n in (
        "scheme", "n_sub", "tile_prisms", "check_every", "blocks_per_sm", "use_graph",
        "persistent_2d")] + [(n, C.c_double) for n in ("forcing_t_a", "forcing_t_b")] + [
        ("forcing", C.c_int), ("vertical", C.c_int)]


class SlimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


_lib = None
_vp, _i, _d, _dp = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double)


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        sig = {
            "slim_params_default": ([C.POINTER(SlimParams)], _i),
            "slim_status_string": ([_i], C.c_char_p),
            "slim_last_error": ([], C.c_char_p),
            "slim_mesh_create": ([_vp, _i, _vp, _i, _vp, _vp, _vp, _i, _vp, _i, C.POINTER(_vp)], _i),
            "slim_mesh_destroy": ([_vp], None),
            "slim_mesh_info": ([_vp, C.POINTER(C.c_int64), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)], _i),
            "slim_state_alloc": ([_vp, _i, C.POINTER(SlimParams), C.POINTER(_vp)], _i),
            "slim_state_free": ([_vp], None),
            "slim_state_set_params": ([_vp, C.POINTER(SlimParams)], _i),
            "slim_state_upload": ([_vp, _i, _vp, _vp], _i),
            "slim_state_download": ([_vp, _i, _vp, _vp], _i),
            "slim_state_field_ptr": ([_vp, _i, C.POINTER(_vp), C.POINTER(_i)], _i),
            "slim_state_check": ([_vp, _vp], _i),
            "slim_rhs3d": ([_vp, _i, _vp, _vp], _i),
            "slim_continuity": ([_vp, _d, _vp], _i),
            "slim_rhs2d": ([_vp, _d, _vp, _vp], _i),
            "slim_vertical_solve": ([_vp, _i, _d, _vp, _vp, _vp], _i),
            "slim_step": ([_vp, _d, _d, _vp], _i),
            "slim_hpg": ([_vp, _vp], _i),
            "slim_tracer_mass": ([_vp, _i, _dp, _vp], _i),
            "slim_step_kernel_count": ([_vp], _i),
            "slim_profile_begin": ([_vp, _i], _i),
            "slim_profile_end": ([_vp, _dp, C.POINTER(_i)], _i),
            "slim_phase_name": ([_i], C.c_char_p),
            "slim_tracer_mass_noalloc": ([_vp, _i, _vp, _vp], _i),
            "slim_selftest_conversions": ([C.c_longlong, C.c_ulonglong, C.POINTER(C.c_longlong),
                                           C.POINTER(C.c_longlong)], _i),
            "slim_selftest_barrier": ([_i, _i, _i, C.POINTER(_i), C.POINTER(_i)], _i),
            "slim_selftest_neighbour_wait": ([_i, _i, _i, C.POINTER(_i), C.POINTER(_i)], _i),
            "slim_selftest_fma_peak": ([_i, C.c_longlong, _dp, _dp], _i),
            "slim_mesh_create_part": ([_vp, _i, _vp, _i, _vp, _vp, _vp, _i, _vp, _i, _vp, C.POINTER(_vp)], _i),
            "slim_halo_create": ([_vp, _i, _vp, _vp, _vp, C.POINTER(_vp)], _i),
            "slim_halo_destroy": ([_vp], None),
            "slim_halo_exchange": ([_vp, _i, _vp], _i),
            "slim_halo_step": ([_vp, _d, _d, _vp], _i),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != 0:
        L = lib()
        raise SlimError(status, f"{L.slim_status_string(status).decode()}: {L.slim_last_error().decode()}")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_vp)


# ---------------------------------------------------------------------------
# functional API (names of the C ABI)
# ---------------------------------------------------------------------------
def slim_params_default(**overrides) -> SlimParams:
    p = SlimParams()
    _check(lib().slim_params_default(C.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def slim_status_string(status: int) -> str:
    return lib().slim_status_string(status).decode()


def slim_mesh_create(xy, tri, h_tri, n_layers, bnd, levels=None, tile_prisms: int = 256) -> int:
    xy = np.ascontiguousarray(xy, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    h_tri = np.ascontiguousarray(h_tri, np.float64)
    n_layers = np.ascontiguousarray(n_layers, np.int32)
    bnd = np.ascontiguousarray(bnd, np.int8)
    lev = None if levels is None else np.ascontiguousarray(levels, np.float64)
    out = _vp()
    _check(lib().slim_mesh_create(_ptr(xy), int(xy.shape[0]), _ptr(tri), int(tri.shape[0]),
                                  _ptr(h_tri), _ptr(n_layers), None if lev is None else _ptr(lev),
                                  0 if lev is None else int(lev.shape[0]), _ptr(bnd),
                                  int(tile_prisms), C.byref(out)))
    return out.value


def slim_mesh_create_part(xy, tri, h_tri, n_layers, bnd, tri_class, levels=None, tile_prisms: int = 256) -> int:
    xy = np.ascontiguousarray(xy, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    h_tri = np.ascontiguousarray(h_tri, np.float64)
    n_layers = np.ascontiguousarray(n_layers, np.int32)
    bnd = np.ascontiguousarray(bnd, np.int8)
    cls = np.ascontiguousarray(tri_class, np.int8)
    lev = None if levels is None else np.ascontiguousarray(levels, np.float64)
    out = _vp()
    _check(lib().slim_mesh_create_part(_ptr(xy), int(xy.shape[0]), _ptr(tri), int(tri.shape[0]),
                                       _ptr(h_tri), _ptr(n_layers), None if lev is None else _ptr(lev),
                                       0 if lev is None else int(lev.shape[0]), _ptr(bnd),
                                       int(tile_prisms), _ptr(cls), C.byref(out)))
    return out.value


def slim_halo_create(states, pair_count, send_tris, recv_tris) -> int:
    arr = (_vp * len(states))(*states)
    pc = np.ascontiguousarray(pair_count, np.int32)
    st = np.ascontiguousarray(send_tris, np.int32)
    rt = np.ascontiguousarray(recv_tris, np.int32)
    out = _vp()
    _check(lib().slim_halo_create(arr, len(states), _ptr(pc), _ptr(st) if st.size else None,
                                  _ptr(rt) if rt.size else None, C.byref(out)))
    return out.value


def slim_halo_destroy(halo: int) -> None:
    lib().slim_halo_destroy(halo)


def slim_halo_exchange(halo: int, field: int, stream: int = 0) -> None:
    _check(lib().slim_halo_exchange(halo, field, stream))


def slim_halo_step(halo: int, t: float, dt: float, stream: int = 0) -> None:
    _check(lib().slim_halo_step(halo, t, dt, stream))


def slim_mesh_destroy(mesh: int) -> None:
    lib().slim_mesh_destroy(mesh)


def slim_mesh_info(mesh: int) -> dict:
    P, nt, ml, ntl = C.c_int64(), _i(), _i(), _i()
    _check(lib().slim_mesh_info(mesh, C.byref(P), C.byref(nt), C.byref(ml), C.byref(ntl)))
    return dict(n_prisms=P.value, n_tri=nt.value, max_layers=ml.value, n_tiles=ntl.value)


def slim_state_alloc(mesh: int, precision: int, params: SlimParams) -> int:
    out = _vp()
    _check(lib().slim_state_alloc(mesh, int(precision), C.byref(params), C.byref(out)))
    return out.value


def slim_state_free(state: int) -> None:
    lib().slim_state_free(state)


def slim_state_set_params(state: int, params: SlimParams) -> None:
    _check(lib().slim_state_set_params(state, C.byref(params)))


def slim_state_upload(state: int, field: int, host: np.ndarray, stream: int = 0) -> None:
    a = np.ascontiguousarray(host, np.float64)
    _check(lib().slim_state_upload(state, int(field), _ptr(a), stream))


def slim_state_upload_ptr(state: int, field: int, host_ptr: int, stream: int = 0) -> None:
    """Upload from a raw host address (e.g. pinned memory) of doubles."""
    _check(lib().slim_state_upload(state, int(field), host_ptr, stream))


def slim_state_download(state: int, field: int, n: int, stream: int = 0) -> np.ndarray:
    out = np.empty(n, np.float64)
    _check(lib().slim_state_download(state, int(field), _ptr(out), stream))
    return out


def slim_state_download_ptr(state: int, field: int, host_ptr: int, stream: int = 0) -> None:
    """Download into a raw host address (e.g. pinned memory) of doubles; synchronises."""
    _check(lib().slim_state_download(state, int(field), host_ptr, stream))


def slim_state_field_ptr(state: int, field: int) -> tuple[int, int]:
    p, es = _vp(), _i()
    _check(lib().slim_state_field_ptr(state, int(field), C.byref(p), C.byref(es)))
    return p.value, es.value


def slim_state_check(state: int, stream: int = 0) -> None:
    _check(lib().slim_state_check(state, stream))


def slim_rhs3d(state: int, field: int, out_dev: int, stream: int = 0) -> None:
    _check(lib().slim_rhs3d(state, int(field), out_dev, stream))


def slim_continuity(state: int, dt: float, stream: int = 0) -> None:
    _check(lib().slim_continuity(state, float(dt), stream))


def slim_rhs2d(state: int, t: float, out_dev: int, stream: int = 0) -> None:
    _check(lib().slim_rhs2d(state, float(t), out_dev, stream))


def slim_vertical_solve(state: int, field: int, beta_dt: float, rhs_dev: int, out_dev: int,
                        stream: int = 0) -> None:
    _check(lib().slim_vertical_solve(state, int(field), float(beta_dt), rhs_dev, out_dev, stream))


def slim_hpg(state: int, stream: int = 0) -> None:
    _check(lib().slim_hpg(state, stream))


def slim_step(state: int, t: float, dt: float, stream: int = 0) -> None:
    _check(lib().slim_step(state, float(t), float(dt), stream))


def slim_tracer_mass(state: int, field: int, stream: int = 0) -> float:
    out = C.c_double()
    _check(lib().slim_tracer_mass(state, int(field), C.byref(out), stream))
    return out.value


def slim_tracer_mass_noalloc(state: int, field: int, mass_dev: int, stream: int = 0) -> None:
    """Tracer mass into one device double at ``mass_dev`` without device allocation
    (asynchronous on ``stream``)."""
    _check(lib().slim_tracer_mass_noalloc(state, int(field), mass_dev, stream))


def slim_selftest_conversions(n: int, seed: int = 0) -> tuple[int, int]:
    """Mismatch counts (binary64->binary32, binary32->binary64) of the library's
    integer-pipe conversions against the GPU's own, over n seeded patterns."""
    a, b = C.c_longlong(-1), C.c_longlong(-1)
    _check(lib().slim_selftest_conversions(int(n), int(seed), C.byref(a), C.byref(b)))
    return a.value, b.value


def slim_selftest_barrier(n_blocks: int, skip_block: int, rounds: int) -> tuple[int, int]:
    """(device error bits, arrivals) of `rounds` rounds of the bounded grid barrier."""
    a, b = C.c_int(-1), C.c_int(-1)
    _check(lib().slim_selftest_barrier(int(n_blocks), int(skip_block), int(rounds), C.byref(a),
                                       C.byref(b)))
    return a.value, b.value


def slim_selftest_neighbour_wait(n_blocks: int, skip_block: int, rounds: int) -> tuple[int, int]:
    """(device error bits, arrivals) of `rounds` rounds of the bounded neighbour waits
    on a ring of blocks."""
    a, b = C.c_int(-1), C.c_int(-1)
    _check(lib().slim_selftest_neighbour_wait(int(n_blocks), int(skip_block), int(rounds), C.byref(a),
                                              C.byref(b)))
    return a.value, b.value


def slim_selftest_fma_peak(precision: int, iters: int = 1 << 16) -> tuple[float, float]:
    """(FLOP/s, milliseconds) of the library's FMA-throughput kernel."""
    f, ms = C.c_double(), C.c_double()
    _check(lib().slim_selftest_fma_peak(precision, C.c_longlong(iters), C.byref(f), C.byref(ms)))
    return f.value, ms.value


def slim_step_kernel_count(state: int) -> int:
    return int(lib().slim_step_kernel_count(state))


def slim_profile_begin(state: int, max_launches: int) -> None:
    _check(lib().slim_profile_begin(state, int(max_launches)))


def slim_profile_end(state: int) -> dict:
    """{phase name: (milliseconds, launches)} of the recorded launches."""
    ms = (C.c_double * len(PHASES))()
    n = (C.c_int * len(PHASES))()
    _check(lib().slim_profile_end(state, ms, n))
    return {PHASES[i]: (ms[i], n[i]) for i in range(len(PHASES)) if n[i] > 0}


def slim_phase_name(phase: int) -> str:
    return lib().slim_phase_name(int(phase)).decode()


# ---------------------------------------------------------------------------
# convenience wrapper owning a mesh and a state
# ---------------------------------------------------------------------------
class Model:
    """A mesh plus one state, freed together.  ``mesh`` is any object with the
    array attributes of ``workloads.Mesh`` (xy, tri, h_tri, n_layers, bnd, levels)."""

    def __init__(self, mesh, precision: int = SLIM_FP64, params: SlimParams | None = None,
                 tile_prisms: int | None = None):
        self.params = params if params is not None else slim_params_default()
        tp = tile_prisms if tile_prisms is not None else (self.params.tile_prisms or 256)
        self.mesh_h = slim_mesh_create(mesh.xy, mesh.tri, mesh.h_tri, mesh.n_layers, mesh.bnd,
                                       mesh.levels, tp)
        self.info = slim_mesh_info(self.mesh_h)
        self.P = self.info["n_prisms"]
        self.n_tri = self.info["n_tri"]
        self.precision = precision
        try:
            self.state = slim_state_alloc(self.mesh_h, precision, self.params)
        except Exception:
            slim_mesh_destroy(self.mesh_h)
            self.mesh_h = None
            self.state = None
            raise

    def n(self, field: str) -> int:
        return 6 * self.P if FIELD_IS_3D[field] else 3 * self.n_tri

    def upload(self, field: str, values, stream: int = 0) -> None:
        a = np.asarray(values, np.float64).reshape(-1)
        if a.shape[0] != self.n(field):
            raise ValueError(f"{field}: expected {self.n(field)} values, got {a.shape[0]}")
        slim_state_upload(self.state, FIELD[field], a, stream)

    def download(self, field: str, stream: int = 0) -> np.ndarray:
        return slim_state_download(self.state, FIELD[field], self.n(field), stream)

    def ptr(self, field: str) -> int:
        return slim_state_field_ptr(self.state, FIELD[field])[0]

    def close(self) -> None:
        if getattr(self, "state", None):
            slim_state_free(self.state)
            self.state = None
        if getattr(self, "mesh_h", None):
            slim_mesh_destroy(self.mesh_h)
            self.mesh_h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PartitionedModel:
    """The partitioned tracer step on one device: one state per partition of
    ``partition.partition(mesh, n_parts)`` and the halo that connects them.  Fields
    are uploaded and downloaded as global arrays (the partitions' owned values)."""

    def __init__(self, mesh, n_parts: int, precision: int = SLIM_FP64, params: SlimParams | None = None,
                 tile_prisms: int = 256):
        from . import partition as pa
        self.mesh = mesh
        self.pt = pa.partition(mesh, n_parts)
        self.params = params if params is not None else slim_params_default()
        self.meshes, self.states, self.halo = [], [], None
        self._pmap = [pa.prism_map(mesh, p) for p in self.pt.parts]
        try:
            for p in self.pt.parts:
                self.meshes.append(slim_mesh_create_part(p.xy, p.tri, p.h_tri, p.n_layers, p.bnd, p.tri_class,
                                                         p.levels, tile_prisms))
                self.states.append(slim_state_alloc(self.meshes[-1], precision, self.params))
            self.halo = slim_halo_create(self.states, self.pt.pair_count, self.pt.send_tris, self.pt.recv_tris)
        except Exception:
            self.close()
            raise

    def upload(self, field: str, values, stream: int = 0) -> None:
        from . import partition as pa
        is3d = FIELD_IS_3D[field]
        for part, st, pm in zip(self.pt.parts, self.states, self._pmap):
            slim_state_upload(st, FIELD[field], pa.to_local(self.mesh, part, values, is3d, pm), stream)

    def download(self, field: str, stream: int = 0) -> np.ndarray:
        from . import partition as pa
        is3d = FIELD_IS_3D[field]
        loc = []
        for part, st, pm in zip(self.pt.parts, self.states, self._pmap):
            n = 6 * len(pm) if is3d else 3 * part.n_tri
            loc.append(slim_state_download(st, FIELD[field], n, stream))
        return pa.owned_to_global(self.mesh, self.pt, loc, is3d)

    def step(self, t: float, dt: float, stream: int = 0) -> None:
        slim_halo_step(self.halo, t, dt, stream)

    def close(self) -> None:
        if getattr(self, "halo", None):
            slim_halo_destroy(self.halo)
            self.halo = None
        for st in getattr(self, "states", []):
            slim_state_free(st)
        for m in getattr(self, "meshes", []):
            slim_mesh_destroy(m)
        self.states, self.meshes = [], []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
