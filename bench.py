#!/usr/bin/env python
"""Throughput of the prismatic DG hot path on one GB300 (or N independent replicas).

Metric: 3D DoF-updates per second = 6 P n_fields3D / (time of one full internal
step), P prisms, reported for the mixed FP32/FP64 form (``value``) with the plain
FP64 form beside it, plus the achieved fraction of the HBM roofline of the
dominant kernel.  ``python bench.py --gpus N --steps K --warmup W``; under
torchrun every rank runs its own replica (independent problem, weak scaling) and
rank 0 prints one JSON line.  ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "3D DoF-updates/s per time step (mixed vs FP64, 1 GB300), % of HBM roofline"
UNIT = "DoF-updates/s"


# ---------------------------------------------------------------------------
def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="basin_baroclinic", choices=sorted(wl.WORKLOADS))
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="prisms per block without the autotuner")
    ap.add_argument("--occ", type=int, default=0, help="blocks per SM without the autotuner")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-accuracy", action="store_true", help="skip the 1000-step mixed-error run")
    ap.add_argument("--layer-sweep", action="store_true",
                    help="time per step against the number of sigma layers (1..64) instead")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the z-level and reef workloads and the tracer-scheme timings")
    return ap.parse_args()


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return dict(hbm_gbs=float(d["hbm_gbs"]), src="measured")
    return dict(hbm_gbs=6800.0, src="fallback")


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
            except Exception:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["no samples"])
        load = [s for s in sm if s > 0.5 * max(sm)]
        return dict(sm_mhz=statistics.median(load), sm_max_mhz=max(mx), reasons=sorted(reasons),
                    samples=len(sm))


# ---------------------------------------------------------------------------
def workload_inputs(name: str):
    """Mesh, parameter overrides, initial fields, time step and the number of 3D
    fields a step updates."""
    W = wl.WORKLOADS[name]
    m = W["mesh"]()
    if W["scheme"] == "tracer":
        if name == "square_tracer":
            u, v = wl.c1_velocity(m)
            T = wl.c1_tracer(m)
        else:
            u, v = wl.basin_velocity(m)
            T = wl.c2_initial_state(m)["T"]
        return m, dict(kappa_v=W["kappa_v"]), dict(U=u, V=v, T=T, ETA=np.zeros(3 * m.n_tri)), W["dt"], 1
    ini = {"basin_baroclinic": wl.c2_initial_state, "basin_baroclinic_small": wl.c2_initial_state,
           "zlevel_baroclinic": wl.c4_initial_state, "reef_baroclinic": wl.c5_initial_state}[name](m)
    fields = dict(U=ini["u"], V=ini["v"], T=ini["T"], S=ini["S"], ETA=ini["eta"], QX=ini["U"], QY=ini["V"])
    par = dict(scheme=1, n_sub=W["n_sub"], kappa_v=W["kappa_v"], nu_v=W["nu_v"],
               kappa_h=W.get("kappa_h", 0.0), nu_h=W.get("nu_h", 0.0))
    dt = W["n_sub"] * wl.fields.dt_2d(m)
    return m, par, fields, dt, 4


def phase_bytes(phase: str, m, esz: int, n_sub: int) -> float:
    """Algorithmic bytes of one launch of a phase: every input read once and every
    output written once (neighbour gathers counted once), per prism P and per
    triangle n_tri.  The 2D kernel of the FP64 form moves 736 B per triangle per
    RK stage (FP64 state, geometry, averages); the mixed form's three stage
    kernels move 332, 452 and 692 B (FP32 stage values and increment sums, FP64
    state and averages only in the last stage), 492 B on average."""
    P, nt = m.n_prisms, m.n_tri
    geo = 160.0 if esz == 4 else 240.0          # per-triangle geometry + adjacency
    if phase == "tracer_stage":                  # T_p, T_n (avg), u, v, W -> T
        return P * 34.0 * esz + nt * (geo + 2 * 3 * esz)
    if phase == "continuity":                    # u, v -> W (+ 2D sums)
        return P * 18.0 * esz + nt * (geo + 9 * 8 + 3 * esz)
    if phase == "hpg":                           # T, S -> r
        return P * 24.0 * esz + nt * (geo + 3 * esz)
    if phase == "mom_pred":                      # u, v, r -> column sums
        return P * 24.0 * esz + nt * (geo + 3 * esz + 12 * 8)
    if phase in ("momentum", "tracers"):         # f_ev(2), f_0(2), u_ev(2, tracers), W, r -> f(2)
        return P * 54.0 * esz + nt * (geo + 3 * 3 * esz + 18 * esz)
    if phase == "ext2d":
        return nt * (492.0 if esz == 4 else 736.0)
    return float("nan")


# phase -> kernel function that runs it (the momentum and tracer updates are two
# instances of one kernel)
KERNEL_OF = {"split": {"continuity": "k_cont_split", "hpg": "k_hpg", "mom_pred": "k_mompred",
                       "ext2d": "k_ext2d", "momentum": "k_update", "tracers": "k_update",
                       "misc": "k_couple2d"},
             "tracer": {"continuity": "k_continuity", "tracer_stage": "k_tracer_stage",
                        "misc": "k_stretch"}}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture, valid only while the kernel sources hash to ``src``; see profiles/.
TRAFFIC = {
    # quarter-size basin capture (4 instances, 232.8 MB per launch) scaled by the prisms
    ("k_update", "mixed", "basin_baroclinic"): dict(bytes=923.2e6, src="ab7ae483b3f24cea"),
}
KSRC = ["paper_2605_16082_gb300/csrc/slim_split.cu", "paper_2605_16082_gb300/csrc/slim_split_device.cuh",
        "paper_2605_16082_gb300/csrc/slim_device.cuh", "paper_2605_16082_gb300/csrc/slim_tracer.cu",
        "paper_2605_16082_gb300/csrc/slim_internal.h"]


def kernel_src_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KSRC:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def rooflines(r: dict, m, scheme: str, pname: str, workload: str, hbm: float, peak_src: str):
    """Achieved GB/s of every kernel function over its launches in the profiled
    steps, and the dominant one (largest share of the step)."""
    esz = 8 if pname == "fp64" else 4
    groups = {}
    for ph, (ms, n) in r["phases"].items():
        k = KERNEL_OF[scheme].get(ph, ph)
        g = groups.setdefault(k, dict(ms=0.0, launches=0, bytes=0.0))
        g["ms"] += ms
        g["launches"] += n
        # the 2D bytes are per RK stage, whatever the number of launches that ran them
        units = (r.get("rk2d_stages") or n) if ph == "ext2d" else n
        g["bytes"] += phase_bytes(ph, m, esz, 0) * units
    out = {}
    for k, g in groups.items():
        if not g["launches"] or not np.isfinite(g["bytes"]):
            continue
        ach = g["bytes"] / (g["ms"] / 1e3) / 1e9
        out[k] = dict(achieved=ach, frac=ach / hbm, launch_ms=g["ms"] / g["launches"],
                      launches=g["launches"], alg_bytes_per_launch=g["bytes"] / g["launches"])
    dom = max(out, key=lambda k: out[k]["launch_ms"] * out[k]["launches"])
    d = out[dom]
    tr = TRAFFIC.get((dom, pname, workload))
    traffic = tr["bytes"] if tr and tr["src"] == kernel_src_hash() else None
    head = dict(kernel=dom, bound="hbm", achieved=d["achieved"], peak=hbm, unit="GB/s",
                frac=d["frac"], traffic=traffic, peak_src=peak_src, launch_ms=d["launch_ms"],
                alg_bytes_per_launch=d["alg_bytes_per_launch"])
    return head, {k: dict(achieved=round(v["achieved"], 1), frac=round(v["frac"], 4),
                          launch_ms=round(v["launch_ms"], 5), launches=v["launches"])
                  for k, v in out.items()}


# FP64 arithmetic of the dominant FP64 kernel per launch, counted by ncu on the same
# sources (2 x DFMA + DADD + DMUL executed, sm__sass_thread_inst_executed_op_d*),
# valid only while the kernel sources hash to ``src``; see profiles/.
FP64_FLOPS = {
    # quarter-size basin capture (2,344 FLOP per prism per launch) scaled by the prisms
    ("k_update", "basin_baroclinic"): dict(flops_per_launch=7.8027e9, src="ab7ae483b3f24cea"),
}


def alu_peaks(slim, sms: int) -> dict:
    """Measured FMA throughput of the library's FMA-loop kernel in FP64 and FP32 with
    the SM clock sampled meanwhile, and the FP64 peak derived from the unit count
    (GB300: 2 FP64 FMA per SM per clock) at that clock."""
    samp = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    samp.start()
    f64, ms64 = slim.slim_selftest_fma_peak(slim.SLIM_FP64, 1 << 15)
    f32, ms32 = slim.slim_selftest_fma_peak(slim.SLIM_MIXED, 1 << 20)
    clk = samp.stop()
    mhz = clk.get("sm_mhz") or 2070.0
    return dict(fp64_measured_tflops=f64 / 1e12, fp32_measured_tflops=f32 / 1e12,
                fp64_derived_tflops=sms * 2 * 2 * mhz * 1e6 / 1e12, sms=sms, sm_mhz=mhz,
                derivation="SMs x 2 FP64 FMA/clock x 2 FLOP x median SM clock under load",
                kernel="8 blocks of 256 threads per SM, 8 independent FMA chains per thread",
                clocks=clk)


def time_workload(slim, torch, name: str, prec: int, steps: int, warmup: int, tile: int, occ: int = 4,
                  profile: bool = True, **extra) -> dict:
    """One workload at a fixed tiling (no autotuner): CUDA-event time of `steps`
    graph-replayed steps after `warmup`, clocks sampled meanwhile, and (profile)
    the per-kernel phase times of as many more launched steps."""
    W = wl.WORKLOADS[name]
    m, over, fields, dt, nf = workload_inputs(name)
    over = dict(over, **extra)
    par = slim.slim_params_default(**over)
    par.tile_prisms, par.blocks_per_sm = tile, occ
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with slim.Model(m, prec, par) as mod:
        torch.cuda.synchronize()
        dev_bytes = free0 - torch.cuda.mem_get_info()[0]
        for k, v in fields.items():
            mod.upload(k, v)
        t = 0.0
        for _ in range(warmup):
            slim.slim_step(mod.state, t, dt, sh); t += dt
        samp = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
        samp.start()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            slim.slim_step(mod.state, t, dt, sh); t += dt
        e1.record(stream)
        torch.cuda.synchronize()
        clk = samp.stop()
        ms = e0.elapsed_time(e1) / steps
        r = dict(n_tri=m.n_tri, n_prisms=m.n_prisms, layers=int(m.n_layers.max()),
                 min_layers=int(m.n_layers.min()), ms_per_step=ms, value=6.0 * m.n_prisms * nf / (ms / 1e3),
                 steps=steps, warmup=warmup, clocks=clk, device_bytes=dev_bytes,
                 tiling=dict(prisms_per_block=tile, blocks_per_sm=occ))
        if profile:
            n_k = slim.slim_step_kernel_count(mod.state)
            slim.slim_profile_begin(mod.state, n_k * steps + 8)
            for _ in range(steps):
                slim.slim_step(mod.state, t, dt, sh); t += dt
            torch.cuda.synchronize()
            r["phases"] = slim.slim_profile_end(mod.state)
            r["rk2d_stages"] = 3 * (par.n_sub // 2 + par.n_sub) * steps if W["scheme"] == "split" else 0
        slim.slim_state_check(mod.state, sh)
    return r


def _build_mesh(name: str) -> None:
    wl.WORKLOADS[name]["mesh"]()


def start_mesh_build(name: str):
    """Build (and cache on disk) a slow-to-generate mesh in a spawned process while
    this one times the GPU."""
    import multiprocessing as mp
    p = mp.get_context("spawn").Process(target=_build_mesh, args=(name,))
    p.start()
    return p


def extra_workloads(slim, torch, args, hbm: float, peak_src: str, reef_proc) -> dict:
    """The z-level basin (uneven columns, 11.4M prisms) and the reef stress mesh
    (41.4M prisms) in the mixed form, each with its roofline and clocks."""
    out = {}
    for name, tile, steps in (("zlevel_baroclinic", 256, 5), ("reef_baroclinic", 512, 3)):
        if name == "reef_baroclinic" and reef_proc is not None:
            reef_proc.join()
        r = time_workload(slim, torch, name, slim.SLIM_MIXED, steps, 2, tile)
        m = types_ns(r)
        head, allk = rooflines(r, m, "split", "mixed", name, hbm, peak_src)
        r.pop("phases"); r.pop("rk2d_stages")
        r.update(roofline=head, roofline_all=allk, precision="mixed")
        out[name] = r
    return out


def types_ns(r: dict):
    import types
    return types.SimpleNamespace(n_prisms=r["n_prisms"], n_tri=r["n_tri"])


def tracer_scheme_times(slim, torch, steps: int = 50) -> dict:
    """Square-basin tracer workload (2048 triangles x 10 layers, dt = 5 s) with the
    lumped 2x2-block and the coupled 6x6-block column systems, both precisions:
    CUDA-event ms per step and DoF-updates/s (one 3D field)."""
    out = {}
    for vname, v in (("lumped", slim.SLIM_VERTICAL_LUMPED), ("coupled", slim.SLIM_VERTICAL_COUPLED)):
        for pname, prec in (("fp64", slim.SLIM_FP64), ("mixed", slim.SLIM_MIXED)):
            r = time_workload(slim, torch, "square_tracer", prec, steps, 5, 256, profile=False, vertical=v)
            out.setdefault(vname, {})[pname] = dict(ms_per_step=r["ms_per_step"], value=r["value"])
    out.update(workload="square_tracer", n_prisms=20480, unit=UNIT, steps=steps)
    return out


def halo_times(slim, torch, steps: int = 10, warmup: int = 3) -> dict:
    """The partitioned tracer step on one device (basin tracer workload: 197,480
    triangles x 20 layers, mixed form): one state launching every kernel, and 2
    and 4 partitions with one ghost layer, boundary tiles first and the halo
    exchange of every stage output overlapping the interior tiles.  CUDA-event ms
    per step; the differences to the single state are the cost of the partitioned
    path (the split launches and the exchanges)."""
    name = "basin_tracer"
    m, over, fields, dt, nf = workload_inputs(name)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    out = dict(workload=name, n_tri=m.n_tri, n_prisms=m.n_prisms, precision="mixed", steps=steps)

    def timed(step):
        for i in range(warmup):
            step(i)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(steps):
            step(warmup + i)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    par = slim.slim_params_default(**over)
    par.use_graph = 0
    with slim.Model(m, slim.SLIM_MIXED, par, tile_prisms=256) as mod:
        for k, v in fields.items():
            mod.upload(k, v)
        out["one_state_ms"] = timed(lambda i: slim.slim_step(mod.state, i * dt, dt, sh))
    for K in (2, 4):
        with slim.PartitionedModel(m, K, slim.SLIM_MIXED, par, tile_prisms=256) as pm:
            for k, v in fields.items():
                pm.upload(k, v)
            ms = timed(lambda i: pm.step(i * dt, dt, sh))
            ghosts = int(sum(p.n_tri - p.n_owned for p in pm.pt.parts))
        out[f"parts{K}_ms"] = ms
        out[f"parts{K}_ghost_triangles"] = ghosts
        out[f"parts{K}_overhead"] = ms / out["one_state_ms"] - 1.0
    return out


def run_ours(args, rank: int, world: int):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2605_16082_gb300 import slim

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    m, over, fields, dt, nf = workload_inputs(args.workload)
    W = wl.WORKLOADS[args.workload]
    dofs = 6.0 * m.n_prisms * nf
    precs = {"both": ["mixed", "fp64"], "mixed": ["mixed"], "fp64": ["fp64"]}[args.precision]
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    res = {}
    clocks = None
    tuned = {}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    res["alu_peaks"] = alu_peaks(slim, sms)
    for pname in precs:
        prec = slim.SLIM_MIXED if pname == "mixed" else slim.SLIM_FP64
        par = slim.slim_params_default(**over)
        if not args.no_tune:
            from paper_2605_16082_gb300 import autotune
            tn = autotune.autotune(m, prec, par, fields, dt, use_cache=False)
            par.tile_prisms = tn["tile_prisms"]
            par.blocks_per_sm = tn["blocks_per_sm"]
            par.persistent_2d = tn.get("persistent_2d", par.persistent_2d)
            tuned[pname] = tn
        else:
            if args.tile:
                par.tile_prisms = args.tile
            if args.occ:
                par.blocks_per_sm = args.occ
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        mod = slim.Model(m, prec, par)
        torch.cuda.synchronize()
        dev_bytes = free0 - torch.cuda.mem_get_info()[0]
        for k, v in fields.items():
            mod.upload(k, v)
        t = 0.0
        for _ in range(args.warmup):
            slim.slim_step(mod.state, t, dt, sh); t += dt
        torch.cuda.synchronize()
        barrier(world)
        sampler = ClockSampler(dev) if pname == precs[0] else None
        if sampler:
            sampler.start()
        n_k = slim.slim_step_kernel_count(mod.state)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        for _ in range(args.steps):
            slim.slim_step(mod.state, t, dt, sh); t += dt
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = e0.elapsed_time(e1)
        # per-kernel durations: the same K steps again with an event pair around
        # every kernel (launched individually while profiling)
        slim.slim_profile_begin(mod.state, n_k * args.steps + 8)
        for _ in range(args.steps):
            slim.slim_step(mod.state, t, dt, sh); t += dt
        torch.cuda.synchronize()
        phases = slim.slim_profile_end(mod.state)
        if sampler:
            clocks = sampler.stop()
        slim.slim_state_check(mod.state, sh)
        ms = allmax(ms, world)
        ms_step = ms / args.steps
        # 2D RK stages in the profiled steps (stage 1 runs n_sub/2 subcycles, stage 2
        # n_sub): the persistent 2D kernel does a whole split stage per launch
        rk2d = 3 * (par.n_sub // 2 + par.n_sub) * args.steps if W["scheme"] == "split" else 0
        r = dict(value=world * dofs / (ms_step / 1e3), ms_per_step=ms_step, phases=phases,
                 gpu_launches=n_k * args.steps, rk2d_stages=rk2d,
                 tile_prisms=par.tile_prisms, blocks_per_sm=par.blocks_per_sm,
                 persistent_2d=int(par.persistent_2d), device_bytes=dev_bytes,
                 autotune=tuned.get(pname, {}).get("all"))
        # end to end through the public API with pinned host buffers
        if not args.no_e2e:
            pin = {k: torch.tensor(v, dtype=torch.float64).pin_memory() for k, v in fields.items()}
            outs = {k: torch.empty(b.numel(), dtype=torch.float64).pin_memory() for k, b in pin.items()
                    if k in ("T", "ETA", "U", "V", "S")}
            ids = {k: slim.FIELD[k] for k in pin}
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                for k, buf in pin.items():
                    slim.slim_state_upload_ptr(mod.state, ids[k], buf.data_ptr(), sh)
                slim.slim_step(mod.state, t, dt, sh); t += dt
                for k, buf in outs.items():
                    slim.slim_state_download_ptr(mod.state, slim.FIELD[k], buf.data_ptr(), sh)
            torch.cuda.synchronize()
            barrier(world)
            e2e_s = allmax(time.perf_counter() - t0, world) / args.steps
            r["e2e"] = dict(value=world * dofs / e2e_s, unit=UNIT,
                            h2d_bytes_per_step=int(sum(b.numel() * 8 for b in pin.values())),
                            d2h_bytes_per_step=int(sum(b.numel() * 8 for b in outs.values())))
        mod.close()
        res[pname] = r
    return m, res, clocks


def mixed_accuracy(steps: int = 1000) -> dict:
    """Mixed against FP64 on the square-basin tracer run (2048 triangles x 10
    layers, dt = 5 s) after ``steps`` steps: tracer relative L2 error and the tracer
    mass drift of both forms (outside the timed region)."""
    from paper_2605_16082_gb300 import slim
    W = wl.WORKLOADS["square_tracer"]
    m = W["mesh"]()
    u, v = wl.c1_velocity(m)
    T = wl.c1_tracer(m)
    out = {}
    for pname, prec in (("fp64", slim.SLIM_FP64), ("mixed", slim.SLIM_MIXED)):
        with slim.Model(m, prec, slim.slim_params_default(kappa_v=W["kappa_v"])) as mod:
            for k, f in (("U", u), ("V", v), ("T", T), ("ETA", np.zeros(3 * m.n_tri))):
                mod.upload(k, f)
            m0 = slim.slim_tracer_mass(mod.state, 0)
            for n in range(steps):
                slim.slim_step(mod.state, n * W["dt"], W["dt"])
            out[pname] = (mod.download("T"), (slim.slim_tracer_mass(mod.state, 0) - m0) / m0)
    a, b = out["mixed"][0], out["fp64"][0]
    res = dict(workload="square_tracer", steps=steps,
               tracer_rel_l2_mixed_vs_fp64=float(np.linalg.norm(a - b) / np.linalg.norm(b)),
               bar=1e-5, mass_drift_mixed=float(out["mixed"][1]), mass_drift_fp64=float(out["fp64"][1]))
    res["split"] = split_accuracy()
    return res


def split_accuracy(steps: int = 200) -> dict:
    """Mixed against FP64 for the split step on a small tidal basin (2,490 triangles
    x 5 sigma layers, n_sub = 20, M2 at the open boundary, about 2.6 h of model
    time) after ``steps`` steps: relative L2 error of every prognostic field, and
    the FP64 run's largest speed."""
    from paper_2605_16082_gb300 import slim
    m = wl.c2_mesh(2500, 5, 0)
    ini = wl.c2_initial_state(m)
    fields = dict(U=ini["u"], V=ini["v"], T=ini["T"], S=ini["S"], ETA=ini["eta"], QX=ini["U"], QY=ini["V"])
    par = dict(scheme=1, n_sub=20, kappa_v=1e-3, nu_v=1e-3, kappa_h=1.0, nu_h=1.0)
    dt = 20 * wl.fields.dt_2d(m)
    names = ("U", "V", "T", "S", "ETA", "QX", "QY")
    out = {}
    for pname, prec in (("fp64", slim.SLIM_FP64), ("mixed", slim.SLIM_MIXED)):
        with slim.Model(m, prec, slim.slim_params_default(**par)) as mod:
            for k, f in fields.items():
                mod.upload(k, f)
            for n in range(steps):
                slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            out[pname] = {k: mod.download(k) for k in names}
    rel = {k: float(np.linalg.norm(out["mixed"][k] - out["fp64"][k]) / np.linalg.norm(out["fp64"][k]))
           for k in names}
    return dict(workload="small tidal basin", steps=steps, rel_l2_mixed_vs_fp64=rel,
                max_abs_u_fp64=float(np.abs(out["fp64"]["U"]).max()))


SWEEP_LAYERS = (1, 2, 3, 4, 6, 8, 10, 12, 16, 20, 24, 32, 40, 48, 56, 64)


def layer_sweep(args) -> dict:
    """Mixed split step against the number of uniform sigma layers on one horizontal
    mesh (the basin generator at ~50k triangles, n_sub = 20): each layer count with
    its autotuned tiling, timed with CUDA events after warm-up; reported per step and
    per prism (the block structure of whole-column tiles shows in the latter)."""
    import dataclasses
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2605_16082_gb300 import autotune, slim
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    base = wl.c2_mesh(50_000, 1, 0)
    stream = torch.cuda.current_stream()
    rows = []
    for N in SWEEP_LAYERS:
        m = dataclasses.replace(base, n_layers=np.full(base.n_tri, N, np.int32))
        ini = wl.c2_initial_state(m)
        fields = dict(U=ini["u"], V=ini["v"], T=ini["T"], S=ini["S"], ETA=ini["eta"], QX=ini["U"],
                      QY=ini["V"])
        par = slim.slim_params_default(scheme=1, n_sub=20, kappa_v=1e-3, nu_v=1e-3, kappa_h=1.0,
                                       nu_h=1.0)
        dt = 20 * wl.fields.dt_2d(m)
        tn = autotune.autotune(m, slim.SLIM_MIXED, par, fields, dt, use_cache=False)
        par.tile_prisms, par.blocks_per_sm = tn["tile_prisms"], tn["blocks_per_sm"]
        par.persistent_2d = tn.get("persistent_2d", par.persistent_2d)
        with slim.Model(m, slim.SLIM_MIXED, par) as mod:
            for k, v in fields.items():
                mod.upload(k, v)
            t = 0.0
            for _ in range(max(3, args.warmup)):
                slim.slim_step(mod.state, t, dt, stream.cuda_stream); t += dt
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                slim.slim_step(mod.state, t, dt, stream.cuda_stream); t += dt
            e1.record(stream)
            torch.cuda.synchronize()
            slim.slim_state_check(mod.state)
            ms = e0.elapsed_time(e1) / args.steps
        P = int(m.n_layers.sum())
        rows.append(dict(layers=N, prisms=P, ms_per_step=ms, ns_per_prism_step=ms * 1e6 / P,
                         dof_updates_per_s=6.0 * P * 4 / (ms / 1e3),
                         prisms_per_block=tn["tile_prisms"], blocks_per_sm=tn["blocks_per_sm"],
                         persistent_2d=int(par.persistent_2d)))
    return dict(layer_sweep=rows, n_tri=base.n_tri, precision="mixed", scheme="split", n_sub=20,
                steps=args.steps)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x: float, world: int) -> float:
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
def host_cpu() -> dict:
    """Host cores and CPU model (lscpu, else /proc/cpuinfo)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as fh:
                for line in fh:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return dict(nproc=os.cpu_count() or 1, model=model or "unknown")


def _patch(workload: str, m, n_patch: int, first: int):
    """Sub-mesh of n_patch consecutive (Hilbert-ordered) columns starting at first;
    cut edges become walls, open-boundary edges stay open."""
    from workloads.meshes import Mesh
    idx = np.arange(first, min(first + n_patch, m.n_tri))
    bnd = m.bnd[idx].copy()
    sub = Mesh(xy=m.xy, tri=m.tri[idx], h_tri=m.h_tri[idx], n_layers=m.n_layers[idx], bnd=bnd,
               levels=m.levels)
    topo = wl.meshes._tag_boundary(sub.xy, sub.tri, None)
    sub.bnd = np.where((topo == 1) & (bnd == 2), 2, topo).astype(np.int8)
    return sub


def _oracle_worker(job):
    """One oracle process: its own patch of the workload, `warm` untimed steps, then
    steps until `seconds` elapse (at least `min_steps`).  Returns (prisms, fields,
    timed steps, timed seconds)."""
    workload, m, n_patch, first, seconds, warm, min_steps, dt_full = job
    from oracle import tracer as otr
    from oracle import baroclinic as obc
    from oracle.mesh import OMesh
    W = wl.WORKLOADS[workload]
    sub = _patch(workload, m, n_patch, first)
    om = OMesh(sub)
    P = om.P
    if W["scheme"] == "tracer":
        if workload == "square_tracer":
            u, v = wl.c1_velocity(sub); T = wl.c1_tracer(sub)
        else:
            u, v = wl.basin_velocity(sub); T = wl.c2_initial_state(sub)["T"]
        state = [np.zeros((3, sub.n_tri)), otr.to3(T, P)]
        u, v = otr.to3(u, P), otr.to3(v, P)
        nf = 1

        def step(k):
            state[0], state[1], _ = otr.tracer_step(om, state[0], state[1], u, v, W["dt"], W["kappa_v"])
    else:
        ini = {"basin_baroclinic": wl.c2_initial_state, "basin_baroclinic_small": wl.c2_initial_state,
               "zlevel_baroclinic": wl.c4_initial_state, "reef_baroclinic": wl.c5_initial_state}[workload](sub)
        st = obc.State(u=otr.to3(ini["u"], P), v=otr.to3(ini["v"], P), T=otr.to3(ini["T"], P),
                       S=otr.to3(ini["S"], P), eta=otr.to2(ini["eta"], sub.n_tri),
                       U=otr.to2(ini["U"], sub.n_tri), V=otr.to2(ini["V"], sub.n_tri))
        st.T_ext, st.S_ext = st.T.copy(), st.S.copy()
        par = obc.Params(n_sub=W["n_sub"], kappa_v=W["kappa_v"], nu_v=W["nu_v"],
                         kappa_h=W.get("kappa_h", 0.0), nu_h=W.get("nu_h", 0.0))
        state = [st]
        nf = 4

        def step(k):
            state[0] = obc.split_step(om, par, state[0], k * dt_full, dt_full)
    for k in range(warm):
        step(k)
    n = 0
    t0 = time.perf_counter()
    while True:
        step(warm + n)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds and n >= min_steps:
            break
    return P, nf, n, el


def oracle_run(workload: str, m, seconds: float, cores: int, warm: int = 0, min_steps: int = 1) -> dict:
    """The oracle as it stands on bounded samples of the workload: `cores` processes
    (spawned: this process may hold a CUDA context), each stepping its own patch of
    consecutive columns.  Throughput is the sum over the processes."""
    import multiprocessing as mp
    W = wl.WORKLOADS[workload]
    n_patch = min(m.n_tri, 1200 if W["scheme"] == "tracer" else 400)
    dt_full = W["n_sub"] * wl.fields.dt_2d(m) if W["scheme"] == "split" else W["dt"]
    n_avail = max(1, m.n_tri // n_patch)
    jobs = [(workload, m, n_patch, (j % n_avail) * n_patch, seconds, warm, min_steps, dt_full)
            for j in range(cores)]
    if cores == 1:
        res = [_oracle_worker(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, jobs)
    value = sum(6.0 * P * nf * n / el for P, nf, n, el in res)
    steps = [n for _, _, n, _ in res]
    el = max(e for _, _, _, e in res)
    P0 = res[0][0]
    return dict(value=value, unit=UNIT, cores=cores, kind="oracle", steps_per_process=steps,
                prisms_per_process=P0,
                seconds=el, ms_per_step=1e3 * sum(e / n for _, _, n, e in res) / len(res),
                sample=f"{cores} process(es) x {n_patch} columns ({P0} prisms) of {workload}, "
                       f"{min(steps)}-{max(steps)} timed steps each in {el:.1f} s, numpy FP64, "
                       f"1 thread per process")


def cpu_baseline(workload: str, m, seconds: float) -> dict:
    """The oracle at every host core (one process per core) and at one core."""
    cpu = host_cpu()
    one = oracle_run(workload, m, 0.4 * seconds, 1)
    allc = oracle_run(workload, m, 0.6 * seconds, cpu["nproc"])
    out = dict(allc)
    out.update(cpu_model=cpu["model"], nproc=cpu["nproc"], value_1core=one["value"],
               sample_1core=one["sample"])
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    W = wl.WORKLOADS[args.workload]
    cfg = dict(workload=args.workload, scheme=W["scheme"], n_sub=W.get("n_sub"),
               l2="working set per step > L2 (no flush needed)")
    if args.impl == "reference":
        if rank != 0:
            return
        m = W["mesh"]()
        cpu = host_cpu()
        # every process steps its own bounded patch of the workload: W untimed steps,
        # then at least K timed ones (about --cpu-seconds of CPU work per process)
        cb = oracle_run(args.workload, m, args.cpu_seconds, cpu["nproc"], warm=args.warmup,
                        min_steps=args.steps)
        cb.update(cpu_model=cpu["model"], nproc=cpu["nproc"])
        cfg.update(n_tri=m.n_tri, n_prisms=m.n_prisms, layers=int(m.n_layers.max()),
                   sample=cb["sample"], sample_prisms_per_process=cb["prisms_per_process"])
        line = dict(impl="reference", metric=METRIC, value=cb["value"], unit=UNIT, n_gpus=args.gpus,
                    steps=args.steps, warmup=args.warmup, ms_per_step=cb["ms_per_step"],
                    higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                    data="synthetic", config=cfg, cpu_baseline=cb,
                    e2e=dict(value=cb["value"], unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line))
        return
    if args.layer_sweep:
        if rank == 0:
            print(json.dumps(layer_sweep(args)))
        return
    reef_proc = None
    if rank == 0 and not args.no_extra and args.workload == "basin_baroclinic":
        reef_proc = start_mesh_build("reef_baroclinic")
    m, res, clocks = run_ours(args, rank, world)
    alu = res.pop("alu_peaks")
    cfg.update(n_tri=m.n_tri, n_prisms=m.n_prisms, layers=int(m.n_layers.max()),
               parallelism=f"replicas{world}")
    if rank != 0:
        return
    pk = peaks()
    head = res.get("mixed") or res["fp64"]
    hname = "mixed" if "mixed" in res else "fp64"

    def roof(r, pname):
        return rooflines(r, m, W["scheme"], pname, args.workload, pk["hbm_gbs"], pk["src"])

    line = dict(metric=METRIC, value=head["value"], unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=head["ms_per_step"], higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32+f64" if hname == "mixed" else "f64",
                data="synthetic", config=cfg, roofline=roof(head, hname)[0],
                roofline_all=roof(head, hname)[1], clocks=clocks,
                gpu_launches=head["gpu_launches"], phases_ms={k: v[0] for k, v in head["phases"].items()},
                device_bytes=head["device_bytes"],
                tiling=dict(prisms_per_block=head["tile_prisms"], blocks_per_sm=head["blocks_per_sm"],
                            persistent_2d=head["persistent_2d"], autotune_ms=head["autotune"]),
                cuda_graph=True)
    if "e2e" in head:
        line["e2e"] = head["e2e"]
    if "fp64" in res and hname != "fp64":
        f = res["fp64"]
        line["fp64"] = dict(value=f["value"], ms_per_step=f["ms_per_step"], roofline=roof(f, "fp64")[0],
                            roofline_all=roof(f, "fp64")[1],
                            e2e=f.get("e2e"), phases_ms={k: v[0] for k, v in f["phases"].items()},
                            device_bytes=f["device_bytes"],
                            tiling=dict(prisms_per_block=f["tile_prisms"], blocks_per_sm=f["blocks_per_sm"]))
        fl = FP64_FLOPS.get((line["fp64"]["roofline"]["kernel"], args.workload))
        flops = fl["flops_per_launch"] if fl and fl["src"] == kernel_src_hash() else None
        lm = line["fp64"]["roofline"]["launch_ms"]
        ach = flops / (lm / 1e3) / 1e12 if flops else None
        line["fp64"]["roofline_alu"] = dict(
            kernel=line["fp64"]["roofline"]["kernel"], bound="alu", unit="TFLOP/s", achieved=ach,
            peak=alu["fp64_derived_tflops"], peak_src="derived (unit count x sampled clock)",
            peak_measured=alu["fp64_measured_tflops"],
            frac=(ach / alu["fp64_derived_tflops"]) if ach else None,
            flops_per_launch=flops, flops_src="ncu executed FP64 instructions (2 DFMA + DADD + DMUL)")
    line["alu_peaks"] = alu
    if not args.no_accuracy and "mixed" in res:
        line["mixed_accuracy"] = mixed_accuracy()
    if not args.no_extra and args.workload == "basin_baroclinic":
        import torch
        from paper_2605_16082_gb300 import slim
        line["extra_workloads"] = extra_workloads(slim, torch, args, pk["hbm_gbs"], pk["src"], reef_proc)
        line["tracer_scheme"] = tracer_scheme_times(slim, torch)
        line["partitioned"] = halo_times(slim, torch)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.workload, m, args.cpu_seconds)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
