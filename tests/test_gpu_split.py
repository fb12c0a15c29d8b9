"""GPU parity of the baroclinic split-IMEX path (C ABI) against the FP64 oracle.

FP64 bar: relative L2 <= 1e-12 per field per step, and every node within 1e-12
of the field's largest magnitude (3D u, v, T, S; 2D eta, U, V; the stage-2
intermediates Qbar, S3, F2D and the vertical flux W; 1e-11 for the pressure
gradient r, see TOL_R).  Cases: a graded basin with an
open tidal boundary (several tiles, ragged last tile), a square basin, and a
z-level basin with uneven columns (1..N layers, walls against shallower
neighbours)."""
import copy

import numpy as np
import pytest

import workloads as wl
from helpers import (assert_close, prisms_of, rel_l2, restrict2, restrict3, ring_submesh,
                     split_case_mesh as case_mesh, split_initial as initial)

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
# The pressure gradient r is a gradient along sloping coordinate surfaces: nodal
# depths of O(100 m) enter through their differences across a triangle.  One
# rounding of its inputs moves r by 1.8e-12 of its norm on the graded basin
# (test_oracle_rounding.py), so r is compared at 1e-11; every other field at 1e-12.
TOL_R = 1e-11


@pytest.fixture(scope="module")
def slim():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2605_16082_gb300 import slim as s
    torch.cuda.init()
    return s


def params(slim, **kw):
    base = dict(scheme=slim.SLIM_SCHEME_SPLIT, n_sub=4, nu_h=0.5, kappa_h=0.5, tide_amp=0.4,
                tide_period=3600.0)
    base.update(kw)
    return slim.slim_params_default(**base)


def oracle_params(p):
    from oracle import baroclinic as bc
    return bc.Params(g=p.g, rho0=p.rho0, f=p.coriolis_f, alpha=p.eos_alpha, beta=p.eos_beta,
                     T0=p.eos_T0, S0=p.eos_S0, kappa_v=p.kappa_v, nu_v=p.nu_v, kappa_h=p.kappa_h,
                     nu_h=p.nu_h, cd=p.drag_cd, penalty_v=p.penalty_v, penalty_h=p.penalty_h,
                     tide_amp=p.tide_amp, tide_period=p.tide_period, n_sub=p.n_sub,
                     forcing=bool(p.forcing))


def oracle_state(m, om, ini):
    from oracle import baroclinic as bc
    from oracle import tracer as tr
    P, nt = om.P, m.n_tri
    st = bc.State(u=tr.to3(ini["U"], P), v=tr.to3(ini["V"], P), T=tr.to3(ini["T"], P),
                  S=tr.to3(ini["S"], P), eta=tr.to2(ini["ETA"], nt), U=tr.to2(ini["QX"], nt),
                  V=tr.to2(ini["QY"], nt))
    st.T_ext = st.T.copy()
    st.S_ext = st.S.copy()
    return st


def model(slim, m, prec, p, ini, tile=256):
    mod = slim.Model(m, prec, p, tile_prisms=tile)
    for k, v in ini.items():
        mod.upload(k, v)
    return mod


@pytest.mark.parametrize("case", ["basin", "square", "zlevel"])
def test_hpg_parity(slim, case):
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m = case_mesh(case)
    ini = initial(m)
    p = params(slim)
    om = OMesh(m)
    st = oracle_state(m, om, ini)
    with model(slim, m, slim.SLIM_FP64, p, ini) as mod:
        assert mod.info["n_tiles"] > 1
        slim.slim_hpg(mod.state)
        rx, ry = mod.download("R_X"), mod.download("R_Y")
    ox, oy = bc.hpg(om, oracle_params(p), st.T, st.S, st.eta)
    assert_close(rx, ox, TOL_R)
    assert_close(ry, oy, TOL_R)


@pytest.mark.parametrize("case", ["basin", "square"])
def test_rhs2d_parity(slim, case):
    import torch
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m = case_mesh(case)
    ini = initial(m)
    p = params(slim)
    om = OMesh(m)
    st = oracle_state(m, om, ini)
    with model(slim, m, slim.SLIM_FP64, p, ini) as mod:
        out = torch.zeros(9 * m.n_tri, dtype=torch.float64, device="cuda")
        slim.slim_rhs2d(mod.state, 1234.5, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(3, 3, m.n_tri)
    Re, RU, RV, _ = bc.mode2d_residual(om, oracle_params(p), st.eta, st.U, st.V, 1234.5)
    assert_close(got[0], Re, TOL64)
    assert_close(got[1], RU, TOL64)
    assert_close(got[2], RV, TOL64)


@pytest.mark.parametrize("case", ["basin", "square", "zlevel"])
def test_rhs3d_momentum_parity(slim, case):
    """slim_rhs3d of U and V: F_3D^h of the state (advection by the uncorrected
    transport, SIPG viscosity, Coriolis, -r/rho0 with r from the state's T and S,
    bed drag) and its FP64 column sums S3, element by element against the oracle;
    the basin and square cases have an open boundary, the z-level case walls
    against shallower columns."""
    import torch
    from oracle import baroclinic as bc
    from oracle import tracer as tr
    from oracle.mesh import OMesh
    m = case_mesh(case)
    ini = initial(m, 2)
    p = params(slim)
    om = OMesh(m)
    st = oracle_state(m, om, ini)
    par = oracle_params(p)
    with model(slim, m, slim.SLIM_FP64, p, ini) as mod:
        assert mod.info["n_tiles"] > 1
        got = []
        for f in (slim.FIELD["U"], slim.FIELD["V"]):
            out = torch.zeros(6 * mod.P, dtype=torch.float64, device="cuda")
            slim.slim_rhs3d(mod.state, f, out.data_ptr())
            torch.cuda.synchronize()
            got.append(out.cpu().numpy())
        s3 = (mod.download("S3_X"), mod.download("S3_Y"))
    dz = om.thickness(st.eta)
    rx, ry = bc.hpg(om, par, st.T, st.S, st.eta)
    qx, qy = tr.transport(dz, st.u, st.v)
    Fx, Fy = bc.momentum_horizontal(om, par, st.u, st.v, qx, qy, rx, ry, dz, ext=(None, None, None, None))
    assert_close(got[0], Fx, TOL64, "Fx")
    assert_close(got[1], Fy, TOL64, "Fy")
    assert_close(s3[0], tr.column_sum(om, Fx), TOL64, "S3x")
    assert_close(s3[1], tr.column_sum(om, Fy), TOL64, "S3y")


FIELDS3 = [("U", "u"), ("V", "v"), ("T", "T"), ("S", "S")]
FIELDS2 = [("ETA", "eta"), ("QX", "U"), ("QY", "V")]


@pytest.mark.parametrize("case", ["basin", "square", "zlevel"])
def test_split_step_parity_fp64(slim, case):
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m = case_mesh(case)
    ini = initial(m)
    p = params(slim)
    om = OMesh(m)
    st = oracle_state(m, om, ini)
    par = oracle_params(p)
    dt = 10.0 * wl.fields.dt_2d(m)
    with model(slim, m, slim.SLIM_FP64, p, ini) as mod:
        for n in range(2):
            d1, d2 = {}, {}
            st = bc.split_step(om, par, st, n * dt, dt, d1, d2)
            slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            for f, o in FIELDS3 + FIELDS2:
                assert_close(mod.download(f), getattr(st, o), TOL64, (n, f))
            assert_close(mod.download("R_X"), d2["r"][0], TOL_R, (n, "r"))
            assert_close(mod.download("W"), d2["W"], TOL64, (n, "W"))
            assert_close(mod.download("QBAR_X"), d2["Qbar"][0], TOL64, (n, "Qbar"))
            assert_close(mod.download("S3_X"), d2["S3"][0], TOL64, (n, "S3"))
            assert_close(mod.download("F2D_Y"), d2["F2D"][1], TOL64, (n, "F2D"))


def test_split_long_run_parity_fp64(slim):
    """100 steps (1.3 h, 1 m tide of period 1 h: currents up to 0.4 m/s, upwind
    directions switching) from the stratified rest state of a small basin
    (550 triangles x 3 layers, n_sub = 20, the workload's step 20 dt_2d): the FP64
    path follows the oracle step after step.  Rounding accumulates over the steps,
    so the bar is 1e-10 instead of the per-step 1e-12."""
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m = wl.c2_mesh(300, 3, 0)
    c2 = wl.c2_initial_state(m)
    ini = dict(U=c2["u"], V=c2["v"], T=c2["T"], S=c2["S"], ETA=c2["eta"], QX=c2["U"], QY=c2["V"])
    p = params(slim, n_sub=20, kappa_v=1e-3, nu_v=1e-3, kappa_h=1.0, nu_h=1.0, tide_amp=1.0)
    om = OMesh(m)
    st = oracle_state(m, om, ini)
    par = oracle_params(p)
    dt = 20.0 * wl.fields.dt_2d(m)
    with model(slim, m, slim.SLIM_FP64, p, ini) as mod:
        for n in range(100):
            st = bc.split_step(om, par, st, n * dt, dt)
            slim.slim_step(mod.state, n * dt, dt)
            if n + 1 in (50, 100):
                slim.slim_state_check(mod.state)
                for f, o in FIELDS3 + FIELDS2:
                    assert_close(mod.download(f), getattr(st, o), 1e-10, (n + 1, f))
        assert np.abs(st.u).max() > 0.2


def test_split_step_parity_tiles(slim):
    """Same step with every tile size gives the oracle's result."""
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m = case_mesh("basin")
    ini = initial(m, 1)
    p = params(slim)
    om = OMesh(m)
    st = bc.split_step(om, oracle_params(p), oracle_state(m, om, ini), 0.0, 30.0)
    for tile in (128, 512):
        with model(slim, m, slim.SLIM_FP64, p, ini, tile=tile) as mod:
            slim.slim_step(mod.state, 0.0, 30.0)
            for f, o in FIELDS3 + FIELDS2:
                assert_close(mod.download(f), getattr(st, o), TOL64, (tile, f))


def test_split_lake_at_rest_gpu(slim):
    m = case_mesh("basin")
    x, y, z, s = wl.fields.node_positions_sigma(m)
    ini = wl.c2_initial_state(m)
    p = params(slim, tide_amp=0.0, kappa_v=0.0, kappa_h=0.0)
    for prec, tol in ((slim.SLIM_FP64, 1e-12), (slim.SLIM_MIXED, 1e-5)):
        up = dict(U=ini["u"], V=ini["v"], T=ini["T"], S=ini["S"], ETA=ini["eta"], QX=ini["U"], QY=ini["V"])
        with model(slim, m, prec, p, up) as mod:
            for n in range(3):
                slim.slim_step(mod.state, n * 40.0, 40.0)
            assert np.abs(mod.download("ETA")).max() < tol
            assert np.abs(mod.download("U")).max() < tol
            assert np.abs(mod.download("T") - ini["T"]).max() < tol * 30


def test_split_mixed_precision_error(slim):
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m = case_mesh("basin")
    ini = initial(m)
    p = params(slim)
    om = OMesh(m)
    st = oracle_state(m, om, ini)
    par = oracle_params(p)
    dt = 10.0 * wl.fields.dt_2d(m)
    with model(slim, m, slim.SLIM_MIXED, p, ini) as mod:
        for n in range(3):
            st = bc.split_step(om, par, st, n * dt, dt)
            slim.slim_step(mod.state, n * dt, dt)
        errs = {f: rel_l2(mod.download(f), getattr(st, o)) for f, o in FIELDS3 + FIELDS2}
    # FP32 residuals: tracers (O(10) values, small increments) stay near 1e-7, the
    # dynamic fields carry the FP32 rounding of their increments
    for f in ("T", "S"):
        assert errs[f] < 1e-6, (f, errs[f])
    for f in ("U", "V", "ETA", "QX", "QY"):
        assert errs[f] < 1e-3, (f, errs[f])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_matches_launches(slim, prec):
    """The captured whole-step graph reproduces the launched step bit for bit,
    including the start time that changes between replays."""
    m = case_mesh("basin")
    ini = initial(m)
    pr = slim.SLIM_FP64 if prec == "fp64" else slim.SLIM_MIXED
    out = []
    for use_graph in (0, 1):
        p = params(slim, use_graph=use_graph)
        with model(slim, m, pr, p, ini) as mod:
            for n in range(3):
                slim.slim_step(mod.state, 100.0 + n * 25.0, 25.0)
            out.append({f: mod.download(f) for f, _ in FIELDS3 + FIELDS2})
    for f in out[0]:
        assert np.array_equal(out[0][f], out[1][f]), f


def test_autotune_returns_a_measured_configuration(slim):
    from paper_2605_16082_gb300 import autotune
    m = case_mesh("basin")
    ini = initial(m)
    p = params(slim)
    res = autotune.autotune(m, slim.SLIM_MIXED, p, ini, 20.0, use_cache=False)
    assert res["tile_prisms"] in autotune.TILES and res["blocks_per_sm"] in autotune.OCCS
    # every (tile, budget) pair except the 3-block budget of 512-prism tiles, and the
    # best of them with the other 2D launch form
    assert len(res["all"]) == len(autotune.TILES) * len(autotune.OCCS)
    assert "512/3" not in res["all"]
    assert sum(k.endswith("persistent0") for k in res["all"]) == 1
    assert res["persistent_2d"] in (0, 1)
    assert res["ms_per_step"] == min(res["all"].values()) > 0


def test_integer_pipe_conversions_match_the_gpu(slim):
    """The mixed 2D update converts between binary32 and binary64 with integer bit
    arithmetic; every pattern class must give the GPU's own result bit for bit."""
    bad_d2f, bad_f2d = slim.slim_selftest_conversions(1 << 24, seed=7)
    assert (bad_d2f, bad_f2d) == (0, 0)


@pytest.fixture(scope="module")
def basin_full():
    """The basin baroclinic workload at full size (197,480 triangles x 20 sigma
    layers, 20 subcycles per step), with the inputs the bench times."""
    W = wl.WORKLOADS["basin_baroclinic"]
    m = W["mesh"]()
    ini = wl.c2_initial_state(m)
    fields = dict(U=ini["u"], V=ini["v"], T=ini["T"], S=ini["S"], ETA=ini["eta"], QX=ini["U"], QY=ini["V"])
    par = dict(scheme=1, n_sub=W["n_sub"], kappa_v=W["kappa_v"], nu_v=W["nu_v"],
               kappa_h=W.get("kappa_h", 0.0), nu_h=W.get("nu_h", 0.0))
    return m, fields, par, W["n_sub"] * wl.fields.dt_2d(m)


def test_split_full_size_in_the_bench_configuration(slim, basin_full):
    """Full size, bench launch configuration (512-prism tiles; mixed with 4 blocks
    per SM): constant tracers stay constant, tracer mass is conserved (open
    boundary closed), the
    hydrostatic pressure gradient matches the oracle at sampled columns, and the
    two forms agree after two steps."""
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m, fields, par, dt = basin_full
    res = {}
    for prec, occ, tol_c, tol_m in ((slim.SLIM_FP64, 2, 1e-12, 1e-13), (slim.SLIM_MIXED, 4, 1e-5, 1e-6)):
        p = slim.slim_params_default(**par)
        p.tile_prisms, p.blocks_per_sm = 512, occ
        const = dict(fields, T=np.full_like(fields["T"], 20.0), S=np.full_like(fields["S"], 35.0))
        with model(slim, m, prec, p, const, tile=512) as mod:
            for n in range(2):
                slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            assert np.abs(mod.download("T") - 20.0).max() < tol_c * 20.0
            assert np.abs(mod.download("S") - 35.0).max() < tol_c * 35.0
        # tracer mass: the same mesh with the open boundary closed (no exchange)
        closed = copy.copy(m)
        closed.bnd = np.where(m.bnd == 2, 1, m.bnd).astype(m.bnd.dtype)
        with model(slim, closed, prec, p, fields, tile=512) as mod:
            m0 = slim.slim_tracer_mass(mod.state, 0)
            for n in range(2):
                slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            assert abs(slim.slim_tracer_mass(mod.state, 0) - m0) < tol_m * abs(m0)
        with model(slim, m, prec, p, fields, tile=512) as mod:
            for n in range(2):
                slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            res[prec] = {f: mod.download(f) for f, _ in FIELDS3 + FIELDS2}
            if prec == slim.SLIM_FP64:
                # hydrostatic pressure gradient of the stepped state at sampled columns
                slim.slim_hpg(mod.state)
                rx, ry = mod.download("R_X"), mod.download("R_Y")
    for f in ("T", "S"):
        assert rel_l2(res[slim.SLIM_MIXED][f], res[slim.SLIM_FP64][f]) < 1e-6, f
    for f in ("U", "V", "ETA", "QX", "QY"):
        assert rel_l2(res[slim.SLIM_MIXED][f], res[slim.SLIM_FP64][f]) < 1e-3, f
    st = res[slim.SLIM_FP64]
    rng = np.random.default_rng(3)
    seeds = np.unique(np.concatenate([rng.choice(m.n_tri, 10, replace=False),
                                      np.nonzero((m.bnd == 2).any(axis=1))[0][:2], [0, m.n_tri - 1]]))
    p = slim.slim_params_default(**par)
    got, ref = [], []
    for sd in seeds:
        sub, tmap, pos = ring_submesh(m, np.array([sd]), 2)
        om = OMesh(sub)
        ox, oy = bc.hpg(om, oracle_params(p), restrict3(st["T"], m, tmap), restrict3(st["S"], m, tmap),
                        restrict2(st["ETA"], m, tmap))
        pr = prisms_of(sub.n_layers, pos)
        got.append(np.concatenate([restrict3(rx, m, np.array([sd])).ravel(),
                                   restrict3(ry, m, np.array([sd])).ravel()]))
        ref.append(np.concatenate([ox[:, :, pr].ravel(), oy[:, :, pr].ravel()]))
    assert_close(np.concatenate(got), np.concatenate(ref), TOL_R)


@pytest.mark.parametrize("mesh", ["basin", "wide"])
def test_persistent_2d_run_matches_stage_launches(slim, mesh):
    """The mixed form's 2D run as one cooperative launch with a grid barrier between
    stages gives the per-stage launches' result bit for bit, with and without the
    CUDA graph; the wide mesh has more triangles than the launch has threads."""
    m = case_mesh("basin") if mesh == "basin" else wl.c2_mesh(140_000, 2, 0)
    ini = initial(m)
    outs = []
    for pers, graph in ((0, 0), (1, 0), (1, 1)):
        p = params(slim)
        p.persistent_2d, p.use_graph = pers, graph
        with model(slim, m, slim.SLIM_MIXED, p, ini) as mod:
            for n in range(3):
                slim.slim_step(mod.state, n * 30.0, 30.0)
            slim.slim_state_check(mod.state)
            outs.append({f: mod.download(f) for f, _ in FIELDS3 + FIELDS2 + [("QBAR_X", "")]})
    for o in outs[1:]:
        for f in o:
            assert np.array_equal(o[f], outs[0][f]), f


def test_grid_barrier_rounds_and_bounded_timeout(slim):
    """The grid barrier of the persistent run: 50 rounds of 8 blocks complete with
    every arrival counted; a block that never arrives makes the others' bounded wait
    run out, which is reported in the error bits (no hang, no fault)."""
    bits, arr = slim.slim_selftest_barrier(8, -1, 50)
    assert (bits, arr) == (0, 8 * 50)
    bits, arr = slim.slim_selftest_barrier(8, 3, 5)
    assert bits & 4 and arr == 7


def test_neighbour_waits_rounds_and_bounded_timeout(slim):
    """The neighbour waits between the stages of the persistent run, on a ring of 8
    blocks: 50 rounds complete with every arrival counted; a block that never arrives
    makes its neighbours' bounded waits run out, then the next ones' a round later,
    which is reported in the error bits (no hang, no fault)."""
    bits, arr = slim.slim_selftest_neighbour_wait(8, -1, 50)
    assert (bits, arr) == (0, 8 * 50)
    bits, arr = slim.slim_selftest_neighbour_wait(8, 3, 3)
    # round 1: the 7 others arrive, blocks 2 and 4 time out; round 2: 1, 5, 6, 7, 0
    # arrive, 1 and 5 time out; round 3: 6, 7, 0 arrive
    assert bits & 4 and arr == 7 + 5 + 3, arr


def _forcing_fields(m, ini):
    """Exterior velocity turning from inflow to outflow between the two forcing
    times, exterior temperature warming by 0.5 (read at open-boundary nodes)."""
    x, y, z, s_ = wl.fields.node_positions_sigma(m)
    ua = (-0.05 * (1.2 - s_)).ravel(); va = (0.01 + 0 * s_).ravel()
    ub = (0.03 * (0.5 + s_)).ravel(); vb = (-0.02 + 0 * s_).ravel()
    return dict(U_EXT=ua, V_EXT=va, U_EXT_B=ub, V_EXT_B=vb, T_EXT_B=ini["T"] + 0.5, S_EXT_B=ini["S"])


def _forced_oracle_state(m, om, ini, fx, p):
    from oracle import baroclinic as bc
    from oracle import tracer as tr
    st = oracle_state(m, om, ini)
    P = om.P
    st.forcing = bc.Forcing(t_a=p.forcing_t_a, t_b=p.forcing_t_b, u_a=tr.to3(fx["U_EXT"], P),
                            v_a=tr.to3(fx["V_EXT"], P), u_b=tr.to3(fx["U_EXT_B"], P),
                            v_b=tr.to3(fx["V_EXT_B"], P), T_a=st.T.copy(), S_a=st.S.copy(),
                            T_b=tr.to3(fx["T_EXT_B"], P), S_b=tr.to3(fx["S_EXT_B"], P))
    return st


@pytest.mark.parametrize("case", ["basin", "square"])
def test_split_forcing_parity_fp64(slim, case):
    """Open-boundary forcing linear in time (exterior velocity and temperature at two
    times, interpolated inside the kernels; the 2D mode with the column sum of the
    exterior transport): two steps against the oracle, every field."""
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m = case_mesh(case)
    ini = initial(m)
    p = params(slim, forcing=1, forcing_t_a=-100.0, forcing_t_b=400.0)
    om = OMesh(m)
    fx = _forcing_fields(m, ini)
    st = _forced_oracle_state(m, om, ini, fx, p)
    par = oracle_params(p)
    dt = 10.0 * wl.fields.dt_2d(m)
    with model(slim, m, slim.SLIM_FP64, p, ini) as mod:
        for k in ("U_EXT", "V_EXT", "U_EXT_B", "V_EXT_B", "T_EXT_B", "S_EXT_B"):
            mod.upload(k, fx[k])
        for n in range(2):
            d1, d2 = {}, {}
            st = bc.split_step(om, par, st, n * dt, dt, d1, d2)
            slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            for f, o in FIELDS3 + FIELDS2:
                assert_close(mod.download(f), getattr(st, o), TOL64, (n, f))
            assert_close(mod.download("W"), d2["W"], TOL64, (n, "W"))
            assert_close(mod.download("QBAR_X"), d2["Qbar"][0], TOL64, (n, "Qbar"))
    # the forcing changed the result (the exterior state enters)
    st0 = bc.split_step(om, oracle_params(params(slim)), oracle_state(m, om, ini), 0.0, dt)
    assert rel_l2(st0.u, bc.split_step(om, par, _forced_oracle_state(m, om, ini, fx, p), 0.0, dt).u) > 1e-6


def test_split_forcing_mixed_and_constants(slim):
    """Forced run in the mixed form against the oracle, and constant tracers with
    constant exterior tracers stay constant under the time-varying exterior flow."""
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m = case_mesh("basin")
    ini = initial(m)
    p = params(slim, forcing=1, forcing_t_a=-100.0, forcing_t_b=400.0)
    om = OMesh(m)
    fx = _forcing_fields(m, ini)
    st = _forced_oracle_state(m, om, ini, fx, p)
    par = oracle_params(p)
    dt = 10.0 * wl.fields.dt_2d(m)
    with model(slim, m, slim.SLIM_MIXED, p, ini) as mod:
        for k in ("U_EXT", "V_EXT", "U_EXT_B", "V_EXT_B", "T_EXT_B", "S_EXT_B"):
            mod.upload(k, fx[k])
        for n in range(2):
            st = bc.split_step(om, par, st, n * dt, dt)
            slim.slim_step(mod.state, n * dt, dt)
        errs = {f: rel_l2(mod.download(f), getattr(st, o)) for f, o in FIELDS3 + FIELDS2}
    for f in ("T", "S"):
        assert errs[f] < 1e-6, (f, errs[f])
    for f in ("U", "V", "ETA", "QX", "QY"):
        assert errs[f] < 1e-3, (f, errs[f])
    const = dict(ini, T=np.full_like(ini["T"], 20.0), S=np.full_like(ini["S"], 35.0))
    fxc = dict(fx, T_EXT_B=const["T"], S_EXT_B=const["S"])
    for prec, tol in ((slim.SLIM_FP64, 1e-12), (slim.SLIM_MIXED, 1e-5)):
        with model(slim, m, prec, p, const) as mod:
            for k in ("U_EXT", "V_EXT", "U_EXT_B", "V_EXT_B", "T_EXT_B", "S_EXT_B"):
                mod.upload(k, fxc[k])
            for n in range(3):
                slim.slim_step(mod.state, n * dt, dt)
            assert np.abs(mod.download("T") - 20.0).max() < tol * 20.0
            assert np.abs(mod.download("S") - 35.0).max() < tol * 35.0


@pytest.fixture(scope="module")
def reef_full():
    """The reef-scale stress workload at full size (~2.4M triangles around 400
    islands, 1-30 z-levels, ~41M prisms; the mesh is cached after its first build)."""
    W = wl.WORKLOADS["reef_baroclinic"]
    m = W["mesh"]()
    ini = wl.c5_initial_state(m)
    fields = dict(U=ini["u"], V=ini["v"], T=ini["T"], S=ini["S"], ETA=ini["eta"], QX=ini["U"], QY=ini["V"])
    par = dict(scheme=1, n_sub=W["n_sub"], kappa_v=W["kappa_v"], nu_v=W["nu_v"],
               kappa_h=W.get("kappa_h", 0.0), nu_h=W.get("nu_h", 0.0))
    return m, fields, par, W["n_sub"] * wl.fields.dt_2d(m)


def test_split_reef_full_size(slim, reef_full):
    """Largest configuration, bench launch shape (512-prism tiles): constant tracers
    stay constant in the mixed form, the pressure gradient of the FP64 step matches
    the oracle at sampled columns (coastline ones included), and the mixed step
    agrees with the FP64 one."""
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m, fields, par, dt = reef_full
    assert m.n_tri > 2_000_000 and int(m.n_layers.sum()) > 40_000_000
    pm = slim.slim_params_default(**par)
    pm.tile_prisms, pm.blocks_per_sm = 512, 4
    const = dict(fields, T=np.full_like(fields["T"], 20.0), S=np.full_like(fields["S"], 35.0))
    with model(slim, m, slim.SLIM_MIXED, pm, const, tile=512) as mod:
        for n in range(2):
            slim.slim_step(mod.state, n * dt, dt)
        slim.slim_state_check(mod.state)
        assert np.abs(mod.download("T") - 20.0).max() < 1e-5 * 20.0
    del const
    res = {}
    for prec in (slim.SLIM_FP64, slim.SLIM_MIXED):
        p = slim.slim_params_default(**par)
        p.tile_prisms, p.blocks_per_sm = 512, 2 if prec == slim.SLIM_FP64 else 4
        with model(slim, m, prec, p, fields, tile=512) as mod:
            slim.slim_step(mod.state, 0.0, dt)
            slim.slim_state_check(mod.state)
            res[prec] = {f: mod.download(f) for f in ("U", "T", "S", "ETA")}
            if prec == slim.SLIM_MIXED:
                for f in ("T", "S"):
                    assert rel_l2(res[prec][f], res[slim.SLIM_FP64][f]) < 1e-6, f
                for f in ("U", "ETA"):
                    assert rel_l2(res[prec][f], res[slim.SLIM_FP64][f]) < 1e-3, f
            if prec == slim.SLIM_FP64:
                # the stepped state is still nearly z-only (its r is the rounding residue
                # of cancelling terms, an absolute floor that grows down 30 z-levels): add
                # a horizontal temperature variation large enough to dominate it
                t_of = np.repeat(np.arange(m.n_tri), m.n_layers)
                xv = m.xy[m.tri[t_of].T, 0]                                   # (3, P) node x
                T_hpg = res[prec]["T"] + 4.0 * np.sin(2 * np.pi * np.broadcast_to(xv[None], (2,) + xv.shape).ravel() / 50e3)
                mod.upload("T", T_hpg)
                slim.slim_hpg(mod.state)
                rx = mod.download("R_X")
    st = res[slim.SLIM_FP64]
    rng = np.random.default_rng(5)
    coast = np.nonzero((m.bnd == 1).any(axis=1))[0]
    seeds = np.unique(np.concatenate([rng.choice(m.n_tri, 6, replace=False), rng.choice(coast, 4, replace=False)]))
    p = slim.slim_params_default(**par)
    got, ref = [], []
    for sd in seeds:
        sub, tmap, pos = ring_submesh(m, np.array([sd]), 2)
        om = OMesh(sub)
        ox, _ = bc.hpg(om, oracle_params(p), restrict3(T_hpg, m, tmap), restrict3(st["S"], m, tmap),
                       restrict2(st["ETA"], m, tmap))
        pr = prisms_of(sub.n_layers, pos)
        got.append(restrict3(rx, m, np.array([sd])).ravel())
        ref.append(ox[:, :, pr].ravel())
    assert_close(np.concatenate(got), np.concatenate(ref), TOL_R)
