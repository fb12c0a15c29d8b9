"""GPU parity of the tracer path (C ABI) against the FP64 CPU oracle.

FP64 bar: relative L2 <= 1e-12 per field per step.  Mixed bar: the FP32
arithmetic's error, stated per test.  Every case spans several thread-block
tiles with a ragged last tile; edge cases cover one-layer columns, uneven
columns, open boundaries and all tile sizes.
"""
import os
import numpy as np
import pytest

import workloads as wl
from helpers import (assert_close, rel_l2, sheared_velocity, random_uneven_mesh, ring_submesh, restrict3,
                     restrict2, prisms_of)

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def slim():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2605_16082_gb300 import slim as s
    torch.cuda.init()
    return s


def _oracle():
    from oracle import tracer as otr
    from oracle.mesh import OMesh
    return otr, OMesh


def _setup(slim, m, u, v, T, prec, eta=None, tile=256, **par):
    p = slim.slim_params_default(**par)
    mod = slim.Model(m, prec, p, tile_prisms=tile)
    mod.upload("U", u); mod.upload("V", v); mod.upload("T", T)
    mod.upload("ETA", np.zeros(3 * m.n_tri) if eta is None else eta)
    return mod


def _torch_out(slim, mod, n):
    import torch
    dt = torch.float64 if mod.precision == slim.SLIM_FP64 else torch.float32
    return torch.zeros(n, dtype=dt, device="cuda")


CASES = {
    "sheared_square": lambda: (wl.c1_mesh(10, 3000.0, 6), 3000.0),
    "one_layer": lambda: (wl.c1_mesh(20, 3000.0, 1), 3000.0),
    "uneven": lambda: (random_uneven_mesh(9, 4000.0, 12, seed=1), 4000.0),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("tile", [128, 256, 512])
def test_rhs3d_parity(slim, case, tile):
    import torch
    otr, OMesh = _oracle()
    m, L = CASES[case]()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.2 * L)
    om = OMesh(m)
    eta = 0.05 * np.sin(np.arange(3 * m.n_tri) * 0.37)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, eta=eta, tile=tile) as mod:
        assert mod.info["n_tiles"] > 1
        out = _torch_out(slim, mod, 6 * mod.P)
        slim.slim_rhs3d(mod.state, 0, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    dz = om.thickness(eta.reshape(3, -1))
    qx, qy = otr.transport(dz, otr.to3(u, om.P), otr.to3(v, om.P))
    ref = otr.horizontal_residual(om, qx, qy, otr.to3(T, om.P))
    assert_close(got, ref, TOL64)


@pytest.mark.parametrize("case", list(CASES))
def test_continuity_parity(slim, case):
    otr, OMesh = _oracle()
    m, L = CASES[case]()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.2 * L)
    om = OMesh(m)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64) as mod:
        slim.slim_continuity(mod.state, 20.0)
        W = mod.download("W")
        e1 = mod.download("ETA_NEXT")
    eo, Wo, _ = otr.continuity(om, np.zeros((3, m.n_tri)), otr.to3(u, om.P), otr.to3(v, om.P), 20.0)
    assert_close(W, Wo, TOL64)
    assert_close(e1, eo, TOL64)


@pytest.mark.parametrize("case", list(CASES))
def test_vertical_solve_parity(slim, case):
    import torch
    otr, OMesh = _oracle()
    m, L = CASES[case]()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.2 * L)
    om = OMesh(m)
    rng = np.random.default_rng(7)
    rhs = rng.standard_normal(6 * om.P)
    kappa, bdt = 5e-3, 30.0
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, kappa_v=kappa, flux_top=1e-4, flux_bot=-2e-4) as mod:
        slim.slim_continuity(mod.state, 20.0)
        W = mod.download("W")
        r = torch.tensor(rhs, dtype=torch.float64, device="cuda")
        out = torch.empty_like(r)
        slim.slim_vertical_solve(mod.state, 0, bdt, r.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # in place (rhs and out alias)
        slim.slim_vertical_solve(mod.state, 0, bdt, r.data_ptr(), r.data_ptr())
        torch.cuda.synchronize()
        got_inplace = r.cpu().numpy()
    ref = otr.stage_solve(om, otr.to3(W, om.P), om.thickness(np.zeros((3, m.n_tri))),
                          otr.to3(rhs, om.P), bdt, kappa, 1e-4, -2e-4)
    assert_close(got, ref, TOL64)
    assert np.array_equal(got, got_inplace)


@pytest.mark.parametrize("case", list(CASES))
def test_step_parity_fp64(slim, case):
    otr, OMesh = _oracle()
    m, L = CASES[case]()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.2 * L)
    om = OMesh(m)
    kappa, dt = 1e-2, 20.0
    eo = np.zeros((3, m.n_tri)); To = otr.to3(T, om.P)
    uo, vo = otr.to3(u, om.P), otr.to3(v, om.P)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, kappa_v=kappa) as mod:
        for n in range(4):
            slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            eo, To, _ = otr.tracer_step(om, eo, To, uo, vo, dt, kappa)
            assert_close(mod.download("T"), To, TOL64, n)
            assert_close(mod.download("ETA"), eo, TOL64, n)


def test_square_basin_workload_parity(slim):
    """The 32x32x10 square-basin workload itself: 3 steps element by element."""
    otr, OMesh = _oracle()
    W = wl.WORKLOADS["square_tracer"]
    m = W["mesh"]()
    u, v = wl.c1_velocity(m)
    T = wl.c1_tracer(m)
    om = OMesh(m)
    eo = np.zeros((3, m.n_tri)); To = otr.to3(T, om.P)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, kappa_v=W["kappa_v"]) as mod:
        for n in range(3):
            slim.slim_step(mod.state, n * W["dt"], W["dt"])
            eo, To, _ = otr.tracer_step(om, eo, To, otr.to3(u, om.P), otr.to3(v, om.P), W["dt"], W["kappa_v"])
            got = mod.download("T")
            assert_close(got, To, TOL64)
            assert np.abs(got - To.ravel()).max() < 1e-12
            assert_close(mod.download("ETA"), eo, TOL64)


def test_open_boundary_inflow_uses_exterior_profile(slim):
    import torch
    otr, OMesh = _oracle()
    m = random_uneven_mesh(8, 3000.0, 6, seed=3, open_x=True)
    assert (m.bnd == 2).any()
    P = int(m.n_layers.sum())
    u = np.full(6 * P, -0.3)          # inflow through the open boundary at x = L
    v = np.full(6 * P, 0.05)
    T = wl.c1_tracer(m, 3000.0, 800.0)
    Text = 0.5 * T + 0.1
    om = OMesh(m)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64) as mod:
        mod.upload("T_EXT", Text)
        out = _torch_out(slim, mod, 6 * mod.P)
        slim.slim_rhs3d(mod.state, 0, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    dz = om.thickness(np.zeros((3, m.n_tri)))
    qx, qy = otr.transport(dz, otr.to3(u, om.P), otr.to3(v, om.P))
    ref = otr.horizontal_residual(om, qx, qy, otr.to3(T, om.P), otr.to3(Text, om.P))
    ref_same = otr.horizontal_residual(om, qx, qy, otr.to3(T, om.P), otr.to3(T, om.P))
    assert rel_l2(ref, ref_same) > 1e-6           # the exterior state matters
    assert_close(got, ref, TOL64)


def test_mass_conservation_and_parity(slim):
    otr, OMesh = _oracle()
    m, L = CASES["uneven"]()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.2 * L)
    om = OMesh(m)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, kappa_v=1e-2) as mod:
        m0 = slim.slim_tracer_mass(mod.state, 0)
        ref0 = otr.tracer_mass(om, np.zeros((3, m.n_tri)), otr.to3(T, om.P))
        assert abs(m0 - ref0) < 1e-14 * abs(ref0)
        for n in range(5):
            slim.slim_step(mod.state, n * 20.0, 20.0)
        m5 = slim.slim_tracer_mass(mod.state, 0)
        assert abs(m5 - m0) < 1e-13 * abs(m0)
        again = slim.slim_tracer_mass(mod.state, 0)
        assert again == m5                         # deterministic


def test_constant_preserved_on_gpu(slim):
    m, L = CASES["uneven"]()
    u, v = sheared_velocity(m, L)
    P = int(m.n_layers.sum())
    with _setup(slim, m, u, v, np.full(6 * P, 2.5), slim.SLIM_FP64, kappa_v=1e-2) as mod:
        for n in range(3):
            slim.slim_step(mod.state, n * 20.0, 20.0)
        T = mod.download("T")
    assert np.abs(T - 2.5).max() < 1e-13 * 2.5


def test_mixed_precision_step_error(slim):
    otr, OMesh = _oracle()
    m, L = CASES["sheared_square"]()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.2 * L)
    om = OMesh(m)
    eo = np.zeros((3, m.n_tri)); To = otr.to3(T, om.P)
    with _setup(slim, m, u, v, T, slim.SLIM_MIXED, kappa_v=1e-2) as mod:
        for n in range(5):
            slim.slim_step(mod.state, n * 20.0, 20.0)
            eo, To, _ = otr.tracer_step(om, eo, To, otr.to3(u, om.P), otr.to3(v, om.P), 20.0, 1e-2)
        errT = rel_l2(mod.download("T"), To)
        erre = rel_l2(mod.download("ETA"), eo)
    assert errT < 1e-5, errT
    assert erre < 1e-5, erre


def test_nonfinite_input_is_reported(slim):
    m, L = CASES["sheared_square"]()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.2 * L)
    T[17] = np.nan
    with _setup(slim, m, u, v, T, slim.SLIM_FP64) as mod:
        slim.slim_step(mod.state, 0.0, 20.0)
        with pytest.raises(slim.SlimError) as ei:
            slim.slim_state_check(mod.state)
        assert ei.value.status == 5
        slim.slim_state_check(mod.state)         # flag was cleared


def test_sampled_parity_at_basin_size(slim):
    """The basin mesh at full size (~200k columns x 20 layers): sampled columns,
    each checked against the oracle run on the 4-ring neighbourhood around it."""
    otr, OMesh = _oracle()
    m = wl.c2_mesh()
    Lx = 200e3
    # a smooth sheared velocity on the basin
    _, _, _, s = wl.fields.node_positions_sigma(m)
    x, y, _, _ = wl.fields.node_positions_sigma(m)
    u = (0.3 * np.sin(np.pi * x / Lx) * (1.5 - s)).ravel()
    v = (0.2 * np.cos(np.pi * y / 1e5) * (0.5 + s)).ravel()
    T = (10 + np.exp(-((x - 0.3 * Lx) ** 2 + (y - 5e4) ** 2) / (2 * (2e4) ** 2)) * (1 - s)).ravel()
    kappa, dt = 1e-3, 10.0
    rng = np.random.default_rng(11)
    seeds = np.unique(np.concatenate([rng.choice(m.n_tri, 24, replace=False), [0, m.n_tri - 1]]))
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, kappa_v=kappa) as mod:
        slim.slim_step(mod.state, 0.0, dt)
        slim.slim_state_check(mod.state)
        T1 = mod.download("T")
        e1 = mod.download("ETA")
    gT, rT, ge, re = [], [], [], []
    for sd in seeds:
        sub, tmap, pos = ring_submesh(m, np.array([sd]), 4)
        om = OMesh(sub)
        eo, To, _ = otr.tracer_step(om, np.zeros((3, sub.n_tri)), restrict3(T, m, tmap),
                                    restrict3(u, m, tmap), restrict3(v, m, tmap), dt, kappa)
        pr = prisms_of(sub.n_layers, pos)
        gT.append(restrict3(T1, m, np.array([sd])).ravel()); rT.append(To[:, :, pr].ravel())
        ge.append(restrict2(e1, m, np.array([sd])).ravel()); re.append(eo[:, pos].ravel())
    # the per-field bar over the sampled outputs
    assert_close(np.concatenate(gT), np.concatenate(rT), TOL64)
    assert_close(np.concatenate(ge), np.concatenate(re), TOL64)


def test_tracer_graph_replay_matches_launches(slim):
    m, L = CASES["uneven"]()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.2 * L)
    res = []
    for g in (0, 1):
        with _setup(slim, m, u, v, T, slim.SLIM_MIXED, kappa_v=1e-2, use_graph=g) as mod:
            for n in range(3):
                slim.slim_step(mod.state, n * 20.0, 20.0)
            res.append(mod.download("T"))
    assert np.array_equal(res[0], res[1])


def _golden_c1_1000():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_tracer_1000.txt")
    vals, idx, smp = {}, [], []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            a, b = line.split()
            if a.isdigit():
                idx.append(int(a)); smp.append(float(b))
            else:
                vals[a] = float(b)
    return vals, np.array(idx), np.array(smp)


def test_mixed_tracer_error_after_1000_steps(slim):
    """Mixed form of the square-basin tracer run against the FP64 form after 1000
    steps: tracer relative L2 error at most 1e-5.  The FP64 form is tied to the
    oracle's own 1000-step run (stored mass and 256 stored nodes)."""
    vals, idx, smp = _golden_c1_1000()
    steps = int(vals["steps"])
    W = wl.WORKLOADS["square_tracer"]
    m = W["mesh"]()
    u, v = wl.c1_velocity(m)
    T = wl.c1_tracer(m)
    res = {}
    for prec in (slim.SLIM_FP64, slim.SLIM_MIXED):
        with _setup(slim, m, u, v, T, prec, kappa_v=W["kappa_v"]) as mod:
            m0 = slim.slim_tracer_mass(mod.state, 0)
            for n in range(steps):
                slim.slim_step(mod.state, n * W["dt"], W["dt"])
            slim.slim_state_check(mod.state)
            res[prec] = (mod.download("T"), m0, slim.slim_tracer_mass(mod.state, 0))
    T64, m0_64, m1_64 = res[slim.SLIM_FP64]
    Tmx, m0_mx, m1_mx = res[slim.SLIM_MIXED]
    scale = np.abs(smp).max()
    assert np.abs(T64[idx] - smp).max() < 1e-10 * scale          # FP64 form = oracle
    assert abs(m0_64 - vals["mass0"]) < 1e-13 * abs(vals["mass0"])
    assert abs(m1_64 - vals["mass"]) < 1e-12 * abs(vals["mass"])
    err = rel_l2(Tmx, T64)
    drift = (m1_mx - m0_mx) / m0_mx
    print(f"mixed vs FP64 after {steps} steps: tracer rel L2 {err:.3e}, mass drift {drift:.3e}")
    assert err <= 1e-5
    assert abs(drift) < 1e-5
