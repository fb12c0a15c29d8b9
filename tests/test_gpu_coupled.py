"""GPU parity of the coupled (consistent-mass, 6x6 per prism) column system of the
tracer scheme (slim_params.vertical = 1) against the FP64 oracle (oracle/coupled.py).

FP64 bar: relative L2 <= 1e-12 per field per step and every node within 1e-12 of
the field's largest magnitude.  Cases span several thread-block tiles with a
ragged last tile: a sheared square basin, one-layer columns, uneven columns
(1..12 layers, walls against shallower neighbours) and an open boundary."""
import numpy as np
import pytest

import workloads as wl
from helpers import assert_close, random_uneven_mesh, rel_l2, sheared_velocity

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


CASES = {
    "sheared_square": lambda: (wl.c1_mesh(10, 3000.0, 6), 3000.0),
    "one_layer": lambda: (wl.c1_mesh(20, 3000.0, 1), 3000.0),
    "uneven": lambda: (random_uneven_mesh(9, 4000.0, 12, seed=1), 4000.0),
    "open": lambda: (random_uneven_mesh(8, 3000.0, 6, seed=3, open_x=True), 3000.0),
}


def _setup(slim, m, u, v, T, prec, eta=None, tile=256, **par):
    p = slim.slim_params_default(vertical=slim.SLIM_VERTICAL_COUPLED, **par)
    mod = slim.Model(m, prec, p, tile_prisms=tile)
    mod.upload("U", u); mod.upload("V", v); mod.upload("T", T)
    mod.upload("ETA", np.zeros(3 * m.n_tri) if eta is None else eta)
    return mod


def _fields(m, L):
    u, v = sheared_velocity(m, L)
    if (m.bnd == 2).any():
        u = u - 0.2                     # inflow through the open side
    T = wl.c1_tracer(m, L, 0.2 * L) + 1.0
    return u, v, T


@pytest.mark.parametrize("case", ["sheared_square", "uneven"])
def test_coupled_continuity_parity(slim, case):
    from oracle import coupled as cp
    from oracle import tracer as otr
    from oracle.mesh import OMesh
    m, L = CASES[case]()
    u, v, T = _fields(m, L)
    om = OMesh(m)
    eta = 0.04 * np.cos(np.arange(3 * m.n_tri) * 0.21)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, eta=eta) as mod:
        assert mod.info["n_tiles"] > 1
        slim.slim_continuity(mod.state, 20.0)
        W = mod.download("W")
        e1 = mod.download("ETA_NEXT")
    eo, Oo, _ = cp.continuity(om, eta.reshape(3, -1), otr.to3(u, om.P), otr.to3(v, om.P), 20.0)
    assert_close(W, Oo, TOL64)
    assert_close(e1, eo, TOL64)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("tile", [128, 256])
def test_coupled_vertical_solve_parity(slim, case, tile):
    import torch
    from oracle import coupled as cp
    from oracle import tracer as otr
    from oracle.mesh import OMesh
    m, L = CASES[case]()
    u, v, T = _fields(m, L)
    om = OMesh(m)
    rng = np.random.default_rng(7)
    rhs = rng.standard_normal(6 * om.P)
    kappa, bdt = 5e-3, 30.0
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, tile=tile, kappa_v=kappa, flux_top=1e-4,
                flux_bot=-2e-4) as mod:
        slim.slim_continuity(mod.state, 20.0)
        W = mod.download("W")
        r = torch.tensor(rhs, dtype=torch.float64, device="cuda")
        out = torch.empty_like(r)
        slim.slim_vertical_solve(mod.state, 0, bdt, r.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        slim.slim_vertical_solve(mod.state, 0, bdt, r.data_ptr(), r.data_ptr())   # rhs and out alias
        torch.cuda.synchronize()
        got_inplace = r.cpu().numpy()
    ref = cp.stage_solve(om, otr.to3(W, om.P), om.thickness(np.zeros((3, m.n_tri))), otr.to3(rhs, om.P),
                         bdt, kappa, 1e-4, -2e-4)
    assert_close(got, ref, TOL64)
    assert np.array_equal(got, got_inplace)


@pytest.mark.parametrize("case", list(CASES))
def test_coupled_step_parity_fp64(slim, case):
    from oracle import coupled as cp
    from oracle import tracer as otr
    from oracle.mesh import OMesh
    m, L = CASES[case]()
    u, v, T = _fields(m, L)
    om = OMesh(m)
    kappa, dt = 1e-2, 20.0
    eo = np.zeros((3, m.n_tri))
    To = otr.to3(T, om.P)
    Tx = To.copy() if (m.bnd == 2).any() else None
    uo, vo = otr.to3(u, om.P), otr.to3(v, om.P)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, kappa_v=kappa) as mod:
        for n in range(4):
            slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            eo, To, Oo = cp.tracer_step(om, eo, To, uo, vo, dt, kappa, T_ext=Tx)
            assert_close(mod.download("T"), To, TOL64, n)
            assert_close(mod.download("ETA"), eo, TOL64, n)
            assert_close(mod.download("W"), Oo, TOL64, n)


def test_coupled_mass_conserved_and_matches_the_oracle(slim):
    from oracle import coupled as cp
    from oracle import tracer as otr
    from oracle.mesh import OMesh
    m, L = CASES["uneven"]()
    u, v, T = _fields(m, L)
    om = OMesh(m)
    with _setup(slim, m, u, v, T, slim.SLIM_FP64, kappa_v=1e-2) as mod:
        m0 = slim.slim_tracer_mass(mod.state, 0)
        ref0 = cp.tracer_mass(om, np.zeros((3, m.n_tri)), otr.to3(T, om.P))
        assert abs(m0 - ref0) < 1e-14 * abs(ref0)
        for n in range(5):
            slim.slim_step(mod.state, n * 20.0, 20.0)
        m5 = slim.slim_tracer_mass(mod.state, 0)
    assert abs(m5 - m0) < 1e-13 * abs(m0)


def test_coupled_constant_tracer_and_graph_replay(slim):
    """Constants stay constant in both precisions; the replayed graph gives the
    launched step's bits."""
    m, L = CASES["uneven"]()
    u, v, _ = _fields(m, L)
    T = np.full(6 * int(m.n_layers.sum()), 2.5)
    for prec, tol in ((slim.SLIM_FP64, 1e-13), (slim.SLIM_MIXED, 2e-6)):
        outs = []
        for g in (0, 1):
            with _setup(slim, m, u, v, T, prec, kappa_v=1e-2, use_graph=g) as mod:
                for n in range(3):
                    slim.slim_step(mod.state, n * 20.0, 20.0)
                outs.append(mod.download("T"))
        assert np.abs(outs[0] - 2.5).max() < tol * 2.5
        assert np.array_equal(outs[0], outs[1])


def test_coupled_mixed_error_after_1000_steps(slim):
    """Square-basin tracer workload (2048 triangles x 10 layers, dt = 5 s), coupled
    column system: the mixed form against the FP64 form after 1000 steps (tracer
    relative L2 <= 1e-5, mass drift <= 1e-5; the FP64 form conserves the mass)."""
    W = wl.WORKLOADS["square_tracer"]
    m = W["mesh"]()
    u, v = wl.c1_velocity(m)
    T = wl.c1_tracer(m)
    out = {}
    for prec in (slim.SLIM_FP64, slim.SLIM_MIXED):
        with _setup(slim, m, u, v, T, prec, kappa_v=W["kappa_v"]) as mod:
            m0 = slim.slim_tracer_mass(mod.state, 0)
            for n in range(1000):
                slim.slim_step(mod.state, n * W["dt"], W["dt"])
            slim.slim_state_check(mod.state)
            out[prec] = (mod.download("T"), (slim.slim_tracer_mass(mod.state, 0) - m0) / m0)
    err = rel_l2(out[slim.SLIM_MIXED][0], out[slim.SLIM_FP64][0])
    assert err <= 1e-5, err
    assert abs(out[slim.SLIM_MIXED][1]) <= 1e-5
    assert abs(out[slim.SLIM_FP64][1]) <= 1e-12


def test_coupled_rejects_the_split_scheme_and_oversized_tiles(slim):
    m, L = CASES["sheared_square"]()
    p = slim.slim_params_default(vertical=slim.SLIM_VERTICAL_COUPLED, scheme=slim.SLIM_SCHEME_SPLIT)
    with pytest.raises(slim.SlimError) as ei:
        slim.Model(m, slim.SLIM_FP64, p)
    assert ei.value.status == 9
    p = slim.slim_params_default(vertical=slim.SLIM_VERTICAL_COUPLED)
    with pytest.raises(slim.SlimError) as ei:
        slim.Model(m, slim.SLIM_FP64, p, tile_prisms=512)
    assert ei.value.status == 9
