"""GPU parity at the layer-count limit: columns of SLIM_MAX_LAYERS (128) layers beside
one-layer and short columns in one tile set (walls against shallower neighbours on
most faces), for the tracer scheme with both column systems and for the split scheme
in both precisions.  FP64 against the oracle per node (relative L2 and every node
within 1e-12 of the field's largest magnitude); the mixed form within the bars of the
other mixed-precision tests."""
import numpy as np
import pytest

import workloads as wl
from helpers import assert_close, rel_l2, sheared_velocity, split_initial
from test_gpu_split import FIELDS2, FIELDS3, model, oracle_params, oracle_state, params

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


def deep_mesh(open_x=False):
    """2 x 2 squares (8 triangles), 300-600 m of water, columns of 128, 1, 7, 128, 2,
    16, 1 and 3 layers (286 prisms; at 128 prisms per tile, four tiles)."""
    L = 4000.0
    op = (lambda x, y: x > L - 1e-6) if open_x else None
    m = wl.meshes.square_mesh(2, L, 1, lambda x, y: 450.0 + 150.0 * np.sin(np.pi * x / L) * np.cos(np.pi * y / L),
                              op)
    m.n_layers = np.array([128, 1, 7, 128, 2, 16, 1, 3], np.int32)
    return m, L


@pytest.mark.parametrize("vertical", [0, 1])
def test_tracer_step_with_128_layer_columns(slim, vertical):
    from oracle import coupled as cp
    from oracle import tracer as otr
    from oracle.mesh import OMesh
    m, L = deep_mesh()
    u, v = sheared_velocity(m, L)
    T = wl.c1_tracer(m, L, 0.3 * L) + 1.0
    om = OMesh(m)
    kappa, dt = 5e-3, 20.0
    par = slim.slim_params_default(kappa_v=kappa, vertical=vertical)
    eo = np.zeros((3, m.n_tri))
    To = otr.to3(T, om.P)
    uo, vo = otr.to3(u, om.P), otr.to3(v, om.P)
    step = cp.tracer_step if vertical else otr.tracer_step
    with slim.Model(m, slim.SLIM_FP64, par, tile_prisms=128) as mod:
        assert mod.info["max_layers"] == 128 and mod.info["n_tiles"] > 1
        for k, f in (("U", u), ("V", v), ("T", T), ("ETA", np.zeros(3 * m.n_tri))):
            mod.upload(k, f)
        for n in range(2):
            slim.slim_step(mod.state, n * dt, dt)
            slim.slim_state_check(mod.state)
            eo, To, _ = step(om, eo, To, uo, vo, dt, kappa)
            assert_close(mod.download("T"), To, TOL64, n)
            assert_close(mod.download("ETA"), eo, TOL64, n)


def test_split_step_with_128_layer_columns(slim):
    from oracle import baroclinic as bc
    from oracle.mesh import OMesh
    m, L = deep_mesh(open_x=True)
    ini = split_initial(m, seed=2)
    p = params(slim)
    om = OMesh(m)
    dt = 10.0 * wl.fields.dt_2d(m)
    st = bc.split_step(om, oracle_params(p), oracle_state(m, om, ini), 0.0, dt)
    for prec in (slim.SLIM_FP64, slim.SLIM_MIXED):
        with model(slim, m, prec, p, ini, tile=128) as mod:
            assert mod.info["max_layers"] == 128
            slim.slim_step(mod.state, 0.0, dt)
            slim.slim_state_check(mod.state)
            got = {f: mod.download(f) for f, _ in FIELDS3 + FIELDS2}
        for f, o in FIELDS3 + FIELDS2:
            if prec == slim.SLIM_FP64:
                assert_close(got[f], getattr(st, o), TOL64, f)
            else:
                assert rel_l2(got[f], getattr(st, o)) < (1e-6 if f in ("T", "S") else 1e-3), f
