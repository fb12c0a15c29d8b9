"""GPU: the partitioned tracer step on one device (slim_halo_*: partitions with one
ghost layer, boundary tiles first, halo exchange overlapping the interior tiles)
gives the single-state step's result.  Every prism's arithmetic is the same and
the ghosts carry exact copies, so the fields agree bit for bit."""
import numpy as np
import pytest

import workloads as wl
from helpers import random_uneven_mesh, sheared_velocity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slim():
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2605_16082_gb300 import slim as s
    torch.cuda.init()
    return s


CASES = {
    "sheared_square": lambda: (wl.c1_mesh(12, 3000.0, 6), 3000.0),
    "uneven_open": lambda: (random_uneven_mesh(10, 3000.0, 8, seed=3, open_x=True), 3000.0),
}


def _fields(m, L):
    u, v = sheared_velocity(m, L)
    if (m.bnd == 2).any():
        u = u - 0.2
    T = wl.c1_tracer(m, L, 0.2 * L) + 1.0
    return dict(U=u, V=v, T=T, ETA=0.02 * np.cos(np.arange(3 * m.n_tri) * 0.3))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("K", [2, 4])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("vertical", [0, 1])
def test_partitioned_step_equals_the_single_state_step(slim, case, K, prec, vertical):
    import torch
    m, L = CASES[case]()
    f = _fields(m, L)
    pr = slim.SLIM_FP64 if prec == "fp64" else slim.SLIM_MIXED
    par = slim.slim_params_default(kappa_v=1e-2, vertical=vertical, use_graph=0)
    with slim.Model(m, pr, par, tile_prisms=128) as one:
        for k, v in f.items():
            one.upload(k, v)
        for n in range(3):
            slim.slim_step(one.state, n * 20.0, 20.0)
        ref = {k: one.download(k) for k in ("T", "ETA", "W")}
    with slim.PartitionedModel(m, K, pr, par, tile_prisms=128) as pm:
        assert len(pm.pt.send_tris) > 0
        for k, v in f.items():
            pm.upload(k, v)
        for n in range(3):
            pm.step(n * 20.0, 20.0)
        torch.cuda.synchronize()
        for st in pm.states:
            slim.slim_state_check(st)
        got = {k: pm.download(k) for k in ("T", "ETA", "W")}
    for k in ref:
        assert np.array_equal(got[k], ref[k]), (k, float(np.abs(got[k] - ref[k]).max()))


def test_exchange_copies_the_owners_values_into_the_ghosts(slim):
    import torch
    m, L = CASES["uneven_open"]()
    f = _fields(m, L)
    from paper_2605_16082_gb300 import partition as pa
    with slim.PartitionedModel(m, 3, slim.SLIM_FP64, slim.slim_params_default()) as pm:
        for k, v in f.items():
            pm.upload(k, v)
        # spoil every ghost column, then exchange
        for part, st, pmap in zip(pm.pt.parts, pm.states, pm._pmap):
            loc = pa.to_local(m, part, f["T"], True, pmap).reshape(6, -1)
            n_own = int(np.asarray(part.n_layers)[:part.n_owned].sum())
            loc[:, n_own:] = -7.0
            slim.slim_state_upload(st, slim.FIELD["T"], loc.ravel())
        slim.slim_halo_exchange(pm.halo, slim.FIELD["T"])
        torch.cuda.synchronize()
        for part, st, pmap in zip(pm.pt.parts, pm.states, pm._pmap):
            got = slim.slim_state_download(st, slim.FIELD["T"], 6 * len(pmap))
            assert np.array_equal(got, pa.to_local(m, part, f["T"], True, pmap))
