"""slim_tracer_mass_noalloc: the tracer mass written to caller device memory with
its scratch in a fixed library array (for callers that cannot allocate device
memory during the call, such as code under a pool allocator that forbids direct
cudaMalloc, or code that must not block the host).  Collected last; must pass
alone in a fresh process and after every other test."""
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_mass_matches_the_allocating_entry_point(slim, prec):
    """Both entry points run the same reduction kernels in the same order, so the
    two results are the same double, bit for bit, on two calls in a row."""
    import torch
    m = random_uneven_mesh(12, 4000.0, 9, seed=5)
    u, v = sheared_velocity(m, 4000.0)
    T = wl.c1_tracer(m, 4000.0, 800.0) + 2.0
    pr = slim.SLIM_FP64 if prec == "fp64" else slim.SLIM_MIXED
    with slim.Model(m, pr, slim.slim_params_default(kappa_v=1e-2)) as mod:
        assert mod.info["n_tiles"] > 1
        for k, f in (("U", u), ("V", v), ("T", T), ("ETA", 0.01 * np.ones(3 * m.n_tri))):
            mod.upload(k, f)
        out = torch.full((2,), np.nan, dtype=torch.float64, device="cuda")
        for call in range(2):
            if call == 1:
                slim.slim_step(mod.state, 0.0, 20.0)       # the mass moves with the step
            ref = slim.slim_tracer_mass(mod.state, 0)
            slim.slim_tracer_mass_noalloc(mod.state, 0, out.data_ptr() + 8 * call)
            torch.cuda.synchronize()
            got = float(out[call].item())
            assert got == ref, (call, got, ref)


def test_noalloc_rejects_bad_arguments(slim):
    import torch
    m = random_uneven_mesh(4, 1000.0, 3, seed=1)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with slim.Model(m, slim.SLIM_FP64, slim.slim_params_default()) as mod:
        with pytest.raises(slim.SlimError) as ei:
            slim.slim_tracer_mass_noalloc(mod.state, 2, out.data_ptr())   # not a tracer field
        assert ei.value.status == 1
        with pytest.raises(slim.SlimError) as ei:
            slim.slim_tracer_mass_noalloc(mod.state, 0, 0)                # null output address
        assert ei.value.status == 1
