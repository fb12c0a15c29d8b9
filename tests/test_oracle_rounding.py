"""Rounding floors of the FP64 oracle: what sets the parity bars.

The GPU FP64 path is held to a relative 1e-12 per field per step, except the
baroclinic pressure gradient r, held to 1e-11.  These tests measure, in the oracle
alone, how far r moves when its inputs move by one rounding (a relative 2^-53):
that spread is the floor any FP64 evaluation of the same formulas can reach, and
for r it is above 1e-12 on the graded basin.  They also pin the cancellation-free
form of the layer-thickness change that enters the continuity (Eq. 17)."""
import numpy as np

from helpers import rel_l2, split_case_mesh, split_initial
from oracle import baroclinic as bc
from oracle import tracer as tr
from oracle.mesh import OMesh


def _perturbed(a, rng):
    return a * (1.0 + 2.0 ** -53 * rng.uniform(-1.0, 1.0, a.shape))


def test_pressure_gradient_floor_is_above_1e12_on_the_graded_basin():
    """r is a horizontal gradient of the hydrostatic pressure along sloping
    coordinate surfaces: nodal depths of O(100 m) enter through their differences
    across a triangle, which cost digits.  One rounding of T, S and eta moves r by
    more than 1e-12 of its norm on the basin case (measured 1.8e-12, max 4e-12), and
    by less than 1e-11 on every case."""
    rng = np.random.default_rng(0)
    par = bc.Params()
    spread = {}
    for case in ("basin", "square", "zlevel"):
        m = split_case_mesh(case)
        om = OMesh(m)
        ini = split_initial(m)
        T, S = tr.to3(ini["T"], om.P), tr.to3(ini["S"], om.P)
        eta = tr.to2(ini["ETA"], m.n_tri)
        r0 = bc.hpg(om, par, T, S, eta)
        r1 = bc.hpg(om, par, _perturbed(T, rng), _perturbed(S, rng), _perturbed(eta, rng))
        spread[case] = max(rel_l2(r1[0], r0[0]), rel_l2(r1[1], r0[1]))
    assert spread["basin"] > 1e-12, spread
    assert max(spread.values()) < 1e-11, spread


def test_thickness_change_is_the_difference_of_thicknesses():
    """dz(eta1) - dz(eta0) = dz_rest (eta1 - eta0)/h (the interfaces stretch
    linearly with eta): the closed form agrees with the subtraction to the
    subtraction's own rounding, vanishes for equal elevations and is exactly
    linear in the elevation change."""
    m = split_case_mesh("zlevel")
    om = OMesh(m)
    rng = np.random.default_rng(1)
    eta0 = 0.3 * rng.standard_normal((3, m.n_tri))
    eta1 = eta0 + 1e-3 * rng.standard_normal((3, m.n_tri))
    d = om.thickness_change(eta0, eta1)
    ref = om.thickness(eta1) - om.thickness(eta0)
    scale = np.abs(om.thickness(eta0)).max()
    assert np.abs(d - ref).max() < 1e-14 * scale
    assert rel_l2(d, ref) < 1e-9
    assert np.abs(om.thickness_change(eta0, eta0)).max() == 0.0
    d2 = om.thickness_change(eta0, eta0 + 2.0 * (eta1 - eta0))
    assert rel_l2(d2, 2.0 * d) < 1e-15
