"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: the matrices
printed in Sec. 2.3 (golden fixtures), exact symbolic integrals, the divergence
theorem, closed-form solutions and conservation identities.
"""
import math
import os

import numpy as np
import pytest

import workloads as wl
from workloads.meshes import Mesh
from oracle import quadrature as Q
from oracle import tracer as tr
from oracle.mesh import OMesh

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def load_gold(name):
    return np.loadtxt(os.path.join(GOLD, name), comments="#")


def tiny_mesh(xy, tri, n_layers, h=None, bnd=None):
    xy = np.asarray(xy, float)
    tri = np.asarray(tri, np.int32)
    nt = tri.shape[0]
    if h is None:
        h = np.full((nt, 3), 10.0)
    if bnd is None:
        bnd = wl.meshes._tag_boundary(xy, tri, None)
    return Mesh(xy=xy, tri=tri, h_tri=np.asarray(h, float),
                n_layers=np.full(nt, n_layers, np.int32) if np.isscalar(n_layers) else np.asarray(n_layers, np.int32),
                bnd=np.asarray(bnd, np.int8))


# ---------------------------------------------------------------------------
# quadrature and basis
# ---------------------------------------------------------------------------
def test_triangle_rule_exact_to_degree_2():
    for i in range(3):
        for j in range(3 - i):
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            approx = 0.5 * sum(w * x ** i * y ** j for (x, y, w) in Q.TRI_RULE)
            assert abs(approx - exact) < 1e-15


def test_gauss_exact_to_degree_3():
    for n in range(4):
        exact = (1 - (-1) ** (n + 1)) / (n + 1)
        assert abs(sum(w * z ** n for z, w in zip(Q.GAUSS_Z, Q.GAUSS_W)) - exact) < 1e-15


def test_consistent_2d_mass_matches_printed():
    # Sec. 2.3: M_h = J_h/24 [[2,1,1],[1,2,1],[1,1,2]]
    m = tiny_mesh([[0, 0], [3, 0.5], [1, 2]], [[0, 1, 2]], 1)
    om = OMesh(m)
    gold = load_gold("mh_p1.txt")
    assert np.allclose(om.mass2d()[0] / om.Jh[0], gold, rtol=0, atol=1e-16)


# ---------------------------------------------------------------------------
# column operators vs the printed 3-layer matrices (Sec. 2.3)
# ---------------------------------------------------------------------------
def test_continuity_rows_match_printed_dvd():
    assert np.array_equal(tr.continuity_rows(3), load_gold("dvd_3layer.txt"))


def test_hpg_rows_match_printed_dvu():
    assert np.array_equal(tr.hpg_rows(3), load_gold("dvu_3layer.txt"))


def _alg1(F, Mh_inv, N):
    """Algorithm 1 (Sec. 2.3) on one column: F (N, 2, 3) per layer (top, bottom) x vertex."""
    r = np.empty_like(F)
    s = np.zeros(3)
    for l in range(N):
        f = np.stack([Mh_inv @ F[l, 0], Mh_inv @ F[l, 1]])
        s = s + f[0] + f[1]
        r[l, 0] = -s + 2 * f[1]
        r[l, 1] = -s
    return r


@pytest.mark.parametrize("N", [1, 2, 3, 7])
def test_algorithm1_solves_printed_dvu(N):
    rng = np.random.default_rng(N)
    Mh = np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]]) * (1.7 / 24)
    D = np.kron(tr.hpg_rows(N), Mh)            # block (2N x 2N) of 3x3 blocks
    F = rng.standard_normal((N, 2, 3))
    r = _alg1(F, np.linalg.inv(Mh), N)
    assert np.allclose(D @ r.reshape(-1), F.reshape(-1), rtol=0, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 5])
def test_dvd_bottom_up_recursion(N):
    # the recursion t = s + f_t + f_b, b = s + f_b - f_t, s = t_below solves D_vd
    rng = np.random.default_rng(10 + N)
    F = rng.standard_normal(2 * N)
    w = np.zeros(2 * N)
    s = 0.0
    for k in range(N - 1, -1, -1):
        ft, fb = F[2 * k], F[2 * k + 1]
        w[2 * k] = s + ft + fb
        w[2 * k + 1] = s + fb - ft
        s = w[2 * k]
    assert np.allclose(tr.continuity_rows(N) @ w, F, atol=1e-14)


# ---------------------------------------------------------------------------
# horizontal residual
# ---------------------------------------------------------------------------
def test_volume_term_matches_exact_symbolic_integral():
    sp = pytest.importorskip("sympy")
    xy = np.array([[0.3, -0.2], [2.1, 0.4], [0.7, 1.9]])
    m = tiny_mesh(xy, [[0, 1, 2]], 1)
    om = OMesh(m)
    rng = np.random.default_rng(3)
    qx, qy, T = (rng.standard_normal((2, 3, 1)) for _ in range(3))
    R = tr.horizontal_residual(om, qx, qy, T)        # single element: walls, no faces
    xi, et, ze = sp.symbols("xi eta zeta")
    ph = [1 - xi - et, xi, et]
    ps = [(1 + ze) / 2, (1 - ze) / 2]
    interp = lambda f: sum(float(f[c, a, 0]) * ph[a] * ps[c] for a in range(3) for c in range(2))
    x = sum(float(xy[a, 0]) * ph[a] for a in range(3))
    y = sum(float(xy[a, 1]) * ph[a] for a in range(3))
    J = sp.Matrix([[sp.diff(x, xi), sp.diff(x, et)], [sp.diff(y, xi), sp.diff(y, et)]])
    Jd = J.det()
    Jinv = J.inv()
    for a in range(3):
        g = Jinv.T * sp.Matrix([sp.diff(ph[a], xi), sp.diff(ph[a], et)])
        for c in range(2):
            f = (interp(qx) * g[0] + interp(qy) * g[1]) * interp(T) * ps[c] * Jd
            val = sp.integrate(sp.integrate(sp.integrate(f, (ze, -1, 1)), (et, 0, 1 - xi)), (xi, 0, 1))
            assert abs(float(val) - R[c, a, 0]) < 1e-12 * (1 + abs(float(val)))


def test_weak_divergence_of_continuous_linear_field():
    # away from walls, R_h(q, 1)_{a,c} = -int phi_a psi_c div(q) J_h = -(div q) J_h / 6
    m = wl.c1_mesh(8, 1000.0, 2)
    om = OMesh(m)
    X = om.X[om.t_of]                                   # (P, 3, 2)
    alpha, beta, gamma, delta = 0.3, -0.7, 1.1, 0.45
    qx = np.empty((2, 3, om.P)); qy = np.empty((2, 3, om.P))
    for a in range(3):
        for c in range(2):
            qx[c, a] = alpha * X[:, a, 0] + beta * X[:, a, 1]
            qy[c, a] = gamma * X[:, a, 0] + delta * X[:, a, 1]
    R = tr.horizontal_residual(om, qx, qy, np.ones_like(qx))
    interior = (om.nbr[om.t_of] >= 0).all(axis=1)
    expect = -(alpha + delta) * om.Jh[om.t_of] / 6.0
    for a in range(3):
        for c in range(2):
            assert np.allclose(R[c, a, interior], expect[interior], rtol=1e-12, atol=1e-9)


def test_upwind_face_flux_direction_and_measure():
    # two triangles sharing the edge x = 1; uniform transport across it
    xy = [[0, 0], [1, 0], [1, 1], [2, 0.5]]
    tri = [[0, 1, 2], [1, 3, 2]]
    m = tiny_mesh(xy, tri, 1)
    om = OMesh(m)
    T = np.zeros((2, 3, 2)); T[:, :, 0] = 1.0            # 1 in the left prism, 0 in the right
    for sign in (+1.0, -1.0):
        qx = np.full((2, 3, 2), 2.5 * sign); qy = np.zeros((2, 3, 2))
        R = tr.horizontal_residual(om, qx, qy, T)
        net_left, net_right = R[..., 0].sum(), R[..., 1].sum()
        # volume terms of a constant field integrate to zero over each element;
        # face |edge| = 1, zeta length 2: flux 2.5 * 2 * T_upwind
        if sign > 0:
            assert abs(net_left + 5.0) < 1e-12 and abs(net_right - 5.0) < 1e-12
        else:
            assert abs(net_left) < 1e-12 and abs(net_right) < 1e-12


def test_horizontal_residual_is_conservative():
    m = wl.c1_mesh(6, 2000.0, 3)
    om = OMesh(m)
    rng = np.random.default_rng(5)
    qx, qy, T = (rng.standard_normal((2, 3, om.P)) for _ in range(3))
    R = tr.horizontal_residual(om, qx, qy, T)
    assert abs(R.sum()) < 1e-12 * np.abs(R).sum()


# ---------------------------------------------------------------------------
# vertical operator
# ---------------------------------------------------------------------------
def _col(N, dz, W=None, kappa=1e-2, omega=2.0):
    Wc = np.zeros((1, 2 * N)) if W is None else np.asarray(W, float)[None]
    return tr.vertical_matrix(Wc, np.asarray(dz, float)[None], kappa, np.array([omega]))[0]


def test_sipg_symmetric_negative_semidefinite_constant_kernel():
    A = _col(5, [1.0, 0.5, 2.0, 0.7, 1.3])
    assert np.allclose(A, A.T, atol=1e-14)
    ev = np.linalg.eigvalsh(A)
    assert ev.max() < 1e-12
    assert np.sum(ev > -1e-10) == 1                      # only the constants
    assert np.allclose(A @ np.ones(10), 0, atol=1e-13)


def test_linear_profile_is_steady_under_vertical_diffusion():
    N, kappa, omega, alpha = 6, 3e-3, 1.5, 0.2
    dz = np.array([0.5, 1.0, 1.5, 0.25, 2.0, 1.0])
    z = np.concatenate([[0.0], -np.cumsum(dz)])
    Tlin = np.empty(2 * N)
    Tlin[0::2] = alpha * z[:-1]
    Tlin[1::2] = alpha * z[1:]
    A = _col(N, dz, kappa=kappa, omega=omega)
    b = tr.neumann_vector(1, N, np.array([omega]), kappa * alpha, kappa * alpha)[0]
    assert np.allclose(A @ Tlin + b, 0, atol=1e-15)


def test_implicit_upwind_advection_direction():
    # upward flux everywhere (W > 0) carries a step profile up with only the small
    # over/undershoots of P1 DG; downward flux never reaches the top layer
    N = 12
    W = np.zeros(2 * N); W[0::2] = 0.3; W[1::2] = 0.3
    A = _col(N, np.ones(N), W=W, kappa=0.0, omega=1.0)
    M = tr.mass_matrix(np.ones((1, N)), np.array([1.0]))[0]
    T = np.zeros(2 * N); T[N:] = 1.0                    # lower half = 1
    for _ in range(50):
        T = np.linalg.solve(M - 0.5 * A, M @ T)
    mean = 0.5 * (T[0::2] + T[1::2])
    assert mean.min() > -2e-2 and mean.max() < 1 + 2e-2
    # the signal moved upward: the top layer gained tracer
    assert mean[0] > 1e-3
    # downward flux leaves the top layer empty
    A2 = _col(N, np.ones(N), W=-W, kappa=0.0, omega=1.0)
    T = np.zeros(2 * N); T[N:] = 1.0
    for _ in range(50):
        T = np.linalg.solve(M - 0.5 * A2, M @ T)
    assert abs(0.5 * (T[0] + T[1])) < 1e-12


def test_vertical_diffusion_converges_at_second_order():
    # T = cos(pi z/H) exp(-kappa pi^2 t/H^2) with no-flux ends; implicit Euler in time
    H, kappa, tend = 10.0, 1.0, 2.0
    errs = []
    for N in (4, 8, 16):
        dz = np.full(N, H / N)
        z = np.concatenate([[0.0], -np.cumsum(dz)])
        T = np.empty(2 * N); T[0::2] = np.cos(np.pi * z[:-1] / H); T[1::2] = np.cos(np.pi * z[1:] / H)
        A = _col(N, dz, kappa=kappa, omega=1.0)
        M = tr.mass_matrix(dz[None], np.array([1.0]))[0]
        nst = 8 * N * N
        dt = tend / nst
        for _ in range(nst):
            T = np.linalg.solve(M - dt * A, M @ T)
        ex = np.empty(2 * N); ex[0::2] = np.cos(np.pi * z[:-1] / H); ex[1::2] = np.cos(np.pi * z[1:] / H)
        ex *= math.exp(-kappa * np.pi ** 2 * tend / H ** 2)
        errs.append(np.sqrt(np.mean((T - ex) ** 2)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 1.8, (errs, orders)


# ---------------------------------------------------------------------------
# whole tracer step
# ---------------------------------------------------------------------------
def _sheared_case(n=6, N=4, L=3000.0):
    m = wl.c1_mesh(n, L, N)
    om = OMesh(m)
    u, v = wl.c1_velocity(m, L)
    u, v = tr.to3(u, om.P), tr.to3(v, om.P)
    # depth shear so that the vertical flux is not zero
    _, _, _, s = wl.fields.node_positions_sigma(m)
    u = u * (1.5 - s); v = v * (0.5 + s)
    return m, om, u, v


def test_constant_tracer_stays_constant():
    m, om, u, v = _sheared_case()
    eta = np.zeros((3, om.n_tri))
    T = np.full((2, 3, om.P), 3.25)
    for _ in range(3):
        eta, T, W = tr.tracer_step(om, eta, T, u, v, 20.0, 1e-2)
    assert np.abs(W).max() > 1e-3                       # the vertical flux is active
    assert np.abs(T - 3.25).max() < 1e-13 * 3.25


def test_tracer_mass_conserved_to_roundoff():
    m, om, u, v = _sheared_case()
    eta = np.zeros((3, om.n_tri))
    T = tr.to3(wl.c1_tracer(m, 3000.0, 500.0), om.P)
    m0 = tr.tracer_mass(om, eta, T)
    for _ in range(5):
        eta, T, _ = tr.tracer_step(om, eta, T, u, v, 20.0, 1e-2)
    assert abs(tr.tracer_mass(om, eta, T) - m0) < 1e-13 * abs(m0)


def test_surface_vertical_flux_vanishes():
    # Eq. 4 (s = 0): the column-integrated continuity and the elevation update agree
    m, om, u, v = _sheared_case()
    eta = np.zeros((3, om.n_tri))
    eta1, W, _ = tr.continuity(om, eta, u, v, 20.0)
    top = W[0][:, om.col_off[:-1]]
    assert np.abs(top).max() < 1e-12 * np.abs(W).max()
    assert np.abs(eta1).max() > 0


def test_step_with_no_flow_is_pure_vertical_diffusion():
    m = wl.c1_mesh(4, 1000.0, 5)
    om = OMesh(m)
    zero = np.zeros((2, 3, om.P))
    _, _, z, _ = wl.fields.node_positions_sigma(m)
    alpha, kappa = 0.05, 2e-3
    eta = np.zeros((3, om.n_tri))
    T = alpha * z
    e1, T1, W = tr.tracer_step(om, eta, T, zero, zero, 50.0, kappa, kappa * alpha, kappa * alpha)
    assert np.abs(W).max() == 0.0 and np.abs(e1).max() == 0.0
    assert np.abs(T1 - T).max() < 1e-13
