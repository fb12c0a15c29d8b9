"""Pins of the coupled (consistent-mass, 6x6 per prism) column system of the
tracer step (Sec. 2.4, oracle/coupled.py).

Each test ties the oracle to something other than itself: an independent
assembly of the column matrices from basis-function values at quadrature points,
the closed-form properties of the discretisation (constants preserved, tracer
mass conserved, a linear profile steady under diffusion, no flux through the
surface), and the P1 rate 2 on a smooth manufactured solution."""
import math

import numpy as np
import pytest

import workloads as wl
from helpers import random_uneven_mesh, sheared_velocity
from oracle import coupled as cp
from oracle import quadrature as Q
from oracle import tracer as tr
from oracle.mesh import OMesh


def test_degree4_rule_is_exact_to_degree_4_and_not_5():
    for i in range(6):
        for j in range(6 - i):
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            approx = 0.5 * sum(w * x ** i * y ** j for (x, y, w) in Q.TRI_RULE4)
            if i + j <= 4:
                assert abs(approx - exact) < 1e-16, (i, j)
    x5 = 0.5 * sum(w * x ** 5 for (x, _, w) in Q.TRI_RULE4)
    assert abs(x5 - 1.0 / 42.0) > 1e-6


# ---------------------------------------------------------------------------
# independent assembly of one column from basis values at quadrature points
# ---------------------------------------------------------------------------
def _rule5():
    """7-point degree-5 rule on the reference triangle (Radon), written from its
    closed form and checked here on the monomials up to degree 5."""
    s = math.sqrt(15.0)
    a1, a2 = (6.0 - s) / 21.0, (6.0 + s) / 21.0
    w1, w2 = (155.0 - s) / 1200.0, (155.0 + s) / 1200.0
    pts = [(1 / 3, 1 / 3, 9 / 40)]
    for a, w in ((a1, w1), (a2, w2)):
        pts += [(a, a, w), (a, 1 - 2 * a, w), (1 - 2 * a, a, w)]
    for i in range(6):
        for j in range(6 - i):
            exact = math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)
            assert abs(0.5 * sum(w * x ** i * y ** j for x, y, w in pts) - exact) < 1e-16
    return pts


def _column_by_quadrature(xy, zt, zb, Om, kappa, penalty, beta_dt):
    """(M - beta_dt A) of one triangle column, assembled from the weak forms:
    xy (3, 2) vertices, zt / zb (N, 3) interface depths at the vertices, Om (N, 2, 3)
    nodal vertical flux [layer][top/bottom][vertex]."""
    N = zt.shape[0]
    d1, d2 = xy[1] - xy[0], xy[2] - xy[0]
    Jh = d1[0] * d2[1] - d1[1] * d2[0]
    phi = lambda x, y: np.array([1 - x - y, x, y])
    psi = lambda z: np.array([(1 + z) / 2, (1 - z) / 2])
    dps = np.array([0.5, -0.5])
    gz, gw = np.polynomial.legendre.leggauss(3)
    n = 6 * N
    ix = lambda k, c, a: (2 * k + c) * 3 + a
    M = np.zeros((n, n))
    A = np.zeros((n, n))
    hz = 0.5 * (zt - zb)                                  # (N, 3)
    for (x, y, w) in _rule5():
        ph = phi(x, y)
        dA = 0.5 * Jh * w
        for k in range(N):
            zz = ph @ hz[k]                               # z_zeta at the point
            for z, wz in zip(gz, gw):
                ps = psi(z)
                Omp = sum(Om[k, f] @ ph * ps[f] for f in range(2))
                for c in range(2):
                    for a in range(3):
                        for d in range(2):
                            for b in range(3):
                                M[ix(k, c, a), ix(k, d, b)] += dA * wz * ph[a] * ps[c] * ph[b] * ps[d] * zz
                                # advection volume: int Omega T dv/dzeta
                                A[ix(k, c, a), ix(k, d, b)] += dA * wz * Omp * ph[b] * ps[d] * ph[a] * dps[c]
        # advection interfaces: F = P1 function of the vertex fluxes Omega^ T^
        for i in range(N):
            for b in range(3):
                Wb = Om[i, 0, b]
                src = ix(i, 0, b) if (i == 0 or Wb > 0) else ix(i - 1, 1, b)
                for a in range(3):
                    v = dA * ph[a] * ph[b] * Wb
                    A[ix(i, 0, a), src] -= v                   # top face of layer i
                    if i > 0:
                        A[ix(i - 1, 1, a), src] += v           # bottom face of layer i - 1
    # diffusion with the degree-4 rule in the horizontal (the reading)
    for (x, y, w) in Q.TRI_RULE4:
        ph = phi(x, y)
        dA = 0.5 * Jh * w
        dz = [ph @ (zt[k] - zb[k]) for k in range(N)]
        for k in range(N):
            for c in range(2):
                for d in range(2):
                    for a in range(3):
                        for b in range(3):
                            # int kappa dT/dz dv/dz dV = int kappa (2/dz)^2 dpsi dpsi (dz/2) dzeta dA
                            A[ix(k, c, a), ix(k, d, b)] -= dA * 2.0 * kappa * (2.0 / dz[k]) * dps[c] * dps[d] * ph[a] * ph[b]
        for i in range(1, N):
            ka, kb = i - 1, i
            sig = penalty * kappa / min(dz[ka], dz[kb])
            # trial functionals at the point: {kappa dT/dz}, [T]; test: the same
            def flux(kk):
                f = np.zeros(n)
                for b in range(3):
                    f[ix(kk, 0, b)] += kappa * ph[b] / dz[kk]
                    f[ix(kk, 1, b)] -= kappa * ph[b] / dz[kk]
                return f
            g = 0.5 * (flux(ka) + flux(kb))
            j = np.zeros(n)
            for b in range(3):
                j[ix(kb, 0, b)] += ph[b]
                j[ix(ka, 1, b)] -= ph[b]
            A -= dA * (-np.outer(j, g) - np.outer(g, j) + sig * np.outer(j, j))
    return M - beta_dt * A


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_coupled_column_matrix_matches_an_independent_assembly(N):
    rng = np.random.default_rng(N)
    xy = np.array([[0.0, 0.0], [700.0, 120.0], [260.0, 540.0]])
    h = np.array([12.0, 19.0, 15.5])
    from workloads.meshes import Mesh
    m = Mesh(xy=xy, tri=np.array([[0, 1, 2]], np.int32), h_tri=h[None], n_layers=np.array([N], np.int32),
             bnd=np.ones((1, 3), np.int8))
    om = OMesh(m)
    eta = np.array([[0.3], [-0.2], [0.1]])
    dz = om.thickness(eta)
    zt, zb = om.interfaces(eta)
    Om = rng.uniform(-0.05, 0.05, (2, 3, N))
    kappa, beta_dt = 3e-2, 40.0
    tris = np.array([0])
    Jh = om.Jh[tris]
    dzc = cp.column_thickness(om, dz, tris, N)
    A = cp.vertical_operator(Jh, dzc, cp.gather6(om, Om, tris, N), kappa, 4.0)[0]
    Mo = cp.mass_column(Jh, dzc)[0]
    got = Mo - beta_dt * A
    ref = _column_by_quadrature(xy, zt.T, zb.T, np.transpose(Om, (2, 0, 1)), kappa, 4.0, beta_dt)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# closed-form properties of the coupled step
# ---------------------------------------------------------------------------
def _uneven_case():
    m = random_uneven_mesh(8, 4000.0, 6, seed=3)
    om = OMesh(m)
    u, v = sheared_velocity(m, 4000.0)
    return m, om, tr.to3(u, om.P), tr.to3(v, om.P)


def test_coupled_constant_tracer_stays_constant():
    m, om, u, v = _uneven_case()
    eta = 0.05 * np.ones((3, m.n_tri))
    T = np.full((2, 3, om.P), 3.25)
    for _ in range(3):
        eta, T, Om = cp.tracer_step(om, eta, T, u, v, 20.0, 1e-2)
    assert np.abs(Om).max() > 1e-4                        # the vertical flux is active
    assert np.abs(eta - 0.05).max() > 1e-6                # the elevation moves
    assert np.abs(T - 3.25).max() < 1e-13 * 3.25


def test_coupled_tracer_mass_conserved_to_roundoff():
    m, om, u, v = _uneven_case()
    eta = np.zeros((3, m.n_tri))
    T = tr.to3(wl.c1_tracer(m, 4000.0, 700.0), om.P) + 1.0
    m0 = cp.tracer_mass(om, eta, T)
    for _ in range(5):
        eta, T, _ = cp.tracer_step(om, eta, T, u, v, 20.0, 1e-2)
    assert abs(cp.tracer_mass(om, eta, T) - m0) < 1e-13 * abs(m0)


def test_coupled_surface_flux_vanishes_and_bed_is_closed():
    m, om, u, v = _uneven_case()
    eta1, Om, _ = cp.continuity(om, np.zeros((3, m.n_tri)), u, v, 20.0)
    top = Om[0][:, om.col_off[:-1]]
    assert np.abs(top).max() < 1e-12 * np.abs(Om).max()
    assert np.abs(eta1).max() > 0


def test_coupled_linear_profile_is_steady_under_vertical_diffusion():
    """No flow, layer thicknesses varying across every triangle: T = alpha z + beta
    with the matching Neumann flux kappa alpha at the surface and the bed stays
    exactly steady."""
    m = wl.c1_mesh(4, 1000.0, 5)
    om = OMesh(m)
    zero = np.zeros((2, 3, om.P))
    _, _, z, _ = wl.fields.node_positions_sigma(m)
    alpha, kappa = 0.05, 2e-3
    eta = np.zeros((3, m.n_tri))
    T = alpha * z.reshape(2, 3, om.P) + 7.0
    e1, T1, Om = cp.tracer_step(om, eta, T, zero, zero, 50.0, kappa, kappa * alpha, kappa * alpha)
    assert np.abs(Om).max() == 0.0 and np.abs(e1).max() == 0.0
    assert np.abs(T1 - T).max() < 1e-13 * np.abs(T).max()


def test_coupled_step_converges_at_second_order():
    """Manufactured solution: the cos^4 bump of radius 2.5 km carried 1 km by a
    uniform current through a channel of depth 20 m while a vertical mode
    1 + 0.3 cos(pi z/H) decays by diffusion (kappa_v = 1e-2):
        T = B(x - u t, y) (1 + 0.3 cos(pi z / H) exp(-kappa (pi/H)^2 t)).
    Horizontal and vertical resolution refined together, dt proportional to h:
    the observed rate of the last refinement is >= 1.8 (the lumped step is first
    order on the same problem, test_oracle_order.py)."""
    L, H, U0, R, XC, YC = 10e3, 20.0, 0.5, 2500.0, 3500.0, 5000.0
    kappa, amp = 1e-2, 0.3
    lam = kappa * (math.pi / H) ** 2

    def exact(om, t):
        X = om.X[om.t_of]
        zt, zb = om.interfaces(np.zeros((3, om.n_tri)))
        out = np.empty((2, 3, om.P))
        for a in range(3):
            r = np.hypot(X[:, a, 0] - U0 * t - XC, X[:, a, 1] - YC)
            B = np.where(r < R, np.cos(0.5 * math.pi * np.minimum(r / R, 1.0)) ** 4, 0.0)
            for c, z in enumerate((zt[a], zb[a])):
                out[c, a] = B * (1.0 + amp * np.cos(math.pi * z / H) * math.exp(-lam * t))
        return out

    errs = []
    t_end = 2000.0
    for n, N in ((8, 2), (16, 4), (32, 8)):
        m = wl.meshes.square_mesh(n, L, N, lambda x, y: H + 0.0 * x, lambda x, y: (x < 1e-6) | (x > L - 1e-6))
        om = OMesh(m)
        u = np.full((2, 3, om.P), U0)
        v = np.zeros((2, 3, om.P))
        eta = np.zeros((3, m.n_tri))
        T = exact(om, 0.0)
        ns = int(math.ceil(t_end / (0.3 * (L / n) / U0)))
        for _ in range(ns):
            eta, T, _ = cp.tracer_step(om, eta, T, u, v, t_end / ns, kappa)
        Te = exact(om, t_end)
        w = cp.apply_mass(om, om.thickness(eta), np.ones_like(T))
        errs.append(math.sqrt(float(np.sum(w * (T - Te) ** 2) / np.sum(w * Te ** 2))))
    order = math.log2(errs[1] / errs[2])
    assert order >= 1.8, errs
