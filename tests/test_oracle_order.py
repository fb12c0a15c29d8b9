"""Order-of-accuracy pins of the CPU oracle on smooth manufactured solutions.

These tie the oracle's horizontal residual (Eq. 6), its horizontal SIPG viscosity
and its SSP-RK3 stage weights to rates that the mathematics fixes:

* the Shu-Osher SSP-RK3 combination is third order in time (a wrong pair of stage
  weights that still sums to one drops the rate);
* the P1 discontinuous-Galerkin advection residual with upwind face fluxes is
  second order in space on a smooth solution when the time derivative carries the
  consistent mass;
* the horizontal SIPG operator solves a smooth Neumann problem at second order,
  and a wrong factor on its face flux makes it inconsistent;
* the SIPG penalty contributes sigma = 6 nu / min(r_in) on a pure jump.

The tracer step of the oracle lumps the mass horizontally onto the vertex columns
(the 2x2-block reading of the vertical system), and the last pin records what
that costs: with the lumped mass the same advection converges at first order.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import tracer as tr
from oracle import baroclinic as bc
from oracle.mesh import OMesh
from oracle.quadrature import int_psi_psi

L = 10e3
H = 20.0
U0 = 0.5
R_BUMP = 2500.0
XC, YC = 3500.0, 5000.0


def bump(x, y):
    """cos^4 bump of radius R_BUMP: three continuous derivatives, compact support, so
    the open boundaries of the channel see exactly zero."""
    r = np.hypot(x - XC, y - YC)
    return np.where(r < R_BUMP, np.cos(0.5 * np.pi * np.minimum(r / R_BUMP, 1.0)) ** 4, 0.0)


def channel(n, n_layers=1):
    """Flat-bottomed square channel: walls at y = 0, L, open at x = 0, L."""
    return wl.meshes.square_mesh(n, L, n_layers, lambda x, y: H + 0.0 * x,
                                 lambda x, y: (x < 1e-6) | (x > L - 1e-6))


def nodal(om, f):
    """(2, 3, P) nodal values of f(x, y) (depth independent)."""
    X = om.X[om.t_of]
    out = np.empty((2, 3, om.P))
    for a in range(3):
        out[:, a] = f(X[:, a, 0], X[:, a, 1])[None]
    return out


def consistent_mass_inverse(om, dz):
    """Inverse of the consistent mass int phi_a phi_b psi_c psi_d (dz/2) J_h of flat
    layers: per prism M_h^-1 (x) G^-1 / (dz/2), M_h = J_h/24 [[2,1,1],[1,2,1],[1,1,2]]
    (Sec. 2.3) and G = int psi psi on [-1, 1]."""
    Mh = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 24.0
    Mhi = np.linalg.inv(Mh)
    Gi = np.linalg.inv(int_psi_psi())
    scale = om.Jh[om.t_of] * 0.5 * dz[0]
    return lambda R: np.einsum("ab,cd,dbp->cap", Mhi, Gi, R) / scale[None, None]


def ssp_rk3(Tn, Lop, dt, alpha=tr.SSP_ALPHA, beta=tr.SSP_BETA):
    T = Tn
    for s in range(3):
        T = alpha[s] * Tn + beta[s] * (T + dt * Lop(T))
    return T


def rel_err(om, T, Te):
    w = tr.apply_mass(om, om.thickness(np.zeros((3, om.n_tri))), np.ones_like(T))
    return math.sqrt(float(np.sum(w * (T - Te) ** 2) / np.sum(w * Te ** 2)))


def orders(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


# ---------------------------------------------------------------------------
# time: SSP-RK3 stage weights
# ---------------------------------------------------------------------------
def _advect_fixed_mesh(n_steps_list, t_end, alpha=tr.SSP_ALPHA, beta=tr.SSP_BETA):
    m = channel(8)
    om = OMesh(m)
    P = om.P
    u = np.full((2, 3, P), U0)
    v = np.zeros((2, 3, P))
    T0 = nodal(om, bump)
    eta = np.zeros((3, m.n_tri))
    out = []
    saved = (tr.SSP_ALPHA, tr.SSP_BETA)
    try:
        tr.SSP_ALPHA, tr.SSP_BETA = alpha, beta
        for ns in n_steps_list:
            T, e = T0, eta
            for _ in range(ns):
                e, T, _ = tr.tracer_step(om, e, T, u, v, t_end / ns, 0.0)
            out.append(T)
    finally:
        tr.SSP_ALPHA, tr.SSP_BETA = saved
    return om, out


def test_tracer_step_is_third_order_in_time():
    """Fixed mesh, transport with no vertical flux (uniform velocity, flat bottom):
    the step is the Shu-Osher SSP-RK3 of the semi-discrete advection, so halving
    the step cuts the error against a 16x finer run by 2^3."""
    om, sols = _advect_fixed_mesh([4, 8, 16, 128], 2000.0)
    ref = sols[-1]
    errs = [rel_err(om, T, ref) for T in sols[:-1]]
    assert min(orders(errs)) >= 2.8, errs


def test_swapped_stage_weights_lose_the_third_order():
    """Planted mistake: exchange the weights of stages 2 and 3 (still convex, so the
    constant-preservation and mass pins cannot see it).  The rate falls below 2.5."""
    om, sols = _advect_fixed_mesh([4, 8, 16, 128], 2000.0, alpha=(0.0, 1.0 / 3.0, 0.75),
                                  beta=(1.0, 2.0 / 3.0, 0.25))
    ref = sols[-1]
    errs = [rel_err(om, T, ref) for T in sols[:-1]]
    assert max(orders(errs)) < 2.5, errs


# ---------------------------------------------------------------------------
# space: upwind DG advection residual
# ---------------------------------------------------------------------------
def _advection_errors(consistent: bool):
    errs = []
    t_end = 2000.0
    for n in (8, 16, 32):
        m = channel(n)
        om = OMesh(m)
        P = om.P
        u = np.full((2, 3, P), U0)
        v = np.zeros((2, 3, P))
        eta = np.zeros((3, m.n_tri))
        dz = om.thickness(eta)
        T = nodal(om, bump)
        ns = int(math.ceil(t_end / (0.3 * (L / n) / U0)))
        dt = t_end / ns
        if consistent:
            qx, qy = tr.transport(dz, u, v)
            minv = consistent_mass_inverse(om, dz)
            Lop = lambda f: minv(tr.horizontal_residual(om, qx, qy, f))
            for _ in range(ns):
                T = ssp_rk3(T, Lop, dt)
        else:
            for _ in range(ns):
                eta, T, _ = tr.tracer_step(om, eta, T, u, v, dt, 0.0)
        errs.append(rel_err(om, T, nodal(om, lambda x, y: bump(x - U0 * t_end, y))))
    return errs


def test_advection_residual_is_second_order_with_the_consistent_mass():
    """The cos^4 bump advected 1 km by a uniform 0.5 m/s current on 8x8, 16x16 and
    32x32 squares (dt proportional to h): the oracle's horizontal residual with the
    consistent mass converges at the P1 rate 2 (observed rate of the last two
    refinements >= 1.8)."""
    errs = _advection_errors(consistent=True)
    assert orders(errs)[-1] >= 1.8, errs
    assert errs[-1] < 0.03, errs


def test_lumped_mass_tracer_step_is_first_order():
    """The same run through the tracer step, whose mass is lumped onto the vertex
    columns (the 2x2-block vertical system): the lumping is O(h) in the evolution
    of every element's slope, and the rate is 1."""
    errs = _advection_errors(consistent=False)
    o = orders(errs)
    assert 0.8 <= o[-1] <= 1.3, errs
    assert errs[-1] > 0.1, errs


# ---------------------------------------------------------------------------
# horizontal SIPG viscosity
# ---------------------------------------------------------------------------
def _probe_matrix(om, op):
    """Sparse matrix of the linear operator op on (2, 3, P) fields, by probing with
    unit values on triangles that are at least three edges apart (distance-2
    colouring of the triangle graph: a probe's image stays within its own triangle
    and its edge neighbours, which no other probe of the same colour reaches)."""
    import scipy.sparse as sp
    nt = om.n_tri
    nbr = om.nbr
    colour = -np.ones(nt, np.int64)
    for t in range(nt):
        near = set()
        for a in nbr[t]:
            if a < 0:
                continue
            near.add(a)
            near.update(int(b) for b in nbr[a] if b >= 0)
        used = {colour[s] for s in near if colour[s] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[t] = c
    rows, cols, vals = [], [], []
    P = om.P
    idx = np.arange(6 * P).reshape(2, 3, P)
    owner = np.empty(nt, np.int64)
    for col in range(colour.max() + 1):
        tris = np.nonzero(colour == col)[0]
        # which probed triangle every triangle's response belongs to
        owner[:] = -1
        owner[tris] = tris
        for t in tris:
            for a in nbr[t]:
                if a >= 0:
                    owner[a] = t
        for c in range(2):
            for a in range(3):
                f = np.zeros((2, 3, P))
                pr = np.concatenate([np.arange(om.col_off[t], om.col_off[t + 1]) for t in tris])
                f[c, a, pr] = 1.0
                g = op(f)
                nz = np.nonzero(g)
                for (cc, aa, p) in zip(*nz):
                    src_t = owner[om.t_of[p]]
                    if src_t < 0:
                        continue
                    k = om.k_of[p]
                    rows.append(idx[cc, aa, p])
                    cols.append(idx[c, a, om.col_off[src_t] + k])
                    vals.append(g[cc, aa, p])
    return sp.csr_matrix((vals, (rows, cols)), shape=(6 * P, 6 * P))


def _sipg_errors(face_factor: float = 1.0, nu: float = 2.0, penalty: float = 6.0):
    """Neumann problem -div(nu grad u) = f on the square, u = cos(pi x/L) cos(pi y/L)
    (zero normal derivative on the boundary, zero mean), one flat layer: solve
    -A u_h = M f_I with A the oracle's SIPG operator (the planted face_factor
    scales its face terms other than the penalty) and M the consistent mass;
    returns the relative L2 errors of three refinements."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    errs = []
    k = math.pi / L
    ue = lambda x, y: np.cos(k * x) * np.cos(k * y)
    for n in (4, 8, 16):
        m = wl.meshes.square_mesh(n, L, 1, lambda x, y: H + 0.0 * x)
        om = OMesh(m)
        dz = om.thickness(np.zeros((3, m.n_tri)))
        Ap = _probe_matrix(om, lambda f: bc.horizontal_viscosity(om, dz, f, nu, penalty))
        A0 = _probe_matrix(om, lambda f: bc.horizontal_viscosity(om, dz, f, nu, 0.0))
        Kv = _probe_matrix(om, lambda f: _volume_only(om, dz, f, nu))
        A = Kv + face_factor * (A0 - Kv) + (Ap - A0)
        P = om.P
        # consistent mass (flat layers) as a sparse block matrix
        Mh = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 24.0
        G = int_psi_psi()
        idx = np.arange(6 * P).reshape(2, 3, P)
        rows, cols, vals = [], [], []
        sc = om.Jh[om.t_of] * 0.5 * dz[0]
        for c in range(2):
            for d in range(2):
                for a in range(3):
                    for b in range(3):
                        rows.append(idx[c, a]); cols.append(idx[d, b]); vals.append(G[c, d] * Mh[a, b] * sc)
        M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(6 * P, 6 * P))
        uI = nodal(om, ue).ravel()
        f = 2.0 * nu * k * k * uI
        # the Neumann operator has the constants of each node layer in its kernel:
        # the load is made orthogonal to them (the discrete compatibility condition)
        # and a small multiple of the mass fixes them at the exact solution's values
        Kn = np.zeros((6 * P, 2))
        Kn[idx[0].ravel(), 0] = 1.0
        Kn[idx[1].ravel(), 1] = 1.0
        b = M @ f
        MK = M @ Kn
        b = b - MK @ np.linalg.solve(Kn.T @ MK, Kn.T @ b)
        eps = 1e-6 * abs(A).max() / abs(M).max()
        uh = spl.spsolve((-A + eps * M).tocsc(), b + eps * (M @ uI))
        d = (uh - uI).reshape(2, 3, P)
        w = tr.apply_mass(om, dz, np.ones((2, 3, P)))
        errs.append(math.sqrt(float(np.sum(w * d ** 2) / np.sum(w * uI.reshape(2, 3, P) ** 2))))
    return errs


def _volume_only(om, dz, f, nu):
    """-int nu z_zeta grad u . grad v of flat layers, written out independently:
    per prism nu (dz/2) (K (x) G) with the P1 stiffness K_ab = (J_h/2) grad phi_a .
    grad phi_b."""
    G = int_psi_psi()
    t = om.t_of
    g = om.grad[t]                                        # (P, 3, 2)
    K = 0.5 * om.Jh[t][:, None, None] * np.einsum("pai,pbi->pab", g, g)
    return -nu * 0.5 * dz[0][None, None] * np.einsum("cd,pab,dbp->cap", G, K, f)


def test_horizontal_sipg_second_order_on_a_smooth_neumann_problem():
    errs = _sipg_errors()
    assert min(orders(errs)) >= 1.8, errs


def test_horizontal_sipg_wrong_face_flux_is_inconsistent():
    """Planted mistake: the face terms (flux and symmetry) doubled.  The operator is
    no longer consistent: refinement stops reducing the error, which ends an order
    of magnitude above the correct operator's."""
    bad = _sipg_errors(face_factor=2.0)
    good = _sipg_errors()
    assert orders(bad)[-1] < 0.5 and bad[-1] > 10.0 * good[-1], (bad, good)


def test_horizontal_sipg_penalty_on_a_pure_jump():
    """Two triangles sharing one edge, u = 1 on the first and 0 on the second, one
    flat layer: the jump is the only thing the penalty sees, and the difference of
    the operator with and without the penalty isolates that term.  On the first
    triangle, node (c, a) of a shared-edge vertex gets
        -sigma (dz/2) int_edge phi_a dl int psi_c dzeta = -sigma (dz/2) (l/2) (1)
    with sigma = penalty nu / min(r_in); the opposite vertex gets nothing."""
    xy = np.array([[0.0, 0.0], [400.0, 0.0], [150.0, 300.0], [450.0, 350.0]])
    tri = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    from workloads.meshes import Mesh
    m = Mesh(xy=xy, tri=tri, h_tri=np.full((2, 3), H), n_layers=np.ones(2, np.int32),
             bnd=wl.meshes._tag_boundary(xy, tri, None))
    om = OMesh(m)
    dz = om.thickness(np.zeros((3, 2)))
    f = np.zeros((2, 3, 2))
    f[:, :, 0] = 1.0
    nu, pen = 3.0, 6.0
    R = bc.horizontal_viscosity(om, dz, f, nu, pen) - bc.horizontal_viscosity(om, dz, f, nu, 0.0)
    per = lambda p: sum(np.hypot(*(p[(i + 1) % 3] - p[i])) for i in range(3))
    area = lambda p: 0.5 * abs((p[1, 0] - p[0, 0]) * (p[2, 1] - p[0, 1]) - (p[1, 1] - p[0, 1]) * (p[2, 0] - p[0, 0]))
    rin = [area(xy[t]) / (0.5 * per(xy[t])) for t in tri]
    sigma = pen * nu / min(rin)
    ledge = np.hypot(*(xy[2] - xy[1]))
    expect = -sigma * 0.5 * H * 0.5 * ledge
    # shared edge 1 -> 2 is edge 1 of triangle 0 (its vertices 1 and 2)
    for c in range(2):
        assert abs(R[c, 1, 0] - expect) < 1e-12 * abs(expect)
        assert abs(R[c, 2, 0] - expect) < 1e-12 * abs(expect)
        assert abs(R[c, 0, 0]) < 1e-12 * abs(expect)
        # the other side gets the opposite sign (conservation)
    assert abs(R[:, :, 1].sum() + R[:, :, 0].sum()) < 1e-12 * abs(expect)
