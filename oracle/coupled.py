"""Oracle of the coupled (consistent-mass) vertical system of the tracer step.

The paper's implicit column systems are fully assembled per prism column
(Sec. 2.4 "Fully-assembled column solvers"): the consistent 2D mass M_h of
Sec. 2.3 couples the three vertices of every layer, so each prism's top three
nodes couple to all six nodes of the prism above and its bottom three nodes to
all six nodes of the prism below, and every layer is a 6x6 block of one
block-tridiagonal system per column.  This module writes that system out: the
time derivative, the vertical advection and the vertical diffusion keep the
trial function's horizontal dependence (no lumping onto the vertex columns), and
every column system is solved by dense LU.  The horizontal residual is the one of
``tracer.py`` (exact, consistent).

Integrals of products of three P1 functions use the exact moments
I_abe = (1/J_h) int phi_a phi_b phi_e (``baroclinic.tri_cubic_moments``):
    K(w)_ab = J_h sum_e I_abe w_e      for a P1 coefficient with nodal values w_e.

Readings (the discrete vertical forms are in the paper's unavailable supporting
information):
* mass: int phi_a phi_b psi_c psi_d z_zeta = G_cd K(dz/2)_ab (exact, z_zeta linear);
* continuity: the printed D_vd pattern of Eq. 17 with the consistent M_h blocks,
  (D_vd (x) M_h) Omega = R_h(q, 1) - d/dt (M 1), and the 2D elevation with the
  consistent 2D mass, M_h (eta' - eta)/dt = column sum of R_h(q, 1), so that the
  surface flux vanishes;
* vertical advection: volume int Omega T dpsi_c/dzeta phi_a exact; at every
  interface the flux F = Omega^ T^ is taken at the vertices (Omega^ the top value
  of the element below, T^ upwind by the sign of Omega^ at that vertex) and
  integrated as the P1 function with those nodal values: int phi_a F = (M_h F)_a;
* vertical diffusion: its coefficient 1/z_zeta and the SIPG penalty
  sigma = penalty kappa / min(dz_above, dz_below) are not polynomials; their
  horizontal integrals use the 6-point degree-4 triangle rule (exact in zeta).
  With point values of 1/z_zeta, kappa/z_zeta dT/dzeta of a linear-in-z profile is
  exactly kappa dT/dz at every point, so that profile stays exactly steady.
Constant preservation, exact tracer mass and the steady linear profile follow
from these forms (pinned in ``tests/test_oracle_coupled.py``).

Column vectors are indexed (2k + c) * 3 + a: layer k, node level c (0 top),
vertex a.  TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from .mesh import OMesh
from .quadrature import TRI_RULE4, dpsi, int_psi_psi, phi, psi
from . import tracer as tr
from .baroclinic import tri_cubic_moments

G = int_psi_psi()
I3 = tri_cubic_moments()
DPSI = dpsi()
PSI_TOP = psi(1.0)      # values of (psi_top, psi_bot) on the top face of a prism
PSI_BOT = psi(-1.0)     # ... and on its bottom face


def kmat(Jh: np.ndarray, w: np.ndarray) -> np.ndarray:
    """K(w)_ab = J_h sum_e I_abe w_e, (n, 3, 3) for Jh (n,), w (n, 3)."""
    return Jh[:, None, None] * np.einsum("abe,ne->nab", I3, w)


PHI4 = np.array([phi(x, y) for (x, y, _) in TRI_RULE4])        # (6 points, 3)
W4 = np.array([w for (_, _, w) in TRI_RULE4])


def qmat(Jh: np.ndarray, f: np.ndarray) -> np.ndarray:
    """int phi_a phi_b f dA by the degree-4 rule, f (n, 6) the values at its points."""
    return 0.5 * Jh[:, None, None] * np.einsum("q,qa,qb,nq->nab", W4, PHI4, PHI4, f)


def at_points(w: np.ndarray) -> np.ndarray:
    """P1 function with vertex values w (n, 3) at the rule's points: (n, 6)."""
    return w @ PHI4.T


def mass2d(Jh: np.ndarray) -> np.ndarray:
    """Consistent P1 mass M_h = K(1), (n, 3, 3) (J_h/24 [[2,1,1],[1,2,1],[1,1,2]])."""
    return kmat(Jh, np.ones((len(Jh), 3)))


def ix(k: int, c: int, a: int) -> int:
    return (2 * k + c) * 3 + a


def gather6(om: OMesh, F: np.ndarray, tris: np.ndarray, N: int) -> np.ndarray:
    """(2, 3, P) nodal array -> (n, 6N) column vectors."""
    p = om.col_off[tris][:, None] + np.arange(N)[None, :]          # (n, N)
    out = np.empty((len(tris), 2 * N * 3))
    for k in range(N):
        for c in range(2):
            for a in range(3):
                out[:, ix(k, c, a)] = F[c, a, p[:, k]]
    return out


def scatter6(om: OMesh, X: np.ndarray, tris: np.ndarray, N: int, out: np.ndarray) -> None:
    p = om.col_off[tris][:, None] + np.arange(N)[None, :]
    for k in range(N):
        for c in range(2):
            for a in range(3):
                out[c, a, p[:, k]] = X[:, ix(k, c, a)]


def column_thickness(om: OMesh, dz: np.ndarray, tris: np.ndarray, N: int) -> np.ndarray:
    """(3, P) layer thickness -> (n, N, 3)."""
    p = om.col_off[tris][:, None] + np.arange(N)[None, :]
    return np.transpose(dz[:, p], (1, 2, 0))


# ---------------------------------------------------------------------------
# mass
# ---------------------------------------------------------------------------
def apply_mass(om: OMesh, dz: np.ndarray, T: np.ndarray) -> np.ndarray:
    """(M T)_{c,a} = sum_d G_cd sum_b K(dz/2)_ab T_{d,b} per prism, (2, 3, P)."""
    K = kmat(om.Jh[om.t_of], (0.5 * dz).T)                          # (P, 3, 3)
    KT = np.einsum("pab,dbp->dap", K, T)
    out = np.empty_like(T)
    for c in range(2):
        out[c] = G[c, 0] * KT[0] + G[c, 1] * KT[1]
    return out


def tracer_mass(om: OMesh, eta: np.ndarray, T: np.ndarray) -> float:
    """Tracer content sum over all nodes of (M T) with the consistent mass, summed
    with math.fsum: the quantity the coupled step conserves in a closed basin."""
    return math.fsum(apply_mass(om, om.thickness(eta), T).ravel().tolist())


def mass_column(Jh: np.ndarray, dzc: np.ndarray) -> np.ndarray:
    """Block-diagonal column mass (n, 6N, 6N): block k = G (x) K(dz_k / 2)."""
    n, N, _ = dzc.shape
    M = np.zeros((n, 6 * N, 6 * N))
    for k in range(N):
        K = kmat(Jh, 0.5 * dzc[:, k])
        for c in range(2):
            for d in range(2):
                M[:, ix(k, c, 0):ix(k, c, 0) + 3, ix(k, d, 0):ix(k, d, 0) + 3] = G[c, d] * K
    return M


# ---------------------------------------------------------------------------
# continuity
# ---------------------------------------------------------------------------
def continuity(om: OMesh, eta_n: np.ndarray, u: np.ndarray, v: np.ndarray, dt: float):
    """Elevation and nodal vertical flux Omega over [t, t+dt], transport frozen at t.

    2D: M_h (eta' - eta)/dt = column sum of R_h(q, 1) per triangle (Eq. 2 with the
    consistent 2D mass).  3D: per column (D_vd (x) M_h) Omega = F with
    F_{k,c,a} = R_h(q,1)_{k,c,a} - sum_e M_h,ae (dz'_k,e - dz_k,e) / (2 dt), the
    printed D_vd pattern of Eq. 17 with the consistent M_h blocks.
    Returns (eta', Omega (2, 3, P), q)."""
    dz_n = om.thickness(eta_n)
    qx, qy = tr.transport(dz_n, u, v)
    R1 = tr.horizontal_residual(om, qx, qy, np.ones_like(u))
    D = tr.column_sum(om, R1)                                       # (3, n_tri)
    Mh = mass2d(om.Jh)
    deta = np.linalg.solve(Mh, D.T[..., None])[..., 0].T            # (3, n_tri)
    eta_np1 = eta_n + dt * deta
    dhz = 0.5 * om.thickness_change(eta_n, eta_np1)                 # (3, P)
    rate = np.einsum("pae,ep->ap", Mh[om.t_of], dhz) / dt           # (3, P)
    F = R1 - rate[None]
    Om = np.zeros_like(F)
    for N, tris in tr.columns_by_depth(om).items():
        A = np.einsum("ij,nab->niajb", tr.continuity_rows(N), Mh[tris]).reshape(len(tris), 6 * N, 6 * N)
        x = np.linalg.solve(A, gather6(om, F, tris, N)[..., None])[..., 0]
        scatter6(om, x, tris, N, Om)
    return eta_np1, Om, (qx, qy)


# ---------------------------------------------------------------------------
# vertical operator
# ---------------------------------------------------------------------------
def vertical_operator(Jh: np.ndarray, dzc: np.ndarray, Om: np.ndarray, kappa: float,
                      penalty: float = 4.0) -> np.ndarray:
    """Vertical operator A (n, 6N, 6N) of a batch of columns with layer thicknesses
    dzc (n, N, 3) and nodal flux Om (n, 6N):

      A T . v = int Omega T dpsi_c/dzeta phi_a J_h - [F v]_top + [F v]_bot     (advection)
                - a_SIPG(T, v)                                                  (diffusion)

    with the interface flux F and the interpolated diffusion coefficients of the
    module docstring.  a_SIPG = element stiffness int kappa/z_zeta dT dv + on every
    interior interface int (-{kappa dT/dz}[v] - {kappa dv/dz}[T] + sigma [T][v]),
    [f] = f_below,top - f_above,bot, natural (Neumann) surface and bed."""
    n, N, _ = dzc.shape
    A = np.zeros((n, 6 * N, 6 * N))
    Mh = mass2d(Jh)
    cols = np.arange(n)
    for k in range(N):
        # advection, volume: A[(k,c,a),(k,d,e)] += dpsi_c K(sum_f G_fd Om_{k,f})_ae
        for d in range(2):
            w = G[0, d] * Om[:, ix(k, 0, 0):ix(k, 0, 0) + 3] + G[1, d] * Om[:, ix(k, 1, 0):ix(k, 1, 0) + 3]
            Kw = kmat(Jh, w)
            for c in range(2):
                A[:, ix(k, c, 0):ix(k, c, 0) + 3, ix(k, d, 0):ix(k, d, 0) + 3] += DPSI[c] * Kw
        # advection, interface k (top face of layer k, bottom face of layer k - 1):
        # F_b = Omega^_b T^_b with Omega^ = Omega_{k,top}, upwind per vertex
        Wk = Om[:, ix(k, 0, 0):ix(k, 0, 0) + 3]                      # (n, 3)
        for b in range(3):
            own = (Wk[:, b] > 0.0) if k > 0 else np.ones(n, bool)
            col_own = ix(k, 0, b)
            col_up = ix(k - 1, 1, b) if k > 0 else col_own
            for a in range(3):
                coef = Mh[:, a, b] * Wk[:, b]
                for c in range(2):
                    if PSI_TOP[c] != 0.0:       # - [F v] on the top face of layer k
                        A[cols, ix(k, c, a), col_own] -= PSI_TOP[c] * np.where(own, coef, 0.0)
                        A[cols, ix(k, c, a), col_up] -= PSI_TOP[c] * np.where(own, 0.0, coef)
                    if k > 0 and PSI_BOT[c] != 0.0:   # + [F v] on the bottom face of k - 1
                        A[cols, ix(k - 1, c, a), col_own] += PSI_BOT[c] * np.where(own, coef, 0.0)
                        A[cols, ix(k - 1, c, a), col_up] += PSI_BOT[c] * np.where(own, 0.0, coef)
        # diffusion, element stiffness: kappa (2 dpsi_c dpsi_d) int phi_a phi_b / z_zeta
        Ki = qmat(Jh, 1.0 / at_points(0.5 * dzc[:, k]))
        for c in range(2):
            for d in range(2):
                A[:, ix(k, c, 0):ix(k, c, 0) + 3, ix(k, d, 0):ix(k, d, 0) + 3] -= \
                    kappa * 2.0 * DPSI[c] * DPSI[d] * Ki
    # diffusion, interior interfaces
    for i in range(1, N):
        ka, kb = i - 1, i
        dza, dzb = at_points(dzc[:, ka]), at_points(dzc[:, kb])
        Ka = qmat(Jh, 1.0 / dza)                         # int phi_a phi_b / dz_above
        Kb = qmat(Jh, 1.0 / dzb)
        Ks = qmat(Jh, penalty * kappa / np.minimum(dza, dzb))
        # test-side factors: [v] (+1 for the top nodes of kb, -1 for the bottom nodes
        # of ka) and {kappa dv/dz} = kappa/2 (+-1/dz) phi_a on the own side
        for a in range(3):
            rows_jump = ((ix(kb, 0, a), 1.0), (ix(ka, 1, a), -1.0))
            for b in range(3):
                # trial functionals at vertex b: {kappa dT/dz} and [T]
                g_terms = ((ix(ka, 0, b), 0.5 * kappa * Ka[:, a, b]), (ix(ka, 1, b), -0.5 * kappa * Ka[:, a, b]),
                           (ix(kb, 0, b), 0.5 * kappa * Kb[:, a, b]), (ix(kb, 1, b), -0.5 * kappa * Kb[:, a, b]))
                j_terms = ((ix(kb, 0, b), 1.0), (ix(ka, 1, b), -1.0))
                for r, sv in rows_jump:
                    for col, gv in g_terms:           # -{kappa dT/dz}[v]
                        A[:, r, col] -= -sv * gv
                    for col, jv in j_terms:           # + sigma [T][v]
                        A[:, r, col] -= sv * jv * Ks[:, a, b]
                # -{kappa dv/dz}[T] for the four test functions next to the face
                for (kk, Kl) in ((ka, Ka), (kb, Kb)):
                    for c in range(2):
                        dv = 0.5 * kappa * (1.0 if c == 0 else -1.0) * Kl[:, a, b]
                        for col, jv in j_terms:
                            A[:, ix(kk, c, a), col] -= -dv * jv
    return A


def neumann_vector(Jh: np.ndarray, N: int, flux_top: float, flux_bot: float) -> np.ndarray:
    """int phi_a (F_s v(surface) - F_b v(bed)) dA, F = kappa dT/dz prescribed: (n, 6N)."""
    b = np.zeros((len(Jh), 6 * N))
    for a in range(3):
        b[:, ix(0, 0, a)] += Jh / 6.0 * flux_top
        b[:, ix(N - 1, 1, a)] -= Jh / 6.0 * flux_bot
    return b


def stage_solve(om: OMesh, Om: np.ndarray, dz_s: np.ndarray, rhs: np.ndarray, beta_dt: float,
                kappa: float, flux_top: float = 0.0, flux_bot: float = 0.0,
                penalty: float = 4.0) -> np.ndarray:
    """Solve (M^(s) - beta dt A^(s)) T = rhs + beta dt b per column (dense LU)."""
    T = np.zeros_like(rhs)
    for N, tris in tr.columns_by_depth(om).items():
        Jh = om.Jh[tris]
        dzc = column_thickness(om, dz_s, tris, N)
        A = vertical_operator(Jh, dzc, gather6(om, Om, tris, N), kappa, penalty)
        M = mass_column(Jh, dzc)
        r = gather6(om, rhs, tris, N) + beta_dt * neumann_vector(Jh, N, flux_top, flux_bot)
        x = np.linalg.solve(M - beta_dt * A, r[..., None])[..., 0]
        scatter6(om, x, tris, N, T)
    return T


def tracer_step(om: OMesh, eta_n: np.ndarray, T_n: np.ndarray, u: np.ndarray, v: np.ndarray,
                dt: float, kappa: float, flux_top: float = 0.0, flux_bot: float = 0.0,
                T_ext: np.ndarray | None = None):
    """One step of the tracer scheme with the coupled vertical system: transport
    frozen at t_n, one continuity solve, three Shu-Osher SSP-RK3 stages

        M^(s) T^(s) = alpha_s M^n T^n + beta_s (M^(s-1) T^(s-1) + dt R_h(T^(s-1)))
                      + beta_s dt A^(s) T^(s) (+ beta_s dt b)

    with the consistent mass M and the stage elevations eta^{n+1},
    (eta^n + eta^{n+1})/2, eta^{n+1} (the same stage weights and elevations as the
    lumped step).  Returns (eta^{n+1}, T^{n+1}, Omega)."""
    eta_np1, Om, (qx, qy) = continuity(om, eta_n, u, v, dt)
    dz_n = om.thickness(eta_n)
    etas = (eta_np1, 0.5 * (eta_n + eta_np1), eta_np1)
    MTn = apply_mass(om, dz_n, T_n)
    T_prev, dz_prev = T_n, dz_n
    for s in range(3):
        dz_s = om.thickness(etas[s])
        Rh = tr.horizontal_residual(om, qx, qy, T_prev, T_ext=T_ext)
        rhs = tr.SSP_ALPHA[s] * MTn + tr.SSP_BETA[s] * (apply_mass(om, dz_prev, T_prev) + dt * Rh)
        T_s = stage_solve(om, Om, dz_s, rhs, tr.SSP_BETA[s] * dt, kappa, flux_top, flux_bot)
        T_prev, dz_prev = T_s, dz_s
    return eta_np1, T_prev, Om
