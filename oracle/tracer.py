"""Oracle for the tracer path: transport, continuity (vertical flux), horizontal
residual, column operators, SSP-RK3 IMEX step and the tracer mass.

Continuous problem (Eqs. 1, 2, 4-6) in the moving coordinate of ``mesh.py``
(a reading of the vertical coordinate): with z_zeta = dz/dzeta, the layer transport q = z_zeta u and the
vertical flux through coordinate surfaces Omega (per unit horizontal area),

    d/dt z_zeta + div_xy q + d/dzeta Omega = 0                      (continuity)
    d/dt (z_zeta T) + div_xy (q T) + d/dzeta (Omega T)
        = d/dzeta (kappa_v / z_zeta dT/dzeta)                       (tracer)

with Omega = 0 on the bed (Eq. 5) and at the surface (Eq. 4 with s = 0).

Test functions v = phi_a psi_c on each prism.  Terms coupling nodes horizontally
are integrated exactly (``quadrature.py``).  Terms coupling nodes vertically
(the time derivative, vertical advection and vertical diffusion) collapse the
horizontal dependence of the trial function onto the test vertex (a reading),
which yields one system per vertex column with 2x2 blocks per layer:

* mass         m_{a,cd} = (J_h/6) (dz_a/2) int psi_c psi_d
* vertical flux weights W_{a,c}: the vertex-weighted Omega nodal values; the
  continuity rows are the D_vd pattern of Eq. 17 with M_h replaced by the vertex
  weight (the same recursion structure), and the tracer uses the very same W
* vertical diffusion: (J_h/6) x 1D SIPG on the vertex's layer thicknesses
  (a reading; the paper does not state its vertical diffusion form)
"""
from __future__ import annotations

import math
import numpy as np

from .quadrature import TRI_RULE, GAUSS_Z, GAUSS_W, phi, psi, dpsi, int_psi_psi
from .mesh import OMesh


# ---------------------------------------------------------------------------
# transport and horizontal residual
# ---------------------------------------------------------------------------
def transport(dz: np.ndarray, u: np.ndarray, v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Nodal layer transport q = (dz/2) u at both nodes of every vertex-layer
    (the nodal transport precomputed at all nodes, Sec. 2.2)."""
    return 0.5 * dz[None] * u, 0.5 * dz[None] * v


def horizontal_residual(om: OMesh, qx: np.ndarray, qy: np.ndarray, T: np.ndarray,
                        T_ext: np.ndarray | None = None,
                        face_corr: np.ndarray | None = None,
                        q_ext: tuple[np.ndarray, np.ndarray] | None = None) -> np.ndarray:
    """R_h(q, T)_{c,a,p} = int_K q T . grad(phi_a) psi_c J_h
                         - sum_lateral faces int phi_a psi_c (q.n)^ T^ dl dzeta

    i.e. the weak form of -div_xy(q T) (Eq. 6, horizontal part).  Face transport is
    the mean of both sides {q}.n; T^ is upwind at each face quadrature point.
    Walls carry no flux.  Open boundaries use the interior transport and, for
    inflow, the exterior state ``T_ext`` (same layout as T; zero-gradient when None).
    With ``q_ext`` (an exterior transport at the own nodes, same layout as qx, qy)
    the open-boundary face transport is the exterior one alone: the exterior state
    comes from data, as in the 2D mode's characteristic open condition, so that the
    interior's baroclinic velocity does not feed the boundary flux (the split
    scheme; the prescribed-velocity tracer scheme passes none).
    ``face_corr`` (P, 3, 2): an additive correction of the normal transport per
    lateral face and edge quadrature point (the same at both zeta points), used
    for the transport that matches the averaged 2D face flux.
    All arrays are (2, 3, P)."""
    R = np.zeros_like(T)
    t = om.t_of
    Jh = om.Jh[t]
    grad = om.grad[t]                                     # (P, 3, 2)
    # volume term
    for (xi, eta, wg) in TRI_RULE:
        ph = phi(xi, eta)
        for zq, wz in zip(GAUSS_Z, GAUSS_W):
            ps = psi(zq)
            qxp = sum(ph[a] * ps[c] * qx[c, a] for a in range(3) for c in range(2))
            qyp = sum(ph[a] * ps[c] * qy[c, a] for a in range(3) for c in range(2))
            Tp = sum(ph[a] * ps[c] * T[c, a] for a in range(3) for c in range(2))
            w = 0.5 * wg * wz * Jh
            for a in range(3):
                qg = qxp * grad[:, a, 0] + qyp * grad[:, a, 1]
                for c in range(2):
                    R[c, a] += w * qg * Tp * ps[c]
    # lateral faces
    gs, gw = GAUSS_Z, GAUSS_W
    for e in range(3):
        pn, ok = om.nbr_prism(e)
        pn_safe = np.where(ok, pn, 0)
        tn = np.where(ok, om.nbr[t, e], 0)
        nx, ny = om.enrm[t, e, 0], om.enrm[t, e, 1]
        L = om.elen[t, e]
        own = (e, (e + 1) % 3)
        loc = om.nloc[t, e]                               # (P, 2)
        is_open = om.bnd[t, e] == 2
        for gi, (sq, ws) in enumerate(zip(gs, gw)):
            lam = 0.5 * (1.0 + sq)
            wv = (1.0 - lam, lam)                         # basis values of the 2 edge vertices
            for zq, wz in zip(GAUSS_Z, GAUSS_W):
                ps = psi(zq)
                qn_own = np.zeros(om.P); T_own = np.zeros(om.P)
                qn_nb = np.zeros(om.P); T_nb = np.zeros(om.P); qn_x = np.zeros(om.P)
                for j in range(2):
                    a = own[j]
                    an = np.where(ok, loc[:, j], 0)
                    for c in range(2):
                        b = wv[j] * ps[c]
                        qn_own += b * (qx[c, a] * nx + qy[c, a] * ny)
                        T_own += b * T[c, a]
                        qn_nb += b * (qx[c, an, pn_safe] * nx + qy[c, an, pn_safe] * ny)
                        T_nb += b * T[c, an, pn_safe]
                        if q_ext is not None:
                            qn_x += b * (q_ext[0][c, a] * nx + q_ext[1][c, a] * ny)
                if T_ext is not None:
                    T_x = sum(wv[j] * ps[c] * T_ext[c, own[j]] for j in range(2) for c in range(2))
                else:
                    T_x = T_own
                qn_open = qn_own if q_ext is None else qn_x
                qn = np.where(ok, 0.5 * (qn_own + qn_nb), np.where(is_open, qn_open, 0.0))
                if face_corr is not None:
                    qn = qn + np.where(ok | is_open, face_corr[:, e, gi], 0.0)
                T_other = np.where(ok, T_nb, T_x)
                flux = qn * np.where(qn > 0.0, T_own, T_other)
                w = 0.5 * L * ws * wz
                for j in range(2):
                    for c in range(2):
                        R[c, own[j]] -= w * flux * wv[j] * ps[c]
    return R


def column_sum(om: OMesh, R: np.ndarray) -> np.ndarray:
    """Sum over the layers and both nodes of each vertex column: (3, n_tri)."""
    s = R.sum(axis=0)                                     # (3, P)
    out = np.zeros((3, om.n_tri))
    for a in range(3):
        np.add.at(out[a], om.t_of, s[a])
    return out


def vertex_weight(om: OMesh) -> np.ndarray:
    """J_h/6 = integral of phi_a over the triangle (vertex quadrature weight), (3, n_tri)."""
    return np.tile(om.Jh / 6.0, (3, 1))


# ---------------------------------------------------------------------------
# column systems
# ---------------------------------------------------------------------------
def continuity_rows(N: int) -> np.ndarray:
    """(2N, 2N) operator of the vertex-weighted vertical flux W on one column,
    derived from  <psi W^int>_top - <psi W^ext>_bot - int W dpsi/dzeta  with W^int the
    element's own top value, W^ext the top value of the element below and 0 on the
    bed (Eq. 17).  Unknown index 2k + c."""
    V = np.zeros((2 * N, 2 * N))
    d = dpsi()
    top, bot = psi(1.0), psi(-1.0)
    for k in range(N):
        for c in range(2):
            r = 2 * k + c
            V[r, 2 * k + 0] += top[c]
            if k + 1 < N:
                V[r, 2 * (k + 1) + 0] -= bot[c]
            for e in range(2):
                V[r, 2 * k + e] -= sum(wz * psi(zq)[e] * d[c] for zq, wz in zip(GAUSS_Z, GAUSS_W))
    return V


def hpg_rows(N: int) -> np.ndarray:
    """(2N, 2N) operator of the top-down column system of Eq. 15/16: r^ext (bottom
    value of the element above) on the top face, r^int on the bottom face; the
    surface value is moved to the right-hand side."""
    V = np.zeros((2 * N, 2 * N))
    d = dpsi()
    top, bot = psi(1.0), psi(-1.0)
    for k in range(N):
        for c in range(2):
            r = 2 * k + c
            if k > 0:
                V[r, 2 * (k - 1) + 1] += top[c]
            V[r, 2 * k + 1] -= bot[c]
            for e in range(2):
                V[r, 2 * k + e] -= sum(wz * psi(zq)[e] * d[c] for zq, wz in zip(GAUSS_Z, GAUSS_W))
    return V


def columns_by_depth(om: OMesh) -> dict[int, np.ndarray]:
    """Triangles grouped by their layer count."""
    out = {}
    for N in np.unique(om.N):
        out[int(N)] = np.nonzero(om.N == N)[0]
    return out


def gather_columns(om: OMesh, F: np.ndarray, tris: np.ndarray, N: int) -> np.ndarray:
    """(2,3,P) nodal array -> (len(tris), 3, 2N) column vectors (index 2k + c)."""
    p = om.col_off[tris][:, None] + np.arange(N)[None, :]           # (nt, N)
    out = np.empty((len(tris), 3, 2 * N))
    for c in range(2):
        out[:, :, c::2] = np.transpose(F[c][:, p], (1, 0, 2))
    return out


def scatter_columns(om: OMesh, X: np.ndarray, tris: np.ndarray, N: int, out: np.ndarray) -> None:
    p = om.col_off[tris][:, None] + np.arange(N)[None, :]
    for c in range(2):
        out[c][:, p] = np.transpose(X[:, :, c::2], (1, 0, 2))


def solve_continuity(om: OMesh, F: np.ndarray) -> np.ndarray:
    """W (2,3,P) from the per-vertex-column systems continuity_rows(N) W = F."""
    W = np.zeros_like(F)
    for N, tris in columns_by_depth(om).items():
        A = continuity_rows(N)
        b = gather_columns(om, F, tris, N)
        x = np.linalg.solve(A[None, None], b[..., None])[..., 0]
        scatter_columns(om, x, tris, N, W)
    return W


def vertical_matrix(Wc: np.ndarray, dzc: np.ndarray, kappa: float, omega: np.ndarray,
                    penalty: float = 4.0) -> np.ndarray:
    """Linear vertical operator A (ncol, 2N, 2N) of one batch of vertex columns.

    R_v(T) = int W T dpsi_c/dzeta - [psi_c W^ T^]_top + [psi_c W^ T^]_bot        (advection)
             - omega * a_SIPG(T, psi_c)                                        (diffusion)

    Wc (ncol, 2N) vertex-weighted fluxes, dzc (ncol, N) layer thicknesses, omega
    (ncol,) the vertex weight J_h/6.  Interface i carries W^_i = W_{i,top} (0 on the
    bed), upwinded: T^ = T_{i,top} if W^_i > 0 else T_{i-1,bot}; the surface uses the
    interior T_{0,top}.  SIPG: element stiffness int kappa/(dz/2) dpsi dpsi, interface
    terms -{kappa dT/dz}[v] - {kappa dv/dz}[T] + sigma [T][v], [v] = v_below,top -
    v_above,bot, sigma = penalty * kappa / min(dz_above, dz_below) (the penalty is a reading)."""
    ncol, twoN = Wc.shape
    N = twoN // 2
    A = np.zeros((ncol, twoN, twoN))
    d = dpsi()
    top, bot = psi(1.0), psi(-1.0)
    # advection, volume
    for k in range(N):
        for c in range(2):
            for dd in range(2):
                acc = np.zeros(ncol)
                for zq, wz in zip(GAUSS_Z, GAUSS_W):
                    ps = psi(zq)
                    Wq = Wc[:, 2 * k] * ps[0] + Wc[:, 2 * k + 1] * ps[1]
                    acc += wz * Wq * ps[dd] * d[c]
                A[:, 2 * k + c, 2 * k + dd] += acc
    # advection, interfaces
    idx = np.arange(ncol)
    for i in range(N):
        What = Wc[:, 2 * i]
        if i == 0:
            src = np.full(ncol, 0)
        else:
            src = np.where(What > 0.0, 2 * i, 2 * (i - 1) + 1)
        for c in range(2):
            A[idx, 2 * i + c, src] -= top[c] * What
            if i > 0:
                A[idx, 2 * (i - 1) + c, src] += bot[c] * What
    # diffusion
    for k in range(N):
        for c in range(2):
            for dd in range(2):
                kl = sum(wz * kappa / (0.5 * dzc[:, k]) * d[c] * d[dd] for zq, wz in zip(GAUSS_Z, GAUSS_W))
                A[:, 2 * k + c, 2 * k + dd] -= omega * kl
    for i in range(1, N):
        ka, kb = i - 1, i                         # layer above, layer below
        g = np.zeros((ncol, twoN))                # {kappa dT/dz}
        g[:, 2 * ka] += 0.5 * kappa / dzc[:, ka]
        g[:, 2 * ka + 1] -= 0.5 * kappa / dzc[:, ka]
        g[:, 2 * kb] += 0.5 * kappa / dzc[:, kb]
        g[:, 2 * kb + 1] -= 0.5 * kappa / dzc[:, kb]
        j = np.zeros((ncol, twoN))                # [T]
        j[:, 2 * kb] += 1.0
        j[:, 2 * ka + 1] -= 1.0
        sig = penalty * kappa / np.minimum(dzc[:, ka], dzc[:, kb])
        a_int = (-np.einsum("ni,nj->nij", j, g) - np.einsum("ni,nj->nij", g, j)
                 + sig[:, None, None] * np.einsum("ni,nj->nij", j, j))
        A -= omega[:, None, None] * a_int
    return A


def neumann_vector(ncol: int, N: int, omega: np.ndarray, flux_top: float, flux_bot: float) -> np.ndarray:
    """omega (F_s v(surface) - F_b v(bed)) with F = kappa dT/dz prescribed."""
    b = np.zeros((ncol, 2 * N))
    b[:, 0] += omega * flux_top
    b[:, 2 * N - 1] -= omega * flux_bot
    return b


def mass_matrix(dzc: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """Block-diagonal lumped mass (ncol, 2N, 2N): omega (dz/2) int psi_c psi_d."""
    ncol, N = dzc.shape
    G = int_psi_psi()
    M = np.zeros((ncol, 2 * N, 2 * N))
    for k in range(N):
        M[:, 2 * k:2 * k + 2, 2 * k:2 * k + 2] = (omega * 0.5 * dzc[:, k])[:, None, None] * G[None]
    return M


def apply_mass(om: OMesh, dz: np.ndarray, T: np.ndarray) -> np.ndarray:
    """(M T) in nodal layout for the lumped mass at layer thicknesses dz (3,P)."""
    G = int_psi_psi()
    w = (om.Jh[om.t_of] / 6.0)[None] * 0.5 * dz         # (3, P)
    out = np.empty_like(T)
    for c in range(2):
        out[c] = w * (G[c, 0] * T[0] + G[c, 1] * T[1])
    return out


def tracer_mass(om: OMesh, eta: np.ndarray, T: np.ndarray) -> float:
    """Discrete tracer content sum over all nodes of (M T): the quantity the scheme
    conserves in a closed basin.  Summed with math.fsum (exactly rounded)."""
    MT = apply_mass(om, om.thickness(eta), T)
    return math.fsum(MT.ravel().tolist())


# ---------------------------------------------------------------------------
# one step: frozen transport, continuity, SSP-RK3 IMEX stages
# ---------------------------------------------------------------------------
def continuity(om: OMesh, eta_n: np.ndarray, u: np.ndarray, v: np.ndarray, dt: float):
    """Advance the elevation with the column-integrated continuity and solve the
    vertical flux W over [t, t+dt] with transport frozen at t.

    2D: (J_h/6) (eta^{n+1} - eta^n)/dt = column sum of R_h(q, 1)  (Eq. 2 with the
    2D mass implied by the lumped 3D mass, so that the surface flux vanishes).
    3D: continuity_rows W = R_h(q, 1) - (m^{n+1} - m^n)/dt per vertex column (Eq. 17),
    m = (J_h/12) dz the lumped mass of T = 1.
    Returns (eta^{n+1}, W, q)."""
    dz_n = om.thickness(eta_n)
    qx, qy = transport(dz_n, u, v)
    R1 = horizontal_residual(om, qx, qy, np.ones_like(u))
    D = column_sum(om, R1)
    eta_np1 = eta_n + dt * D / vertex_weight(om)
    w12 = (om.Jh[om.t_of] / 12.0)[None]
    F = R1 - (w12 * om.thickness_change(eta_n, eta_np1) / dt)[None]
    W = solve_continuity(om, F)
    return eta_np1, W, (qx, qy)


SSP_ALPHA = (0.0, 0.75, 1.0 / 3.0)
SSP_BETA = (1.0, 0.25, 2.0 / 3.0)


def stage_solve(om: OMesh, W: np.ndarray, dz_s: np.ndarray, rhs: np.ndarray, beta_dt: float,
                kappa: float, flux_top: float = 0.0, flux_bot: float = 0.0) -> np.ndarray:
    """Solve (M^(s) - beta dt A^(s)) T = rhs + beta dt b per vertex column."""
    T = np.zeros_like(rhs)
    for N, tris in columns_by_depth(om).items():
        ncol = len(tris)
        Wc = gather_columns(om, W, tris, N).reshape(ncol * 3, 2 * N)
        p = om.col_off[tris][:, None] + np.arange(N)[None, :]
        dzc = np.transpose(dz_s[:, p], (1, 0, 2)).reshape(ncol * 3, N)
        omega = np.repeat(om.Jh[tris] / 6.0, 3)
        A = vertical_matrix(Wc, dzc, kappa, omega)
        M = mass_matrix(dzc, omega)
        b = neumann_vector(ncol * 3, N, omega, flux_top, flux_bot)
        r = gather_columns(om, rhs, tris, N).reshape(ncol * 3, 2 * N) + beta_dt * b
        x = np.linalg.solve(M - beta_dt * A, r[..., None])[..., 0]
        scatter_columns(om, x.reshape(ncol, 3, 2 * N), tris, N, T)
    return T


def tracer_step(om: OMesh, eta_n: np.ndarray, T_n: np.ndarray, u: np.ndarray, v: np.ndarray,
                dt: float, kappa: float, flux_top: float = 0.0, flux_bot: float = 0.0):
    """One step of the tracer scheme: transport frozen at t_n, one continuity solve,
    three Shu-Osher SSP-RK3 stages with explicit horizontal and implicit vertical terms

        M^(s) T^(s) = alpha_s M^n T^n + beta_s (M^(s-1) T^(s-1) + dt R_h(T^(s-1)))
                      + beta_s dt R_v(T^(s))

    (alpha, beta) = (0,1), (3/4,1/4), (1/3,2/3); stage elevations eta^{n+1},
    (eta^n + eta^{n+1})/2, eta^{n+1} (the masses the continuity implies).
    Arrays in (2,3,P) / (3,n_tri) layout.  Returns (eta^{n+1}, T^{n+1}, W)."""
    eta_np1, W, (qx, qy) = continuity(om, eta_n, u, v, dt)
    dz_n = om.thickness(eta_n)
    etas = (eta_np1, 0.5 * (eta_n + eta_np1), eta_np1)
    MTn = apply_mass(om, dz_n, T_n)
    T_prev, dz_prev = T_n, dz_n
    for s in range(3):
        dz_s = om.thickness(etas[s])
        Rh = horizontal_residual(om, qx, qy, T_prev)
        rhs = SSP_ALPHA[s] * MTn + SSP_BETA[s] * (apply_mass(om, dz_prev, T_prev) + dt * Rh)
        T_s = stage_solve(om, W, dz_s, rhs, SSP_BETA[s] * dt, kappa, flux_top, flux_bot)
        T_prev, dz_prev = T_s, dz_s
    return eta_np1, T_prev, W


def to3(f: np.ndarray, P: int) -> np.ndarray:
    return np.asarray(f, dtype=np.float64).reshape(2, 3, P)


def to2(f: np.ndarray, n_tri: int) -> np.ndarray:
    return np.asarray(f, dtype=np.float64).reshape(3, n_tri)
