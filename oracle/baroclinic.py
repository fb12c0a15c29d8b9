"""Oracle of the baroclinic step: density and horizontal pressure gradient, 3D
momentum residual, 2D external mode, mode coupling and the split-IMEX step.

Readings: the paper defers the discrete forms to its supporting information,
so every form below is written from the
continuous equations (Eqs. 1-10) in the moving coordinate of ``mesh.py`` with the
structure the paper states: the column systems of Eqs. 15-17 / Algorithm 1, the
discrete momentum step of Eqs. 11-14, the 2D/3D coupling F2D of Sec. 2.2 and the
transport consistency of Sec. 2.5.

Arrays: 3D nodal fields (2, 3, P) [c][a][p]; 2D nodal fields (3, n_tri) [a][t];
2D face data (n_tri, 3, 2) [t][edge][edge Gauss point] in the edge's own
orientation (point 0 nearer vertex e).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .mesh import OMesh
from .quadrature import TRI_RULE, GAUSS_Z, GAUSS_W, GRAD_REF, phi, psi, dpsi, int_psi_psi
from . import tracer as tr


@dataclasses.dataclass
class Params:
    g: float = 9.81
    rho0: float = 1025.0
    f: float = 1e-4
    alpha: float = 2e-4
    beta: float = 7.6e-4
    T0: float = 10.0
    S0: float = 35.0
    kappa_v: float = 1e-3
    nu_v: float = 1e-3
    kappa_h: float = 0.0
    nu_h: float = 0.0
    cd: float = 2.5e-3
    penalty_v: float = 4.0
    penalty_h: float = 6.0
    tide_amp: float = 1.0
    tide_period: float = 44712.0
    n_sub: int = 20
    forcing: bool = False        # prescribed exterior velocity / tracers (Forcing)


@dataclasses.dataclass
class Forcing:
    """Open-boundary forcing given at two times t_a < t_b and linear in time between
    them (Sec. 3, data management: forcing fields vary linearly between two input
    states and are interpolated where they are used): exterior velocity (u, v) and
    tracers (T, S) at the open-boundary nodes, (2, 3, P) like the state.  theta(t) =
    (t - t_a)/(t_b - t_a) is not clamped, so the data stay linear in time."""
    t_a: float
    t_b: float
    u_a: np.ndarray
    v_a: np.ndarray
    u_b: np.ndarray
    v_b: np.ndarray
    T_a: np.ndarray
    S_a: np.ndarray
    T_b: np.ndarray
    S_b: np.ndarray

    def theta(self, t: float) -> float:
        return (t - self.t_a) / (self.t_b - self.t_a)

    def at(self, t: float):
        th = self.theta(t)
        lerp = lambda a, b: a + th * (b - a)
        return lerp(self.u_a, self.u_b), lerp(self.v_a, self.v_b), lerp(self.T_a, self.T_b), lerp(self.S_a, self.S_b)


def exterior_transport(om: OMesh, u_x, v_x):
    """Exterior layer transport q_ext = (dz_rest/2) u_ext at the nodes (the rest
    thickness, so that its column sum is linear in time with the data)."""
    return tr.transport(om.thickness(np.zeros((3, om.n_tri))), u_x, v_x)


def exterior_column_transport(om: OMesh, u_x, v_x):
    """Q_ext = column sum of q_ext (3, n_tri): the 2D exterior transport as the
    vertical sum of the 3D one (the linear-transport consistency of Sec. 2.5)."""
    qx, qy = exterior_transport(om, u_x, v_x)
    return tr.column_sum(om, qx), tr.column_sum(om, qy)


@dataclasses.dataclass
class State:
    u: np.ndarray
    v: np.ndarray
    T: np.ndarray
    S: np.ndarray
    eta: np.ndarray
    U: np.ndarray
    V: np.ndarray
    T_ext: np.ndarray | None = None
    S_ext: np.ndarray | None = None
    forcing: Forcing | None = None


# 2-point Gauss along edges: parameter lam from vertex e (0) to vertex e+1 (1)
EDGE_LAM = 0.5 * (1.0 + GAUSS_Z)
EDGE_W = GAUSS_W                      # weights on [-1, 1]; |edge|/2 scales them


# ---------------------------------------------------------------------------
# density and horizontal pressure gradient (Eqs. 7-8, Eqs. 15-16, Algorithm 1)
# ---------------------------------------------------------------------------
def density_anomaly(par: Params, T: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Linear equation of state rho' = rho0 (-alpha (T - T0) + beta (S - S0))."""
    return par.rho0 * (-par.alpha * (T - par.T0) + par.beta * (S - par.S0))


def _z_nodes(om: OMesh, eta: np.ndarray):
    zt, zb = om.interfaces(eta)          # (3, P)
    return zt, zb


def hpg_rhs(om: OMesh, par: Params, rho: np.ndarray, eta: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """F = -int_K v g grad_h rho' dV for v = phi_a psi_c (physical horizontal gradient at
    constant z), the right-hand side of dr/dz = -g grad_h rho': r is the horizontal
    gradient of the baroclinic hydrostatic pressure p' = g int_z^eta rho' dz' (Eq. 7),
    so it grows downward by g grad_h rho' per metre (Eq. 8 integrated from the top
    down).  In the weak form
        +g int_K rho' grad_h v dV - g oint_dK v {rho'} n_h dS
    with grad_h v|_z = grad(phi_a) psi_c - phi_a psi_c' grad_xy z / z_zeta and
    dV = J_h z_zeta dA dzeta.  Lateral faces: normal n_e, dS = z_zeta dl dzeta (own
    geometry), central {rho'} (own value on boundaries).  Top/bottom faces:
    n_h dS = -grad z_top dA / +grad z_bot dA, central {rho'} with the element above
    / below (own value at the surface and the bed).  The surface condition
    r = g rho'(eta) grad(eta) (Eq. 8) enters through the top row of layer 0:
    F_top -= M_h r_surface.  Returns (Fx, Fy), each (2, 3, P)."""
    Fx = np.zeros_like(rho); Fy = np.zeros_like(rho)
    t = om.t_of
    Jh = om.Jh[t]
    grad = om.grad[t]                                      # (P, 3, 2)
    zt, zb = _z_nodes(om, eta)
    # grad_xy z at the top and bottom interface: linear in xy per prism
    gzt = np.stack([sum(zt[a] * grad[:, a, d] for a in range(3)) for d in range(2)], -1)  # (P, 2)
    gzb = np.stack([sum(zb[a] * grad[:, a, d] for a in range(3)) for d in range(2)], -1)
    dz = zt - zb                                           # (3, P)
    ds = dpsi()
    g = par.g
    # volume
    for (xi, et, wg) in TRI_RULE:
        ph = phi(xi, et)
        zz = 0.5 * sum(ph[a] * dz[a] for a in range(3))   # z_zeta
        for zq, wz in zip(GAUSS_Z, GAUSS_W):
            ps = psi(zq)
            rp = sum(ph[a] * ps[c] * rho[c, a] for a in range(3) for c in range(2))
            gz = ps[0] * gzt + ps[1] * gzb                 # grad_xy z at (xi, eta, zeta)
            w = 0.5 * wg * wz * Jh
            for a in range(3):
                for c in range(2):
                    # rho' (grad phi_a psi_c z_zeta - phi_a dpsi_c grad z)
                    for d, F in ((0, Fx), (1, Fy)):
                        F[c, a] += g * w * rp * (grad[:, a, d] * ps[c] * zz - ph[a] * ds[c] * gz[:, d])
    # lateral faces
    for e in range(3):
        pn, ok = om.nbr_prism(e)
        pn_safe = np.where(ok, pn, 0)
        n = om.enrm[t, e]                                  # (P, 2)
        L = om.elen[t, e]
        own = (e, (e + 1) % 3)
        loc = om.nloc[t, e]
        for lam, ws in zip(EDGE_LAM, EDGE_W):
            wv = (1.0 - lam, lam)
            zz = 0.5 * (wv[0] * dz[own[0]] + wv[1] * dz[own[1]])
            for zq, wz in zip(GAUSS_Z, GAUSS_W):
                ps = psi(zq)
                r_own = sum(wv[j] * ps[c] * rho[c, own[j]] for j in range(2) for c in range(2))
                r_nb = np.zeros(om.P)
                for j in range(2):
                    an = np.where(ok, loc[:, j], 0)
                    for c in range(2):
                        r_nb += wv[j] * ps[c] * rho[c, an, pn_safe]
                rh = np.where(ok, 0.5 * (r_own + r_nb), r_own)
                w = 0.5 * L * ws * wz * zz
                for j in range(2):
                    for c in range(2):
                        Fx[c, own[j]] -= g * w * rh * n[:, 0] * wv[j] * ps[c]
                        Fy[c, own[j]] -= g * w * rh * n[:, 1] * wv[j] * ps[c]
    # top and bottom faces (zeta = +1: psi_top = 1; zeta = -1: psi_bot = 1)
    above = np.where(om.k_of > 0, np.arange(om.P) - 1, -1)
    below = np.where(om.k_of + 1 < om.N[t], np.arange(om.P) + 1, -1)
    for (xi, et, wg) in TRI_RULE:
        ph = phi(xi, et)
        w = 0.5 * wg * Jh
        r_top_own = sum(ph[a] * rho[0, a] for a in range(3))
        r_top_up = sum(ph[a] * rho[1, a][np.where(above >= 0, above, 0)] for a in range(3))
        r_top = np.where(above >= 0, 0.5 * (r_top_own + r_top_up), r_top_own)
        r_bot_own = sum(ph[a] * rho[1, a] for a in range(3))
        r_bot_dn = sum(ph[a] * rho[0, a][np.where(below >= 0, below, 0)] for a in range(3))
        r_bot = np.where(below >= 0, 0.5 * (r_bot_own + r_bot_dn), r_bot_own)
        for a in range(3):
            for d, F in ((0, Fx), (1, Fy)):
                F[0, a] -= g * w * ph[a] * r_top * (-gzt[:, d])
                F[1, a] -= g * w * ph[a] * r_bot * (+gzb[:, d])
    # surface condition: r^ext on the top face of layer 0 = g rho'(top) grad eta
    Mh = om.mass2d()[t]                                    # (P, 3, 3)
    geta = np.stack([sum(eta[a, t] * grad[:, a, d] for a in range(3)) for d in range(2)], -1)
    top = om.k_of == 0
    for d, F in ((0, Fx), (1, Fy)):
        rs = g * rho[0] * geta[:, d][None]                 # (3, P) nodal r_surface
        MR = np.einsum("pab,bp->ap", Mh, rs)
        F[0] -= np.where(top[None], MR, 0.0)
    return Fx, Fy


def hpg_solve(om: OMesh, Fx: np.ndarray, Fy: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """r from D_vu r = F per column (Eq. 16): the block operator hpg_rows(N) with the
    consistent 2D mass M_h in every block, solved densely."""
    Mh = om.mass2d()
    rx = np.zeros_like(Fx); ry = np.zeros_like(Fy)
    for N, tris in tr.columns_by_depth(om).items():
        D = tr.hpg_rows(N)
        p = om.col_off[tris][:, None] + np.arange(N)[None, :]
        for F, r in ((Fx, rx), (Fy, ry)):
            # unknown ordering (k, c, a): (2N * 3)
            b = np.transpose(F[:, :, p], (2, 3, 0, 1)).reshape(len(tris), 6 * N)   # (nt, N, 2, 3)
            A = np.einsum("ij,tab->tiajb", D, Mh[tris]).reshape(len(tris), 6 * N, 6 * N)
            x = np.linalg.solve(A, b[..., None])[..., 0].reshape(len(tris), N, 2, 3)
            r[:, :, p] = np.transpose(x, (2, 3, 0, 1))
    return rx, ry


def hpg(om: OMesh, par: Params, T: np.ndarray, S: np.ndarray, eta: np.ndarray):
    rho = density_anomaly(par, T, S)
    Fx, Fy = hpg_rhs(om, par, rho, eta)
    return hpg_solve(om, Fx, Fy)


# ---------------------------------------------------------------------------
# 3D momentum horizontal terms F_3D^h (Sec. 2.2)
# ---------------------------------------------------------------------------
def lumped_source(om: OMesh, dz: np.ndarray, fx: np.ndarray) -> np.ndarray:
    """(M f) for a nodal source f with the lumped 2x2-per-layer mass."""
    return tr.apply_mass(om, dz, fx)


def tri_cubic_moments() -> np.ndarray:
    """I[a, b, e] = (1/J_h) int_K phi_a phi_b phi_e dA for the P1 basis of a triangle:
    1/20 when a = b = e, 1/60 when exactly two indices agree, 1/120 when all differ
    (the barycentric moments 2A p! q! r! / (p + q + r + 2)! with J_h = 2A)."""
    I = np.empty((3, 3, 3))
    for a in range(3):
        for b in range(3):
            for e in range(3):
                n_eq = len({a, b, e})
                I[a, b, e] = {1: 1.0 / 20.0, 2: 1.0 / 60.0, 3: 1.0 / 120.0}[n_eq]
    return I


def pressure_source(om: OMesh, dz: np.ndarray, r: np.ndarray) -> np.ndarray:
    """int_K phi_a psi_c r dV for the nodal field r (2, 3, P), integrated exactly: r is
    P1 x P1 and z_zeta = sum_e phi_e dz_e / 2 is linear over the triangle, so
        S[c, a] = J_h sum_d G_cd sum_b (sum_e I_abe dz_e / 2) r[d, b].
    With the consistent M_h of the r solve (Eq. 16) this makes the momentum source
    the weak pressure gradient itself, the negative adjoint of the weak divergence of
    the continuity; the horizontally lumped product instead leaves M_l M_c^-1 between
    them, and a stratified rest state then grows a slow mode on irregular meshes."""
    G = tr.int_psi_psi()
    I = tri_cubic_moments()
    hz = 0.5 * dz                                                  # (3, P)
    K = om.Jh[om.t_of][:, None, None] * np.einsum("abe,ep->pab", I, hz)   # (P, 3, 3)
    Kr = np.einsum("pab,dbp->dap", K, r)                           # (2, 3, P)
    out = np.empty_like(r)
    for c in range(2):
        out[c] = G[c, 0] * Kr[0] + G[c, 1] * Kr[1]
    return out


def horizontal_viscosity(om: OMesh, dz: np.ndarray, u: np.ndarray, nu: float, penalty: float) -> np.ndarray:
    """SIPG for div_zeta(nu z_zeta grad_zeta u) on coordinate surfaces, tested with
    phi_a psi_c:
      -int nu z_zeta grad u . grad v J_h
      + oint ({nu z_zeta grad u}.n v + 1/2 nu z_zeta^- grad v.n [u] - sigma {z_zeta} [u] v)
    sigma = penalty nu / r_in (min over both sides); walls and open boundaries:
    natural (zero flux).  Face z_zeta: own for the own-gradient terms, mean for the
    penalty."""
    R = np.zeros_like(u)
    if nu == 0.0:
        return R
    t = om.t_of
    Jh = om.Jh[t]
    grad = om.grad[t]
    rin = om.Jh / om.elen.sum(axis=1)
    # grad u at zeta points: linear in zeta, constant in xy
    def gradu(f, idx, gr):
        return [np.stack([sum(f[c, a][idx] * gr[:, a, d] for a in range(3)) for d in range(2)], -1)
                for c in range(2)]                                   # per node layer c: (P, 2)
    gu = gradu(u, slice(None), grad)
    for (xi, et, wg) in TRI_RULE:
        ph = phi(xi, et)
        zz = 0.5 * sum(ph[a] * dz[a] for a in range(3))
        for zq, wz in zip(GAUSS_Z, GAUSS_W):
            ps = psi(zq)
            g_ = ps[0] * gu[0] + ps[1] * gu[1]
            w = 0.5 * wg * wz * Jh * nu * zz
            for a in range(3):
                for c in range(2):
                    R[c, a] -= w * (g_[:, 0] * grad[:, a, 0] + g_[:, 1] * grad[:, a, 1]) * ps[c]
    for e in range(3):
        pn, ok = om.nbr_prism(e)
        pn_safe = np.where(ok, pn, 0)
        tn = np.where(ok, om.nbr[t, e], 0)
        n = om.enrm[t, e]
        L = om.elen[t, e]
        own = (e, (e + 1) % 3)
        loc = om.nloc[t, e]
        grn = om.grad[tn]
        gu_n = [np.stack([sum(u[c, a][pn_safe] * grn[:, a, d] for a in range(3)) for d in range(2)], -1)
                for c in range(2)]
        sig = penalty * nu / np.minimum(rin[t], rin[tn])
        for lam, ws in zip(EDGE_LAM, EDGE_W):
            wv = (1.0 - lam, lam)
            zz_o = 0.5 * (wv[0] * dz[own[0]] + wv[1] * dz[own[1]])
            zz_n = np.zeros(om.P)
            for j in range(2):
                an = np.where(ok, loc[:, j], 0)
                zz_n += 0.5 * wv[j] * dz[an, pn_safe]
            for zq, wz in zip(GAUSS_Z, GAUSS_W):
                ps = psi(zq)
                u_o = sum(wv[j] * ps[c] * u[c, own[j]] for j in range(2) for c in range(2))
                u_n = np.zeros(om.P)
                for j in range(2):
                    an = np.where(ok, loc[:, j], 0)
                    for c in range(2):
                        u_n += wv[j] * ps[c] * u[c, an, pn_safe]
                go = ps[0] * gu[0] + ps[1] * gu[1]
                gn = ps[0] * gu_n[0] + ps[1] * gu_n[1]
                flux = 0.5 * nu * ((zz_o * (go * n).sum(-1)) + (zz_n * (gn * n).sum(-1)))
                jump = u_o - u_n
                w = np.where(ok, 0.5 * L * ws * wz, 0.0)
                # every test function of the element: phi_a vanishes on the face for
                # the opposite vertex, but its gradient does not
                for a in range(3):
                    va = wv[own.index(a)] if a in own else 0.0
                    for c in range(2):
                        v = va * ps[c]
                        gv = (grad[:, a] * n).sum(-1) * ps[c]     # grad v . n on the own side
                        R[c, a] += w * (flux * v + 0.5 * nu * zz_o * gv * jump
                                        - sig * 0.5 * (zz_o + zz_n) * jump * v)
    return R


def bottom_drag(om: OMesh, par: Params, u: np.ndarray, v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Quadratic bed stress -C_d |u_b| u_b on the bed face of every bottom layer, by
    vertex quadrature (J_h/6 per bottom node)."""
    Dx = np.zeros_like(u); Dy = np.zeros_like(v)
    bot = (om.k_of + 1) == om.N[om.t_of]
    w = om.Jh[om.t_of] / 6.0
    ub, vb = u[1], v[1]
    sp = np.sqrt(ub ** 2 + vb ** 2)
    Dx[1] = np.where(bot[None], -par.cd * w[None] * sp * ub, 0.0)
    Dy[1] = np.where(bot[None], -par.cd * w[None] * sp * vb, 0.0)
    return Dx, Dy


def momentum_horizontal(om: OMesh, par: Params, u, v, qx, qy, rx, ry, dz, face_corr=None, ext=None):
    """F_3D^h(u, q, r) (Eq. 11): advection -div(q u) (upwind), horizontal viscosity,
    Coriolis -f e_z x u, baroclinic pressure gradient -r/rho0, bottom
    drag (Coriolis with the lumped mass, the pressure gradient integrated exactly:
    pressure_source).  dz: layer thickness of the transport geometry.  ext = (u_ext, v_ext,
    qx_ext, qy_ext): exterior velocity (None: zero-gradient) and transport at open
    boundaries (None: the own transport, as in the prediction with the uncorrected
    transport q)."""
    ux = vx = qe = None
    if ext is not None:
        ux, vx = ext[0], ext[1]
        qe = None if ext[2] is None else (ext[2], ext[3])
    Fx = tr.horizontal_residual(om, qx, qy, u, T_ext=ux, face_corr=face_corr, q_ext=qe)
    Fy = tr.horizontal_residual(om, qx, qy, v, T_ext=vx, face_corr=face_corr, q_ext=qe)
    Fx += horizontal_viscosity(om, dz, u, par.nu_h, par.penalty_h)
    Fy += horizontal_viscosity(om, dz, v, par.nu_h, par.penalty_h)
    Fx += lumped_source(om, dz, par.f * v) - pressure_source(om, dz, rx) / par.rho0
    Fy += lumped_source(om, dz, -par.f * u) - pressure_source(om, dz, ry) / par.rho0
    Dx, Dy = bottom_drag(om, par, u, v)
    return Fx + Dx, Fy + Dy


# ---------------------------------------------------------------------------
# 2D external mode (Eqs. 2, 10): P1 DG, lumped mass J_h/6, upwind linear-wave flux
# ---------------------------------------------------------------------------
def tide(par: Params, t: float) -> float:
    return par.tide_amp * math.cos(2.0 * math.pi * t / par.tide_period)


def mode2d_residual(om: OMesh, par: Params, eta, U, V, time: float, Q_ext=None):
    """(R_eta, R_U, R_V) (3, n_tri) and the numerical eta flux at every edge point
    (n_tri, 3, 2) for the state (eta, Q = (U, V)):
      R_eta,a = int Q . grad phi_a - oint phi_a F_eta
      R_Q,a   = int g eta (H grad phi_a + phi_a grad H) - oint phi_a g H^- eta^ n
    with H = h + eta, c = sqrt(g (h^- + h^+)/2) (rest depth) at each edge point,
      F_eta = {Q}.n + c/2 (eta^- - eta^+),   eta^ = {eta} + (q^- - q^+)/(2c)
    (upwind flux of the linear wave system).  Walls: eta^+ = eta^-, q^+ = -q^-.
    Open boundary: the exterior state comes from data alone, eta^+ = A cos(2 pi t /
    T_M2) and Q^+ = 0 (or the prescribed exterior transport Q_ext = (Qx, Qy) at
    this time, (3, n_tri)): with the upwind flux this is a characteristic
    (radiating) condition whose boundary energy flux g eta^ F_eta = (g/4c)
    (q^- + c eta^-)^2 >= 0 for zero data, so the boundary only removes energy.
    Q^+ = Q^- instead feeds the interior's incoming characteristic back and leaves
    a weakly growing boundary mode."""
    nt = om.n_tri
    g = par.g
    h = om.h.T                                             # (3, n_tri)
    H = h + eta
    gr = om.grad                                           # (n_tri, 3, 2)
    Re = np.zeros((3, nt)); RU = np.zeros((3, nt)); RV = np.zeros((3, nt))
    gH = np.stack([sum(H[b] * gr[:, b, d] for b in range(3)) for d in range(2)], -1)   # (n_tri, 2)
    for (xi, et, wg) in TRI_RULE:
        ph = phi(xi, et)
        w = 0.5 * wg * om.Jh
        Qx = sum(ph[b] * U[b] for b in range(3)); Qy = sum(ph[b] * V[b] for b in range(3))
        e_ = sum(ph[b] * eta[b] for b in range(3)); H_ = sum(ph[b] * H[b] for b in range(3))
        for a in range(3):
            Re[a] += w * (Qx * gr[:, a, 0] + Qy * gr[:, a, 1])
            RU[a] += w * g * e_ * (H_ * gr[:, a, 0] + ph[a] * gH[:, 0])
            RV[a] += w * g * e_ * (H_ * gr[:, a, 1] + ph[a] * gH[:, 1])
    Fe = np.zeros((nt, 3, 2))
    A_tide = tide(par, time)
    tt = np.arange(nt)
    for e in range(3):
        nb = om.nbr[:, e]
        ok = nb >= 0
        nbs = np.where(ok, nb, 0)
        n = om.enrm[:, e]
        L = om.elen[:, e]
        own = (e, (e + 1) % 3)
        loc = om.nloc[:, e]
        is_open = om.bnd[:, e] == 2
        for gi, (lam, ws) in enumerate(zip(EDGE_LAM, EDGE_W)):
            wv = (1.0 - lam, lam)
            eo = wv[0] * eta[own[0]] + wv[1] * eta[own[1]]
            Ho = wv[0] * H[own[0]] + wv[1] * H[own[1]]
            qo = (wv[0] * (U[own[0]] * n[:, 0] + V[own[0]] * n[:, 1])
                  + wv[1] * (U[own[1]] * n[:, 0] + V[own[1]] * n[:, 1]))
            l0, l1 = np.where(ok, loc[:, 0], 0), np.where(ok, loc[:, 1], 0)
            en = wv[0] * eta[l0, nbs] + wv[1] * eta[l1, nbs]
            Hn = wv[0] * H[l0, nbs] + wv[1] * H[l1, nbs]
            qn = (wv[0] * (U[l0, nbs] * n[:, 0] + V[l0, nbs] * n[:, 1])
                  + wv[1] * (U[l1, nbs] * n[:, 0] + V[l1, nbs] * n[:, 1]))
            # exterior states
            q_open = np.zeros_like(qo)
            if Q_ext is not None:
                q_open = (wv[0] * (Q_ext[0][own[0]] * n[:, 0] + Q_ext[1][own[0]] * n[:, 1])
                          + wv[1] * (Q_ext[0][own[1]] * n[:, 0] + Q_ext[1][own[1]] * n[:, 1]))
            e_ext = np.where(ok, en, np.where(is_open, A_tide, eo))
            q_ext = np.where(ok, qn, np.where(is_open, q_open, -qo))
            # wave speed of the rest depth (the linear-wave Riemann problem)
            ho = wv[0] * h[own[0]] + wv[1] * h[own[1]]
            hn = wv[0] * h[l0, nbs] + wv[1] * h[l1, nbs]
            h_ext = np.where(ok, hn, ho)
            c = np.sqrt(g * 0.5 * (ho + h_ext))
            F_eta = 0.5 * (qo + q_ext) + 0.5 * c * (eo - e_ext)
            e_hat = 0.5 * (eo + e_ext) + (qo - q_ext) / (2.0 * c)
            Fe[:, e, gi] = F_eta
            w = 0.5 * L * ws
            for j in range(2):
                a = own[j]
                Re[a] -= w * wv[j] * F_eta
                RU[a] -= w * wv[j] * g * Ho * e_hat * n[:, 0]
                RV[a] -= w * wv[j] * g * Ho * e_hat * n[:, 1]
    return Re, RU, RV, Fe


SSP_A = (0.0, 0.75, 1.0 / 3.0)
SSP_B = (1.0, 0.25, 2.0 / 3.0)
SSP_BUTCHER_B = (1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0)


def mode2d_run(om: OMesh, par: Params, eta0, U0, V0, S3x, S3y, t0: float, T_total: float, n: int,
               Q_ab=None, forcing: Forcing | None = None):
    """n SSP-RK3 subcycles of length T_total/n of the 2D mode with the frozen 3D
    source S3 (column sums of F_3D^h).  Returns the end state, the time-averaged
    transport Qbar = (1/n) sum_m sum_s b_s Q^(m,s) (b = 1/6, 1/6, 2/3: the weights
    with which the stage inputs enter the update, so that eta_end - eta0 =
    -T_total (6/J_h) div(Qbar, Gbar)) and the matching average eta face flux Gbar.
    With forcing, Q_ab = (Q_ext at t_a, Q_ext at t_b) and the open boundary takes
    Q_ext(t) = Q_a + theta(t)(Q_b - Q_a) at each stage time."""
    w = np.tile(om.Jh / 6.0, (3, 1))
    dts = T_total / n
    eta, U, V = eta0.copy(), U0.copy(), V0.copy()
    Qbx = np.zeros_like(U); Qby = np.zeros_like(V); Gb = np.zeros((om.n_tri, 3, 2))
    time = t0
    stage_t = (0.0, 1.0, 0.5)
    for m in range(n):
        e_n, U_n, V_n = eta, U, V
        e_s, U_s, V_s = eta, U, V
        for s in range(3):
            ts = time + stage_t[s] * dts
            Qx = None
            if forcing is not None:
                th = forcing.theta(ts)
                Qx = (Q_ab[0][0] + th * (Q_ab[1][0] - Q_ab[0][0]), Q_ab[0][1] + th * (Q_ab[1][1] - Q_ab[0][1]))
            Re, RU, RV, Fe = mode2d_residual(om, par, e_s, U_s, V_s, ts, Q_ext=Qx)
            bw = SSP_BUTCHER_B[s] / n
            Qbx += bw * U_s; Qby += bw * V_s; Gb += bw * Fe
            e_new = SSP_A[s] * e_n + SSP_B[s] * (e_s + dts * Re / w)
            U_new = SSP_A[s] * U_n + SSP_B[s] * (U_s + dts * (RU + S3x) / w)
            V_new = SSP_A[s] * V_n + SSP_B[s] * (V_s + dts * (RV + S3y) / w)
            e_s, U_s, V_s = e_new, U_new, V_new
        eta, U, V = e_s, U_s, V_s
        time += dts
    return eta, U, V, Qbx, Qby, Gb


# ---------------------------------------------------------------------------
# corrected transport (Sec. 2.2: sum_vertical qbar = Qbar) and face correction
# ---------------------------------------------------------------------------
def column_sum_q(om: OMesh, qx, qy):
    return tr.column_sum(om, qx), tr.column_sum(om, qy)


def corrected_transport(om: OMesh, dz, qx, qy, Qbx, Qby):
    """qbar = q + (dz_k / H)(Qbar - sum_column q)/2 at both nodes of every vertex-layer,
    so that the column sum of int qbar dzeta equals Qbar exactly."""
    Sx, Sy = column_sum_q(om, qx, qy)
    H = np.zeros((3, om.n_tri))
    for a in range(3):
        np.add.at(H[a], om.t_of, dz[a])
    t = om.t_of
    frac = dz / H[:, t]
    Dx = (Qbx - Sx)[:, t]; Dy = (Qby - Sy)[:, t]
    return qx + 0.5 * (frac * Dx)[None], qy + 0.5 * (frac * Dy)[None]


def face_correction(om: OMesh, dz, Qbx, Qby, Gb, Q_ext):
    """Per prism and lateral-face quadrature point, the additive correction of the
    normal transport c_k (Gbar - {Qbar}.n)/2 (units of q.n) that makes the column sum
    of the 3D lateral fluxes equal the 2D averaged face flux Gbar.  c_k = layer
    fraction of the face: (dz_k^- + dz_k^+) / sum over paired layers (own only at an
    open boundary).  {Qbar} on an open boundary is the exterior transport Q_ext
    (3, n_tri) alone, matching the 3D open-face transport q_ext, so that the open
    face carries q_ext + c_k (Gbar - Q_ext.n)/2 (zero data: the 2D face flux spread
    over the layers by thickness).  Walls: 0.
    Returns (P, 3, 2) [p][edge][edge point]."""
    P = om.P
    t, k = om.t_of, om.k_of
    corr = np.zeros((P, 3, 2))
    for e in range(3):
        pn, ok = om.nbr_prism(e)
        pn_safe = np.where(ok, pn, 0)
        tn = np.where(om.nbr[t, e] >= 0, om.nbr[t, e], 0)
        n = om.enrm[t, e]
        own = (e, (e + 1) % 3)
        loc = om.nloc[t, e]
        is_open = om.bnd[t, e] == 2
        has_nb = om.nbr[t, e] >= 0
        for gi, lam in enumerate(EDGE_LAM):
            wv = (1.0 - lam, lam)
            dz_o = wv[0] * dz[own[0]] + wv[1] * dz[own[1]]
            l0, l1 = np.where(ok, loc[:, 0], 0), np.where(ok, loc[:, 1], 0)
            dz_n = wv[0] * dz[l0, pn_safe] + wv[1] * dz[l1, pn_safe]
            # paired-layer sums per prism's column pair
            pair = np.where(ok, dz_o + dz_n, np.where(is_open, dz_o, 0.0))
            tot = np.zeros(P)
            key_t = t
            sums = np.zeros(om.n_tri)
            np.add.at(sums, key_t, pair)
            tot = sums[t]
            Qo = (wv[0] * (Qbx[own[0], t] * n[:, 0] + Qby[own[0], t] * n[:, 1])
                  + wv[1] * (Qbx[own[1], t] * n[:, 0] + Qby[own[1], t] * n[:, 1]))
            ln0, ln1 = np.where(has_nb, loc[:, 0], 0), np.where(has_nb, loc[:, 1], 0)
            Qn = (wv[0] * (Qbx[ln0, tn] * n[:, 0] + Qby[ln0, tn] * n[:, 1])
                  + wv[1] * (Qbx[ln1, tn] * n[:, 0] + Qby[ln1, tn] * n[:, 1]))
            Q_open = (wv[0] * (Q_ext[0][own[0], t] * n[:, 0] + Q_ext[1][own[0], t] * n[:, 1])
                      + wv[1] * (Q_ext[0][own[1], t] * n[:, 0] + Q_ext[1][own[1], t] * n[:, 1]))
            Qavg = np.where(has_nb, 0.5 * (Qo + Qn), Q_open)
            delta = Gb[t, e, gi] - Qavg
            ck = np.where(tot > 0, pair / np.where(tot > 0, tot, 1.0), 0.0)
            corr[:, e, gi] = np.where(ok | is_open, 0.5 * ck * delta, 0.0)
    return corr


# ---------------------------------------------------------------------------
# the split-IMEX internal step (Sec. 2, Eqs. 11-14)
# ---------------------------------------------------------------------------
def _col_sum3(om, F):
    return tr.column_sum(om, F)


def _explicit_vertical(om, W, dz, f, kappa, penalty):
    """R_v(f) = A f for the vertical operator (explicit evaluation)."""
    out = np.zeros_like(f)
    for N, tris in tr.columns_by_depth(om).items():
        ncol = len(tris)
        Wc = tr.gather_columns(om, W, tris, N).reshape(ncol * 3, 2 * N)
        p = om.col_off[tris][:, None] + np.arange(N)[None, :]
        dzc = np.transpose(dz[:, p], (1, 0, 2)).reshape(ncol * 3, N)
        omega = np.repeat(om.Jh[tris] / 6.0, 3)
        A = tr.vertical_matrix(Wc, dzc, kappa, omega, penalty)
        x = tr.gather_columns(om, f, tris, N).reshape(ncol * 3, 2 * N)
        y = np.einsum("nij,nj->ni", A, x)
        tr.scatter_columns(om, y.reshape(ncol, 3, 2 * N), tris, N, out)
    return out


def split_stage(om: OMesh, par: Params, st0: State, ev: State, t0: float, dt: float, n_sub: int,
                implicit: bool, diag: dict | None = None):
    """One stage of the split-IMEX step from st0 (the state at t0) over dt, with the
    horizontal terms evaluated at ev: hpg -> F_3D^h prediction with q -> 2D
    subcycles -> F2D -> corrected transport qbar and vertical flux W -> momentum ->
    tracers (the component order of Sec. 2, Fig. 1a; turbulence is not built)."""
    dz_ev = om.thickness(ev.eta)
    dz0 = om.thickness(st0.eta)
    # open-boundary forcing: the 2D run of this stage spans [t0, t0 + dt] and sees
    # Q_ext(t) linear in t; the 3D terms take the exterior state at the middle of
    # that run, whose column transport is the run's average of Q_ext
    # (unforced: zero exterior transport, zero-gradient exterior velocity)
    Fo = st0.forcing if par.forcing else None
    Q_ab = None
    T_x, S_x = st0.T_ext, st0.S_ext
    qe = (np.zeros_like(st0.u), np.zeros_like(st0.v))
    Q_mid = (np.zeros((3, om.n_tri)), np.zeros((3, om.n_tri)))
    ext3 = (None, None, qe[0], qe[1])
    if Fo is not None:
        ux, vx, T_x, S_x = Fo.at(t0 + 0.5 * dt)
        qe = exterior_transport(om, ux, vx)
        ext3 = (ux, vx, qe[0], qe[1])
        Q_mid = exterior_column_transport(om, ux, vx)
        Q_ab = (exterior_column_transport(om, Fo.u_a, Fo.v_a), exterior_column_transport(om, Fo.u_b, Fo.v_b))
    # 1. density and horizontal pressure gradient
    rx, ry = hpg(om, par, ev.T, ev.S, ev.eta)
    # 2. prediction of F_3D^h with the uncorrected transport q of the evaluation
    # state on every face (open faces: the own q, the estimate of the 2D flux there)
    qx, qy = tr.transport(dz_ev, ev.u, ev.v)
    Fpx, Fpy = momentum_horizontal(om, par, ev.u, ev.v, qx, qy, rx, ry, dz_ev, ext=(ext3[0], ext3[1], None, None))
    S3x, S3y = _col_sum3(om, Fpx), _col_sum3(om, Fpy)
    # 3. external mode from the state at t0
    eta1, U1, V1, Qbx, Qby, Gb = mode2d_run(om, par, st0.eta, st0.U, st0.V, S3x, S3y, t0, dt, n_sub,
                                            Q_ab=Q_ab, forcing=Fo)
    # 4. 2D momentum forcing F2D = (Q1 - (Q0 + dt S3/w))/dt
    w = np.tile(om.Jh / 6.0, (3, 1))
    F2x = (U1 - (st0.U + dt * S3x / w)) / dt
    F2y = (V1 - (st0.V + dt * S3y / w)) / dt
    # 5. corrected transport and the vertical flux (continuity over [t0, t0 + dt])
    qbx, qby = corrected_transport(om, dz_ev, qx, qy, Qbx, Qby)
    corr = face_correction(om, dz_ev, Qbx, Qby, Gb, Q_ext=Q_mid)
    dz1 = om.thickness(eta1)
    R1 = tr.horizontal_residual(om, qbx, qby, np.ones_like(qbx), face_corr=corr, q_ext=qe)
    F = R1 - ((om.Jh[om.t_of] / 12.0)[None] * om.thickness_change(st0.eta, eta1) / dt)[None]
    W = tr.solve_continuity(om, F)
    # 6. momentum: M1 u1 = M0 u0 + dt (F_3D^h(u_ev, qbar, r) + M1 F2D/H1 + [A u1 | A u_ev])
    Fx, Fy = momentum_horizontal(om, par, ev.u, ev.v, qbx, qby, rx, ry, dz_ev, face_corr=corr, ext=ext3)
    H1 = np.zeros((3, om.n_tri))
    for a in range(3):
        np.add.at(H1[a], om.t_of, dz1[a])
    H1n = H1[:, om.t_of]
    cpl_x = lumped_source(om, dz1, np.broadcast_to((F2x[:, om.t_of] / H1n)[None], st0.u.shape))
    cpl_y = lumped_source(om, dz1, np.broadcast_to((F2y[:, om.t_of] / H1n)[None], st0.u.shape))
    rhs_u = tr.apply_mass(om, dz0, st0.u) + dt * (Fx + cpl_x)
    rhs_v = tr.apply_mass(om, dz0, st0.v) + dt * (Fy + cpl_y)
    # tracers: M1 T1 = M0 T0 + dt (R_h(T_ev, qbar) + [A T1 | A T_ev])
    RT = tr.horizontal_residual(om, qbx, qby, ev.T, T_ext=T_x, face_corr=corr, q_ext=qe)
    RS = tr.horizontal_residual(om, qbx, qby, ev.S, T_ext=S_x, face_corr=corr, q_ext=qe)
    RT += horizontal_viscosity(om, dz_ev, ev.T, par.kappa_h, par.penalty_h)
    RS += horizontal_viscosity(om, dz_ev, ev.S, par.kappa_h, par.penalty_h)
    rhs_T = tr.apply_mass(om, dz0, st0.T) + dt * RT
    rhs_S = tr.apply_mass(om, dz0, st0.S) + dt * RS
    if implicit:
        u1 = tr.stage_solve(om, W, dz1, rhs_u, dt, par.nu_v)
        v1 = tr.stage_solve(om, W, dz1, rhs_v, dt, par.nu_v)
        T1 = tr.stage_solve(om, W, dz1, rhs_T, dt, par.kappa_v)
        S1 = tr.stage_solve(om, W, dz1, rhs_S, dt, par.kappa_v)
    else:
        def expl(rhs, f, kap):
            y = rhs + dt * _explicit_vertical(om, W, dz_ev, f, kap, par.penalty_v)
            return tr.stage_solve(om, np.zeros_like(W), dz1, y, 0.0, 0.0)   # M1^-1 y
        u1 = expl(rhs_u, ev.u, par.nu_v)
        v1 = expl(rhs_v, ev.v, par.nu_v)
        T1 = expl(rhs_T, ev.T, par.kappa_v)
        S1 = expl(rhs_S, ev.S, par.kappa_v)
    if diag is not None:
        diag.update(W=W, r=(rx, ry), S3=(S3x, S3y), F2D=(F2x, F2y), Qbar=(Qbx, Qby), Gbar=Gb,
                    qbar=(qbx, qby), corr=corr, F3h=(Fx, Fy), R1=R1)
    return State(u=u1, v=v1, T=T1, S=S1, eta=eta1, U=U1, V=V1, T_ext=st0.T_ext, S_ext=st0.S_ext,
                 forcing=st0.forcing)


def split_step(om: OMesh, par: Params, st: State, t: float, dt: float, diag1=None, diag2=None) -> State:
    """Two-stage split-IMEX step (a reading of Sec. 2 and Fig. 1): stage 1 over dt/2, vertically implicit,
    n_sub/2 external subcycles; stage 2 over dt from the same start state with the
    horizontal terms at the stage-1 state, vertically explicit, n_sub subcycles.

    Pinned by what the structure fixes (lake at rest, constant tracers, the
    column sum of the corrected transport, the vanishing surface flux, tracer mass
    in a closed basin); agreement with the coefficients of the paper's own
    split-IMEX scheme is parity unpinned (they are in its unavailable supporting
    information)."""
    half = split_stage(om, par, st, st, t, 0.5 * dt, par.n_sub // 2, True, diag1)
    return split_stage(om, par, st, half, t, dt, par.n_sub, False, diag2)
