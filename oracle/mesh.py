"""Oracle mesh: connectivity, 2D geometry and the moving vertical coordinate.

The 3D mesh is the 2D triangulation extruded into columns of prisms (Sec. 1,
Sec. 2.1).  Prism ``p = col_off[t] + k`` is layer ``k`` (0 at the surface) of the
column under triangle ``t``.  The oracle builds its own edge adjacency from the
triangle list (it does not use any table of the CUDA library).

Vertical coordinate (a reading: the paper leaves the vertical coordinate to its
supporting information): each triangle vertex ``a`` of
triangle ``t`` has rest interface depths ``zhat_i`` (``-i h/N`` for sigma layers;
the level table, with the column's own depth at the bottom, for z-levels) and the
interfaces move with the triangle's own (discontinuous) elevation as
``z_i = eta + (1 + eta/h) zhat_i``.
"""
from __future__ import annotations

import numpy as np


class OMesh:
    def __init__(self, m):
        self.m = m
        self.n_tri = m.n_tri
        self.N = m.n_layers.astype(np.int64)
        self.col_off = np.concatenate([[0], np.cumsum(self.N)]).astype(np.int64)
        self.P = int(self.col_off[-1])
        self.t_of = np.repeat(np.arange(self.n_tri), self.N)
        self.k_of = np.arange(self.P) - self.col_off[self.t_of]
        X = m.xy[m.tri]                      # (n_tri, 3, 2)
        self.X = X
        d1 = X[:, 1] - X[:, 0]
        d2 = X[:, 2] - X[:, 0]
        # x = X0 + xi d1 + eta d2: Jacobian [[d1x, d2x], [d1y, d2y]]
        self.Jh = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
        if (self.Jh <= 0).any():
            raise ValueError("triangles must be counter-clockwise")
        Jm = np.stack([np.stack([d1[:, 0], d2[:, 0]], -1), np.stack([d1[:, 1], d2[:, 1]], -1)], 1)
        Jinv = np.linalg.inv(Jm)            # (n_tri, 2, 2): d(xi,eta)/d(x,y)
        from .quadrature import GRAD_REF
        # grad_x phi_a = Jinv^T grad_ref phi_a
        self.grad = np.einsum("tji,aj->tai", Jinv, GRAD_REF)  # (n_tri, 3, 2)
        # edges e: vertex e -> vertex e+1; outward unit normal for CCW triangles
        self.elen = np.zeros((self.n_tri, 3))
        self.enrm = np.zeros((self.n_tri, 3, 2))
        for e in range(3):
            dxy = X[:, (e + 1) % 3] - X[:, e]
            L = np.hypot(dxy[:, 0], dxy[:, 1])
            self.elen[:, e] = L
            self.enrm[:, e, 0] = dxy[:, 1] / L
            self.enrm[:, e, 1] = -dxy[:, 0] / L
        # adjacency by shared global vertex pairs
        self.nbr = -np.ones((self.n_tri, 3), dtype=np.int64)
        self.nloc = -np.ones((self.n_tri, 3, 2), dtype=np.int64)  # nbr-local index of own vertices e, e+1
        table: dict[tuple[int, int], list[tuple[int, int]]] = {}
        tri = m.tri
        for t in range(self.n_tri):
            for e in range(3):
                a, b = int(tri[t, e]), int(tri[t, (e + 1) % 3])
                table.setdefault((min(a, b), max(a, b)), []).append((t, e))
        for lst in table.values():
            if len(lst) == 2:
                (t1, e1), (t2, e2) = lst
                for (ta, ea), (tb, _) in (((t1, e1), (t2, e2)), ((t2, e2), (t1, e1))):
                    self.nbr[ta, ea] = tb
                    for j, a in enumerate((ea, (ea + 1) % 3)):
                        gv = tri[ta, a]
                        self.nloc[ta, ea, j] = int(np.nonzero(tri[tb] == gv)[0][0])
            elif len(lst) > 2:
                raise ValueError("non-manifold edge")
        self.bnd = m.bnd.astype(np.int64)
        self.h = m.h_tri                      # (n_tri, 3)
        self.levels = m.levels

    # ------------------------------------------------------------------
    def mass2d(self) -> np.ndarray:
        """Consistent 2D P1 mass matrix int phi_a phi_b J_h of every triangle,
        (n_tri, 3, 3), by the triangle rule (Sec. 2.3 prints its closed form)."""
        from .quadrature import TRI_RULE, phi
        M = np.zeros((self.n_tri, 3, 3))
        for (xi, eta, w) in TRI_RULE:
            ph = phi(xi, eta)
            M += 0.5 * w * self.Jh[:, None, None] * np.outer(ph, ph)[None]
        return M

    def rest_interfaces(self) -> tuple[np.ndarray, np.ndarray]:
        """Rest depths of the top and bottom interface of every prism at every
        vertex, each (3, P)."""
        t, k = self.t_of, self.k_of
        zt = np.empty((3, self.P))
        zb = np.empty((3, self.P))
        for a in range(3):
            h = self.h[t, a]
            N = self.N[t].astype(np.float64)
            if self.levels is None:
                zt[a] = -(k / N) * h
                zb[a] = -((k + 1) / N) * h
            else:
                zt[a] = self.levels[k]
                zb[a] = np.where(k + 1 >= self.N[t], -h, self.levels[np.minimum(k + 1, len(self.levels) - 1)])
        return zt, zb

    def interfaces(self, eta: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """Interface depths z_top, z_bot (3, P) for the 2D elevation eta (3, n_tri)."""
        zt0, zb0 = self.rest_interfaces()
        e = eta[:, self.t_of]
        h = self.h[self.t_of].T
        s = 1.0 + e / h
        return e + s * zt0, e + s * zb0

    def thickness(self, eta: np.ndarray) -> np.ndarray:
        zt, zb = self.interfaces(eta)
        return zt - zb

    def thickness_change(self, eta0: np.ndarray, eta1: np.ndarray) -> np.ndarray:
        """dz(eta1) - dz(eta0) (3, P), written as dz_rest (eta1 - eta0)/h: the
        interfaces stretch linearly with eta, so this is the same quantity without
        the cancellation of subtracting two thicknesses (whose rounding, relative to
        the small change, is eps h / |eta1 - eta0|)."""
        zt0, zb0 = self.rest_interfaces()
        h = self.h[self.t_of].T
        return (zt0 - zb0) * (eta1 - eta0)[:, self.t_of] / h

    def nbr_prism(self, e: int) -> tuple[np.ndarray, np.ndarray]:
        """For edge e of every prism: the lateral neighbour prism (or -1) and a mask."""
        t, k = self.t_of, self.k_of
        tn = self.nbr[t, e]
        ok = (tn >= 0)
        tn_safe = np.where(ok, tn, 0)
        ok &= k < self.N[tn_safe]
        pn = np.where(ok, self.col_off[tn_safe] + k, -1)
        return pn, ok
