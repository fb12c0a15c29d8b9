"""Initial nodal fields and workload definitions.

3D nodal fields use the layout of the C-ABI: a flat float64 array of length 6P
indexed ``(c * 3 + a) * P + p`` with ``c`` = 0 for the top node and 1 for the bottom
node of a prism, ``a`` the triangle vertex (0..2) and ``p = col_off[t] + k`` the prism
(layer ``k`` = 0 at the surface), ``col_off`` the exclusive prefix sum of the
per-triangle layer counts.  Reshaped to ``(2, 3, P)`` it reads ``[c][a][p]``.

2D nodal fields (elevation, transport) are ``(3, n_tri)`` arrays ``[a][t]`` flattened.

Initial conditions are evaluated at the nodes' rest positions (elevation zero): the
reference interface depths are ``-i h / N`` for sigma layers and the level table
(with the column's own depth at the bottom) for z-levels.  This is input
preparation, not part of the discretisation.
"""
from __future__ import annotations

import numpy as np

from .meshes import Mesh, c1_mesh, c2_mesh, c4_mesh, c5_mesh, cached_mesh


def col_offsets(m: Mesh) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(m.n_layers)]).astype(np.int64)


def prism_tri_layer(m: Mesh) -> tuple[np.ndarray, np.ndarray]:
    """(triangle, layer) of every prism in column-contiguous order."""
    t = np.repeat(np.arange(m.n_tri), m.n_layers)
    off = col_offsets(m)
    k = np.arange(off[-1]) - off[t]
    return t, k


def node_positions_sigma(m: Mesh) -> tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """Rest positions x, y, z and depth fraction s = -z/h of every node, each (2, 3, P)."""
    t, k = prism_tri_layer(m)
    P = t.shape[0]
    x = np.empty((2, 3, P)); y = np.empty((2, 3, P)); z = np.empty((2, 3, P)); s = np.empty((2, 3, P))
    N = m.n_layers[t].astype(np.float64)
    for a in range(3):
        v = m.tri[t, a]
        h = m.h_tri[t, a]
        for c in range(2):
            i = (k + c).astype(np.float64)
            x[c, a] = m.xy[v, 0]
            y[c, a] = m.xy[v, 1]
            if m.levels is None:
                z[c, a] = -i / N * h
            else:
                ii = (k + c).astype(np.int64)
                zl = m.levels[np.minimum(ii, len(m.levels) - 1)]
                z[c, a] = np.where(ii >= m.n_layers[t], -h, zl)
            s[c, a] = -z[c, a] / h
    return x, y, z, s


def flat(f: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(f.reshape(-1))


# ----------------------------------------------------------------------------
# square basin tracer workload
# ----------------------------------------------------------------------------
def c1_velocity(m: Mesh, L: float = 10e3, umax: float = 0.5) -> tuple[np.ndarray, np.ndarray]:
    """Depth-uniform velocity u = Q/h with the closed-basin transport Q = curl psi,
    psi = Psi0 sin^2(pi x/L) sin^2(pi y/L), scaled so max |u| = umax at the vertices."""
    t, _ = prism_tri_layer(m)
    P = t.shape[0]
    u = np.empty((2, 3, P)); v = np.empty((2, 3, P))
    xs, ys = m.xy[:, 0], m.xy[:, 1]
    k = np.pi / L
    dpsi_dx = k * np.sin(2 * k * xs) * np.sin(k * ys) ** 2
    dpsi_dy = k * np.sin(k * xs) ** 2 * np.sin(2 * k * ys)
    for a in range(3):
        vid = m.tri[t, a]
        h = m.h_tri[t, a]
        for c in range(2):
            u[c, a] = -dpsi_dy[vid] / h
            v[c, a] = dpsi_dx[vid] / h
    scale = umax / np.sqrt(u ** 2 + v ** 2).max()
    return flat(u * scale), flat(v * scale)


def c1_tracer(m: Mesh, L: float = 10e3, sigma_h: float = 1e3, sigma_v: float = 0.2) -> np.ndarray:
    """Gaussian blob of unit amplitude, horizontal width sigma_h centred at (0.3L, 0.3L),
    vertical width sigma_v (fraction of the local depth) centred at mid-depth."""
    x, y, _, s = node_positions_sigma(m)
    r2 = (x - 0.3 * L) ** 2 + (y - 0.3 * L) ** 2
    return flat(np.exp(-r2 / (2 * sigma_h ** 2)) * np.exp(-(s - 0.5) ** 2 / (2 * sigma_v ** 2)))


def basin_velocity(m: Mesh, Lx: float = 200e3, Ly: float = 100e3, umax: float = 0.5,
                   shear: bool = True) -> tuple[np.ndarray, np.ndarray]:
    """Velocity with zero normal component on the basin boundary, from the
    streamfunction psi = sin^2(pi x/Lx) sin^2(pi y/Ly); optional depth shear."""
    x, y, _, s = node_positions_sigma(m)
    kx, ky = np.pi / Lx, np.pi / Ly
    u = -np.sin(kx * x) ** 2 * ky * np.sin(2 * ky * y)
    v = kx * np.sin(2 * kx * x) * np.sin(ky * y) ** 2
    scale = umax / np.sqrt(u ** 2 + v ** 2).max()
    if shear:
        u = u * (1.5 - s)
        v = v * (1.5 - s)
    return flat(u * scale), flat(v * scale)


# ----------------------------------------------------------------------------
# baroclinic basin workload
# ----------------------------------------------------------------------------
def c2_initial_state(m: Mesh, h_max: float = 200.0) -> dict:
    """Rest state with linear stratification T = 28 + 13 z/h_max, S = 34 - 2 z/h_max."""
    _, _, z, _ = node_positions_sigma(m)
    P = z.shape[2]
    zero3 = np.zeros(6 * P)
    return dict(u=zero3.copy(), v=zero3.copy(),
                T=flat(28.0 + 13.0 * z / h_max), S=flat(34.0 - 2.0 * z / h_max),
                eta=np.zeros(3 * m.n_tri), U=np.zeros(3 * m.n_tri), V=np.zeros(3 * m.n_tri))


def c4_initial_state(m: Mesh) -> dict:
    return c2_initial_state(m, h_max=600.0)


def dt_2d(m: Mesh, g: float = 9.81, cfl: float = 0.25) -> float:
    """0.25 min_t r_in / (sqrt(g h_t) + 1): the external-mode step of the basin workloads."""
    p = m.xy[m.tri]
    e = np.stack([np.hypot(*(p[:, (i + 1) % 3] - p[:, i]).T) for i in range(3)], axis=1)
    u = p[:, 1] - p[:, 0]; w = p[:, 2] - p[:, 0]
    area = 0.5 * np.abs(u[:, 0] * w[:, 1] - u[:, 1] * w[:, 0])
    r_in = 2 * area / e.sum(axis=1)
    c = np.sqrt(g * m.h_tri.max(axis=1)) + 1.0
    return float(cfl * (r_in / c).min())


# name -> description used by tests and the bench
WORKLOADS = {
    "basin_tracer": dict(mesh=lambda: c2_mesh(200_000, 20, 0), dt=10.0, steps=100,
                         kappa_v=1e-3, scheme="tracer"),
    "square_tracer": dict(mesh=lambda: c1_mesh(32, 10e3, 10), dt=5.0, steps=100,
                          kappa_v=1e-3, scheme="tracer"),
    "basin_baroclinic": dict(mesh=lambda: c2_mesh(200_000, 20, 0), steps=1000, n_sub=20,
                             kappa_v=1e-3, nu_v=1e-3, kappa_h=1.0, nu_h=1.0, scheme="split"),
    # the same basin at a quarter of the triangles (~1M prisms): profiler captures
    "basin_baroclinic_small": dict(mesh=lambda: c2_mesh(50_000, 20, 0), steps=1000, n_sub=20,
                                   kappa_v=1e-3, nu_v=1e-3, kappa_h=1.0, nu_h=1.0, scheme="split"),
    "zlevel_baroclinic": dict(mesh=lambda: c4_mesh(500_000, 0), steps=3, n_sub=20,
                              kappa_v=1e-3, nu_v=1e-3, kappa_h=1.0, nu_h=1.0, scheme="split"),
    # reef-scale stress run: ~2.4M triangles around 400 islands, 1-30 z-levels (~41M prisms)
    "reef_baroclinic": dict(mesh=lambda: cached_mesh("reef_c5_v1", c5_mesh), steps=2000, n_sub=20,
                            kappa_v=1e-3, nu_v=1e-3, kappa_h=1.0, nu_h=1.0, scheme="split"),
}


def c5_initial_state(m: Mesh) -> dict:
    return c2_initial_state(m, h_max=1000.0)
