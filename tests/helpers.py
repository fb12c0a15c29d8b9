"""Shared test helpers: seeded cases, sub-meshes for sampled checks, norms."""
from __future__ import annotations

import numpy as np

import workloads as wl
from workloads.meshes import Mesh


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def sheared_velocity(m: Mesh, L: float, umax: float = 0.5):
    """Closed-basin velocity with depth shear, so the vertical flux is active."""
    u, v = wl.c1_velocity(m, L, umax)
    _, _, _, s = wl.fields.node_positions_sigma(m)
    s = s.reshape(-1)
    return u * (1.5 - s), v * (0.5 + s)


def random_uneven_mesh(n: int = 10, L: float = 4000.0, n_max: int = 12, seed: int = 0,
                       open_x: bool = False) -> Mesh:
    """Square mesh with a random number of layers per column (1..n_max), jittered depths."""
    rng = np.random.default_rng(seed)
    bathy = lambda x, y: 20.0 + 10.0 * np.sin(2 * np.pi * x / L) * np.cos(np.pi * y / L)
    op = (lambda x, y: x > L - 1e-6) if open_x else None
    m = wl.meshes.square_mesh(n, L, 1, bathy, op)
    m.n_layers = rng.integers(1, n_max + 1, size=m.n_tri).astype(np.int32)
    return m


def edge_adjacency(m: Mesh) -> np.ndarray:
    """(n_tri, 3) neighbour across each edge or -1 (test-side, from the triangle list)."""
    tri = m.tri.astype(np.int64)
    a = tri.ravel()
    b = np.roll(tri, -1, axis=1).ravel()
    key = np.minimum(a, b) * (m.n_vert + 1) + np.maximum(a, b)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    nbr = -np.ones(3 * m.n_tri, dtype=np.int64)
    same = ks[1:] == ks[:-1]
    i = np.nonzero(same)[0]
    e1, e2 = order[i], order[i + 1]
    nbr[e1] = e2 // 3
    nbr[e2] = e1 // 3
    return nbr.reshape(m.n_tri, 3)


def ring_submesh(m: Mesh, seeds: np.ndarray, rings: int):
    """Sub-mesh of the seed triangles and ``rings`` rings of edge neighbours around
    them.  Cut edges become walls.  Returns (sub-mesh, triangle map sub -> full,
    positions of the seeds in the sub-mesh)."""
    nbr = edge_adjacency(m)
    sel = np.zeros(m.n_tri, bool)
    sel[seeds] = True
    front = np.asarray(seeds)
    for _ in range(rings):
        nb = nbr[front].ravel()
        nb = nb[nb >= 0]
        nb = nb[~sel[nb]]
        sel[nb] = True
        front = np.unique(nb)
    tmap = np.nonzero(sel)[0]
    inv = -np.ones(m.n_tri, np.int64)
    inv[tmap] = np.arange(len(tmap))
    bnd = m.bnd[tmap].copy()
    cut = (nbr[tmap] >= 0) & (~sel[np.where(nbr[tmap] >= 0, nbr[tmap], 0)])
    bnd[cut] = 1
    sub = Mesh(xy=m.xy, tri=np.ascontiguousarray(m.tri[tmap]), h_tri=np.ascontiguousarray(m.h_tri[tmap]),
               n_layers=np.ascontiguousarray(m.n_layers[tmap]), bnd=np.ascontiguousarray(bnd),
               levels=m.levels, name=m.name + "-sub")
    return sub, tmap, inv[seeds]


def col_offsets(n_layers: np.ndarray) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(n_layers)]).astype(np.int64)


def restrict3(f: np.ndarray, m: Mesh, tmap: np.ndarray) -> np.ndarray:
    """3D nodal field of the full mesh -> (2, 3, P_sub) of the sub-mesh triangles."""
    off = col_offsets(m.n_layers)
    P = off[-1]
    f = np.asarray(f).reshape(2, 3, P)
    idx = np.concatenate([np.arange(off[t], off[t + 1]) for t in tmap])
    return f[:, :, idx]


def restrict2(f: np.ndarray, m: Mesh, tmap: np.ndarray) -> np.ndarray:
    return np.asarray(f).reshape(3, m.n_tri)[:, tmap]


def prisms_of(n_layers: np.ndarray, tris: np.ndarray) -> np.ndarray:
    off = col_offsets(n_layers)
    return np.concatenate([np.arange(off[t], off[t + 1]) for t in tris])


def assert_close(got, ref, tol: float, what=None) -> None:
    """Parity bar: relative L2 over the field AND every node within tol of the
    field's largest magnitude (a single wrong node -- a wall face, a ragged last
    tile, the last layer of a short column -- fails the second even when the norm
    hides it)."""
    g = np.asarray(got, np.float64).ravel()
    r = np.asarray(ref, np.float64).ravel()
    assert g.shape == r.shape, (what, g.shape, r.shape)
    e2 = rel_l2(g, r)
    d = np.abs(g - r)
    scale = float(np.abs(r).max()) or 1.0
    emax = float(d.max()) / scale if d.size else 0.0
    assert e2 < tol and emax <= tol, dict(what=what, rel_l2=e2, max_rel=emax, at=int(np.argmax(d)) if d.size else -1,
                                          tol=tol)


def split_case_mesh(name):
    """Meshes of the split-scheme parity cases: a graded basin with an open tidal
    boundary, a square basin with an open side, a z-level basin with uneven columns."""
    if name == "basin":
        return wl.c2_mesh(2500, 5, 0)
    if name == "square":
        return wl.meshes.square_mesh(10, 4000.0, 4, lambda x, y: 15.0 + 20.0 * x / 4000.0,
                                     lambda x, y: x > 4000.0 - 1e-6)
    if name == "zlevel":
        return wl.c4_mesh(3000, 0, n_max=12, h_max=60.0)
    raise KeyError(name)


def split_initial(m, seed=0):
    """Seeded smooth state of the split-scheme parity cases (velocity with depth
    shear, T and S varying in x, y and z, sloped elevation and transport)."""
    rng = np.random.default_rng(seed)
    x, y, z, s = wl.fields.node_positions_sigma(m)
    Lx = max(m.xy[:, 0].max(), 1.0)
    Ly = max(m.xy[:, 1].max(), 1.0)
    u = 0.2 * np.sin(np.pi * x / Lx) * np.cos(np.pi * y / Ly) * (1.2 - s)
    v = 0.1 * np.cos(np.pi * x / Lx) * (0.4 + s)
    T = 15.0 + 10.0 * np.exp(z / 40.0) + 0.5 * np.sin(3 * x / Lx)
    S = 34.0 - 2.0 * z / 60.0 + 0.3 * np.cos(2 * y / Ly)
    xt, yt = m.xy[m.tri][:, :, 0].T, m.xy[m.tri][:, :, 1].T
    eta = 0.05 * np.cos(np.pi * xt / Lx) + 0.02 * np.sin(2 * np.pi * yt / Ly)
    U = 1.0 * np.sin(np.pi * xt / Lx)
    V = 0.3 * np.cos(np.pi * yt / Ly) * np.sin(np.pi * xt / Lx)
    return dict(U=u.ravel(), V=v.ravel(), T=T.ravel(), S=S.ravel(), ETA=eta.ravel(), QX=U.ravel(), QY=V.ravel())
