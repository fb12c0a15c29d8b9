"""Synthetic triangle meshes, bathymetry and vertical layering.

A mesh is described by plain arrays (the same arrays the C-ABI takes):

* ``xy``        (n_vert, 2) float64  vertex coordinates [m]
* ``tri``       (n_tri, 3)  int32    counter-clockwise vertex indices
* ``h_tri``     (n_tri, 3)  float64  water depth at rest at each triangle vertex [m]
                                     (equal to the bathymetry for sigma layers; the
                                     staircase depth for z-levels)
* ``n_layers``  (n_tri,)    int32    prisms in the column under each triangle
* ``levels``    (n_levels,) float64 or None: reference interface depths (0 > z_1 > ...)
                                     for z-level layering, None for uniform sigma layers
* ``bnd``       (n_tri, 3)  int8     per triangle edge e (vertex e -> vertex e+1):
                                     0 interior, 1 closed wall, 2 open boundary

Triangles are returned in Hilbert-curve order of their centroids (the ordering the
paper uses for cache locality of lateral neighbour accesses, Sec. 2.1).
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Mesh:
    xy: np.ndarray
    tri: np.ndarray
    h_tri: np.ndarray
    n_layers: np.ndarray
    bnd: np.ndarray
    levels: np.ndarray | None = None
    name: str = ""

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])

    @property
    def n_vert(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_prisms(self) -> int:
        return int(self.n_layers.sum())


# ----------------------------------------------------------------------------
# Hilbert ordering
# ----------------------------------------------------------------------------
def _hilbert_d(x: np.ndarray, y: np.ndarray, order: int) -> np.ndarray:
    """Hilbert index of integer points (x, y) in [0, 2^order)^2 (vectorised xy->d)."""
    x = x.astype(np.int64).copy()
    y = y.astype(np.int64).copy()
    d = np.zeros_like(x)
    n = 1 << order
    s = n >> 1
    while s > 0:
        rx = ((x & s) > 0).astype(np.int64)
        ry = ((y & s) > 0).astype(np.int64)
        d += s * s * ((3 * rx) ^ ry)
        # rotate the quadrant
        flip = ry == 0
        swap_x = np.where(flip & (rx == 1), n - 1 - x, x)
        swap_y = np.where(flip & (rx == 1), n - 1 - y, y)
        x = np.where(flip, swap_y, x)
        y = np.where(flip, swap_x, y)
        s >>= 1
    return d


def hilbert_order(xy: np.ndarray, tri: np.ndarray, order: int = 16) -> np.ndarray:
    """Permutation of triangles along a Hilbert curve through their centroids."""
    c = xy[tri].mean(axis=1)
    lo = c.min(axis=0)
    span = max(float((c.max(axis=0) - lo).max()), 1e-30)
    n = (1 << order) - 1
    ix = np.clip(((c[:, 0] - lo[0]) / span * n).astype(np.int64), 0, n)
    iy = np.clip(((c[:, 1] - lo[1]) / span * n).astype(np.int64), 0, n)
    return np.argsort(_hilbert_d(ix, iy, order), kind="stable")


def permute_triangles(m: Mesh, perm: np.ndarray) -> Mesh:
    return dataclasses.replace(m, tri=np.ascontiguousarray(m.tri[perm]),
                               h_tri=np.ascontiguousarray(m.h_tri[perm]),
                               n_layers=np.ascontiguousarray(m.n_layers[perm]),
                               bnd=np.ascontiguousarray(m.bnd[perm]))


# ----------------------------------------------------------------------------
# boundary tagging (topology only)
# ----------------------------------------------------------------------------
def _tag_boundary(xy: np.ndarray, tri: np.ndarray, is_open) -> np.ndarray:
    """0 for edges shared by two triangles, 2 for boundary edges whose midpoint
    satisfies ``is_open``, 1 for the other boundary edges."""
    n_tri = tri.shape[0]
    a = tri
    b = np.roll(tri, -1, axis=1)
    lo = np.minimum(a, b).ravel().astype(np.int64)
    hi = np.maximum(a, b).ravel().astype(np.int64)
    key = lo * (xy.shape[0] + 1) + hi
    _, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
    bnd_edge = cnt[inv] == 1
    mid = 0.5 * (xy[a.ravel()] + xy[b.ravel()])
    tags = np.zeros(3 * n_tri, dtype=np.int8)
    tags[bnd_edge] = 1
    if is_open is not None:
        op = bnd_edge & is_open(mid[:, 0], mid[:, 1])
        tags[op] = 2
    return tags.reshape(n_tri, 3)


# ----------------------------------------------------------------------------
# structured square mesh (32 x 32 squares each split along the same diagonal)
# ----------------------------------------------------------------------------
def square_mesh(n: int, L: float, n_layers: int, bathy, open_pred=None,
                hilbert: bool = True, name: str = "") -> Mesh:
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    xy = np.stack([i.ravel() * (L / n), j.ravel() * (L / n)], axis=1).astype(np.float64)
    vid = lambda ii, jj: jj * (n + 1) + ii
    tris = []
    for jj in range(n):
        for ii in range(n):
            v00, v10, v11, v01 = vid(ii, jj), vid(ii + 1, jj), vid(ii + 1, jj + 1), vid(ii, jj + 1)
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    tri = np.asarray(tris, dtype=np.int32)
    h_vert = bathy(xy[:, 0], xy[:, 1])
    m = Mesh(xy=xy, tri=tri, h_tri=np.ascontiguousarray(h_vert[tri]),
             n_layers=np.full(tri.shape[0], n_layers, dtype=np.int32),
             bnd=_tag_boundary(xy, tri, open_pred), levels=None, name=name)
    if hilbert:
        m = permute_triangles(m, hilbert_order(m.xy, m.tri))
    return m


def c1_bathymetry(L: float):
    return lambda x, y: 30.0 + 20.0 * np.sin(np.pi * x / L) * np.cos(np.pi * y / L)


def c1_mesh(n: int = 32, L: float = 10e3, n_layers: int = 10) -> Mesh:
    """Square basin of side L, n x n squares split in 2 triangles, closed walls,
    h = 30 + 20 sin(pi x/L) cos(pi y/L), uniform sigma layers."""
    return square_mesh(n, L, n_layers, c1_bathymetry(L), None, name=f"square{n}x{n}x{n_layers}")


# ----------------------------------------------------------------------------
# graded unstructured basin: newest-vertex bisection refined toward x = 0
# ----------------------------------------------------------------------------
def _nvb_refine(xy: list, tris: list, target) -> tuple[list, list]:
    """Conforming newest-vertex bisection.  ``tris`` holds (a, b, c) with the
    refinement edge (b, c); a triangle is marked while its refinement edge is
    longer than ``target`` at its centroid.  Hanging nodes are closed by further
    bisection until the mesh is conforming."""
    mid: dict[tuple[int, int], int] = {}

    def midpoint(u, v):
        k = (u, v) if u < v else (v, u)
        m = mid.get(k)
        if m is None:
            m = len(xy)
            xy.append(((xy[u][0] + xy[v][0]) * 0.5, (xy[u][1] + xy[v][1]) * 0.5))
            mid[k] = m
        return m

    def key(u, v):
        return (u, v) if u < v else (v, u)

    while True:
        P = np.asarray(xy)
        T = np.asarray(tris)
        eb = P[T[:, 1]] - P[T[:, 2]]
        elen = np.hypot(eb[:, 0], eb[:, 1])
        cen = P[T].mean(axis=1)
        marked = elen > target(cen[:, 0], cen[:, 1])
        if not marked.any():
            break
        # bisect the marked triangles, then close hanging nodes
        new = []
        for idx, (a, b, c) in enumerate(tris):
            if marked[idx]:
                m = midpoint(b, c)
                new.append((m, a, b))
                new.append((m, c, a))
            else:
                new.append((a, b, c))
        tris = new
        while True:
            changed = False
            new = []
            for (a, b, c) in tris:
                if key(a, b) in mid or key(b, c) in mid or key(c, a) in mid:
                    m = midpoint(b, c)
                    new.append((m, a, b))
                    new.append((m, c, a))
                    changed = True
                else:
                    new.append((a, b, c))
            tris = new
            if not changed:
                break
    return xy, tris


def _jitter(xy: np.ndarray, tri: np.ndarray, frac: float, rng, fixed: np.ndarray) -> np.ndarray:
    """Move every free vertex by at most ``frac`` x its shortest incident edge,
    rejecting moves that shrink an incident triangle's area below 0.3 x its original."""
    n = xy.shape[0]
    a, b = tri.ravel(), np.roll(tri, -1, axis=1).ravel()
    el = np.hypot(*(xy[a] - xy[b]).T)
    hmin = np.full(n, np.inf)
    np.minimum.at(hmin, a, el)
    np.minimum.at(hmin, b, el)

    def area(p):
        u = p[tri[:, 1]] - p[tri[:, 0]]
        v = p[tri[:, 2]] - p[tri[:, 0]]
        return u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]

    a0 = area(xy)
    r = frac * hmin * np.sqrt(rng.random(n))
    th = 2 * np.pi * rng.random(n)
    d = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    d[fixed] = 0.0
    out = xy + d
    for _ in range(8):
        bad_t = area(out) < 0.3 * a0
        if not bad_t.any():
            break
        bad_v = np.unique(tri[bad_t].ravel())
        out[bad_v] = xy[bad_v]
    return out


def basin_mesh(Lx: float, Ly: float, nx0: int, ny0: int, s_min: float, s_max: float,
               seed: int, jitter: float = 0.2, hilbert: bool = True) -> tuple[np.ndarray, np.ndarray]:
    """Graded conforming triangulation of [0,Lx] x [0,Ly], finest (edge ~ s_min) at x = 0,
    coarsening linearly to s_max at x = Lx.  Returns (xy, tri), tri CCW."""
    target = lambda x, y: s_min + (s_max - s_min) * np.clip(x / Lx, 0.0, 1.0)
    return graded_mesh(Lx, Ly, nx0, ny0, target, seed, jitter, hilbert)


def graded_mesh(Lx: float, Ly: float, nx0: int, ny0: int, target, seed: int, jitter: float = 0.2,
                hilbert: bool = True, keep=None) -> tuple[np.ndarray, np.ndarray]:
    """Conforming newest-vertex-bisection triangulation of [0,Lx] x [0,Ly] refined until
    every edge is below the size field target(x, y); ``keep(cx, cy)`` (optional) selects
    the triangles to keep by their centroids (holes).  Returns (xy, tri), tri CCW."""
    i, j = np.meshgrid(np.arange(nx0 + 1), np.arange(ny0 + 1), indexing="xy")
    xy = [(float(ii * Lx / nx0), float(jj * Ly / ny0)) for ii, jj in zip(i.ravel(), j.ravel())]
    vid = lambda ii, jj: jj * (nx0 + 1) + ii
    tris = []
    for jj in range(ny0):
        for ii in range(nx0):
            v00, v10, v11, v01 = vid(ii, jj), vid(ii + 1, jj), vid(ii + 1, jj + 1), vid(ii, jj + 1)
            # newest vertex first; the shared diagonal (v00, v11) is both triangles' refinement edge
            tris.append((v10, v11, v00))
            tris.append((v01, v00, v11))
    xy, tris = _nvb_refine(xy, tris, target)
    P = np.asarray(xy, dtype=np.float64)
    T = np.asarray(tris, dtype=np.int64)
    if keep is not None:
        c = P[T].mean(axis=1)
        T = T[keep(c[:, 0], c[:, 1])]
        used = np.unique(T)
        remap = -np.ones(P.shape[0], np.int64)
        remap[used] = np.arange(used.size)
        P, T = P[used], remap[T]
    # orient counter-clockwise
    u = P[T[:, 1]] - P[T[:, 0]]
    v = P[T[:, 2]] - P[T[:, 0]]
    cw = (u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]) < 0
    T[cw] = T[cw][:, [0, 2, 1]]
    eps = 1e-6 * min(Lx, Ly)
    fixed = (P[:, 0] < eps) | (P[:, 0] > Lx - eps) | (P[:, 1] < eps) | (P[:, 1] > Ly - eps)
    rng = np.random.default_rng(seed)
    P = _jitter(P, T, jitter, rng, fixed)
    T = T.astype(np.int32)
    if hilbert:
        T = T[hilbert_order(P, T)]
    return P, T


def c2_mesh(target_tri: int = 200_000, n_layers: int = 20, seed: int = 0,
            s_min: float | None = None) -> Mesh:
    """200 km x 100 km basin, coast (wall) at x = 0 with refinement toward it, open
    boundary at x = 200 km, walls at y = 0 and y = 100 km; linear shelf
    h = 10 + 190 x / 200 km; uniform sigma layers."""
    Lx, Ly = 200e3, 100e3
    if s_min is None:
        # the triangle count scales like 1/s_min for a linear size ramp
        s_min = 146.0 * (200_000 / target_tri)
    xy, tri = basin_mesh(Lx, Ly, 20, 10, s_min, 4000.0, seed)
    h_vert = 10.0 + 190.0 * (xy[:, 0] / Lx)
    bnd = _tag_boundary(xy, tri, lambda x, y: x > Lx - 1e-3)
    return Mesh(xy=xy, tri=tri, h_tri=np.ascontiguousarray(h_vert[tri]),
                n_layers=np.full(tri.shape[0], n_layers, dtype=np.int32), bnd=bnd,
                levels=None, name=f"basin{tri.shape[0]}x{n_layers}")


# ----------------------------------------------------------------------------
# z-level-like layering with uneven columns
# ----------------------------------------------------------------------------
def zlevels(n_max: int, dz0: float, depth: float) -> np.ndarray:
    """Interface depths 0 = z_0 > z_1 > ... > z_n_max = -depth with geometric
    thicknesses dz0 * r^k (r solved by bisection)."""
    lo, hi = 1.0 + 1e-9, 2.0
    for _ in range(200):
        r = 0.5 * (lo + hi)
        tot = dz0 * (r ** n_max - 1.0) / (r - 1.0)
        if tot > depth:
            hi = r
        else:
            lo = r
    dz = dz0 * r ** np.arange(n_max)
    z = -np.concatenate([[0.0], np.cumsum(dz)])
    z[-1] = -depth
    return z


def zlevel_columns(h_vert: np.ndarray, tri: np.ndarray, levels: np.ndarray,
                   merge: float = 0.3) -> tuple[np.ndarray, np.ndarray]:
    """Per-vertex level counts N_v (levels above -h, thin partial bottom layers merged
    upward), per-triangle N_t = min_v N_v and the triangle's staircase depth at each
    vertex: -levels[N_t] when N_v > N_t, else h_v."""
    dzl = levels[:-1] - levels[1:]
    n_lev = len(dzl)
    # number of full or partial layers above -h
    nv = np.searchsorted(-levels, h_vert, side="left")  # first interface with depth >= h
    nv = np.clip(nv, 1, n_lev)
    # merge thin partial bottom layer
    part = h_vert + levels[nv - 1]  # thickness of the partial bottom layer
    thin = (part < merge * dzl[nv - 1]) & (nv > 1)
    nv = np.where(thin, nv - 1, nv)
    nt = nv[tri].min(axis=1).astype(np.int32)
    hv = h_vert[tri]
    stair = -levels[nt][:, None] * np.ones((1, 3))
    h_tri = np.where(nv[tri] > nt[:, None], stair, hv)
    return nt, np.ascontiguousarray(h_tri)


def c4_mesh(target_tri: int = 500_000, seed: int = 0, n_max: int = 60,
            h_min: float = 2.0, h_max: float = 600.0) -> Mesh:
    """Basin generator at ~500k triangles with log-uniform smooth bathymetry in
    [2, 600] m (a smooth seeded noise field, rank-mapped to a uniform variable so
    that the depth is log-uniform) and z-level layering (geometric levels from 1 m)
    of 1..60 layers per column: ~12M prisms at the default size."""
    Lx, Ly = 200e3, 100e3
    s_min = 146.0 * (200_000 / target_tri)
    xy, tri = basin_mesh(Lx, Ly, 20, 10, s_min, 4000.0, seed)
    rng = np.random.default_rng(seed + 1)
    noise = np.zeros(xy.shape[0])
    for _ in range(8):
        kx, ky = rng.uniform(1, 6, size=2) * 2 * np.pi / np.array([Lx, Ly])
        ph = rng.uniform(0, 2 * np.pi)
        noise += np.sin(kx * xy[:, 0] + ky * xy[:, 1] + ph)
    u = (np.argsort(np.argsort(noise)) + 0.5) / noise.size      # uniform on (0, 1)
    h_vert = np.exp(np.log(h_min) + u * (np.log(h_max) - np.log(h_min)))
    levels = zlevels(n_max, 1.0, h_max)
    nt, h_tri = zlevel_columns(h_vert, tri, levels)
    bnd = _tag_boundary(xy, tri, lambda x, y: x > Lx - 1e-3)
    return Mesh(xy=xy, tri=tri, h_tri=h_tri, n_layers=nt, bnd=bnd, levels=levels,
                name=f"zlevel{tri.shape[0]}")


# ----------------------------------------------------------------------------
# reef-scale stress mesh: islands, multiscale coastline, uneven columns
# ----------------------------------------------------------------------------
def reef_islands(n: int, Lx: float, Ly: float, seed: int, r_min: float = 100.0, r_max: float = 2000.0):
    """n circular islands (centres uniform, 5 km from the outer boundary; radii
    log-uniform in [r_min, r_max])."""
    rng = np.random.default_rng(seed + 7)
    cx = rng.uniform(5e3, Lx - 5e3, n)
    cy = rng.uniform(5e3, Ly - 5e3, n)
    r = np.exp(rng.uniform(np.log(r_min), np.log(r_max), n))
    return cx, cy, r


def _coast_distance(x, y, isl, k: int = 16):
    """Distance to the nearest island coastline (0 inside an island): the minimum of
    |p - c_i| - r_i over the k nearest centres, exact whenever the nearest coast
    belongs to one of them; a point whose k-th centre is nearer than its best
    coast distance plus the largest radius is checked against all islands."""
    from scipy.spatial import cKDTree
    cx, cy, r = isl
    x = np.asarray(x, np.float64).ravel(); y = np.asarray(y, np.float64).ravel()
    pts = np.stack([x, y], axis=1)
    tree = cKDTree(np.stack([cx, cy], axis=1))
    kk = min(k, cx.size)
    dist, idx = tree.query(pts, k=kk)
    dist = dist.reshape(pts.shape[0], kk); idx = idx.reshape(pts.shape[0], kk)
    d = np.maximum(dist - r[idx], 0.0).min(axis=1)
    unsure = dist[:, -1] < d + r.max()
    if unsure.any() and kk < cx.size:
        q = pts[unsure]
        dx = q[:, 0:1] - cx[None]; dy = q[:, 1:2] - cy[None]
        d[unsure] = np.maximum(np.sqrt(dx * dx + dy * dy) - r[None], 0.0).min(axis=1)
    return d


def c5_mesh(n_islands: int = 400, Lx: float = 400e3, Ly: float = 200e3, seed: int = 0,
            s_min: float = 50.0, s_max: float = 5000.0, ramp: float = 0.15, n_max: int = 30,
            h_min: float = 1.0, h_max: float = 1000.0, h_scale: float = 6e3) -> Mesh:
    """Reef-scale stress mesh: edge ~ s_min at the island coastlines growing by
    ``ramp`` per metre of distance to s_max, triangles inside the islands removed
    (their coastlines are walls), open boundary at x = Lx, walls elsewhere; depth
    h = h_min + (h_max - h_min) tanh(d / h_scale) with d the distance to the nearest
    coast; z-levels (geometric from 1 m) with at most n_max layers per column."""
    isl = reef_islands(n_islands, Lx, Ly, seed)
    target = lambda x, y: np.minimum(s_max, s_min + ramp * _coast_distance(x, y, isl))
    cx, cy, r = isl
    keep = lambda x, y: _coast_distance(x, y, isl) > 0.0
    xy, tri = graded_mesh(Lx, Ly, 40, 20, target, seed, keep=keep)
    d = _coast_distance(xy[:, 0], xy[:, 1], isl)
    h_vert = h_min + (h_max - h_min) * np.tanh(d / h_scale)
    levels = zlevels(n_max, 1.0, h_max)
    nt, h_tri = zlevel_columns(h_vert, tri, levels)
    bnd = _tag_boundary(xy, tri, lambda x, y: x > Lx - 1e-3)
    return Mesh(xy=xy, tri=tri, h_tri=h_tri, n_layers=nt, bnd=bnd, levels=levels,
                name=f"reef{tri.shape[0]}")


def cached_mesh(name: str, build) -> Mesh:
    """``build()`` once per machine: the mesh is kept as an .npz file in the system
    temporary directory under ``name`` (large generated meshes take minutes)."""
    import os
    import tempfile
    d = os.path.join(tempfile.gettempdir(), "slim_gb300_meshes")
    path = os.path.join(d, name + ".npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        lv = z["levels"]
        return Mesh(xy=z["xy"], tri=z["tri"], h_tri=z["h_tri"], n_layers=z["n_layers"], bnd=z["bnd"],
                    levels=lv if lv.size else None, name=str(z["name"]))
    m = build()
    os.makedirs(d, exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, xy=m.xy, tri=m.tri, h_tri=m.h_tri, n_layers=m.n_layers, bnd=m.bnd,
             levels=m.levels if m.levels is not None else np.zeros(0), name=m.name)
    os.replace(tmp, path)
    return m
