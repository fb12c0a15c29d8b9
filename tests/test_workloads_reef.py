"""The reef-scale stress mesh generator on a reduced domain (the full mesh takes
about a minute and a half): a valid conforming CCW triangulation with the islands
carved out, uneven z-level columns of 1..30 layers, depth rising away from the
coasts, an open boundary only at x = Lx."""
import numpy as np

from workloads import meshes


def test_reduced_reef_mesh_is_valid():
    Lx, Ly = 40e3, 20e3
    m = meshes.c5_mesh(n_islands=6, Lx=Lx, Ly=Ly, seed=3)
    xy, tri = m.xy, m.tri
    u = xy[tri[:, 1]] - xy[tri[:, 0]]
    v = xy[tri[:, 2]] - xy[tri[:, 0]]
    assert ((u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]) > 0).all()          # counter-clockwise
    e = np.sort(np.stack([tri, np.roll(tri, -1, axis=1)], axis=2).reshape(-1, 2), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert cnt.max() <= 2                                                 # conforming
    cx, cy, r = meshes.reef_islands(6, Lx, Ly, 3)
    c = xy[tri].mean(axis=1)
    # islands carved (the node jitter after carving moves coastline vertices by at
    # most 0.2 of a ~50 m edge)
    inside = np.hypot(c[:, 0:1] - cx[None], c[:, 1:2] - cy[None]) < r[None] - 25.0
    assert not inside.any()
    assert m.n_layers.min() >= 1 and m.n_layers.max() <= 30
    assert m.levels is not None and len(m.levels) == 31
    # coastline edges are walls, the open boundary lies at x = Lx only
    for t_, ed in zip(*np.nonzero(m.bnd == 2)):
        a, b = tri[t_, ed], tri[t_, (ed + 1) % 3]
        assert xy[a, 0] > Lx - 1e-3 and xy[b, 0] > Lx - 1e-3
    assert (m.bnd == 1).sum() > 0
    # shallow at the coasts, deep offshore
    d = meshes._coast_distance(xy[:, 0], xy[:, 1], (cx, cy, r))
    near = d[tri].mean(axis=1) < 200.0
    assert m.h_tri[near].mean() < 0.2 * m.h_tri[~near].mean()


def test_coast_distance_matches_brute_force():
    isl = meshes.reef_islands(50, 100e3, 50e3, 1)
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 100e3, 5000), rng.uniform(0, 50e3, 5000)
    cx, cy, r = isl
    brute = np.maximum(np.hypot(x[:, None] - cx[None], y[:, None] - cy[None]) - r[None], 0).min(axis=1)
    assert np.allclose(meshes._coast_distance(x, y, isl, k=4), brute, rtol=0, atol=1e-9)
