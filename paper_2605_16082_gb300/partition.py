"""Horizontal partitioning of a prismatic mesh for the partitioned step (Sec. 3,
"Multi-GPU": horizontal partitions, each with one layer of ghost triangles, halo
exchanges after every neighbour-access phase, boundary kernels ahead of the
interior ones).

The triangles of the generated meshes are in Hilbert order, so contiguous ranges
of it are compact partitions; the ranges are cut at equal numbers of prisms.
Each partition's local mesh lists

    its owned triangles next to a ghost (class 0), its other owned triangles
    (class 1), then its ghosts (class 2: the other partitions' triangles across
    its edges),

each group in global order.  A ghost's edges that leave the partition become
walls.  The pair lists say, for every ordered pair of partitions (i, j), which
owned triangles of i are ghosts of j (local ids on both sides).  Host-side set-up
only; the step and the exchanges run in the library (slim_halo_*).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def edge_neighbours(tri: np.ndarray, n_vert: int) -> np.ndarray:
    """(n_tri, 3) triangle across each edge e (vertices e, e+1), or -1."""
    tri = np.asarray(tri, np.int64)
    a = tri.ravel()
    b = np.roll(tri, -1, axis=1).ravel()
    key = np.minimum(a, b) * (n_vert + 1) + np.maximum(a, b)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    nbr = -np.ones(3 * tri.shape[0], np.int64)
    i = np.nonzero(ks[1:] == ks[:-1])[0]
    e1, e2 = order[i], order[i + 1]
    nbr[e1] = e2 // 3
    nbr[e2] = e1 // 3
    return nbr.reshape(-1, 3)


@dataclasses.dataclass
class Part:
    """One partition: its local mesh (the arrays of slim_mesh_create_part) and maps."""
    xy: np.ndarray
    tri: np.ndarray
    h_tri: np.ndarray
    n_layers: np.ndarray
    bnd: np.ndarray
    levels: np.ndarray | None
    tri_class: np.ndarray      # int8, 0 / 1 / 2 per local triangle
    glob: np.ndarray           # local -> global triangle id
    n_owned: int

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])


@dataclasses.dataclass
class Partitioning:
    parts: list
    owner: np.ndarray          # global triangle -> partition
    pair_count: np.ndarray     # (K, K) triangles i sends to j
    send_tris: np.ndarray      # concatenated local ids in the sender, row-major (i, j)
    recv_tris: np.ndarray      # the matching local ghost ids in the receiver


def partition(mesh, n_parts: int) -> Partitioning:
    """Split the (Hilbert-ordered) triangles into n_parts contiguous ranges of about
    equal prism counts, each with one ghost layer."""
    nt = mesh.tri.shape[0]
    if not 1 <= n_parts <= nt:
        raise ValueError("n_parts must be between 1 and the number of triangles")
    nl = np.asarray(mesh.n_layers, np.int64)
    cum = np.concatenate([[0], np.cumsum(nl)])
    cuts = np.searchsorted(cum, np.arange(1, n_parts) * cum[-1] / n_parts, side="left")
    bounds = np.concatenate([[0], np.clip(cuts, 1, nt - 1), [nt]])
    bounds = np.maximum.accumulate(bounds)
    owner = np.zeros(nt, np.int64)
    for p in range(n_parts):
        owner[bounds[p]:bounds[p + 1]] = p
    nbr = edge_neighbours(mesh.tri, mesh.xy.shape[0])
    parts = []
    local_of = []
    for p in range(n_parts):
        own = np.arange(bounds[p], bounds[p + 1])
        nb = nbr[own]
        foreign = (nb >= 0) & (owner[np.where(nb >= 0, nb, 0)] != p)
        ghosts = np.unique(nb[foreign])
        touches = foreign.any(axis=1)
        order = np.concatenate([own[touches], own[~touches], ghosts])
        cls = np.concatenate([np.zeros(touches.sum(), np.int8), np.ones((~touches).sum(), np.int8),
                              np.full(len(ghosts), 2, np.int8)])
        loc = -np.ones(nt, np.int64)
        loc[order] = np.arange(len(order))
        bnd = np.asarray(mesh.bnd, np.int8)[order].copy()
        # ghost edges whose neighbour is outside the local mesh: walls
        gnb = nbr[ghosts]
        cut = (gnb >= 0) & (loc[np.where(gnb >= 0, gnb, 0)] < 0)
        gb = bnd[len(own):]
        gb[cut] = 1
        bnd[len(own):] = gb
        parts.append(Part(xy=mesh.xy, tri=np.ascontiguousarray(mesh.tri[order]),
                          h_tri=np.ascontiguousarray(mesh.h_tri[order]),
                          n_layers=np.ascontiguousarray(np.asarray(mesh.n_layers)[order]),
                          bnd=np.ascontiguousarray(bnd), levels=mesh.levels, tri_class=cls,
                          glob=order, n_owned=len(own)))
        local_of.append(loc)
    pair_count = np.zeros((n_parts, n_parts), np.int64)
    send, recv = [], []
    for i in range(n_parts):
        for j in range(n_parts):
            if i == j:
                continue
            g = parts[j].glob[parts[j].tri_class == 2]
            g = g[owner[g] == i]
            pair_count[i, j] = len(g)
            send.append(local_of[i][g])
            recv.append(local_of[j][g])
    cat = lambda xs: np.concatenate(xs).astype(np.int32) if xs else np.zeros(0, np.int32)
    return Partitioning(parts=parts, owner=owner, pair_count=pair_count.astype(np.int32),
                        send_tris=cat(send), recv_tris=cat(recv))


def prism_map(mesh, part: Part) -> np.ndarray:
    """Global prism index of every local prism of the partition."""
    goff = np.concatenate([[0], np.cumsum(np.asarray(mesh.n_layers, np.int64))])
    return np.concatenate([np.arange(goff[t], goff[t + 1]) for t in part.glob]) if part.n_tri else \
        np.zeros(0, np.int64)


def to_local(mesh, part: Part, f: np.ndarray, is3d: bool, pmap: np.ndarray | None = None) -> np.ndarray:
    """A global nodal field (6P or 3 n_tri values) restricted to the partition's
    local mesh (owned and ghost triangles)."""
    f = np.asarray(f, np.float64)
    if is3d:
        P = int(np.asarray(mesh.n_layers).sum())
        pm = prism_map(mesh, part) if pmap is None else pmap
        return f.reshape(6, P)[:, pm].ravel()
    nt = mesh.tri.shape[0]
    return f.reshape(3, nt)[:, part.glob].ravel()


def owned_to_global(mesh, pt: Partitioning, locals_: list, is3d: bool) -> np.ndarray:
    """Assemble a global field from the owned triangles of every partition."""
    nt = mesh.tri.shape[0]
    if is3d:
        P = int(np.asarray(mesh.n_layers).sum())
        out = np.empty((6, P))
        for part, f in zip(pt.parts, locals_):
            pm = prism_map(mesh, part)
            Pl = len(pm)
            n_own = int(np.asarray(part.n_layers)[:part.n_owned].sum())
            out[:, pm[:n_own]] = np.asarray(f).reshape(6, Pl)[:, :n_own]
        return out.ravel()
    out = np.empty((3, nt))
    for part, f in zip(pt.parts, locals_):
        out[:, part.glob[:part.n_owned]] = np.asarray(f).reshape(3, part.n_tri)[:, :part.n_owned]
    return out.ravel()
