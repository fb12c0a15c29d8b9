"""Partitioner of the partitioned step (Sec. 3 horizontal decomposition with one
ghost layer): owned sets, ghost layers, triangle classes and the pair lists,
checked against adjacency found by brute force (every pair of triangles compared
by their shared vertices)."""
import itertools

import numpy as np
import pytest

import workloads as wl
from helpers import random_uneven_mesh
from paper_2605_16082_gb300 import partition as pa


def brute_neighbours(tri):
    """Set of neighbours of every triangle: triangles sharing two vertices."""
    nb = [set() for _ in range(len(tri))]
    sets = [set(map(int, t)) for t in tri]
    for i, j in itertools.combinations(range(len(tri)), 2):
        if len(sets[i] & sets[j]) == 2:
            nb[i].add(j)
            nb[j].add(i)
    return nb


CASES = {
    "basin": lambda: wl.c2_mesh(600, 3, 0),
    "uneven_open": lambda: random_uneven_mesh(8, 3000.0, 6, seed=3, open_x=True),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("K", [2, 3, 4])
def test_partitions_and_ghost_tables_match_brute_force_adjacency(case, K):
    m = CASES[case]()
    nb = brute_neighbours(m.tri)
    pt = pa.partition(m, K)
    owned = np.concatenate([p.glob[:p.n_owned] for p in pt.parts])
    assert np.array_equal(np.sort(owned), np.arange(m.n_tri))          # the owned sets partition the mesh
    prisms = [int(np.asarray(p.n_layers)[:p.n_owned].sum()) for p in pt.parts]
    assert max(prisms) - min(prisms) <= 2 * int(m.n_layers.max())       # balanced by prisms
    pos = 0
    for i, j in itertools.product(range(K), range(K)):
        n = int(pt.pair_count[i, j])
        if i == j:
            assert n == 0
            continue
        send = pt.send_tris[pos:pos + n]
        recv = pt.recv_tris[pos:pos + n]
        pos += n
        gi, gj = pt.parts[i].glob, pt.parts[j].glob
        # the same global triangles on both sides: owned by i, ghosts of j
        assert np.array_equal(gi[send], gj[recv])
        assert (send < pt.parts[i].n_owned).all()
        assert (pt.parts[j].tri_class[recv] == 2).all()
    assert pos == len(pt.send_tris) == len(pt.recv_tris)
    for p, part in enumerate(pt.parts):
        own = set(map(int, part.glob[:part.n_owned]))
        ghosts = set(map(int, part.glob[part.n_owned:]))
        want = set().union(*(nb[t] for t in own)) - own
        assert ghosts == want                                           # exactly one ghost layer
        for l, t in enumerate(part.glob[:part.n_owned]):                # class 0 iff a ghost neighbour
            assert part.tri_class[l] == (0 if nb[t] & ghosts else 1)
        assert (np.diff(part.tri_class) >= 0).all()
        # every ghost is sent by its owner to this partition exactly once
        got = sorted(int(g) for i in range(K) if i != p
                     for g in pt.parts[p].glob[pt.recv_tris[_pair_slice(pt, i, p)]])
        assert got == sorted(ghosts)
        # local boundary tags: owned edges keep theirs, ghost edges leaving the
        # partition become walls, and the local mesh is consistent
        local_nb = pa.edge_neighbours(part.tri, part.xy.shape[0])
        for l in range(part.n_tri):
            for e in range(3):
                if local_nb[l, e] >= 0:
                    assert part.bnd[l, e] == 0
                elif l < part.n_owned:
                    assert part.bnd[l, e] == m.bnd[part.glob[l], e] != 0
                else:
                    assert part.bnd[l, e] != 0


def _pair_slice(pt, i, j):
    K = pt.pair_count.shape[0]
    start = int(pt.pair_count.ravel()[:i * K + j].sum())
    return slice(start, start + int(pt.pair_count[i, j]))


def test_fields_round_trip_through_the_partitions():
    m = CASES["uneven_open"]()
    pt = pa.partition(m, 3)
    rng = np.random.default_rng(0)
    f3 = rng.standard_normal(6 * int(m.n_layers.sum()))
    f2 = rng.standard_normal(3 * m.n_tri)
    loc3 = [pa.to_local(m, p, f3, True) for p in pt.parts]
    loc2 = [pa.to_local(m, p, f2, False) for p in pt.parts]
    assert np.array_equal(pa.owned_to_global(m, pt, loc3, True), f3)
    assert np.array_equal(pa.owned_to_global(m, pt, loc2, False), f2)
