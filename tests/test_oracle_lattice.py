"""Pins of the oracle's lattice (Sec. 2: 16-site cubic cell, periodic,
coordination six) against an independent construction: the pyrochlore
lattice as the bond midpoints of the diamond lattice, neighbours by O(N^2)
distance search."""
import json
import os

import numpy as np
import pytest

import oracle
import refmath

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_sizes.json")


def test_site_counts_match_paper():
    g = json.load(open(GOLDEN))
    for L, N in g["sizes"].items():
        assert 16 * int(L) ** 3 == N
    for L in (1, 2, 3):
        assert oracle.Oracle(L, oracle.ISING, 1).N == 16 * L ** 3


@pytest.mark.parametrize("L", [1, 2, 3])
def test_positions_are_diamond_bond_midpoints(L):
    ours = np.array([oracle.site_position(L, i) for i in range(16 * L ** 3)]) * 2  # 1/8 units
    ref = refmath.diamond_midpoint_positions(L)
    P = 8 * L
    # equal as sets up to one global translation
    shift = (ref[0] - ours[0]) % P
    moved = (ours + shift) % P
    key = lambda a: set(map(tuple, a.tolist()))
    ok = key(moved) == key(ref)
    if not ok:  # try every translation that maps ours[0] onto some ref point
        for r in ref:
            moved = (ours + (r - ours[0])) % P
            if key(moved) == key(ref):
                ok = True
                break
    assert ok
    assert len(key(ours)) == 16 * L ** 3


@pytest.mark.parametrize("L", [1, 2, 3])
def test_nn_table_matches_brute_force(L):
    o = oracle.Oracle(L, oracle.ISING, 1)
    pos = np.array([oracle.site_position(L, i) for i in range(o.N)])
    nbrs, dmin = refmath.brute_force_neighbours(pos, 4 * L)
    assert dmin == 2  # |d|^2 = 2 in quarter-cell units
    nn = o.nn()
    for i in range(o.N):
        assert set(nn[i].tolist()) == nbrs[i]
        assert len(nbrs[i]) == json.load(open(GOLDEN))["coordination"]


@pytest.mark.parametrize("L", [1, 2, 3])
def test_bonds_form_corner_sharing_tetrahedra(L):
    o = oracle.Oracle(L, oracle.ISING, 1)
    bi, bj = o.bonds()
    N = o.N
    assert len(bi) == 3 * N
    pairs = set()
    for a, b in zip(bi.tolist(), bj.tolist()):
        assert a != b
        pairs.add((min(a, b), max(a, b)))
    assert len(pairs) == 3 * N  # no duplicate bonds, even at L = 1
    nn = o.nn()
    want = {(min(i, j), max(i, j)) for i in range(N) for j in nn[i].tolist()}
    assert pairs == want  # the bonds are exactly the nearest-neighbour pairs
    # every group of six consecutive bonds is a complete graph on 4 sites
    tets = []
    for t in range(N // 2):
        sites = set(bi[6 * t:6 * t + 6].tolist()) | set(bj[6 * t:6 * t + 6].tolist())
        assert len(sites) == 4
        tets.append(sites)
    # corner sharing: each site lies in exactly two tetrahedra, one "up"
    # (even group) and one "down" (odd group); each tetrahedron has one
    # site of each basis index
    count = np.zeros((N, 2), dtype=int)
    for t, s in enumerate(tets):
        assert sorted(x & 3 for x in s) == [0, 1, 2, 3]
        for x in s:
            count[x, t % 2] += 1
    assert (count == 1).all()


def test_l1_graph_degree_and_size():
    o = oracle.Oracle(1, oracle.ISING, 1)
    nn = o.nn()
    assert nn.shape == (16, 6)
    deg = np.bincount(np.concatenate(o.bonds()), minlength=16)
    assert (deg == 6).all()
