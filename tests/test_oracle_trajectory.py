"""Second-implementation checks of one oracle sweep.

A sweep is recomputed step by step in numpy from the spins before it, with
random numbers from cuRAND's Philox (not the oracle's), clusters from
scipy.sparse.csgraph, and the bond list from the geometry test's pinned
tetrahedra.  This pins the index conventions (bond random-number id, call
index, byte / word / bit slots, tags, sweep field), the bond rule of each model,
the canonical root, the flip and the reflection s -> s - 2 (s.r) r (Wolff
embedding, Sec. 2)."""
import math

import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle
import refmath

BOND, FLIP, AXIS, INIT, TIE = 1, 2, 3, 4, 5


@pytest.fixture(scope="module", autouse=True)
def probe():
    if refmath.curand_philox_lib() is None:
        pytest.skip("nvcc not available to build the cuRAND host probe")


def min_index_labels(N, bi, bj, active):
    g = coo_matrix((np.ones(int(active.sum())), (bi[active], bj[active])), shape=(N, N))
    nc, comp = connected_components(g, directed=False)
    mins = np.full(nc, N, dtype=np.int64)
    np.minimum.at(mins, comp, np.arange(N))
    return mins[comp].astype(np.int32)


def axis_from_curand(seed, sweep, n):
    for a in range(256):
        w = refmath.curand_philox(np.array([[a, 0, sweep, AXIS]]),
                                  np.array([[seed & 0xFFFFFFFF, seed >> 32]]))[0]
        u0 = float(w[0].view(np.int32)) / 2 ** 31
        u1 = float(w[1].view(np.int32)) / 2 ** 31
        s = u0 * u0 + u1 * u1
        if 0 < s < 1:
            if n == 2:
                q = math.sqrt(s)
                return np.array([u0 / q, u1 / q])
            t = math.sqrt(1 - s)
            return np.array([2 * u0 * t, 2 * u1 * t, 1 - 2 * s])
    raise AssertionError


@pytest.mark.parametrize("L,T,seed", [(1, 4.21394, 1), (2, 4.21394, 7), (3, 3.0, 0x123456789ABC)])
def test_ising_sweep_recomputed(L, T, seed):
    beta = 1 / T
    o = oracle.Oracle(L, oracle.ISING, seed=seed, start="random")
    o.sweep(beta, 3)
    bi, bj = o.bonds()
    N = o.N
    for _ in range(3):
        k = o.sweep_count
        s0 = o.spins().astype(np.int64)
        o.sweep(beta, 1)
        sat = s0[bi] == s0[bj]
        w = refmath.bond_words(seed, k, 3 * N)
        thr = math.floor(-math.expm1(-2 * beta) * 2 ** 32)
        act = sat & (w.astype(np.int64) < thr)
        assert (o.active().astype(bool) == act).all()
        lab = min_index_labels(N, bi, bj, act)
        assert (o.labels() == lab).all()
        fb = refmath.stream_bits(seed, k, FLIP, lab)
        s1 = np.where(fb == 1, -s0, s0)
        assert (o.spins() == s1).all()
        E, m2, m4 = o.measure()
        assert E == -float((s1[bi] * s1[bj]).sum())
        m = abs(float(s1.sum())) / N
        assert m2 == m * m and m4 == (m * m) * (m * m)


def test_random_ising_start_recomputed():
    o = oracle.Oracle(2, oracle.ISING, seed=99, start="random")
    b = refmath.stream_bits(99, 0xFFFFFFFF, INIT, np.arange(o.N))
    assert (o.spins() == np.where(b == 1, -1, 1)).all()


@pytest.mark.parametrize("model", [2, 3])
@pytest.mark.parametrize("L,T", [(1, 1.5), (2, 1.0)])
def test_vector_sweep_recomputed(model, L, T):
    beta = 1 / T
    seed = 31
    o = oracle.Oracle(L, model, seed=seed, start="random")
    o.sweep(beta, 2)
    bi, bj = o.bonds()
    N = o.N
    for _ in range(3):
        k = o.sweep_count
        s0 = o.spins()
        o.sweep(beta, 1)
        r = axis_from_curand(seed, k, model)
        assert (o.axis() == r).all()
        proj = s0 @ r
        x = proj[bi] * proj[bj]
        w = refmath.bond_words(seed, k, 3 * N).astype(np.float64)
        p = -np.expm1(-2 * beta * np.maximum(x, 0))
        thr = np.floor(p * 2 ** 32)
        act = (x > 0) & (w < thr)
        # a threshold within 1e-4 of an integer may legitimately differ in
        # the last bit of p between numpy and libm; none are expected here
        frac = p * 2 ** 32 - thr
        assert (np.minimum(frac, 1 - frac)[x > 0] > 1e-4).all()
        assert (o.active().astype(bool) == act).all()
        lab = min_index_labels(N, bi, bj, act)
        assert (o.labels() == lab).all()
        flip = refmath.stream_bits(seed, k, FLIP, lab) == 1
        s1 = s0.copy()
        refl = s0 - 2 * proj[:, None] * r[None, :]
        refl /= np.linalg.norm(refl, axis=1, keepdims=True)
        s1[flip] = refl[flip]
        assert np.abs(o.spins() - s1).max() < 1e-14
        # the reflection reverses the projection on r and keeps |s| = 1
        assert np.allclose(o.spins()[flip] @ r, -proj[flip], atol=1e-14)
        assert np.allclose(np.linalg.norm(o.spins(), axis=1), 1, atol=1e-14)


# The documented (g, q) -> (tetrahedron, vertex pair) table of the bond ids
# (include/pyro.h), written out here from that text.
DOC_ID_TABLE = {(0, 0): ("up", (0, 1)), (0, 1): ("up", (1, 2)), (0, 2): ("up", (2, 3)), (0, 3): ("up", (0, 3)),
                (1, 0): ("up", (0, 2)), (1, 1): ("up", (1, 3)), (1, 2): ("down", (0, 2)), (1, 3): ("down", (1, 3)),
                (2, 0): ("down", (0, 1)), (2, 1): ("down", (1, 2)), (2, 2): ("down", (2, 3)), (2, 3): ("down", (0, 3))}


def test_bond_rng_ids_are_a_permutation():
    # every cell's 48 bonds use 48 distinct ids 48 c .. 48 c + 47
    o = oracle.Oracle(2, oracle.ISING, 1)
    ids = np.array([oracle.bond_rng_id(b) for b in range(3 * o.N)])
    assert (np.sort(ids) == np.arange(3 * o.N)).all()
    # and each id 48 c + 16 g + 4 f + q names the bond the documentation
    # says: the oracle's own bond list gives each bond's cell, FCC point,
    # tetrahedron (both ends among sites 4r .. 4r + 3: up) and vertex pair
    # (the ends' basis indices)
    bi, bj = o.bonds()
    for b in range(3 * o.N):
        r = b // 12
        i, j = int(bi[b]), int(bj[b])
        tet = "up" if i >> 2 == r and j >> 2 == r else "down"
        pair = tuple(sorted((i & 3, j & 3)))
        c, rest = divmod(int(ids[b]), 48)
        g, fq = divmod(rest, 16)
        f, q = divmod(fq, 4)
        assert c == r >> 2 and f == (r & 3), b
        assert DOC_ID_TABLE[(g, q)] == (tet, pair), b


def test_clusters_match_scipy_on_random_graphs():
    rng = np.random.default_rng(0)
    for trial in range(20):
        N = int(rng.integers(1, 400))
        B = int(rng.integers(0, 3 * N + 1))
        bi = rng.integers(0, N, B).astype(np.int32)
        bj = rng.integers(0, N, B).astype(np.int32)
        act = rng.random(B) < rng.random()
        lab = oracle.clusters(N, bi, bj, act)
        assert (lab == min_index_labels(N, bi, bj, act)).all()
