"""Full-size parity: the L = 256 Ising lattice of the benchmark (N = 2^28
sites, random start, T = 4.21394), in the benchmark's launch configuration.
The oracle cannot hold this lattice, so outputs are checked on samples the
oracle's definitions can compute one by one (bond decisions, flips from
cuRAND's Philox with the documented layout) and through properties that hold
at any size (canonical labels are cluster minima and roots label themselves;
E and M recomputed exactly from the returned spins)."""
import math

import numpy as np
import pytest

import lattice_np
import paper_1612_08312_gb300 as pyro
import refmath
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def probe():
    if refmath.curand_philox_lib() is None:
        pytest.skip("nvcc not available to build the cuRAND host probe")


@pytest.mark.parametrize("tile", ["default", "auto"])
def test_l256_sweep_sampled(probe, tile):
    cfg = workloads.ISING_L256
    L, T, seed = cfg["L"], cfg["T"][1], cfg["seeds"][0]
    beta = 1.0 / T
    lat = pyro.Lattice(L, pyro.ISING, seed, start="random", tile=(0, 0, 0) if tile == "default" else "auto")
    N = lat.N
    assert N == 16 * 256 ** 3
    # random start from the INIT stream, sampled
    rng = np.random.default_rng(0)
    s0 = lat.spins()
    idx = rng.integers(0, N, 200000)
    init = refmath.stream_bits(seed, 0xFFFFFFFF, 4, idx)
    assert (s0[idx] == np.where(init == 1, -1, 1)).all()
    lat.sweep(beta, 2)
    s0 = lat.spins()
    k = lat.sweep_count
    lat.sweep(beta, 1)
    s1 = lat.spins()
    lab = lat.labels()
    # canonical labels: minimum of the cluster, roots label themselves
    assert (lab <= np.arange(N, dtype=np.int64)).all()
    assert (lab[lab] == lab).all()
    # sampled bonds: an active bond joins two sites of one cluster
    b = rng.integers(0, 3 * N, 300000)
    bi, bj = lattice_np.bond_endpoints(L, b)
    thr = math.floor(-math.expm1(-2 * beta) * 2 ** 32)
    w = refmath.bond_words_of(seed, k, b).astype(np.int64)
    active = (s0[bi] == s0[bj]) & (w < thr)
    assert active.sum() > 1000
    assert (lab[bi[active]] == lab[bj[active]]).all()
    # sampled flips: a site flips iff its cluster root's flip bit is set
    i = rng.integers(0, N, 300000)
    fb = refmath.stream_bits(seed, k, 2, lab[i].astype(np.int64))
    assert (s1[i] == np.where(fb == 1, -s0[i], s0[i])).all()
    # measurement recomputed exactly from the spins
    # more sweeps: the label invariants must hold after every one
    ar = np.arange(N, dtype=np.int64)
    for _ in range(3):
        lat.sweep(beta, 1)
        lb = lat.labels()
        assert (lb <= ar).all() and (lb[lb] == lb).all()
    s1 = lat.spins()
    E, m2, m4 = lat.measure()
    M = int(s1.astype(np.int64).sum())
    anti = 0
    for start in range(0, 3 * N, 1 << 26):
        bb = np.arange(start, min(3 * N, start + (1 << 26)), dtype=np.int64)
        ei, ej = lattice_np.bond_endpoints(L, bb)
        anti += int((s1[ei] != s1[ej]).sum())
    assert E == -float(3 * N - 2 * anti)
    m = abs(M) / N
    assert m2 == m * m and m4 == (m * m) * (m * m)
    lat.close()
