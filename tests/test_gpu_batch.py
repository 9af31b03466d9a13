"""Batched replicas: every phase of a sweep is one launch over all replicas'
tiles and long runs replay captured CUDA graphs; each replica must still be
exactly the chain of a single lattice with the replica's seed (and so the
oracle's chain)."""
import numpy as np
import pytest

import oracle
import paper_1612_08312_gb300 as pyro

pytestmark = pytest.mark.gpu


def test_ising_batch_matches_single_lattices_and_oracle():
    Ls = [4, 8, 8, 12, 16]
    Ts = [4.19, 4.21, 4.22, 4.23, 4.24]
    b = pyro.Replicas(Ls, [1 / T for T in Ts], pyro.ISING, start="random", seed=1)
    b.sweep(37)
    for r, (L, T) in enumerate(zip(Ls, Ts)):
        seed = pyro.replica_seed(1, r)
        o = oracle.Oracle(L, oracle.ISING, seed, "random")
        o.sweep(1 / T, 37)
        assert (b.spins(r) == o.spins()).all(), r
        assert b.stats(r) == o.stats(), r
        assert b.measure(r) == o.measure(), r


@pytest.mark.parametrize("model", [2, 3])
def test_vector_fp64_batch_matches_oracle(model):
    Ls = [2, 4, 4]
    Ts = [1.2, 1.3, 2.0]
    b = pyro.Replicas(Ls, [1 / T for T in Ts], model, precision=pyro.FP64, start="random", seed=5)
    b.sweep(3)
    for r, (L, T) in enumerate(zip(Ls, Ts)):
        o = oracle.Oracle(L, model, pyro.replica_seed(5, r), "random")
        o.sweep(1 / T, 3)
        assert np.abs(b.spins(r) - o.spins()).max() < 1e-12


def test_batch_graph_chunks_and_launch_accounting():
    b = pyro.Replicas([8, 8], [0.23, 0.24], pyro.ISING, start="random", seed=9)
    l0 = b.launches
    b.sweep(70)  # two 32-sweep graphs plus six single-sweep graphs
    b.sync()
    # per sweep: local labelling, crossing unions, crossing roots, flip,
    # measurement, accumulation
    assert b.launches - l0 == 70 * 6
    s = b.stats(0)
    assert s["count"] == 70


def test_folded_accumulation_matches_the_oracle_and_counts_its_launch():
    """A lattice of 2048 tiles or more sums its measurement partials in
    groups first (one more launch per sweep); its statistics must still be
    the oracle's, bit for bit."""
    L = 32
    g = pyro.Lattice(L, pyro.ISING, 5, start="random", tile=(4, 2, 2))  # 32^3 / 16 = 2048 tiles
    o = oracle.Oracle(L, oracle.ISING, 5, "random")
    g.set_graphs(False)
    g.sweep(1 / 4.21394, 1)  # the first sweep at a new beta also sets the lattice's parameters
    l0 = g.launches
    g.sweep(1 / 4.21394, 3)
    g.sync()
    assert g.launches - l0 == 3 * 7
    o.sweep(1 / 4.21394, 4)
    assert g.stats() == o.stats()
    assert g.measure() == o.measure()
    g.close()


def test_mixed_sizes_uneven_tiles():
    Ls = [16, 24, 32]
    b = pyro.Replicas(Ls, [1 / 4.21394] * 3, pyro.ISING, start="random", seed=2)
    b.sweep(5)
    for r, L in enumerate(Ls):
        o = oracle.Oracle(L, oracle.ISING, pyro.replica_seed(2, r), "random")
        o.sweep(1 / 4.21394, 5)
        assert (b.spins(r) == o.spins()).all()


def test_batch_tile_autotune_and_single_reads():
    """A batch created with the batch autotuner's tile runs the same chains;
    all replicas' statistics and measurements come back in one read each and
    equal the per-replica reads."""
    Ls = [8, 16, 24]
    betas = [1 / 4.2, 1 / 4.21394, 1 / 4.23]
    tile, ms = pyro.pyro_batch_autotune(Ls, betas, pyro.ISING, pyro.FP64, 2)
    assert all(L % t == 0 for L in Ls for t in tile) and ms > 0
    b = pyro.Replicas(Ls, betas, pyro.ISING, start="random", seed=4, tile=tile)
    b.sweep(6)
    allm = b.measure_all()
    alls = b.stats_all()
    for r, L in enumerate(Ls):
        o = oracle.Oracle(L, oracle.ISING, pyro.replica_seed(4, r), "random")
        o.sweep(betas[r], 6)
        assert (b.spins(r) == o.spins()).all()
        assert tuple(allm[r]) == o.measure() == b.measure(r)
        assert alls[r] == o.stats() == b.stats(r)
    b.close()
