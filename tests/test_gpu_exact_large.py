"""Bit-exact oracle parity at the workloads' own sizes.

The smaller parity tests stop at L = 48.  Here the CUDA sweep is compared
with the oracle, sweep by sweep, on the lattices the benchmark workloads
run: the L = 64 and L = 96 replicas of the batched Ising workload, L = 128,
and the L = 256 headline lattice in the benchmark's launch configurations
(default tile and the 8 x 8 x 8 tile the autotuner picks); one FP64 XY sweep
at L = 64; and one FP64 Heisenberg replica at L = 64 inside a batch.

Ising: spins, canonical cluster labels and (E, m^2, m^4) identical after
every sweep.  n-vector FP64: labels identical, spins and E within 1e-12.
The oracle runs at about 0.01 site updates per ns on one core, so the L =
256 case costs a few minutes of host time and about 15 GB of host memory."""
import numpy as np
import pytest

import oracle
import paper_1612_08312_gb300 as pyro
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def ising_exact(L, T, seed, sweeps, tile=(0, 0, 0)):
    beta = 1.0 / T
    o = oracle.Oracle(L, oracle.ISING, seed, "random")
    g = pyro.Lattice(L, pyro.ISING, seed, start="random", tile=tile)
    assert (g.spins() == o.spins()).all()
    for s in range(sweeps):
        o.sweep(beta, 1)
        g.sweep(beta, 1)
        assert (g.spins() == o.spins()).all(), f"spins differ after sweep {s}"
        assert (g.labels() == o.labels()).all(), f"labels differ after sweep {s}"
        assert g.measure() == o.measure(), f"measurement differs after sweep {s}"
    assert g.stats() == o.stats()
    g.close()


@pytest.mark.parametrize("L,T", [(64, 4.19), (64, 4.21394), (96, 4.24)])
def test_ising_batch_sizes(L, T):
    ising_exact(L, T, seed=31 + L, sweeps=3)


def test_ising_l128():
    ising_exact(128, 4.21394, seed=7, sweeps=2)


@pytest.mark.parametrize("tile", [(0, 0, 0), (8, 8, 8)])
def test_ising_l256_headline(tile):
    cfg = workloads.ISING_L256
    ising_exact(cfg["L"], cfg["T"][1], seed=cfg["seeds"][0], sweeps=2, tile=tile)


def test_xy_fp64_l64():
    L, T, seed = 64, 2.0285, 3
    o = oracle.Oracle(L, oracle.XY, seed, "random")
    g = pyro.Lattice(L, pyro.XY, seed, precision=pyro.FP64, start="random")
    o.sweep(1 / T, 1)
    g.sweep(1 / T, 1)
    assert (g.labels() == o.labels()).all()
    assert np.abs(g.spins() - o.spins()).max() <= 1e-12
    Eg, _, _ = g.measure()
    Eo, _, _ = o.measure()
    assert abs(Eg - Eo) <= 1e-12 * abs(Eo)
    g.close()


def test_heisenberg_fp64_batch_replica_l64():
    Ls, Ts = [32, 64], [1.30, 1.3171]
    b = pyro.Replicas(Ls, [1 / T for T in Ts], pyro.HEIS, precision=pyro.FP64, start="random", seed=11)
    b.sweep(1)
    o = oracle.Oracle(64, oracle.HEIS, pyro.replica_seed(11, 1), "random")
    o.sweep(1 / Ts[1], 1)
    assert np.abs(b.spins(1) - o.spins()).max() <= 1e-12
    E, _, _ = b.measure(1)
    Eo, _, _ = o.measure()
    assert abs(E - Eo) <= 1e-12 * abs(Eo)
    b.close()
