"""Ising parity: the CUDA sweep against the oracle, bit for bit.

After every sweep the spins, the canonical cluster labels (minimum site
index of each cluster) and the measurement (E, m^2, m^4 of Eq. 1-2) must be
identical, and so must the compensated accumulators, which both sides sum in
sweep order.  Sizes span one tile up to many tiles with ragged tile shapes,
every legal tile edge, both starts, beta = 0 (no bond active) and beta large
(one cluster)."""
import numpy as np
import pytest

import oracle
import paper_1612_08312_gb300 as pyro
import workloads

pytestmark = pytest.mark.gpu


def run_pair(L, T, seed, start, sweeps, tile=(0, 0, 0), per_sweep=True):
    beta = 0.0 if T == float("inf") else (1.0 / T if T > 0 else 1e3)
    o = oracle.Oracle(L, oracle.ISING, seed, start)
    g = pyro.Lattice(L, pyro.ISING, seed, start=start, tile=tile)
    assert (g.spins() == o.spins()).all()
    for s in range(sweeps):
        o.sweep(beta, 1)
        g.sweep(beta, 1)
        if per_sweep or s == sweeps - 1:
            assert (g.spins() == o.spins()).all(), f"spins differ after sweep {s}"
            assert (g.labels() == o.labels()).all(), f"labels differ after sweep {s}"
            assert g.measure() == o.measure()
    so, sg = o.stats(), g.stats()
    assert sg == so
    return o, g


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("start", ["up", "random"])
def test_small_lattices_every_sweep(L, start):
    run_pair(L, 4.21394, seed=L * 7 + 1, start=start, sweeps=6)


@pytest.mark.parametrize("tile", [(1, 1, 1), (2, 2, 2), (4, 2, 1), (2, 4, 8), (8, 8, 4), (8, 8, 8), (16, 8, 4),
                                  (16, 16, 2)])
def test_tile_shapes(tile):
    run_pair(16, 4.21394, seed=3, start="random", sweeps=4, tile=tile)


@pytest.mark.parametrize("T", [2.0, 4.0, 4.21394, 4.5, 8.0])
def test_temperatures_l12(T):
    run_pair(12, T, seed=11, start="random", sweeps=5)


def test_l24_many_tiles():
    run_pair(24, 4.21394, seed=5, start="random", sweeps=3)


def test_l48_many_sweeps_near_tc():
    # 216 tiles of 512 cells, every sweep compared (rare interleavings of
    # the shared-memory union-find must never change a label)
    run_pair(48, 4.21394, seed=17, start="random", sweeps=8)


def test_tile_over_512_cells_is_rejected():
    with pytest.raises(pyro.PyroError) as ei:
        pyro.Lattice(16, pyro.ISING, 1, tile=(16, 16, 4))
    assert ei.value.code == pyro.E_INVAL


def test_beta_zero_has_no_active_bond():
    o, g = run_pair(4, float("inf"), seed=2, start="random", sweeps=3)
    assert (g.labels() == np.arange(g.N)).all()


def test_large_beta_single_cluster():
    o, g = run_pair(8, 0.0, seed=2, start="up", sweeps=3)
    assert (g.labels() == 0).all()
    E, m2, m4 = g.measure()
    assert E == -3.0 * g.N and m2 == 1.0 and m4 == 1.0


def test_multi_sweep_calls_and_graph_chunks_match():
    # a long call runs through captured CUDA graphs; the trajectory must be
    # the same chain as one-sweep calls
    L, T, seed = 8, 4.21394, 9
    o = oracle.Oracle(L, oracle.ISING, seed, "random")
    g = pyro.Lattice(L, pyro.ISING, seed, start="random")
    o.sweep(1 / T, 70)
    g.sweep(1 / T, 70)
    assert (g.spins() == o.spins()).all()
    assert (g.labels() == o.labels()).all()
    assert g.stats() == o.stats()
    assert g.sweep_count == 70


def test_checkpoint_resume_is_bit_exact():
    L, T = 8, 4.21394
    a = pyro.Lattice(L, pyro.ISING, 4, start="random")
    a.sweep(1 / T, 10)
    s = a.spins()
    k = a.sweep_count
    a.sweep(1 / T, 10)
    b = pyro.Lattice(L, pyro.ISING, 4, start="up")
    b.set_spins(s)
    b.sweep_count = k
    b.sweep(1 / T, 10)
    assert (a.spins() == b.spins()).all()
    assert (a.labels() == b.labels()).all()


def test_trace_records_each_sweep():
    L, T = 4, 4.21394
    o = oracle.Oracle(L, oracle.ISING, 8, "random")
    g = pyro.Lattice(L, pyro.ISING, 8, start="random")
    pyro.pyro_set_trace(g.h, 16)
    g.sweep(1 / T, 40)
    tr = o.sweep(1 / T, 40, trace=True)
    got = pyro.pyro_get_trace(g.h, 100)
    assert got.shape == (16, 4)
    assert (got == tr[-16:]).all()


def test_config_l8_workload_first_sweeps():
    cfg = workloads.ISING_L8
    run_pair(cfg["L"], cfg["T"][0], seed=cfg["seed"], start=cfg["start"], sweeps=20, per_sweep=False)
