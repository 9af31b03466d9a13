"""Failure handling without faulting the GPU: simulated allocation failure
on the host, and a union-find bound lowered to zero so that the kernels'
bounded loops give up at once and report through the device status word."""
import numpy as np
import pytest

import oracle
import paper_1612_08312_gb300 as pyro

pytestmark = pytest.mark.gpu


def test_allocation_failure_is_reported_and_leaves_no_state():
    for k in (1, 3, 6):
        pyro.pyro_debug_set(pyro.DEBUG_FAIL_ALLOCS, k)
        with pytest.raises(pyro.PyroError) as ei:
            pyro.Lattice(8, pyro.ISING, 1)
        assert ei.value.code == pyro.E_NOMEM
    pyro.pyro_debug_set(pyro.DEBUG_FAIL_ALLOCS, 0)
    g = pyro.Lattice(8, pyro.ISING, 1, start="random")
    o = oracle.Oracle(8, oracle.ISING, 1, "random")
    g.sweep(0.2, 3)
    o.sweep(0.2, 3)
    assert (g.spins() == o.spins()).all()


def test_union_bound_exhaustion_reports_noconverge():
    g = pyro.Lattice(8, pyro.ISING, 2, start="random")
    try:
        pyro.pyro_debug_set(pyro.DEBUG_UNITE_BOUND, 0)
        g.sweep(1 / 4.21394, 2)
        with pytest.raises(pyro.PyroError) as ei:
            g.sync()
        assert ei.value.code == pyro.E_NOCONVERGE
    finally:
        pyro.pyro_debug_set(pyro.DEBUG_UNITE_BOUND, 4096)
    h = pyro.Lattice(8, pyro.ISING, 2, start="random")
    o = oracle.Oracle(8, oracle.ISING, 2, "random")
    h.sweep(1 / 4.21394, 2)
    o.sweep(1 / 4.21394, 2)
    assert (h.spins() == o.spins()).all() and (h.labels() == o.labels()).all()


@pytest.mark.parametrize("model", [1, 2])
def test_autotuned_tile_is_valid_and_exact(model):
    tile, ms = pyro.pyro_autotune(16, model, pyro.FP64, 0.25, 2)
    assert all(16 % t == 0 for t in tile) and ms > 0
    g = pyro.Lattice(16, model, 3, precision=pyro.FP64, start="random", tile=tile)
    o = oracle.Oracle(16, model, 3, "random")
    g.sweep(0.25, 2)
    o.sweep(0.25, 2)
    assert (g.labels() == o.labels()).all()
    assert np.abs(g.spins().astype(np.float64) - o.spins()).max() <= 1e-12


def test_chain_crosses_the_link_stamp_wraparound():
    """Links of clusters that cross tile faces are stamped with a per-sweep
    epoch; before the 32-bit stamps would wrap, every link array is cleared
    and the epochs restart.  A lattice started just below that point must
    follow the oracle's chain bit for bit through it, with single sweeps and
    with a multi-sweep call."""
    try:
        pyro.pyro_debug_set(pyro.DEBUG_EPOCH_START, 0xFFFFFFF0 - 3)
        g = pyro.Lattice(16, pyro.ISING, 9, start="random")
    finally:
        pyro.pyro_debug_set(pyro.DEBUG_EPOCH_START, 0)
    o = oracle.Oracle(16, oracle.ISING, 9, "random")
    for n in (1, 1, 1, 1, 1, 3, 40):
        g.sweep(1 / 4.21394, n)
        o.sweep(1 / 4.21394, n)
        assert (g.spins() == o.spins()).all()
        assert (g.labels() == o.labels()).all()
    g.close()
