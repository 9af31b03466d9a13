"""The allocation-free Ising sweep (pyro_ising_sweep_noalloc).

It exists for callers that must not allocate device memory themselves (a
framework that owns the device memory budget, a plugin barred from
allocating after start-up, a loop where cudaMalloc would stall other
streams): they pass device buffers in and the sweep's scratch lives in a
fixed array inside the library.  Here two calls in a row, through the C ABI,
must give the same spins, canonical labels and measurement as the library's
allocating entry points (pyro_sweep and friends) on the same chain -- the
tolerance of the Ising tests, which is bit-exact equality.

This file is collected last on purpose, so that a run that stops at the
first failure has run every other test first; it also passes when run on
its own in a fresh process."""
import numpy as np
import pytest

import paper_1612_08312_gb300 as pyro

pytestmark = pytest.mark.gpu


def packed(spins_pm1: np.ndarray) -> np.ndarray:
    """+-1 spins in site order -> one uint16 per cell, bit set for -1."""
    bits = (spins_pm1 == -1).astype(np.uint16).reshape(-1, 16)
    return (bits << np.arange(16, dtype=np.uint16)).sum(1).astype(np.uint16)


@pytest.mark.parametrize("L,T,seed", [(8, 4.21394, 3), (12, 4.5, 7), (32, 4.21394, 11)])
def test_noalloc_matches_allocating_entry_points(L, T, seed):
    import torch
    dev = torch.device("cuda", 0)
    beta = 1.0 / T
    ref = pyro.Lattice(L, pyro.ISING, seed, start="random")
    ref.sweep(beta, 3)  # start from an equilibrating configuration at sweep 3
    s0 = ref.spins()
    k0 = ref.sweep_count
    N = 16 * L ** 3
    spins_a = torch.from_numpy(packed(s0).view(np.int16)).to(dev)
    spins_b = torch.empty_like(spins_a)
    labels = torch.empty(N, dtype=torch.int32, device=dev)
    meas = torch.empty(4, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for step in range(2):  # two calls in a row: a -> b, then b -> b in place
        src, dst = (spins_a, spins_b) if step == 0 else (spins_b, spins_b)
        pyro.pyro_ising_sweep_noalloc(src.data_ptr(), dst.data_ptr(), labels.data_ptr(), meas.data_ptr(), L,
                                      beta, seed, k0 + step, stream.cuda_stream)
        ref.sweep(beta, 1)
        got_spins = dst.cpu().numpy().view(np.uint16)
        assert (got_spins == packed(ref.spins())).all(), f"spins differ on call {step}"
        assert (labels.cpu().numpy() == ref.labels()).all(), f"labels differ on call {step}"
        E, m2, m4, M = meas.cpu().numpy().tolist()
        assert (E, m2, m4) == ref.measure(), f"measurement differs on call {step}"
        assert M == float(ref.spins().astype(np.int64).sum())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    p = x.data_ptr()
    with pytest.raises(pyro.PyroError) as ei:
        pyro.pyro_ising_sweep_noalloc(p, p, p, p, pyro.NOALLOC_MAX_L + 1, 0.2, 1, 0, None)
    assert ei.value.code == pyro.E_INVAL
    assert "L must be in" in str(ei.value)


def _packed_device(spins_pm1, dev):
    import torch
    return torch.from_numpy(packed(spins_pm1).view(np.int16)).to(dev)


def test_noalloc_allocates_nothing_and_crosses_the_stamp_wraparound():
    """The links of clusters that cross tile faces carry a per-call stamp in
    the fixed array; before the stamps would wrap, the array's links are
    cleared and the stamps restart.  Two calls taken across that point must
    still match the allocating entry points bit for bit, and a call (after a
    first one has loaded everything it needs) must leave the device's free
    memory unchanged."""
    import torch
    dev = torch.device("cuda", 0)
    L, T, seed = 16, 4.21394, 23
    beta = 1.0 / T
    ref = pyro.Lattice(L, pyro.ISING, seed, start="random")
    ref.sweep(beta, 2)
    k0 = ref.sweep_count
    N = 16 * L ** 3
    spins = _packed_device(ref.spins(), dev)
    labels = torch.empty(N, dtype=torch.int32, device=dev)
    meas = torch.empty(4, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    # a first call on a scratch copy loads every kernel the entry point uses
    # (module loading may take device memory once per process)
    warm = spins.clone()
    pyro.pyro_ising_sweep_noalloc(warm.data_ptr(), warm.data_ptr(), labels.data_ptr(), meas.data_ptr(), L, beta, seed,
                                  0, stream.cuda_stream)
    try:
        pyro.pyro_debug_set(pyro.DEBUG_NOALLOC_STAMP, 0xFFFFFFEF)
        for step in range(2):  # stamps 0xFFFFFFF0, then cleared links and stamp 1
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info(dev)[0]
            pyro.pyro_ising_sweep_noalloc(spins.data_ptr(), spins.data_ptr(), labels.data_ptr(), meas.data_ptr(), L,
                                          beta, seed, k0 + step, stream.cuda_stream)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info(dev)[0]
            assert free1 == free0, "the call changed the device's free memory"
            ref.sweep(beta, 1)
            assert (spins.cpu().numpy().view(np.uint16) == packed(ref.spins())).all(), f"spins differ on call {step}"
            assert (labels.cpu().numpy() == ref.labels()).all(), f"labels differ on call {step}"
    finally:
        pyro.pyro_debug_set(pyro.DEBUG_NOALLOC_STAMP, 0)
    ref.close()


def test_noalloc_rejects_partially_overlapping_spin_buffers():
    import torch
    L = 4
    buf = torch.zeros(2 * L ** 3, dtype=torch.int16, device="cuda")
    x = torch.zeros(16 * L ** 3 + 8, dtype=torch.int32, device="cuda")
    with pytest.raises(pyro.PyroError) as ei:
        pyro.pyro_ising_sweep_noalloc(buf.data_ptr(), buf.data_ptr() + 2, x.data_ptr(), x.data_ptr(), L, 0.2, 1, 0,
                                      None)
    assert ei.value.code == pyro.E_INVAL
    assert "overlap" in str(ei.value)
