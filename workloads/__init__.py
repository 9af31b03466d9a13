"""Seeded synthetic workloads shared by the oracle tests, the CUDA parity
tests and the benchmark.

This module holds no step of the Swendsen-Wang method: only the lattice
sizes, temperatures and sweep counts of the workloads, and numpy-seeded
generators of starting spin configurations that both sides are given as
inputs.  (Random numbers drawn inside a sweep come from each side's own
Philox4x32-10; they are not generated here.)

The workloads are the paper's kind of run (Sec. 2: pyrochlore lattice,
N = 16 L^3, J = 1, periodic boundaries; temperatures around the critical
points of Sec. 3).  There is no dataset.
"""
from __future__ import annotations

import numpy as np

ISING, XY, HEIS = 1, 2, 3

# Critical temperatures reported in the abstract / Sec. 3 (context values).
TC = {ISING: 4.21394, XY: 2.02850, HEIS: 1.31695}


def n_sites(L: int) -> int:
    """Sec. 2: N = 16 L^3."""
    return 16 * L ** 3


ISING_L8 = dict(name="ising_L8", model=ISING, L=8, T=[4.21394], start="up", seed=1,
                equil=1000, sweeps=10000)
ISING_L256 = dict(name="ising_L256", model=ISING, L=256, T=[4.20, 4.21394, 4.23], start="random",
                  seeds=[1, 2, 3], equil=200, sweeps=2000)
ISING_BATCH = dict(name="ising_batch48", model=ISING, L=[16, 24, 32, 48, 64, 96],
                   T=[4.19 + k * 0.05 / 7 for k in range(8)], start="random", seed=1, sweeps=5000)
XY_L64 = dict(name="xy_L64", model=XY, L=64, T=[2.01, 2.0285, 2.05], start="random", seed=1,
              sweeps=3000)
HEIS_BATCH = dict(name="heis_batch24", model=HEIS, L=[32, 64, 128],
                  T=[1.30 + k * 0.03 / 7 for k in range(8)], start="random", seed=1, sweeps=3000)

CONFIGS = [ISING_L8, ISING_L256, ISING_BATCH, XY_L64, HEIS_BATCH]

# Generic lattices (Sec. 2 neighbour table; Sec. 3.4 simple cubic, whose
# critical temperatures the paper quotes: Ising 4.511524, XY 2.20182,
# Heisenberg 1.4430; Sec. 4 dilution).  The simple-cubic L = 640 lattice
# has N = 262,144,000 sites, about the pyrochlore L = 256 lattice's count.
TC_SC = {ISING: 4.511524, XY: 2.20182, HEIS: 1.4430}
SC_L640 = dict(name="sc_L640", model=ISING, L=640, T=TC_SC[ISING], start="random", seed=1)
# site-diluted simple cubic, occupation 0.8, near its transition (T about 3.5)
SC_DIL_L512 = dict(name="sc_dil_L512", model=ISING, L=512, T=3.5, p_site=0.8, mask_seed=7, start="random", seed=1)
# the simple-cubic lattice handed over as an explicit bond list
SC_LIST_L512 = dict(name="sc_list_L512", model=ISING, L=512, T=TC_SC[ISING], start="random", seed=1)
GRAPH_CONFIGS = [SC_L640, SC_DIL_L512, SC_LIST_L512]


def site_mask(N: int, p: float, seed: int) -> np.ndarray:
    """Occupied (1) / vacant (0) sites, i.i.d. with occupation p (PCG64)."""
    return (np.random.default_rng(seed).random(N) < p).astype(np.uint8)


def sc_bond_list(L: int):
    """The periodic simple-cubic L^3 lattice as an explicit bond list (an
    input in the neighbour-table form): site i = x + L (y + L z), bonds
    3 i + d to the next site along +x, +y, +z."""
    i = np.arange(L ** 3, dtype=np.int64)
    x, y, z = i % L, (i // L) % L, i // (L * L)
    nb = np.stack([(x + 1) % L + L * (y + L * z), x + L * ((y + 1) % L + L * z),
                   x + L * (y + L * ((z + 1) % L))], axis=1)
    return np.repeat(i, 3).astype(np.int32), nb.reshape(-1).astype(np.int32)


def batch_replicas(cfg: dict):
    """(L, T) of every replica of a batched workload, L-major."""
    return [(L, T) for L in cfg["L"] for T in cfg["T"]]


def random_ising(N: int, seed: int) -> np.ndarray:
    """i.i.d. +-1 spins (int8) from numpy's PCG64."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random(N) < 0.5, 1, -1).astype(np.int8)


def random_unit_vectors(N: int, n: int, seed: int, fp32_exact: bool = True) -> np.ndarray:
    """N unit n-vectors uniform on the sphere (normalised Gaussians), shape
    (N, n), float64.  With fp32_exact every entry is rounded to the nearest
    float32 so that an FP32 and an FP64 consumer start from identical values."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((N, n))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    if fp32_exact:
        v = v.astype(np.float32).astype(np.float64)
    return v
