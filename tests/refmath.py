"""Independent brute-force mathematics used to pin the oracle.

Nothing here calls the oracle or the CUDA library.  Everything is numpy /
scipy written from textbook definitions:
  - the pyrochlore lattice as the bond midpoints of the diamond lattice;
  - exact Boltzmann averages of the L = 1 Ising cell by enumerating all
    2^16 states (Eq. 1 Hamiltonian, Eq. 2 moments);
  - closed forms for independent unit n-vectors (beta = 0);
  - a Metropolis sampler for n-vector spins (a different Markov chain with
    the same stationary distribution as Swendsen-Wang);
  - cuRAND's Philox4x32-10, called on the host from the CUDA toolkit header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- lattice --
def diamond_midpoint_positions(L: int) -> np.ndarray:
    """Pyrochlore sites as midpoints of the diamond-lattice bonds, in units of
    1/8 of the cubic cell (so all coordinates are integers), periodic mod 8L.

    Diamond = FCC (cell edge 8 in these units: points 8c + {0,(0,4,4),(4,0,4),
    (4,4,0)}) plus a second FCC shifted by (2,2,2).  Each first-sublattice atom
    has four bonds along (+-1,+-1,+-1)*2 with an even number of minus signs;
    their midpoints are at offsets (1,1,1), (1,-1,-1), (-1,1,-1), (-1,-1,1)."""
    fcc = np.array([[0, 0, 0], [0, 4, 4], [4, 0, 4], [4, 4, 0]])
    mids = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]])
    pts = []
    for z in range(L):
        for y in range(L):
            for x in range(L):
                for a in fcc:
                    for m in mids:
                        pts.append(8 * np.array([x, y, z]) + a + m)
    return np.mod(np.array(pts), 8 * L)


def brute_force_neighbours(pos: np.ndarray, period: int) -> list[set]:
    """All pairs at the minimum periodic distance, by O(N^2) search."""
    d = pos[:, None, :] - pos[None, :, :]
    d = (d + period // 2) % period - period // 2
    # when the period is small, also try the other images
    r2 = np.full(d.shape[:2], np.iinfo(np.int64).max, dtype=np.int64)
    for sx in (-period, 0, period):
        for sy in (-period, 0, period):
            for sz in (-period, 0, period):
                dd = d + np.array([sx, sy, sz])
                r2 = np.minimum(r2, (dd * dd).sum(-1))
    np.fill_diagonal(r2, np.iinfo(np.int64).max)
    dmin = r2.min()
    return [set(np.nonzero(r2[i] == dmin)[0].tolist()) for i in range(len(pos))], dmin


# ------------------------------------------------------------ enumeration --
def enumerate_ising(bonds_i: np.ndarray, bonds_j: np.ndarray, N: int, beta: float):
    """Exact <E>, <m^2>, <m^4> of the Ising model on a graph of N <= 20
    sites by summing over all 2^N states (H of Eq. 1 with J = 1)."""
    states = np.arange(2 ** N, dtype=np.int64)
    sig = 1 - 2 * ((states[:, None] >> np.arange(N)) & 1)
    E = -(sig[:, bonds_i] * sig[:, bonds_j]).sum(1).astype(np.float64)
    M = sig.sum(1).astype(np.float64)
    logw = -beta * E
    w = np.exp(logw - logw.max())
    Z = w.sum()
    m = np.abs(M) / N
    return dict(E=(w * E).sum() / Z, E2=(w * E * E).sum() / Z, m2=(w * m ** 2).sum() / Z,
                m4=(w * m ** 4).sum() / Z)


def independent_moments(N: int, n: int):
    """<m^2>, <m^4> of N independent uniform unit n-vectors (beta = 0):
    <M.M> = N, <(M.M)^2> = N^2 + 2 N (N - 1) / n."""
    m2 = 1.0 / N
    m4 = (N * N + 2.0 * N * (N - 1) / n) / N ** 4
    return m2, m4


# ------------------------------------------------------------- statistics --
def binned_mean_se(x: np.ndarray, nbins: int = 50):
    """Mean and standard error from nbins consecutive bins (autocorrelation
    shorter than a bin)."""
    x = np.asarray(x, dtype=np.float64)
    nb = len(x) // nbins
    b = x[: nb * nbins].reshape(nbins, nb).mean(1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nbins)


def jackknife_ratio(m2: np.ndarray, m4: np.ndarray, nbins: int = 50):
    """U = <m^4>/<m^2>^2 (Eq. 2) with its jackknife error over nbins bins."""
    nb = len(m2) // nbins
    b2 = m2[: nb * nbins].reshape(nbins, nb).mean(1)
    b4 = m4[: nb * nbins].reshape(nbins, nb).mean(1)
    U = b4.mean() / b2.mean() ** 2
    s2, s4 = b2.sum(), b4.sum()
    Uj = ((s4 - b4) / (nbins - 1)) / ((s2 - b2) / (nbins - 1)) ** 2
    err = np.sqrt((nbins - 1) / nbins * ((Uj - Uj.mean()) ** 2).sum())
    return U, err


# -------------------------------------------------------------- Metropolis --
def metropolis_nvector(nbr: np.ndarray, n: int, beta: float, chains: int, sweeps: int,
                       burn: int, seed: int):
    """Single-site Metropolis for unit n-vectors on a graph given by its
    neighbour table nbr (N x z), run on `chains` independent chains in
    parallel.  Proposal: a fresh uniform unit vector (symmetric).  Returns the
    per-sweep chain averages of E, m^2, m^4."""
    rng = np.random.default_rng(seed)
    N = nbr.shape[0]

    def unit(size):
        v = rng.standard_normal(size + (n,))
        return v / np.linalg.norm(v, axis=-1, keepdims=True)

    s = unit((chains, N))
    out = []
    ar = np.arange(chains)
    for t in range(burn + sweeps):
        for i in range(N):
            h = s[:, nbr[i], :].sum(1)
            new = unit((chains,))
            dE = -((new - s[:, i, :]) * h).sum(-1)
            acc = rng.random(chains) < np.exp(np.minimum(0.0, -beta * dE))
            s[ar[acc], i, :] = new[acc]
        if t >= burn:
            E = -0.5 * (s[:, :, None, :] * s[:, nbr, :]).sum((-1, -2, -3))
            m = np.linalg.norm(s.sum(1), axis=-1) / N
            out.append((E, m ** 2, m ** 4))
    return np.array(out)  # (sweeps, 3, chains)


# -------------------------------------------------------- cuRAND Philox ----
_probe = None


def curand_philox_lib():
    """Build (once) and load a host shared library that calls cuRAND's
    curand_Philox4x32_10 from the CUDA toolkit header.  Returns None when
    nvcc is not available."""
    global _probe
    if _probe is not None:
        return _probe
    src = os.path.join(HERE, "helpers", "curand_philox_probe.cu")
    out_dir = tempfile.mkdtemp(prefix="philox_probe_")
    so = os.path.join(out_dir, "probe.so")
    nvcc = os.environ.get("NVCC", "nvcc")
    try:
        subprocess.check_call([nvcc, "-shared", "-Xcompiler", "-fPIC", "-o", so, src],
                              stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    except (OSError, subprocess.CalledProcessError):
        return None
    lib = ctypes.CDLL(so)
    lib.probe_philox.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_long]
    _probe = lib
    return lib


def curand_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Batched cuRAND Philox4x32-10: ctr (n,4) uint32, key (n,2) uint32."""
    lib = curand_philox_lib()
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.zeros_like(ctr)
    lib.probe_philox(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, len(ctr))
    return out


def _stream_calls(seed: int, sweep_field: int, tag: int, j: np.ndarray) -> np.ndarray:
    j = np.asarray(j, dtype=np.uint64)
    ctr = np.stack([(j & np.uint64(0xFFFFFFFF)).astype(np.uint32),
                    (j >> np.uint64(32)).astype(np.uint32),
                    np.full(len(j), sweep_field, dtype=np.uint32),
                    np.full(len(j), tag, dtype=np.uint32)], 1)
    key = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32), (len(j), 1))
    return curand_philox(ctr, key)


def stream_bytes(seed: int, sweep_field: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """Byte x of a (seed, sweep, tag) stream via cuRAND: byte x & 15 (bits
    8 (x & 3) and up of output word (x & 15) >> 2) of call x >> 4."""
    idx = np.asarray(idx, dtype=np.uint64)
    out = _stream_calls(seed, sweep_field, tag, idx >> np.uint64(4))
    t = (idx & np.uint64(15)).astype(np.int64)
    w = out[np.arange(len(idx)), t >> 2]
    return ((w >> (8 * (t & 3)).astype(np.uint32)) & np.uint32(0xFF)).astype(np.uint32)


def stream_words(seed: int, sweep_field: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """Word x of a stream via cuRAND: output word x & 3 of call x >> 2."""
    idx = np.asarray(idx, dtype=np.uint64)
    out = _stream_calls(seed, sweep_field, tag, idx >> np.uint64(2))
    return out[np.arange(len(idx)), (idx & np.uint64(3)).astype(np.int64)]


def stream_bits(seed: int, sweep_field: int, tag: int, idx: np.ndarray) -> np.ndarray:
    """Bit x of a stream via cuRAND: bit x & 31 of output word (x & 127) >> 5
    of call x >> 7."""
    idx = np.asarray(idx, dtype=np.uint64)
    out = _stream_calls(seed, sweep_field, tag, idx >> np.uint64(7))
    t = (idx & np.uint64(127)).astype(np.int64)
    w = out[np.arange(len(idx)), t >> 5]
    return ((w >> (t & 31).astype(np.uint32)) & np.uint32(1)).astype(np.uint32)


# Random-number id of bond 12 r + k: 48 c + 16 g + 4 f + q (r = 4 c + f), with
# (g, q) per pair k: up (0,1) (0,2) (0,3) (1,2) (1,3) (2,3), then down likewise.
RNG_G = np.array([0, 1, 0, 0, 1, 0, 2, 1, 2, 2, 1, 2])
RNG_Q = np.array([0, 0, 3, 1, 1, 2, 0, 2, 3, 1, 3, 2])


def bond_rng_ids(nbonds: int) -> np.ndarray:
    b = np.arange(nbonds, dtype=np.int64)
    r, k = b // 12, b % 12
    return (48 * (r >> 2) + 16 * RNG_G[k] + 4 * (r & 3) + RNG_Q[k]).astype(np.uint64)


def bond_rng_ids_of(b: np.ndarray) -> np.ndarray:
    b = np.asarray(b, dtype=np.int64)
    r, k = b // 12, b % 12
    return (48 * (r >> 2) + 16 * RNG_G[k] + 4 * (r & 3) + RNG_Q[k]).astype(np.uint64)


def bond_words_of(seed: int, sweep: int, bonds: np.ndarray) -> np.ndarray:
    """32-bit uniforms of the given bonds 12 r + k."""
    ids = bond_rng_ids_of(bonds)
    hi = stream_bytes(seed, sweep, 1, ids).astype(np.uint64)
    lo = stream_words(seed, sweep, 5, ids).astype(np.uint64) & np.uint64(0xFFFFFF)
    return (hi << np.uint64(24)) | lo


def bond_words(seed: int, sweep: int, nbonds: int) -> np.ndarray:
    """32-bit uniform of each bond 12 r + k: its id's BOND-stream byte as the
    top 8 bits, the low 24 bits of its TIE-stream word (tag 5) below."""
    ids = bond_rng_ids(nbonds)
    hi = stream_bytes(seed, sweep, 1, ids).astype(np.uint64)
    lo = stream_words(seed, sweep, 5, ids).astype(np.uint64) & np.uint64(0xFFFFFF)
    return (hi << np.uint64(24)) | lo
