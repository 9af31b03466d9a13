"""CPU oracle for the pyrochlore Swendsen-Wang sweep (test infrastructure).

This package is test infrastructure, not part of the product path: only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import it.  It wraps ``pyro_oracle.c`` -- a plain,
single-threaded C implementation written from the paper (Soldatov et al.,
arXiv:1612.08312: Sec. 2 lattice and method, Eq. 1 Hamiltonian, Eq. 2
moment ratio) -- through ctypes.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pyro_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ISING, XY, HEIS = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            c = ctypes
            L.orc_new.restype = c.c_void_p
            L.orc_new.argtypes = [c.c_int, c.c_int, c.c_uint64, c.c_int, c.c_double]
            L.orc_free.argtypes = [c.c_void_p]
            L.orc_sweep.restype = c.c_int
            L.orc_sweep.argtypes = [c.c_void_p, c.c_double, c.c_int64, c.c_void_p]
            L.orc_measure.argtypes = [c.c_void_p] + [c.POINTER(c.c_double)] * 3 + [c.c_void_p]
            L.orc_stats.argtypes = [c.c_void_p, c.c_void_p]
            L.orc_reset_stats.argtypes = [c.c_void_p]
            L.orc_num_sites.restype = c.c_int64
            L.orc_num_sites.argtypes = [c.c_void_p]
            L.orc_get_sweep.restype = c.c_uint64
            L.orc_get_sweep.argtypes = [c.c_void_p]
            L.orc_set_sweep.argtypes = [c.c_void_p, c.c_uint64]
            for name in ("orc_get_axis", "orc_get_labels", "orc_get_active", "orc_get_nn",
                         "orc_get_spins", "orc_set_spins"):
                getattr(L, name).argtypes = [c.c_void_p, c.c_void_p]
            L.orc_get_bonds.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p]
            L.orc_philox.argtypes = [c.c_void_p, c.c_void_p, c.c_void_p]
            L.orc_bond_word.restype = c.c_uint32
            L.orc_bond_word.argtypes = [c.c_uint64, c.c_uint32, c.c_uint64]
            L.orc_bond_rng_id.restype = c.c_uint64
            L.orc_bond_rng_id.argtypes = [c.c_uint64]
            L.orc_threshold.restype = c.c_uint64
            L.orc_threshold.argtypes = [c.c_double, c.c_double]
            L.orc_unit_vector.restype = c.c_int
            L.orc_unit_vector.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint64, c.c_int,
                                          c.c_void_p]
            L.orc_clusters.restype = c.c_int
            L.orc_clusters.argtypes = [c.c_int64, c.c_int64, c.c_void_p, c.c_void_p, c.c_void_p,
                                       c.c_void_p]
            L.orc_build_nn.restype = c.c_int
            L.orc_build_nn.argtypes = [c.c_int, c.c_void_p]
            L.orc_site_position.argtypes = [c.c_int, c.c_int64, c.c_void_p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(counter, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def bond_word(seed: int, sweep: int, b: int) -> int:
    """The 32-bit uniform of the bond with random-number id b in a sweep."""
    return int(lib().orc_bond_word(seed, sweep, b))


def bond_rng_id(bond: int) -> int:
    """Random-number id of bond 12 r + k."""
    return int(lib().orc_bond_rng_id(bond))


def threshold(beta: float, J: float = 1.0) -> int:
    return int(lib().orc_threshold(beta, J))


def unit_vector(seed: int, sweep_field: int, tag: int, call_base: int, n: int):
    r = np.zeros(3, dtype=np.float64)
    att = lib().orc_unit_vector(seed, sweep_field, tag, call_base, n, _ptr(r))
    return r[:n].copy(), att


def clusters(nsites: int, bi: np.ndarray, bj: np.ndarray, active: np.ndarray) -> np.ndarray:
    bi = np.ascontiguousarray(bi, dtype=np.int32)
    bj = np.ascontiguousarray(bj, dtype=np.int32)
    act = np.ascontiguousarray(active, dtype=np.uint8)
    lab = np.zeros(nsites, dtype=np.int32)
    lib().orc_clusters(nsites, len(bi), _ptr(bi), _ptr(bj), _ptr(act), _ptr(lab))
    return lab


def site_position(L: int, i: int) -> np.ndarray:
    p = np.zeros(3, dtype=np.int32)
    lib().orc_site_position(L, i, _ptr(p))
    return p


class Oracle:
    """One pyrochlore lattice of n-vector spins (model 1 Ising, 2 XY, 3 Heisenberg)."""

    def __init__(self, L: int, model: int, seed: int, start: str = "up", J: float = 1.0):
        self._lib = lib()
        self.L, self.model, self.seed, self.J = L, model, seed, J
        self.ncomp = model
        self.h = self._lib.orc_new(L, model, seed, 1 if start == "random" else 0, J)
        if not self.h:
            raise RuntimeError(f"oracle init failed for L={L} model={model}")
        self.N = int(self._lib.orc_num_sites(self.h))
        self.NB = 3 * self.N

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.orc_free(h)
            self.h = None

    def sweep(self, beta: float, n: int = 1, trace: bool = False):
        buf = np.zeros((n, 4), dtype=np.float64) if trace else None
        rc = self._lib.orc_sweep(self.h, beta, n, _ptr(buf) if trace else None)
        if rc != 0:
            raise ValueError("oracle sweep rejected its arguments")
        return buf

    def measure(self):
        E, m2, m4 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        M = np.zeros(3, dtype=np.float64)
        self._lib.orc_measure(self.h, ctypes.byref(E), ctypes.byref(m2), ctypes.byref(m4), _ptr(M))
        return E.value, m2.value, m4.value

    def magnetization(self) -> np.ndarray:
        E, m2, m4 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        M = np.zeros(3, dtype=np.float64)
        self._lib.orc_measure(self.h, ctypes.byref(E), ctypes.byref(m2), ctypes.byref(m4), _ptr(M))
        return M[: self.ncomp]

    def stats(self) -> dict:
        out = np.zeros(6, dtype=np.float64)
        self._lib.orc_stats(self.h, _ptr(out))
        return dict(count=int(out[0]), sum_E=out[1], sum_E2=out[2], sum_m2=out[3], sum_m4=out[4],
                    sum_absm=out[5])

    def reset_stats(self):
        self._lib.orc_reset_stats(self.h)

    @property
    def sweep_count(self) -> int:
        return int(self._lib.orc_get_sweep(self.h))

    @sweep_count.setter
    def sweep_count(self, s: int):
        self._lib.orc_set_sweep(self.h, s)

    def spins(self) -> np.ndarray:
        if self.model == ISING:
            out = np.zeros(self.N, dtype=np.int8)
        else:
            out = np.zeros((self.N, self.ncomp), dtype=np.float64)
        self._lib.orc_get_spins(self.h, _ptr(out))
        return out

    def set_spins(self, s: np.ndarray):
        if self.model == ISING:
            a = np.ascontiguousarray(s, dtype=np.int8).reshape(self.N)
        else:
            a = np.ascontiguousarray(s, dtype=np.float64).reshape(self.N, self.ncomp)
        self._lib.orc_set_spins(self.h, _ptr(a))

    def labels(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.int32)
        self._lib.orc_get_labels(self.h, _ptr(out))
        return out

    def active(self) -> np.ndarray:
        out = np.zeros(self.NB, dtype=np.uint8)
        self._lib.orc_get_active(self.h, _ptr(out))
        return out

    def axis(self) -> np.ndarray:
        out = np.zeros(3, dtype=np.float64)
        self._lib.orc_get_axis(self.h, _ptr(out))
        return out[: self.ncomp]

    def nn(self) -> np.ndarray:
        out = np.zeros((self.N, 6), dtype=np.int32)
        self._lib.orc_get_nn(self.h, _ptr(out))
        return out

    def bonds(self):
        bi = np.zeros(self.NB, dtype=np.int32)
        bj = np.zeros(self.NB, dtype=np.int32)
        self._lib.orc_get_bonds(self.h, _ptr(bi), _ptr(bj))
        return bi, bj
