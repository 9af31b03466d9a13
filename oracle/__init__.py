"""CPU oracle for the pyrochlore Swendsen-Wang sweep (test infrastructure).

This package is test infrastructure, not part of the product path: only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import it.  It wraps ``pyro_oracle.c`` -- a plain,
single-threaded C implementation written from the paper (Soldatov et al.,
arXiv:1612.08312: Sec. 2 lattice and method, Eq. 1 Hamiltonian, Eq. 2
moment ratio) -- and ``graph_oracle.c`` (the same sweep on any bond list:
Sec. 2 neighbour table, Sec. 3.4 simple-cubic lattice, Sec. 4 dilution)
through ctypes.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "pyro_oracle.c"), os.path.join(_HERE, "graph_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ISING, XY, HEIS = 1, 2, 3


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-Wall", "-o", tmp] + _SRCS + ["-lm"])
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
            L.gorc_new.restype = c.c_void_p
            L.gorc_new.argtypes = [c.c_int64, c.c_int64, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p, c.c_int,
                                   c.c_uint64, c.c_int, c.c_double]
            L.gorc_free.argtypes = [c.c_void_p]
            L.gorc_sweep.restype = c.c_int
            L.gorc_sweep.argtypes = [c.c_void_p, c.c_double, c.c_int64, c.c_void_p]
            L.gorc_measure.argtypes = [c.c_void_p] + [c.POINTER(c.c_double)] * 3 + [c.c_void_p]
            L.gorc_stats.argtypes = [c.c_void_p, c.c_void_p]
            L.gorc_reset_stats.argtypes = [c.c_void_p]
            for name in ("gorc_num_sites", "gorc_num_bonds"):
                getattr(L, name).restype = c.c_int64
                getattr(L, name).argtypes = [c.c_void_p]
            L.gorc_get_sweep.restype = c.c_uint64
            L.gorc_get_sweep.argtypes = [c.c_void_p]
            L.gorc_set_sweep.argtypes = [c.c_void_p, c.c_uint64]
            for name in ("gorc_get_labels", "gorc_get_active", "gorc_get_axis", "gorc_get_spins",
                         "gorc_set_spins"):
                getattr(L, name).argtypes = [c.c_void_p, c.c_void_p]
            L.gorc_edges_from_table.restype = c.c_int64
            L.gorc_edges_from_table.argtypes = [c.c_int64, c.c_int, c.c_void_p, c.c_void_p, c.c_void_p]
            L.gorc_sc_edges.restype = c.c_int
            L.gorc_sc_edges.argtypes = [c.c_int, c.c_void_p, c.c_void_p]
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


# ---------------------------------------------------------------- graphs --

def sc_edges(L: int):
    """Bond list of the periodic simple-cubic L^3 lattice (bond 3 i + d)."""
    N = L ** 3
    bi = np.zeros(3 * N, dtype=np.int32)
    bj = np.zeros(3 * N, dtype=np.int32)
    if lib().gorc_sc_edges(L, _ptr(bi), _ptr(bj)) != 0:
        raise ValueError("simple-cubic lattice needs L >= 2")
    return bi, bj


def edges_from_table(nbr: np.ndarray):
    """Bond list of a symmetric neighbour table (N x z, -1 = none): slot
    (i, k) with i < nbr[i, k], in the order of (i, k)."""
    t = np.ascontiguousarray(nbr, dtype=np.int32)
    N, z = t.shape
    E = int(lib().gorc_edges_from_table(N, z, _ptr(t), None, None))
    if E < 0:
        raise ValueError("neighbour table is out of range, has a self entry, or is not symmetric")
    bi = np.zeros(max(E, 1), dtype=np.int32)
    bj = np.zeros(max(E, 1), dtype=np.int32)
    lib().gorc_edges_from_table(N, z, _ptr(t), _ptr(bi), _ptr(bj))
    return bi[:E], bj[:E]


def pyrochlore_edges(L: int):
    """The pyrochlore lattice's bonds as a list whose position is each
    bond's random-number id, so that the graph sweep on it runs the
    pyrochlore chain of the same seed."""
    o = Oracle(L, ISING, 0)
    bi, bj = o.bonds()
    ids = np.array([bond_rng_id(b) for b in range(len(bi))], dtype=np.int64)
    order = np.argsort(ids)
    return bi[order].copy(), bj[order].copy()


class GraphOracle:
    """Swendsen-Wang on an arbitrary bond list (model 1 Ising, 2 XY, 3
    Heisenberg), with optional site and bond masks (dilution)."""

    def __init__(self, N: int, bi, bj, model: int, seed: int, start: str = "up", J: float = 1.0,
                 site_mask=None, edge_mask=None):
        self._lib = lib()
        self.N, self.model, self.ncomp, self.seed, self.J = N, model, model, seed, J
        self._bi = np.ascontiguousarray(bi, dtype=np.int32)
        self._bj = np.ascontiguousarray(bj, dtype=np.int32)
        self.NB = len(self._bi)
        sm = None if site_mask is None else np.ascontiguousarray(site_mask, dtype=np.uint8)
        em = None if edge_mask is None else np.ascontiguousarray(edge_mask, dtype=np.uint8)
        self.h = self._lib.gorc_new(N, self.NB, _ptr(self._bi), _ptr(self._bj),
                                    None if sm is None else _ptr(sm), None if em is None else _ptr(em),
                                    model, seed, 1 if start == "random" else 0, J)
        if not self.h:
            raise ValueError("graph oracle rejected its arguments")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._lib.gorc_free(h)
            self.h = None

    def sweep(self, beta: float, n: int = 1, trace: bool = False):
        buf = np.zeros((n, 4), dtype=np.float64) if trace else None
        if self._lib.gorc_sweep(self.h, beta, n, _ptr(buf) if trace else None) != 0:
            raise ValueError("graph oracle sweep rejected its arguments")
        return buf

    def measure(self):
        E, m2, m4 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        M = np.zeros(3, dtype=np.float64)
        self._lib.gorc_measure(self.h, ctypes.byref(E), ctypes.byref(m2), ctypes.byref(m4), _ptr(M))
        return E.value, m2.value, m4.value

    def magnetization(self) -> np.ndarray:
        E, m2, m4 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        M = np.zeros(3, dtype=np.float64)
        self._lib.gorc_measure(self.h, ctypes.byref(E), ctypes.byref(m2), ctypes.byref(m4), _ptr(M))
        return M[: self.ncomp]

    def stats(self) -> dict:
        out = np.zeros(6, dtype=np.float64)
        self._lib.gorc_stats(self.h, _ptr(out))
        return dict(count=int(out[0]), sum_E=out[1], sum_E2=out[2], sum_m2=out[3], sum_m4=out[4],
                    sum_absm=out[5])

    def reset_stats(self):
        self._lib.gorc_reset_stats(self.h)

    @property
    def sweep_count(self) -> int:
        return int(self._lib.gorc_get_sweep(self.h))

    @sweep_count.setter
    def sweep_count(self, s: int):
        self._lib.gorc_set_sweep(self.h, s)

    def spins(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.int8) if self.model == ISING else np.zeros((self.N, self.ncomp))
        self._lib.gorc_get_spins(self.h, _ptr(out))
        return out

    def set_spins(self, s: np.ndarray):
        if self.model == ISING:
            a = np.ascontiguousarray(s, dtype=np.int8).reshape(self.N)
        else:
            a = np.ascontiguousarray(s, dtype=np.float64).reshape(self.N, self.ncomp)
        self._lib.gorc_set_spins(self.h, _ptr(a))

    def labels(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.int32)
        self._lib.gorc_get_labels(self.h, _ptr(out))
        return out

    def active(self) -> np.ndarray:
        out = np.zeros(max(self.NB, 1), dtype=np.uint8)
        self._lib.gorc_get_active(self.h, _ptr(out))
        return out[: self.NB]

    def axis(self) -> np.ndarray:
        out = np.zeros(3, dtype=np.float64)
        self._lib.gorc_get_axis(self.h, _ptr(out))
        return out[: self.ncomp]
