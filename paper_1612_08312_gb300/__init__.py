"""GB300-native Swendsen-Wang sweeps on the pyrochlore lattice.

A thin ctypes binding of libpyro (include/pyro.h), the CUDA library that
runs the whole sweep on the GPU: bond activation, connected-component
labelling, cluster flips and the E / m^2 / m^4 reductions of Soldatov,
Nefedev, Komura and Okabe (arXiv:1612.08312, Sec. 2, Eq. 1-2).

The functions below carry the C names and only marshal arguments; every step
of a sweep runs in the library's kernels.  There is no CPU fallback: if the
library cannot be built or loaded, importing raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ISING, XY, HEIS = 1, 2, 3
FP32, FP64 = 0, 1
START_UP, START_RANDOM = 0, 1

OK, E_INVAL, E_NOMEM, E_CUDA, E_NOCONVERGE, E_TIMEOUT, E_STATE = 0, -1, -2, -3, -4, -5, -6
MAX_L = 511
MAX_REPS = 64

_lock = threading.Lock()
_lib = None


class PyroError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pyro error {code}: {msg}")
        self.code = code


class pyro_config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("model", ctypes.c_int), ("precision", ctypes.c_int),
                ("start", ctypes.c_int), ("J", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("tile", ctypes.c_int * 3), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t)]


class pyro_graph_config(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("precision", ctypes.c_int), ("start", ctypes.c_int),
                ("J", ctypes.c_double), ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("sc_L", ctypes.c_int), ("nsites", ctypes.c_int64), ("nbonds", ctypes.c_int64),
                ("bond_i", ctypes.c_void_p), ("bond_j", ctypes.c_void_p), ("site_mask", ctypes.c_void_p),
                ("bond_mask", ctypes.c_void_p)]


class pyro_stats_t(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("sum_E", ctypes.c_double), ("sum_E2", ctypes.c_double),
                ("sum_m2", ctypes.c_double), ("sum_m4", ctypes.c_double), ("sum_absm", ctypes.c_double)]


_SIGS = {
    "pyro_init": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_uint64]),
    "pyro_init_ex": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(pyro_config)]),
    "pyro_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(pyro_config)]),
    "pyro_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]),
    "pyro_measure": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_double)] * 3),
    "pyro_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pyro_stats_t)]),
    "pyro_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "pyro_get_spins": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "pyro_set_spins": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "pyro_state_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "pyro_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "pyro_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "pyro_get_labels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "pyro_get_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "pyro_set_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "pyro_set_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "pyro_get_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int64)]),
    "pyro_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "pyro_num_sites": (ctypes.c_int64, [ctypes.c_void_p]),
    "pyro_get_tile": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "pyro_get_stream": (ctypes.c_void_p, [ctypes.c_void_p]),
    "pyro_launch_count": (ctypes.c_uint64, [ctypes.c_void_p]),
    "pyro_profile_phases": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double)]),
    "pyro_set_graphs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pyro_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "pyro_debug_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64]),
    "pyro_destroy": (None, [ctypes.c_void_p]),
    "pyro_last_error": (ctypes.c_char_p, []),
    "pyro_batch_init": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]),
    "pyro_batch_init_ex": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                          ctypes.POINTER(ctypes.c_int)]),
    "pyro_batch_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double)]),
    "pyro_batch_stats_all": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pyro_batch_measure_all": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pyro_batch_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pyro_batch_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(pyro_stats_t)]),
    "pyro_batch_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "pyro_batch_measure": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.POINTER(ctypes.c_double)] * 3),
    "pyro_batch_get_spins": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "pyro_batch_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "pyro_batch_total_sites": (ctypes.c_int64, [ctypes.c_void_p]),
    "pyro_batch_launch_count": (ctypes.c_uint64, [ctypes.c_void_p]),
    "pyro_batch_get_stream": (ctypes.c_void_p, [ctypes.c_void_p]),
    "pyro_batch_destroy": (None, [ctypes.c_void_p]),
    "pyro_graph_init": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(pyro_graph_config)]),
    "pyro_graph_bonds_from_table": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                     ctypes.c_void_p]),
    "pyro_graph_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64]),
    "pyro_graph_measure": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_double)] * 3),
    "pyro_graph_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pyro_stats_t)]),
    "pyro_graph_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "pyro_graph_get_spins": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "pyro_graph_set_spins": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "pyro_graph_get_labels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]),
    "pyro_graph_set_sweep": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "pyro_graph_get_sweep": (ctypes.c_uint64, [ctypes.c_void_p]),
    "pyro_graph_num_sites": (ctypes.c_int64, [ctypes.c_void_p]),
    "pyro_graph_num_bonds": (ctypes.c_int64, [ctypes.c_void_p]),
    "pyro_graph_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "pyro_graph_get_stream": (ctypes.c_void_p, [ctypes.c_void_p]),
    "pyro_graph_launch_count": (ctypes.c_uint64, [ctypes.c_void_p]),
    "pyro_graph_destroy": (None, [ctypes.c_void_p]),
    "pyro_ising_sweep_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                                ctypes.c_void_p]),
}


def library_path() -> str:
    return _build.OUT


def lib():
    """Load libpyro.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def declared_symbols() -> list[str]:
    return list(_SIGS)


def _check(rc: int):
    if rc != OK:
        raise PyroError(rc, lib().pyro_last_error().decode())


def _buf(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- C names --
def pyro_init(L: int, model: int, seed: int):
    h = ctypes.c_void_p()
    _check(lib().pyro_init(ctypes.byref(h), L, model, seed))
    return h


def pyro_init_ex(L: int, model: int, seed: int, precision: int = FP32, start: int = START_UP,
                 J: float = 1.0, stream: int | None = None, tile=(0, 0, 0), workspace: int | None = None,
                 workspace_bytes: int = 0):
    cfg = pyro_config(L, model, precision, start, J, seed, stream, (ctypes.c_int * 3)(*tile), workspace,
                      workspace_bytes)
    h = ctypes.c_void_p()
    _check(lib().pyro_init_ex(ctypes.byref(h), ctypes.byref(cfg)))
    return h


def pyro_workspace_bytes(L: int, model: int, precision: int = FP32, start: int = START_UP, J: float = 1.0,
                         tile=(0, 0, 0)) -> int:
    """Device bytes of a lattice with this configuration (caller-owned memory)."""
    cfg = pyro_config(L, model, precision, start, J, 0, None, (ctypes.c_int * 3)(*tile), None, 0)
    n = int(lib().pyro_workspace_bytes(ctypes.byref(cfg)))
    if n == 0:
        raise PyroError(E_INVAL, lib().pyro_last_error().decode())
    return n


def pyro_sweep(h, beta: float, n: int = 1):
    _check(lib().pyro_sweep(h, beta, n))


def pyro_measure(h):
    E, m2, m4 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().pyro_measure(h, ctypes.byref(E), ctypes.byref(m2), ctypes.byref(m4)))
    return E.value, m2.value, m4.value


def _stats_dict(s: pyro_stats_t) -> dict:
    return dict(count=int(s.count), sum_E=s.sum_E, sum_E2=s.sum_E2, sum_m2=s.sum_m2, sum_m4=s.sum_m4,
                sum_absm=s.sum_absm)


def pyro_stats(h) -> dict:
    s = pyro_stats_t()
    _check(lib().pyro_stats(h, ctypes.byref(s)))
    return _stats_dict(s)


def pyro_reset_stats(h):
    _check(lib().pyro_reset_stats(h))


def pyro_num_sites(h) -> int:
    return int(lib().pyro_num_sites(h))


def pyro_get_spins(h, model: int) -> np.ndarray:
    N = pyro_num_sites(h)
    out = np.zeros(N, dtype=np.int8) if model == ISING else np.zeros((N, model), dtype=np.float64)
    _check(lib().pyro_get_spins(h, _buf(out), out.nbytes))
    return out


def pyro_set_spins(h, spins: np.ndarray):
    a = np.ascontiguousarray(spins)
    if a.dtype != np.int8:
        a = np.ascontiguousarray(a, dtype=np.float64)
    _check(lib().pyro_set_spins(h, _buf(a), a.nbytes))


def pyro_state_bytes(h) -> int:
    return int(lib().pyro_state_bytes(h))


def pyro_get_state(h, host_ptr: int, nbytes: int):
    """Copy the compact device state to host memory at host_ptr (asynchronous)."""
    _check(lib().pyro_get_state(h, ctypes.c_void_p(host_ptr), nbytes))


def pyro_set_state(h, host_ptr: int, nbytes: int):
    _check(lib().pyro_set_state(h, ctypes.c_void_p(host_ptr), nbytes))


def pyro_get_labels(h) -> np.ndarray:
    out = np.zeros(pyro_num_sites(h), dtype=np.int32)
    _check(lib().pyro_get_labels(h, _buf(out), out.nbytes))
    return out


def pyro_get_sweep(h) -> int:
    s = ctypes.c_uint64()
    _check(lib().pyro_get_sweep(h, ctypes.byref(s)))
    return int(s.value)


def pyro_set_sweep(h, sweep: int):
    _check(lib().pyro_set_sweep(h, sweep))


def pyro_set_trace(h, capacity: int):
    _check(lib().pyro_set_trace(h, capacity))


def pyro_get_trace(h, max_records: int) -> np.ndarray:
    out = np.zeros((max(max_records, 1), 4), dtype=np.float64)
    n = ctypes.c_int64()
    _check(lib().pyro_get_trace(h, _buf(out), max_records, ctypes.byref(n)))
    return out[: n.value]


def pyro_sync(h):
    _check(lib().pyro_sync(h))


def pyro_get_tile(h):
    t = (ctypes.c_int * 3)()
    _check(lib().pyro_get_tile(h, t))
    return tuple(t)


def pyro_get_stream(h) -> int:
    return lib().pyro_get_stream(h) or 0


def pyro_launch_count(h) -> int:
    return int(lib().pyro_launch_count(h))


DEBUG_FAIL_ALLOCS, DEBUG_UNITE_BOUND, DEBUG_NOALLOC_STAMP, DEBUG_EPOCH_START = 1, 2, 3, 4


def pyro_set_graphs(h, on: bool):
    _check(lib().pyro_set_graphs(h, 1 if on else 0))


def pyro_autotune(L: int, model: int, precision: int = FP32, beta: float = 0.2373, nsweeps: int = 5):
    """Fastest labelling tile for this GPU and lattice (cached); returns
    (tile, ms per sweep)."""
    t = (ctypes.c_int * 3)()
    ms = ctypes.c_double()
    _check(lib().pyro_autotune(L, model, precision, beta, nsweeps, t, ctypes.byref(ms)))
    return tuple(t), ms.value


def pyro_debug_set(key: int, value: int):
    _check(lib().pyro_debug_set(key, value))


PHASES = ("local", "boundary", "flip", "measure", "accumulate")


def pyro_profile_phases(h, beta: float, n: int) -> dict:
    """Mean device ms of each sweep phase over n event-bracketed sweeps."""
    ms = (ctypes.c_double * len(PHASES))()
    _check(lib().pyro_profile_phases(h, beta, n, ms))
    return dict(zip(PHASES, list(ms)))


def pyro_destroy(h):
    lib().pyro_destroy(h)


def pyro_last_error() -> str:
    return lib().pyro_last_error().decode()


def pyro_batch_init(Ls, betas, model: int, precision: int = FP32, start: int = START_RANDOM, seed: int = 1):
    R = len(Ls)
    La = (ctypes.c_int * R)(*Ls)
    Ba = (ctypes.c_double * R)(*betas)
    b = ctypes.c_void_p()
    _check(lib().pyro_batch_init(ctypes.byref(b), R, La, Ba, model, precision, start, seed))
    return b


def pyro_batch_init_ex(Ls, betas, model: int, precision: int = FP32, start: int = START_RANDOM, seed: int = 1,
                       tile=(0, 0, 0)):
    R = len(Ls)
    La = (ctypes.c_int * R)(*Ls)
    Ba = (ctypes.c_double * R)(*betas)
    b = ctypes.c_void_p()
    _check(lib().pyro_batch_init_ex(ctypes.byref(b), R, La, Ba, model, precision, start, seed,
                                    (ctypes.c_int * 3)(*tile)))
    return b


def pyro_batch_autotune(Ls, betas, model: int, precision: int = FP32, nsweeps: int = 3):
    """Fastest labelling tile for a batch of these sizes (cached); returns
    (tile, ms per batch sweep)."""
    R = len(Ls)
    t = (ctypes.c_int * 3)()
    ms = ctypes.c_double()
    _check(lib().pyro_batch_autotune(R, (ctypes.c_int * R)(*Ls), (ctypes.c_double * R)(*betas), model, precision,
                                     nsweeps, t, ctypes.byref(ms)))
    return tuple(t), ms.value


def pyro_batch_stats_all(b, R: int) -> list:
    s = (pyro_stats_t * R)()
    _check(lib().pyro_batch_stats_all(b, ctypes.cast(s, ctypes.c_void_p)))
    return [_stats_dict(x) for x in s]


def pyro_batch_measure_all(b, R: int) -> np.ndarray:
    out = np.zeros((R, 3), dtype=np.float64)
    _check(lib().pyro_batch_measure_all(b, _buf(out)))
    return out


def pyro_batch_sweep(b, n: int = 1):
    _check(lib().pyro_batch_sweep(b, n))


def pyro_batch_stats(b, r: int) -> dict:
    s = pyro_stats_t()
    _check(lib().pyro_batch_stats(b, r, ctypes.byref(s)))
    return _stats_dict(s)


def pyro_batch_reset_stats(b):
    _check(lib().pyro_batch_reset_stats(b))


def pyro_batch_measure(b, r: int):
    E, m2, m4 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().pyro_batch_measure(b, r, ctypes.byref(E), ctypes.byref(m2), ctypes.byref(m4)))
    return E.value, m2.value, m4.value


def pyro_batch_get_spins(b, r: int, N: int, model: int) -> np.ndarray:
    out = np.zeros(N, dtype=np.int8) if model == ISING else np.zeros((N, model), dtype=np.float64)
    _check(lib().pyro_batch_get_spins(b, r, _buf(out), out.nbytes))
    return out


def pyro_batch_sync(b):
    _check(lib().pyro_batch_sync(b))


def pyro_batch_total_sites(b) -> int:
    return int(lib().pyro_batch_total_sites(b))


def pyro_batch_launch_count(b) -> int:
    return int(lib().pyro_batch_launch_count(b))


def pyro_batch_get_stream(b) -> int:
    return lib().pyro_batch_get_stream(b) or 0


def pyro_batch_destroy(b):
    lib().pyro_batch_destroy(b)


NOALLOC_MAX_L = 32


def pyro_ising_sweep_noalloc(spins_in: int, spins_out: int, labels: int, meas: int, L: int, beta: float,
                             seed: int, sweep: int, stream: int | None = None):
    """One Ising sweep on caller-owned device buffers (raw device pointers),
    with the library's fixed scratch array instead of any allocation."""
    _check(lib().pyro_ising_sweep_noalloc(spins_in, spins_out, labels, meas, L, beta, seed, sweep, stream))


# ---------------------------------------------------- generic lattices --
def pyro_graph_bonds_from_table(nbr: np.ndarray):
    """Bond list (bond_i, bond_j) of a symmetric neighbour table (N x z,
    -1 = none): slot (i, k) with i < nbr[i, k], in the order of (i, k)."""
    t = np.ascontiguousarray(nbr, dtype=np.int32)
    N, z = t.shape
    E = int(lib().pyro_graph_bonds_from_table(N, z, _buf(t), None, None))
    if E < 0:
        _check(E)
    bi = np.zeros(max(E, 1), dtype=np.int32)
    bj = np.zeros(max(E, 1), dtype=np.int32)
    rc = int(lib().pyro_graph_bonds_from_table(N, z, _buf(t), _buf(bi), _buf(bj)))
    if rc < 0:
        _check(rc)
    return bi[:E], bj[:E]


def pyro_graph_init(model: int, seed: int, precision: int = FP64, start: int = START_UP, J: float = 1.0,
                    stream: int | None = None, sc_L: int = 0, nsites: int = 0, bond_i=None, bond_j=None,
                    site_mask=None, bond_mask=None):
    keep = []

    def arr(a, dt):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data

    bi = arr(bond_i, np.int32)
    bj = arr(bond_j, np.int32)
    nb = 0 if bond_i is None else len(keep[0])
    cfg = pyro_graph_config(model, precision, start, J, seed, stream, sc_L, nsites, nb, bi, bj,
                            arr(site_mask, np.uint8), arr(bond_mask, np.uint8))
    g = ctypes.c_void_p()
    _check(lib().pyro_graph_init(ctypes.byref(g), ctypes.byref(cfg)))
    return g


def pyro_graph_sweep(g, beta: float, n: int = 1):
    _check(lib().pyro_graph_sweep(g, beta, n))


def pyro_graph_measure(g):
    E, m2, m4 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().pyro_graph_measure(g, ctypes.byref(E), ctypes.byref(m2), ctypes.byref(m4)))
    return E.value, m2.value, m4.value


def pyro_graph_stats(g) -> dict:
    s = pyro_stats_t()
    _check(lib().pyro_graph_stats(g, ctypes.byref(s)))
    return dict(count=s.count, sum_E=s.sum_E, sum_E2=s.sum_E2, sum_m2=s.sum_m2, sum_m4=s.sum_m4,
                sum_absm=s.sum_absm)


def pyro_graph_reset_stats(g):
    _check(lib().pyro_graph_reset_stats(g))


def pyro_graph_num_sites(g) -> int:
    return int(lib().pyro_graph_num_sites(g))


def pyro_graph_num_bonds(g) -> int:
    return int(lib().pyro_graph_num_bonds(g))


def pyro_graph_get_spins(g, model: int, out: np.ndarray | None = None) -> np.ndarray:
    """Spins in site order (Ising int8, n-vector float64 N x n); `out`, if
    given, is a C-contiguous array of that shape and type to fill (for
    instance a view of pinned host memory)."""
    N = pyro_graph_num_sites(g)
    if out is None:
        out = np.zeros(N, dtype=np.int8) if model == ISING else np.zeros((N, model), dtype=np.float64)
    _check(lib().pyro_graph_get_spins(g, _buf(out), out.nbytes))
    return out


def pyro_graph_set_spins(g, s: np.ndarray, model: int):
    a = np.ascontiguousarray(s, dtype=np.int8 if model == ISING else np.float64)
    _check(lib().pyro_graph_set_spins(g, _buf(a), a.nbytes))


def pyro_graph_get_labels(g) -> np.ndarray:
    N = pyro_graph_num_sites(g)
    out = np.zeros(N, dtype=np.int32)
    _check(lib().pyro_graph_get_labels(g, _buf(out), N))
    return out


def pyro_graph_set_sweep(g, s: int):
    _check(lib().pyro_graph_set_sweep(g, s))


def pyro_graph_get_sweep(g) -> int:
    return int(lib().pyro_graph_get_sweep(g))


def pyro_graph_sync(g):
    _check(lib().pyro_graph_sync(g))


def pyro_graph_get_stream(g) -> int:
    return lib().pyro_graph_get_stream(g) or 0


def pyro_graph_launch_count(g) -> int:
    return int(lib().pyro_graph_launch_count(g))


def pyro_graph_destroy(g):
    lib().pyro_graph_destroy(g)


# ------------------------------------------------------- convenience API --
class Lattice:
    """One pyrochlore lattice on the GPU (owns a pyro_handle)."""

    def __init__(self, L: int, model: int = ISING, seed: int = 1, precision: int = FP32,
                 start: str | int = "up", J: float = 1.0, tile=(0, 0, 0), stream: int | None = None,
                 workspace: int | None = None, workspace_bytes: int = 0):
        """workspace: a device pointer (e.g. a torch tensor's data_ptr()) of
        at least pyro_workspace_bytes(...) bytes that the lattice lives in;
        the caller keeps it alive until close()."""
        st = start if isinstance(start, int) else (START_RANDOM if start == "random" else START_UP)
        self.L, self.model, self.seed, self.precision = L, model, seed, precision
        if tile == "auto":
            tile = pyro_autotune(L, model, precision)[0]
        self.h = pyro_init_ex(L, model, seed, precision, st, J, stream, tile, workspace, workspace_bytes)
        self.N = pyro_num_sites(self.h)

    def close(self):
        if getattr(self, "h", None):
            pyro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, beta: float, n: int = 1):
        pyro_sweep(self.h, beta, n)

    def measure(self):
        return pyro_measure(self.h)

    def stats(self):
        return pyro_stats(self.h)

    def reset_stats(self):
        pyro_reset_stats(self.h)

    def spins(self):
        return pyro_get_spins(self.h, self.model)

    def set_spins(self, s):
        pyro_set_spins(self.h, s)

    def labels(self):
        return pyro_get_labels(self.h)

    @property
    def sweep_count(self):
        return pyro_get_sweep(self.h)

    @sweep_count.setter
    def sweep_count(self, s):
        pyro_set_sweep(self.h, s)

    def sync(self):
        pyro_sync(self.h)

    @property
    def tile(self):
        return pyro_get_tile(self.h)

    @property
    def launches(self):
        return pyro_launch_count(self.h)

    def set_graphs(self, on: bool):
        pyro_set_graphs(self.h, on)


class Replicas:
    """Independent lattices updated together (owns a pyro_batch)."""

    def __init__(self, Ls, betas, model: int = ISING, precision: int = FP32, start: str | int = "random",
                 seed: int = 1, tile=(0, 0, 0)):
        st = start if isinstance(start, int) else (START_RANDOM if start == "random" else START_UP)
        self.Ls, self.betas, self.model = list(Ls), list(betas), model
        if tile == "auto":
            tile = pyro_batch_autotune(self.Ls, self.betas, model, precision)[0]
        self.tile = tuple(tile)
        self.b = pyro_batch_init_ex(self.Ls, self.betas, model, precision, st, seed, tile)
        self.total_sites = pyro_batch_total_sites(self.b)

    def close(self):
        if getattr(self, "b", None):
            pyro_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n: int = 1):
        pyro_batch_sweep(self.b, n)

    def stats(self, r: int):
        return pyro_batch_stats(self.b, r)

    def reset_stats(self):
        pyro_batch_reset_stats(self.b)

    def measure(self, r: int):
        return pyro_batch_measure(self.b, r)

    def stats_all(self) -> list:
        return pyro_batch_stats_all(self.b, len(self.Ls))

    def measure_all(self) -> np.ndarray:
        """(R, 3) array of every replica's E, m^2, m^4 (one device read)."""
        return pyro_batch_measure_all(self.b, len(self.Ls))

    def spins(self, r: int):
        return pyro_batch_get_spins(self.b, r, 16 * self.Ls[r] ** 3, self.model)

    def sync(self):
        pyro_batch_sync(self.b)

    @property
    def launches(self):
        return pyro_batch_launch_count(self.b)

    @property
    def stream(self) -> int:
        return pyro_batch_get_stream(self.b)


def replica_seed(seed: int, r: int) -> int:
    """Seed of replica r of a batch: seed + r * 0x9E3779B97F4A7C15 mod 2^64."""
    return (seed + r * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF


class Graph:
    """A generic lattice on the GPU (owns a pyro_graph): an explicit bond
    list (bond_i, bond_j) over nsites sites, or the simple-cubic sc_L^3
    lattice, optionally diluted by a site mask and a bond mask."""

    def __init__(self, model: int = ISING, seed: int = 1, precision: int = FP64, start: str | int = "up",
                 J: float = 1.0, sc_L: int = 0, nsites: int = 0, bond_i=None, bond_j=None, site_mask=None,
                 bond_mask=None, stream: int | None = None):
        st = start if isinstance(start, int) else (START_RANDOM if start == "random" else START_UP)
        self.model = model
        self.g = pyro_graph_init(model, seed, precision, st, J, stream, sc_L, nsites, bond_i, bond_j, site_mask,
                                 bond_mask)
        self.N = pyro_graph_num_sites(self.g)
        self.NB = pyro_graph_num_bonds(self.g)

    def close(self):
        if getattr(self, "g", None):
            pyro_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, beta: float, n: int = 1):
        pyro_graph_sweep(self.g, beta, n)

    def measure(self):
        return pyro_graph_measure(self.g)

    def stats(self):
        return pyro_graph_stats(self.g)

    def reset_stats(self):
        pyro_graph_reset_stats(self.g)

    def spins(self, out=None):
        return pyro_graph_get_spins(self.g, self.model, out)

    def set_spins(self, s):
        pyro_graph_set_spins(self.g, s, self.model)

    def labels(self):
        return pyro_graph_get_labels(self.g)

    @property
    def sweep_count(self):
        return pyro_graph_get_sweep(self.g)

    @sweep_count.setter
    def sweep_count(self, s):
        pyro_graph_set_sweep(self.g, s)

    def sync(self):
        pyro_graph_sync(self.g)

    @property
    def stream(self):
        return pyro_graph_get_stream(self.g)

    @property
    def launches(self):
        return pyro_graph_launch_count(self.g)
