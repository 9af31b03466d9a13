"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/pyro.h declares; the Python binding covers the same names.
Argument checks that run before any CUDA call are exercised on the CPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1612_08312_gb300 as pyro

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(pyro_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("pyro_init", "pyro_sweep", "pyro_measure"):
        assert core in names


def test_library_exports_every_declared_symbol():
    path = pyro._build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (pyro_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_uses_the_c_names():
    assert sorted(pyro.declared_symbols()) == declared_functions()
    for n in declared_functions():
        assert callable(getattr(pyro, n))


def test_build_targets_sm_103a_only():
    assert pyro._build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("L,model", [(0, 1), (512, 1), (4, 0), (4, 4), (-3, 2)])
def test_init_rejects_bad_arguments(L, model):
    with pytest.raises(pyro.PyroError) as ei:
        pyro.pyro_init_ex(L, model, 1)
    assert ei.value.code == pyro.E_INVAL


def test_init_rejects_bad_tile_and_options():
    for kw in (dict(tile=(3, 8, 4)), dict(tile=(8, 8, 32)), dict(precision=7), dict(start=5), dict(J=0.0),
               dict(J=float("nan"))):
        with pytest.raises(pyro.PyroError) as ei:
            pyro.pyro_init_ex(8, pyro.ISING, 1, **kw)
        assert ei.value.code == pyro.E_INVAL


def test_null_handle_calls_fail_cleanly():
    L = pyro.lib()
    assert L.pyro_sweep(None, 0.2, 1) == pyro.E_INVAL
    assert L.pyro_sync(None) == pyro.E_INVAL
    assert L.pyro_measure(None, None, None, None) == pyro.E_INVAL
    assert L.pyro_num_sites(None) == 0
    assert "NULL" in pyro.pyro_last_error()
    L.pyro_destroy(None)


def test_batch_rejects_bad_arguments():
    for Ls, betas in (([8] * 65, [0.2] * 65), ([8, 0], [0.2, 0.2]), ([8], [-1.0]), ([8], [float("inf")])):
        with pytest.raises(pyro.PyroError) as ei:
            pyro.pyro_batch_init(Ls, betas, pyro.ISING)
        assert ei.value.code == pyro.E_INVAL


def test_debug_hook_rejects_bad_keys_without_a_gpu():
    with pytest.raises(pyro.PyroError):
        pyro.pyro_debug_set(99, 1)
    with pytest.raises(pyro.PyroError):
        pyro.pyro_debug_set(pyro.DEBUG_FAIL_ALLOCS, -1)
    pyro.pyro_debug_set(pyro.DEBUG_FAIL_ALLOCS, 0)


def test_workspace_bytes_is_host_only_and_checks_its_config():
    # the size of a lattice's device arrays is computed on the host
    n8 = pyro.pyro_workspace_bytes(8, pyro.ISING)
    n16 = pyro.pyro_workspace_bytes(16, pyro.ISING)
    assert n8 > 0 and 7 * n8 < n16 < 9 * n8
    assert pyro.pyro_workspace_bytes(8, pyro.XY, pyro.FP64) > pyro.pyro_workspace_bytes(8, pyro.XY, pyro.FP32)
    with pytest.raises(pyro.PyroError):
        pyro.pyro_workspace_bytes(0, pyro.ISING)
    with pytest.raises(pyro.PyroError):
        pyro.pyro_workspace_bytes(8, pyro.ISING, tile=(3, 1, 1))


def test_graph_bonds_from_table_on_the_host():
    """pyro_graph_bonds_from_table runs on the host: the simple-cubic table
    gives the oracle's bond list, and bad tables are refused."""
    import numpy as np
    import oracle
    L = 4
    bi, bj = oracle.sc_edges(L)
    rows = [[] for _ in range(L ** 3)]
    for a, b in zip(bi.tolist(), bj.tolist()):
        rows[a].append(b)
        rows[b].append(a)
    nbr = np.full((L ** 3, 7), -1, dtype=np.int32)  # one spare empty column
    for i, r in enumerate(rows):
        nbr[i, :len(r)] = r
    gi, gj = pyro.pyro_graph_bonds_from_table(nbr)
    oi, oj = oracle.edges_from_table(nbr)
    assert (gi == oi).all() and (gj == oj).all() and len(gi) == 3 * L ** 3
    for bad in ([[0, -1], [0, -1]], [[1, -1], [-1, -1]], [[5, -1], [0, -1]]):  # self entry, asymmetric, out of range
        with pytest.raises(pyro.PyroError) as ei:
            pyro.pyro_graph_bonds_from_table(np.array(bad, dtype=np.int32))
        assert ei.value.code == pyro.E_INVAL


def test_graph_init_rejects_bad_arguments_on_the_host():
    import numpy as np
    cases = [dict(model=4, sc_L=8), dict(model=1, sc_L=1), dict(model=1, sc_L=1291),
             dict(model=1, nsites=3, bond_i=np.array([0]), bond_j=np.array([0])),      # self-loop
             dict(model=1, nsites=3, bond_i=np.array([0]), bond_j=np.array([3])),      # out of range
             dict(model=1, sc_L=8, bond_i=np.array([0]), bond_j=np.array([1])),        # list with sc_L
             dict(model=2, precision=5, sc_L=8), dict(model=1, sc_L=8, start=3), dict(model=1, sc_L=8, J=-1.0),
             dict(model=1, nsites=0)]
    for kw in cases:
        with pytest.raises(pyro.PyroError) as ei:
            pyro.pyro_graph_init(kw.pop("model"), 1, **kw)
        assert ei.value.code == pyro.E_INVAL, kw
    L = pyro.lib()
    assert L.pyro_graph_sweep(None, 0.2, 1) == pyro.E_INVAL
    assert L.pyro_graph_num_sites(None) == 0
    L.pyro_graph_destroy(None)
