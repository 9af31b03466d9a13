"""Caller-owned device memory (pyro_config.workspace): a lattice carved
from a torch tensor's memory, with no library allocation at all, runs the
same chain as a library-allocated lattice and as the oracle, bit for bit;
the spins it reports are those that lie in the caller's buffer."""
import numpy as np
import pytest

import oracle
import paper_1612_08312_gb300 as pyro

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,L,prec", [(1, 12, pyro.FP64), (1, 24, pyro.FP64), (2, 8, pyro.FP64), (3, 8, pyro.FP32)])
def test_lattice_in_torch_memory(model, L, prec):
    import torch
    nbytes = pyro.pyro_workspace_bytes(L, model, prec, pyro.START_RANDOM)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    # any device allocation by the library would now fail
    pyro.pyro_debug_set(pyro.DEBUG_FAIL_ALLOCS, 1000)
    try:
        g = pyro.Lattice(L, model, 5, precision=prec, start="random", workspace=buf.data_ptr(), workspace_bytes=nbytes)
    finally:
        pyro.pyro_debug_set(pyro.DEBUG_FAIL_ALLOCS, 0)
    h = pyro.Lattice(L, model, 5, precision=prec, start="random")
    o = oracle.Oracle(L, model, 5, "random")
    beta = 1 / (4.21394 if model == 1 else 2.0285 if model == 2 else 1.31695)
    for _ in range(3):
        g.sweep(beta, 1)
        h.sweep(beta, 1)
        o.sweep(beta, 1)
        assert (g.spins() == h.spins()).all()
        assert (g.labels() == h.labels()).all() and (g.labels() == o.labels()).all()
        if model == 1:
            assert (g.spins() == o.spins()).all()
        elif prec == pyro.FP64:
            assert np.abs(g.spins() - o.spins()).max() <= 1e-12
    assert g.stats() == h.stats()
    # the spins follow the 256-byte statistics record in the workspace
    n = pyro.pyro_state_bytes(g.h)
    g.sync()
    dev_state = buf[256:256 + n].cpu().numpy()
    host_state = np.zeros(n, dtype=np.uint8)
    pyro.pyro_get_state(g.h, host_state.ctypes.data, n)
    g.sync()
    assert (dev_state == host_state).all()
    g.close()
    h.close()


def test_workspace_errors():
    import torch
    nbytes = pyro.pyro_workspace_bytes(8, pyro.ISING)
    buf = torch.empty(nbytes + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(pyro.PyroError) as ei:
        pyro.Lattice(8, pyro.ISING, 1, workspace=buf.data_ptr(), workspace_bytes=nbytes - 1)
    assert ei.value.code == pyro.E_NOMEM
    with pytest.raises(pyro.PyroError) as ei:
        pyro.Lattice(8, pyro.ISING, 1, workspace=buf.data_ptr() + 8, workspace_bytes=nbytes)
    assert ei.value.code == pyro.E_INVAL
