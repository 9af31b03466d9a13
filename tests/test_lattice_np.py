"""The numpy closed-form bond list used by the full-size tests equals the
oracle's geometrically built bond list (Sec. 2 lattice)."""
import numpy as np
import pytest

import lattice_np
import oracle


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_closed_form_bonds_match_oracle(L):
    o = oracle.Oracle(L, oracle.ISING, 1)
    bi, bj = o.bonds()
    ci, cj = lattice_np.bond_endpoints(L, np.arange(3 * o.N))
    assert (ci == bi).all() and (cj == bj).all()
