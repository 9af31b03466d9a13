"""The generic-lattice sweep (pyro_graph_*) against the graph oracle, sweep
by sweep: the simple-cubic lattice (implicit bonds, Sec. 3.4), explicit bond
lists and neighbour tables (Sec. 2), site and bond dilution (Sec. 4).

Ising: spins, canonical labels and (E, m^2, m^4) identical.  n-vector FP64:
labels identical, spins within 1e-12, E within 1e-12 relative (the bond sum
is taken in another order).  FP32: the chain is not bit-compatible with an
FP64 one, so it is checked where no bond decides (beta = 0) and by the
state it reaches."""
import numpy as np
import pytest

import oracle
import paper_1612_08312_gb300 as pyro

pytestmark = pytest.mark.gpu

T_SC = {1: 4.511524, 2: 2.20182, 3: 1.4430}  # simple-cubic critical temperatures quoted in Sec. 3.4


def exact(g, o, beta, sweeps, model=1):
    for s in range(sweeps):
        g.sweep(beta, 1)
        o.sweep(beta, 1)
        assert (g.labels() == o.labels()).all(), f"labels differ after sweep {s}"
        if model == 1:
            assert (g.spins() == o.spins()).all(), f"spins differ after sweep {s}"
            assert g.measure() == o.measure(), f"measurement differs after sweep {s}"
        else:
            assert np.abs(g.spins() - o.spins()).max() <= 1e-12
            Eg, m2g, _ = g.measure()
            Eo, m2o, _ = o.measure()
            assert abs(Eg - Eo) <= 1e-12 * max(1.0, abs(Eo))
            assert abs(m2g - m2o) <= 1e-12


@pytest.mark.parametrize("L", [2, 3, 4, 8, 13, 16, 32])
def test_simple_cubic_ising(L):
    bi, bj = oracle.sc_edges(L)
    g = pyro.Graph(pyro.ISING, 7 + L, sc_L=L, start="random")
    o = oracle.GraphOracle(L ** 3, bi, bj, 1, 7 + L, "random")
    assert (g.spins() == o.spins()).all()
    exact(g, o, 1 / T_SC[1], 4)
    assert g.stats() == o.stats()


@pytest.mark.parametrize("model", [2, 3])
@pytest.mark.parametrize("L", [4, 7, 16])
def test_simple_cubic_vector_fp64(model, L):
    bi, bj = oracle.sc_edges(L)
    g = pyro.Graph(model, 3, precision=pyro.FP64, sc_L=L, start="random")
    o = oracle.GraphOracle(L ** 3, bi, bj, model, 3, "random")
    exact(g, o, 1 / T_SC[model], 3, model)


def test_explicit_bond_list_matches_implicit_simple_cubic():
    L = 12
    bi, bj = oracle.sc_edges(L)
    a = pyro.Graph(pyro.ISING, 5, sc_L=L, start="random")
    b = pyro.Graph(pyro.ISING, 5, nsites=L ** 3, bond_i=bi, bond_j=bj, start="random")
    for _ in range(3):
        a.sweep(1 / T_SC[1])
        b.sweep(1 / T_SC[1])
        assert (a.spins() == b.spins()).all() and (a.labels() == b.labels()).all()
        assert a.measure() == b.measure()


@pytest.mark.parametrize("model", [1, 3])
def test_pyrochlore_bond_list_reproduces_the_pyrochlore_kernels(model):
    """Sec. 2: with the pyrochlore neighbour table the generic program runs
    the pyrochlore chain -- here the bond list ordered by random-number id,
    against the dedicated pyrochlore kernels."""
    L = 6
    bi, bj = oracle.pyrochlore_edges(L)
    prec = pyro.FP64
    g = pyro.Graph(model, 11, precision=prec, nsites=16 * L ** 3, bond_i=bi, bond_j=bj, start="random")
    p = pyro.Lattice(L, model, 11, precision=prec, start="random")
    beta = 1 / (4.21394 if model == 1 else 1.31695)
    for _ in range(3):
        g.sweep(beta)
        p.sweep(beta)
        assert (g.labels() == p.labels()).all()
        if model == 1:
            assert (g.spins() == p.spins()).all()
            assert g.measure() == p.measure()
        else:
            assert np.abs(g.spins() - p.spins()).max() <= 1e-12
    p.close()


def test_neighbour_table_random_graph():
    """An irregular graph given as a neighbour table (degrees 0 to 8)."""
    rng = np.random.default_rng(2)
    N = 3000
    pairs = set()
    while len(pairs) < 6000:
        a, b = rng.integers(0, N, 2)
        if a != b:
            pairs.add((int(min(a, b)), int(max(a, b))))
    rows = [[] for _ in range(N)]
    for a, b in pairs:
        if len(rows[a]) < 8 and len(rows[b]) < 8:
            rows[a].append(b)
            rows[b].append(a)
    nbr = np.full((N, 8), -1, dtype=np.int32)
    for i, r in enumerate(rows):
        nbr[i, :len(r)] = r
    bi, bj = pyro.pyro_graph_bonds_from_table(nbr)
    obi, obj = oracle.edges_from_table(nbr)
    assert (bi == obi).all() and (bj == obj).all()
    g = pyro.Graph(pyro.ISING, 8, nsites=N, bond_i=bi, bond_j=bj, start="random")
    o = oracle.GraphOracle(N, obi, obj, 1, 8, "random")
    exact(g, o, 0.7, 5)


@pytest.mark.parametrize("model", [1, 2])
def test_site_and_bond_dilution(model):
    L = 16
    N = L ** 3
    rng = np.random.default_rng(11)
    site = (rng.random(N) < 0.7).astype(np.uint8)
    bond = (rng.random(3 * N) < 0.9).astype(np.uint8)
    bi, bj = oracle.sc_edges(L)
    g = pyro.Graph(model, 4, precision=pyro.FP64, sc_L=L, start="random", site_mask=site, bond_mask=bond)
    o = oracle.GraphOracle(N, bi, bj, model, 4, "random", site_mask=site, edge_mask=bond)
    exact(g, o, 1 / (3.2 if model == 1 else 1.5), 4, model)
    s = g.spins()
    s0 = oracle.GraphOracle(N, bi, bj, model, 4, "random").spins()
    assert (s[site == 0] == s0[site == 0]).all()  # vacant sites never move


def test_infinite_beta_and_degenerate_graphs():
    L = 10
    site = (np.random.default_rng(1).random(L ** 3) < 0.35).astype(np.uint8)  # below percolation
    bi, bj = oracle.sc_edges(L)
    g = pyro.Graph(pyro.ISING, 2, sc_L=L, site_mask=site)
    o = oracle.GraphOracle(L ** 3, bi, bj, 1, 2, site_mask=site)
    exact(g, o, 50.0, 2)
    # one site, no bonds
    g = pyro.Graph(pyro.HEIS, 3, nsites=1, bond_i=np.zeros(0, np.int32), bond_j=np.zeros(0, np.int32),
                   start="random")
    o = oracle.GraphOracle(1, np.zeros(0, np.int32), np.zeros(0, np.int32), 3, 3, "random")
    exact(g, o, 1.0, 2, 3)
    # every site vacant
    g = pyro.Graph(pyro.ISING, 2, sc_L=L, site_mask=np.zeros(L ** 3, np.uint8), start="random")
    s0 = g.spins()
    g.sweep(0.3, 3)
    assert (g.spins() == s0).all() and g.measure() == (0.0, 0.0, 0.0)


@pytest.mark.parametrize("model", [2, 3])
def test_fp32_vector(model):
    L = 12
    bi, bj = oracle.sc_edges(L)
    g = pyro.Graph(model, 6, precision=pyro.FP32, sc_L=L, start="random")
    o = oracle.GraphOracle(L ** 3, bi, bj, model, 6, "random")
    assert np.abs(g.spins() - o.spins()).max() <= 1e-7
    # beta = 0: no bond is active, every site flips with its own bit
    g.sweep(0.0, 2)
    o.sweep(0.0, 2)
    assert (g.labels() == o.labels()).all()
    assert np.abs(g.spins() - o.spins()).max() <= 1e-5
    # at T_c the FP32 chain keeps unit spins and a finite energy near the FP64 chain's mean
    g.sweep(1 / T_SC[model], 50)
    s = g.spins()
    assert np.abs(np.linalg.norm(s, axis=1) - 1).max() <= 1e-5
    E, _, _ = g.measure()
    assert -3 * L ** 3 < E < 0


def test_simple_cubic_l128_two_sweeps():
    L = 128
    bi, bj = oracle.sc_edges(L)
    g = pyro.Graph(pyro.ISING, 13, sc_L=L, start="random")
    o = oracle.GraphOracle(L ** 3, bi, bj, 1, 13, "random")
    exact(g, o, 1 / T_SC[1], 2)


def test_errors_and_union_bound():
    with pytest.raises(pyro.PyroError) as ei:
        pyro.Graph(pyro.ISING, 1, nsites=3, bond_i=np.array([0]), bond_j=np.array([0]))
    assert ei.value.code == pyro.E_INVAL and "self-loop" in str(ei.value)
    with pytest.raises(pyro.PyroError) as ei:
        pyro.Graph(pyro.ISING, 1, nsites=3, bond_i=np.array([0]), bond_j=np.array([3]))
    assert ei.value.code == pyro.E_INVAL
    with pytest.raises(pyro.PyroError):
        pyro.Graph(pyro.ISING, 1, sc_L=1)
    bad = np.array([[1, -1], [-1, -1]], dtype=np.int32)  # 0 -> 1 without 1 -> 0
    with pytest.raises(pyro.PyroError) as ei:
        pyro.pyro_graph_bonds_from_table(bad)
    assert "symmetric" in str(ei.value)
    g = pyro.Graph(pyro.ISING, 2, sc_L=8, start="random")
    try:
        pyro.pyro_debug_set(pyro.DEBUG_UNITE_BOUND, 0)
        g.sweep(0.5, 1)
        with pytest.raises(pyro.PyroError) as ei:
            g.sync()
        assert ei.value.code == pyro.E_NOCONVERGE
    finally:
        pyro.pyro_debug_set(pyro.DEBUG_UNITE_BOUND, 4096)
    bi, bj = oracle.sc_edges(8)
    h = pyro.Graph(pyro.ISING, 2, sc_L=8, start="random")
    o = oracle.GraphOracle(512, bi, bj, 1, 2, "random")
    exact(h, o, 0.5, 2)
