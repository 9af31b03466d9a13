"""Pins of the generic-lattice oracle (oracle/graph_oracle.c): the sweep on
an arbitrary bond list (Sec. 2: the program needs only the neighbour
table), the simple-cubic lattice (Sec. 3.4) and dilution (Sec. 4).

Each pin comes from outside the oracle itself:
  - the pyrochlore bond list in random-number-id order must reproduce the
    pyrochlore oracle (pinned by its own tests) sweep by sweep;
  - the simple-cubic bond list must be networkx's periodic grid graph;
  - at beta = infinity every satisfied present bond is active, so from an
    ordered start the clusters are scipy's connected components of the
    occupied sub-lattice;
  - on rings the Ising energy and <M^2> have closed forms (transfer
    matrix), and the XY and Heisenberg energies per bond are I1/I0 and the
    Langevin function, up to corrections of order u^N;
  - on a small diluted graph the chain samples the Boltzmann distribution
    of its occupied part, enumerated exactly."""
import numpy as np
import pytest

import oracle

T_SC = 4.511524  # simple-cubic Ising critical temperature quoted by the paper (Sec. 3.4)


@pytest.mark.parametrize("model", [1, 2, 3])
@pytest.mark.parametrize("L", [1, 2])
def test_pyrochlore_bond_list_reproduces_the_pyrochlore_chain(model, L):
    bi, bj = oracle.pyrochlore_edges(L)
    N = 16 * L ** 3
    g = oracle.GraphOracle(N, bi, bj, model, 17, "random")
    o = oracle.Oracle(L, model, 17, "random")
    beta = {1: 0.23, 2: 0.5, 3: 0.75}[model]
    for s in range(6):
        g.sweep(beta)
        o.sweep(beta)
        assert (g.labels() == o.labels()).all(), f"labels differ after sweep {s}"
        if model == 1:
            assert (g.spins() == o.spins()).all()
            assert g.measure() == o.measure()
        else:
            assert (g.spins() == o.spins()).all()  # same per-site arithmetic
            Eg, m2g, _ = g.measure()
            Eo, m2o, _ = o.measure()
            assert abs(Eg - Eo) <= 1e-12 * max(1.0, abs(Eo))  # bond sums in another order
            assert abs(m2g - m2o) <= 1e-12


@pytest.mark.parametrize("L", [3, 4, 5])
def test_simple_cubic_bonds_are_the_periodic_grid(L):
    nx = pytest.importorskip("networkx")
    bi, bj = oracle.sc_edges(L)
    assert len(bi) == 3 * L ** 3
    G = nx.grid_graph(dim=[L, L, L], periodic=True)
    # networkx nodes are (z, y, x) tuples for dim=[L, L, L] listed x first;
    # map every node to the index x + L (y + L z) with x the first listed axis
    want = set()
    for a, b in G.edges():
        ia = a[0] + L * (a[1] + L * a[2])
        ib = b[0] + L * (b[1] + L * b[2])
        want.add((min(ia, ib), max(ia, ib)))
    got = {(min(a, b), max(a, b)) for a, b in zip(bi.tolist(), bj.tolist())}
    assert got == want
    # bond 3 i + d starts at site i
    assert (bi == np.repeat(np.arange(L ** 3), 3)).all()


def test_simple_cubic_l2_has_double_bonds():
    bi, bj = oracle.sc_edges(2)
    pairs = [(min(a, b), max(a, b)) for a, b in zip(bi.tolist(), bj.tolist())]
    from collections import Counter
    c = Counter(pairs)
    assert len(c) == 12 and set(c.values()) == {2}


def _table_of(N, bi, bj, z):
    rows = [[] for _ in range(N)]
    for a, b in zip(bi.tolist(), bj.tolist()):
        rows[a].append(b)
        rows[b].append(a)
    t = np.full((N, z), -1, dtype=np.int32)
    for i, r in enumerate(rows):
        t[i, :len(r)] = sorted(r)
    return t


def test_edges_from_table():
    L = 4
    bi, bj = oracle.sc_edges(L)
    t = _table_of(L ** 3, bi, bj, 7)  # one spare -1 column
    ei, ej = oracle.edges_from_table(t)
    assert len(ei) == 3 * L ** 3
    assert sorted(zip(ei.tolist(), ej.tolist())) == sorted((min(a, b), max(a, b)) for a, b in zip(bi.tolist(), bj.tolist()))
    assert (np.diff(ei) >= 0).all() and (ei < ej).all()
    bad = t.copy()
    bad[0, 0] = 0  # names its own row
    with pytest.raises(ValueError):
        oracle.edges_from_table(bad)
    bad = t.copy()
    bad[0, 6] = 2  # 0 -> 2 without 2 -> 0
    with pytest.raises(ValueError):
        oracle.edges_from_table(bad)


def test_infinite_beta_clusters_are_connected_components():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    L = 6
    N = L ** 3
    bi, bj = oracle.sc_edges(L)
    rng = np.random.default_rng(5)
    site = (rng.random(N) < 0.6).astype(np.uint8)
    bond = (rng.random(3 * N) < 0.8).astype(np.uint8)
    g = oracle.GraphOracle(N, bi, bj, 1, 3, "up", site_mask=site, edge_mask=bond)
    g.sweep(50.0)  # p = 1 - exp(-100) rounds to 1: every satisfied bond is active
    keep = (bond == 1) & (site[bi] == 1) & (site[bj] == 1)
    A = sp.coo_matrix((np.ones(keep.sum()), (bi[keep], bj[keep])), shape=(N, N))
    _, comp = csgraph.connected_components(A, directed=False)
    # canonical label = the minimum site of the component
    mins = np.full(comp.max() + 1, N)
    np.minimum.at(mins, comp, np.arange(N))
    assert (g.labels() == mins[comp]).all()
    lab = g.labels()
    s = g.spins()
    # vacant sites never flip; every cluster is uniform
    assert (s[site == 0] == 1).all()
    for c in np.unique(lab[site == 1]):
        assert len(np.unique(s[lab == c])) == 1
    # E counts present bonds only; all satisfied, clusters flip together,
    # but bonds between two clusters may now be unsatisfied
    E, m2, _ = g.measure()
    sat = (s[bi] == s[bj])[keep]
    assert E == -float(sat.sum() - (~sat).sum())
    assert m2 == (abs(float(s[site == 1].sum())) / site.sum()) ** 2


def test_beta_zero_and_empty_cases():
    L = 3
    bi, bj = oracle.sc_edges(L)
    g = oracle.GraphOracle(L ** 3, bi, bj, 1, 9, "random")
    g.sweep(0.0, 3)
    assert (g.labels() == np.arange(L ** 3)).all()
    # no bonds at all
    g = oracle.GraphOracle(5, np.zeros(0, np.int32), np.zeros(0, np.int32), 3, 1, "random")
    g.sweep(1.0, 2)
    E, m2, m4 = g.measure()
    assert E == 0.0 and (g.labels() == np.arange(5)).all()
    # every site vacant: nothing moves, m = 0
    g = oracle.GraphOracle(L ** 3, bi, bj, 1, 9, "random", site_mask=np.zeros(L ** 3, np.uint8))
    s0 = g.spins()
    g.sweep(0.3, 2)
    assert (g.spins() == s0).all() and g.measure() == (0.0, 0.0, 0.0)
    with pytest.raises(ValueError):
        oracle.GraphOracle(3, np.array([0], np.int32), np.array([0], np.int32), 1, 1)  # self-loop


def _ring(N):
    i = np.arange(N, dtype=np.int32)
    return i, ((i + 1) % N).astype(np.int32)


def _binned_mean(x, nbin=50):
    b = np.asarray(x).reshape(nbin, -1).mean(1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nbin)


def test_ising_ring_closed_forms():
    N, beta = 12, 0.45
    bi, bj = _ring(N)
    g = oracle.GraphOracle(N, bi, bj, 1, 21, "random")
    g.sweep(beta, 200)
    tr = g.sweep(beta, 40000, trace=True)
    t = np.tanh(beta)
    E_exact = -N * (t + t ** (N - 1)) / (1 + t ** N)
    M2_exact = N * sum((t ** r + t ** (N - r)) / (1 + t ** N) for r in range(N))
    Em, Ee = _binned_mean(tr[:, 0])
    mm, me = _binned_mean(tr[:, 1])
    assert abs(Em - E_exact) < 5 * Ee
    assert abs(mm - M2_exact / N ** 2) < 5 * me


@pytest.mark.parametrize("model,beta", [(2, 1.2), (3, 1.5)])
def test_vector_ring_energy(model, beta):
    special = pytest.importorskip("scipy.special")
    N = 32
    bi, bj = _ring(N)
    g = oracle.GraphOracle(N, bi, bj, model, 4, "random")
    g.sweep(beta, 200)
    tr = g.sweep(beta, 20000, trace=True)
    u = special.i1(beta) / special.i0(beta) if model == 2 else 1 / np.tanh(beta) - 1 / beta
    Em, Ee = _binned_mean(tr[:, 0])
    assert abs(Em + N * u) < 5 * Ee + 1e-6


def test_diluted_graph_samples_the_boltzmann_distribution_of_its_occupied_part():
    """On a small irregular graph with a vacant site and a masked bond, the
    chain's states of the occupied sites are distributed as exp(-beta E)
    with E over the present bonds only (exact enumeration), and the vacant
    site's spin never changes."""
    edges = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (3, 4), (4, 5), (1, 5)]
    bi = np.array([e[0] for e in edges], dtype=np.int32)
    bj = np.array([e[1] for e in edges], dtype=np.int32)
    site = np.array([1, 1, 1, 1, 0, 1], dtype=np.uint8)
    bond = np.array([1, 1, 1, 1, 0, 1, 1, 1], dtype=np.uint8)  # (0, 2) absent
    present = [e for k, e in enumerate(edges) if bond[k] and site[e[0]] and site[e[1]]]
    occ = [i for i in range(6) if site[i]]
    beta = 0.6
    g = oracle.GraphOracle(6, bi, bj, 1, 31, "random", site_mask=site, edge_mask=bond)
    s4 = g.spins()[4]
    n = 60000
    counts = np.zeros(2 ** len(occ))
    for _ in range(n):
        g.sweep(beta)
        s = g.spins()
        assert s[4] == s4
        counts[sum(((1 - s[i]) // 2) << k for k, i in enumerate(occ))] += 1
    E = np.zeros(2 ** len(occ))
    for a in range(2 ** len(occ)):
        sig = {i: 1 - 2 * ((a >> k) & 1) for k, i in enumerate(occ)}
        E[a] = -sum(sig[i] * sig[j] for i, j in present)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    f = counts / n
    sigma = np.sqrt(pi * (1 - pi) / (n / 4))  # a generous autocorrelation allowance
    assert (np.abs(f - pi) < 5 * sigma + 1e-4).all()
