"""Statistical and closed-form pins of the oracle's Swendsen-Wang chain.

* Ising, L = 1 (16 sites, 48 bonds): exact Boltzmann averages by enumerating
  all 2^16 states (Eq. 1, Eq. 2) against long oracle runs.
* beta = 0: independent spins, closed-form <m^2>, <m^4>, U = 1 + 2(N-1)/(nN)
  -> (n+2)/n (Sec. 3: the high-temperature limit of U).
* beta large from the ordered state: one cluster, E = -3JN (ground state of
  Eq. 1), U = 1 (Sec. 3: the T -> 0 limit of U).
* XY / Heisenberg, L = 1: long oracle runs against an independent
  single-site Metropolis chain with the same stationary distribution.
"""
import numpy as np
import pytest

import oracle
import refmath


def l1_bonds():
    pos = np.array([oracle.site_position(1, i) for i in range(16)])
    nbrs, _ = refmath.brute_force_neighbours(pos, 4)
    bi, bj = [], []
    for i in range(16):
        for j in sorted(nbrs[i]):
            if j > i:
                bi.append(i)
                bj.append(j)
    return np.array(bi), np.array(bj)


@pytest.mark.parametrize("T", [4.21394, 2.0, 8.0])
def test_ising_l1_matches_enumeration(T):
    bi, bj = l1_bonds()
    assert len(bi) == 48
    beta = 1.0 / T
    ex = refmath.enumerate_ising(bi, bj, 16, beta)
    o = oracle.Oracle(1, oracle.ISING, seed=11, start="random")
    o.sweep(beta, 2000)
    tr = o.sweep(beta, 300000, trace=True)
    for col, key in ((0, "E"), (1, "m2"), (2, "m4")):
        mean, se = refmath.binned_mean_se(tr[:, col], 100)
        assert abs(mean - ex[key]) < 4 * se + 1e-12, (key, mean, ex[key], se)
    # the accumulated compensated sums equal the correctly rounded sums of
    # the per-sweep values (math.fsum) to within an ulp or two
    import math
    o.reset_stats()
    tr = o.sweep(beta, 50000, trace=True)
    st = o.stats()
    assert st["count"] == 50000
    for key, col in (("sum_E", tr[:, 0]), ("sum_E2", tr[:, 0] ** 2), ("sum_m2", tr[:, 1]),
                     ("sum_m4", tr[:, 2]), ("sum_absm", np.sqrt(tr[:, 1]))):
        exact = math.fsum(col.tolist())
        assert abs(st[key] - exact) <= 4 * np.spacing(abs(exact)), key


def test_ising_l1_enumeration_limits():
    bi, bj = l1_bonds()
    hot = refmath.enumerate_ising(bi, bj, 16, 1e-9)
    assert abs(hot["m4"] / hot["m2"] ** 2 - 2.875) < 1e-6  # 1 + 2*15/16
    cold = refmath.enumerate_ising(bi, bj, 16, 50.0)
    assert abs(cold["E"] + 48.0) < 1e-9 and abs(cold["m4"] / cold["m2"] ** 2 - 1.0) < 1e-12


@pytest.mark.parametrize("model", [1, 2, 3])
def test_beta_zero_independent_spins(model):
    L = 1
    N = 16
    o = oracle.Oracle(L, model, seed=5, start="random")
    tr = o.sweep(0.0, 200000, trace=True)
    # no bond is ever active: every site is its own cluster
    assert (o.labels() == np.arange(N)).all()
    assert o.active().sum() == 0
    m2, m4 = refmath.independent_moments(N, model)
    for col, want in ((1, m2), (2, m4)):
        mean, se = refmath.binned_mean_se(tr[:, col], 100)
        assert abs(mean - want) < 4 * se, (col, mean, want, se)
    U = tr[:, 2].mean() / tr[:, 1].mean() ** 2
    assert abs(U - (1 + 2 * (N - 1) / (model * N))) < 0.02


@pytest.mark.parametrize("model", [1, 2, 3])
@pytest.mark.parametrize("L", [1, 2])
def test_ordered_state_at_large_beta(model, L):
    o = oracle.Oracle(L, model, seed=3, start="up")
    E0, m2, m4 = o.measure()
    assert E0 == -3.0 * o.N and m2 == 1.0 and m4 == 1.0
    for _ in range(5):
        o.sweep(40.0, 1)
        assert (o.labels() == 0).all()  # one cluster, canonical label 0
        E, m2, m4 = o.measure()
        assert abs(E + 3.0 * o.N) < 1e-9 * o.N
        assert abs(m2 - 1.0) < 1e-12 and abs(m4 - 1.0) < 1e-12


@pytest.mark.parametrize("model", [1, 2, 3])
def test_measure_matches_definition(model):
    L = 2
    o = oracle.Oracle(L, model, seed=2, start="random")
    o.sweep(0.3, 3)
    s = o.spins().astype(np.float64).reshape(o.N, -1)
    pos = np.array([oracle.site_position(L, i) for i in range(o.N)])
    nbrs, _ = refmath.brute_force_neighbours(pos, 4 * L)
    E = -0.5 * sum(float(s[i] @ s[j]) for i in range(o.N) for j in nbrs[i])
    M = s.sum(0)
    m = np.linalg.norm(M) / o.N
    E_o, m2_o, m4_o = o.measure()
    assert abs(E_o - E) < 1e-10 * o.N
    assert abs(m2_o - m * m) < 1e-14 and abs(m4_o - m ** 4) < 1e-14


@pytest.mark.parametrize("model,T", [(2, 1.2), (3, 0.9)])
def test_vector_l1_matches_metropolis(model, T):
    beta = 1.0 / T
    o = oracle.Oracle(1, model, seed=21, start="random")
    o.sweep(beta, 2000)
    tr = o.sweep(beta, 200000, trace=True)
    pos = np.array([oracle.site_position(1, i) for i in range(16)])
    nbrs, _ = refmath.brute_force_neighbours(pos, 4)
    nbr = np.array([sorted(s) for s in nbrs])
    mc = refmath.metropolis_nvector(nbr, model, beta, chains=1024, sweeps=400, burn=100, seed=4)
    for col in range(3):
        a, sa = refmath.binned_mean_se(tr[:, col], 100)
        per_chain = mc[:, col, :].mean(0)  # independent chains
        b, sb = per_chain.mean(), per_chain.std(ddof=1) / np.sqrt(per_chain.size)
        assert abs(a - b) < 4 * np.hypot(sa, sb), (col, a, b, sa, sb)
