"""Exact detailed balance of the Swendsen-Wang Ising rule (SW87, Sec. 1-2)
with the oracle's own bond probability (threshold / 2^32) and cluster
routine, on one tetrahedron (K4) and on two corner-sharing tetrahedra (the
pyrochlore motif, Sec. 2).  The full transition matrix is built by
enumerating every state, every subset of satisfied bonds and every flip
pattern of the resulting clusters.  Balance is exact at the inverse
temperature that the 32-bit threshold realises."""
import itertools

import numpy as np
import pytest

import oracle

K4 = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
TWO_TETS = K4 + [(3, 4), (3, 5), (3, 6), (4, 5), (4, 6), (5, 6)]


def transition_matrix(n, edges, beta):
    p = oracle.threshold(beta) / 2 ** 32
    bi = np.array([e[0] for e in edges], dtype=np.int32)
    bj = np.array([e[1] for e in edges], dtype=np.int32)
    S = 2 ** n
    T = np.zeros((S, S))
    for a in range(S):
        sig = np.array([1 - 2 * ((a >> k) & 1) for k in range(n)])
        sat = [b for b, (i, j) in enumerate(edges) if sig[i] == sig[j]]
        for r in range(len(sat) + 1):
            for sub in itertools.combinations(sat, r):
                prob = p ** r * (1 - p) ** (len(sat) - r)
                act = np.zeros(len(edges), dtype=np.uint8)
                act[list(sub)] = 1
                lab = oracle.clusters(n, bi, bj, act)
                roots = sorted(set(lab.tolist()))
                for fl in range(2 ** len(roots)):
                    flipped = {roots[k] for k in range(len(roots)) if (fl >> k) & 1}
                    b = a
                    for i in range(n):
                        if lab[i] in flipped:
                            b ^= 1 << i
                    T[a, b] += prob / 2 ** len(roots)
    return T


@pytest.mark.parametrize("n,edges", [(4, K4), (7, TWO_TETS)])
@pytest.mark.parametrize("beta", [0.2, 1 / 4.21394, 0.9])
def test_detailed_balance(n, edges, beta):
    T = transition_matrix(n, edges, beta)
    assert np.allclose(T.sum(1), 1.0, atol=1e-12)
    E = np.array([-sum((1 - 2 * ((a >> i) & 1)) * (1 - 2 * ((a >> j) & 1)) for i, j in edges)
                  for a in range(2 ** n)], dtype=np.float64)
    # The 32-bit threshold realises p_q = floor(p 2^32) / 2^32, i.e. the SW rule
    # at beta_eff = -log(1 - p_q) / 2, within 2^-32 / (2 (1 - p)) of beta.
    p_q = oracle.threshold(beta) / 2 ** 32
    beta_eff = -np.log1p(-p_q) / 2
    assert abs(beta_eff - beta) < 2.0 ** -32 / (2 * (1 - p_q))
    pi = np.exp(-beta_eff * (E - E.min()))
    pi /= pi.sum()
    F = pi[:, None] * T
    assert np.abs(F - F.T).max() < 1e-14
    # and the chain is ergodic on the state space (irreducible)
    R = (T > 0) | np.eye(len(T), dtype=bool)
    reach = R.copy()
    for _ in range(len(T)):
        reach = (reach.astype(np.int64) @ R.astype(np.int64)) > 0
    assert reach.all()
