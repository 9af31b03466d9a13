"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11) against
cuRAND's implementation from the CUDA toolkit header, called on the host;
and of the derived quantities (Ising threshold, random unit axis)."""
import math

import numpy as np
import pytest

import oracle
import refmath


@pytest.fixture(scope="module")
def probe():
    lib = refmath.curand_philox_lib()
    if lib is None:
        pytest.skip("nvcc not available to build the cuRAND host probe")
    return lib


def test_philox_matches_curand(probe):
    rng = np.random.default_rng(123)
    n = 2000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = 0
    key[:2] = 0
    ctr[4] = 0xFFFFFFFF
    want = refmath.curand_philox(ctr, key)
    got = np.array([oracle.philox(ctr[t], key[t]) for t in range(n)])
    assert (got == want).all()


def test_threshold_reading():
    # T_beta = floor(p 2^32), p = 1 - exp(-2 beta J); 2^32 at p = 1, 0 at beta = 0
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(1e3) == 2 ** 32
    for beta in (0.1, 1 / 4.21394, 0.5, 2.0):
        p = 1.0 - math.exp(-2.0 * beta)
        t = oracle.threshold(beta)
        assert abs(t / 2 ** 32 - p) < 2e-9
        assert t == math.floor(-math.expm1(-2.0 * beta) * 2 ** 32)


@pytest.mark.parametrize("n", [2, 3])
def test_unit_vector_uniform_on_sphere(n, probe):
    # unit norm, isotropic first and second moments: <r> = 0, <r r^T> = I/n
    rs = np.array([oracle.unit_vector(7, s, 3, 0, n)[0] for s in range(20000)])
    assert np.allclose(np.linalg.norm(rs, axis=1), 1.0, atol=1e-15)
    assert np.abs(rs.mean(0)).max() < 4 / np.sqrt(20000)
    C = rs.T @ rs / len(rs)
    assert np.abs(C - np.eye(n) / n).max() < 6 / np.sqrt(20000)
    if n == 3:  # Archimedes: z uniform on [-1, 1]
        h, _ = np.histogram(rs[:, 2], bins=10, range=(-1, 1))
        assert np.abs(h / len(rs) - 0.1).max() < 0.01


def test_unit_vector_uses_stream_words(probe):
    # recompute attempt 0 from cuRAND words: u = signed word * 2^-31
    for s in range(50):
        w = refmath.curand_philox(np.array([[0, 0, s, 3]]), np.array([[9, 0]]))[0]
        u0 = float(np.int32(w[0].view(np.int32))) / 2 ** 31
        u1 = float(np.int32(w[1].view(np.int32))) / 2 ** 31
        ss = u0 * u0 + u1 * u1
        r, att = oracle.unit_vector(9, s, 3, 0, 2)
        if 0 < ss < 1:
            assert att == 1
            assert r[0] == u0 / math.sqrt(ss) and r[1] == u1 / math.sqrt(ss)
        else:
            assert att > 1
