"""The finite-size-scaling harness through the batched GPU sweep.

The binned runs of fss.run_bins on the GPU reproduce the exact enumeration
of the L = 1 cell, agree with the oracle's binned run at L = 2 within three
combined standard errors, give the beta = 0 closed form
U = 1 + 2 (N - 1)/(n N), and feed the crossing and collapse analysis."""
import numpy as np
import pytest

import refmath
from paper_1612_08312_gb300 import fss
from test_fss import OracleRunner
from test_oracle_equilibrium import l1_bonds

pytestmark = pytest.mark.gpu

T = 4.21394


def test_gpu_binned_run_matches_enumeration_and_oracle():
    run = fss.run_bins([1, 2], [T], model=1, eq_sweeps=500, nbins=40, bin_sweeps=1000, seed=3)
    U, Uerr, _ = fss.moment_ratio(run)
    bi, bj = l1_bonds()
    ex = refmath.enumerate_ising(bi, bj, 16, 1.0 / T)
    assert abs(U[0, 0] - ex["m4"] / ex["m2"] ** 2) < 4 * Uerr[0, 0]
    ref = fss.run_bins([2], [T], model=1, eq_sweeps=500, nbins=40, bin_sweeps=1000,
                       runner=OracleRunner([2], [T], 1))
    Ur, Urerr, _ = fss.moment_ratio(ref)
    assert abs(U[1, 0] - Ur[0, 0]) < 3 * np.hypot(Uerr[1, 0], Urerr[0, 0])
    for name in ("m2", "e"):
        g, ge, _ = fss.jackknife(lambda a: a, getattr(run, name))
        o, oe, _ = fss.jackknife(lambda a: a, getattr(ref, name))
        assert abs(g[1, 0] - o[0, 0]) < 3 * np.hypot(ge[1, 0], oe[0, 0]), name


@pytest.mark.parametrize("model", [1, 2, 3])
def test_gpu_binned_run_at_beta_zero_gives_the_closed_form(model):
    L, N = 2, 128
    run = fss.run_bins([L], [float("inf")], model=model, eq_sweeps=20, nbins=40, bin_sweeps=500, seed=9)
    U, Uerr, _ = fss.moment_ratio(run)
    m2, m4 = refmath.independent_moments(N, model)
    assert abs(U[0, 0] - m4 / m2 ** 2) < 4 * Uerr[0, 0]


def test_gpu_analysis_of_a_small_grid():
    Ts = [4.16, 4.19, 4.22, 4.25, 4.28]
    run = fss.run_bins([4, 6, 8], Ts, model=1, eq_sweeps=200, nbins=20, bin_sweeps=200, seed=5)
    out = fss.analyse(run, Tc0=4.21)
    assert len(out["table"]) == 15 and len(out["crossings"]) == 2
    U = np.array([row["U"] for row in out["table"]]).reshape(3, 5)
    # U grows with T (towards 3) at every size
    assert (np.diff(U, axis=1) > 0).all()
    assert np.isfinite(out["collapse"]["Tc"]) and np.isfinite(out["collapse"]["nu"])
