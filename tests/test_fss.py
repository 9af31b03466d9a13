"""The finite-size-scaling harness (Sec. 3, Eq. 2-4) on the CPU.

Pins: the jackknife of a plain mean equals the standard error exactly, and
a ratio's jackknife equals a brute-force leave-one-out evaluation; crossings
of straight lines are exact; the collapse fits recover the T_c, nu and
beta/nu that synthetic data were generated with; and the binned-run
pipeline, driven by the oracle, reproduces the exact enumeration of the
L = 1 cell and the beta = 0 closed form U = 1 + 2 (N - 1)/(n N)."""
import numpy as np
import pytest

import oracle
import refmath
from paper_1612_08312_gb300 import fss
from test_oracle_equilibrium import l1_bonds


class OracleRunner:
    """The oracle behind the runner interface of fss.run_bins (replica r =
    iL * len(Ts) + iT, as there)."""

    def __init__(self, Ls, Ts, model, seed=7):
        self.reps = []
        for L in Ls:
            for T in Ts:
                self.reps.append((oracle.Oracle(L, model, seed + len(self.reps), "random"), 1.0 / T))

    def sweep(self, n):
        for o, beta in self.reps:
            o.sweep(beta, n)

    def reset_stats(self):
        for o, _ in self.reps:
            o.reset_stats()

    def stats(self, r):
        return self.reps[r][0].stats()

    def close(self):
        pass


def test_jackknife_of_a_mean_is_the_standard_error():
    x = np.random.default_rng(3).normal(size=(4, 5, 37))
    full, err, _ = fss.jackknife(lambda a: a, x)
    assert np.allclose(full, x.mean(-1), rtol=0, atol=1e-15)
    assert np.allclose(err, x.std(-1, ddof=1) / np.sqrt(37), rtol=1e-12, atol=0)


def test_jackknife_of_a_ratio_equals_brute_force_leave_one_out():
    rng = np.random.default_rng(4)
    m2 = rng.uniform(0.2, 0.3, size=23)
    m4 = m2 ** 2 * rng.uniform(1.2, 1.4, size=23)
    U, err, _ = fss.jackknife(lambda a, b: b / (a * a), m2, m4)
    vals = []
    for k in range(23):
        keep = np.arange(23) != k
        vals.append(m4[keep].mean() / m2[keep].mean() ** 2)
    vals = np.array(vals)
    ref = np.sqrt(22 / 23 * ((vals - vals.mean()) ** 2).sum())
    assert U == pytest.approx(m4.mean() / m2.mean() ** 2, rel=1e-14)
    assert err == pytest.approx(ref, rel=1e-10)


def test_crossing_of_straight_lines_is_exact():
    Ts = [4.17, 4.19, 4.23, 4.25]
    Ua = [1.2 + 2.0 * (T - 4.2) for T in Ts]
    Ub = [1.2 + 3.5 * (T - 4.2) for T in Ts]
    assert fss.crossing_temperature(Ts, Ua, Ub) == pytest.approx(4.2, abs=1e-12)
    assert np.isnan(fss.crossing_temperature(Ts, [1, 1, 1, 1], [2, 2, 2, 2]))


def synthetic_run(Tc=4.2, nu=0.63, bnu=0.52, Ls=(8, 12, 16, 24), noise=2e-3, nbins=12, seed=5):
    """Bins whose means follow U = f1(x) (Eq. 3) and <m^2> = size^(-2 beta/nu) f2(x)
    (Eq. 4) exactly, x = t size^(1/nu), with relative noise per bin.  The
    temperature window keeps |x| below about 1.6, as a grid around T_c does."""
    Ts = np.linspace(4.19, 4.21, 9)
    rng = np.random.default_rng(seed)
    m2 = np.zeros((len(Ls), len(Ts), nbins))
    m4 = np.zeros_like(m2)
    for i, L in enumerate(Ls):
        size = fss.linear_size(L)
        x = (Ts - Tc) / Tc * size ** (1.0 / nu)
        U = 2.0 + 0.8 * np.tanh(0.9 * x - 0.3)
        M2 = size ** (-2 * bnu) * np.exp(-0.7 * x)
        for b in range(nbins):
            a = M2 * (1 + noise * rng.standard_normal(len(Ts)))
            m2[i, :, b] = a
            m4[i, :, b] = U * a * a * (1 + noise * rng.standard_normal(len(Ts)))
    return fss.BinnedRun(list(Ls), list(Ts), 1, m2, m4, np.zeros_like(m2), 100)


def test_collapse_fit_recovers_the_scaling_parameters():
    run = synthetic_run()
    fit = fss.fit_collapse(run, Tc0=4.197, nu0=0.7)
    assert fit["Tc"] == pytest.approx(4.2, abs=1e-4)
    assert fit["nu"] == pytest.approx(0.63, abs=0.01)
    assert fit["beta_over_nu"] == pytest.approx(0.52, abs=5e-3)
    assert fit["Tc_err"] < 1e-3 and fit["nu_err"] < 0.01
    # errors of the size of the noise: the criterion sits near 1 at the minimum
    assert 0.2 < fit["S_U"] < 5
    # wrong parameters collapse worse
    U, Uerr, _ = fss.moment_ratio(run)
    assert fss._u_collapse(run.Ls, run.Ts, U, Uerr, 4.205, 0.63) > 10 * fit["S_U"]


def test_crossings_of_synthetic_curves_sit_at_tc():
    # U depends on t size^(1/nu) only, so every pair of sizes crosses at T_c exactly
    run = synthetic_run(noise=1e-6)
    for c in fss.crossings(run):
        assert c["T"] == pytest.approx(4.2, abs=1e-4)
        assert c["err"] < 1e-4


def test_binned_oracle_run_matches_exact_enumeration():
    T = 4.21394
    bi, bj = l1_bonds()
    ex = refmath.enumerate_ising(bi, bj, 16, 1.0 / T)
    run = fss.run_bins([1], [T], model=1, eq_sweeps=500, nbins=40, bin_sweeps=1000,
                       runner=OracleRunner([1], [T], 1))
    U, Uerr, _ = fss.moment_ratio(run)
    M2, M2err, _ = fss.jackknife(lambda a: a, run.m2)
    E, Eerr, _ = fss.jackknife(lambda a: a, run.e)
    assert abs(U[0, 0] - ex["m4"] / ex["m2"] ** 2) < 4 * Uerr[0, 0]
    assert abs(M2[0, 0] - ex["m2"]) < 4 * M2err[0, 0]
    assert abs(E[0, 0] - ex["E"] / 16) < 4 * Eerr[0, 0]


@pytest.mark.parametrize("model", [1, 2])
def test_binned_oracle_run_at_beta_zero_gives_the_closed_form(model):
    N = 16
    run = fss.run_bins([1], [float("inf")], model=model, eq_sweeps=10, nbins=40, bin_sweeps=500,
                       runner=OracleRunner([1], [float("inf")], model))
    U, Uerr, _ = fss.moment_ratio(run)
    m2, m4 = refmath.independent_moments(N, model)
    assert abs(U[0, 0] - m4 / m2 ** 2) < 4 * Uerr[0, 0]
    assert m4 / m2 ** 2 == pytest.approx(1 + 2 * (N - 1) / (model * N))


def test_run_bins_rejects_a_single_bin():
    with pytest.raises(ValueError):
        fss.run_bins([1], [4.2], nbins=1, runner=OracleRunner([1], [4.2], 1))
