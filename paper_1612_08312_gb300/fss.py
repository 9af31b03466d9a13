"""Finite-size-scaling analysis of the moment ratio (Sec. 3, Eq. 2-4).

The paper locates each critical point with the moment ratio
U = <m^4>/<m^2>^2 of Eq. 2.  Curves U(T) of different sizes cross near T_c
(Fig. 2); with the right T_c and nu they collapse onto one function of
t (N^{1/3})^{1/nu}, t = (T - T_c)/T_c (Eq. 3), and <m^2> (N^{1/3})^{2 beta/nu}
collapses the same way (Eq. 4).  The linear size is N^{1/3} = 16^{1/3} L.

This module runs replicas over a grid of sizes and temperatures through the
batched GPU sweep, in bins of sweeps, and evaluates
  - U and <m^2> per (L, T), with jackknife errors over the bins;
  - the crossing temperature of U(T) for each pair of successive sizes (the
    root of U_a - U_b, linearly interpolated between grid temperatures);
  - T_c and nu that best collapse U (Eq. 3), then beta/nu that best
    collapses <m^2> (Eq. 4).  The paper gives the best choices but not how
    they were found; here they minimise a collapse criterion: the mean, over
    every point and every other size whose curve spans the point's scaling
    variable, of the squared distance to that curve (interpolated
    quadratically through its three nearest points) over the summed
    variances.  Near the minimum this mean is about 1 when the sizes agree
    within their errors.
Errors of crossings and fits are jackknife errors over the bins.

Usage: python -m paper_1612_08312_gb300.fss --model 1 --L 32 48 64 96
       --T 4.205 4.21 4.2125 4.215 4.2175 4.22 [--eq 2000 --bins 40 --bin-sweeps 500]
prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np

N_COMPONENTS = {1: 1, 2: 2, 3: 3}  # Ising, XY, Heisenberg


@dataclass
class BinnedRun:
    """Bin means of one run: arrays indexed (size, temperature, bin)."""

    Ls: list
    Ts: list
    model: int
    m2: np.ndarray
    m4: np.ndarray
    e: np.ndarray  # energy per site
    bin_sweeps: int
    seconds: float = 0.0
    meta: dict = field(default_factory=dict)


def linear_size(L) -> np.ndarray:
    """N^{1/3} = 16^{1/3} L, the linear size the paper's scaling forms use."""
    return np.cbrt(16.0) * np.asarray(L, dtype=np.float64)


def run_bins(Ls, Ts, model: int = 1, precision: int = 0, eq_sweeps: int = 1000, nbins: int = 40,
             bin_sweeps: int = 200, seed: int = 1, runner=None) -> BinnedRun:
    """Run one replica per (L, T), row-major (replica r = iL * len(Ts) + iT),
    for eq_sweeps unmeasured sweeps and then nbins bins of bin_sweeps sweeps.
    `runner` is any object with sweep(n), reset_stats(), stats(r) (a dict
    with count, sum_E, sum_m2, sum_m4) and close(); by default the batched
    GPU sweep (Replicas) with replica seeds derived from `seed`."""
    from . import Replicas

    Ls, Ts = [int(L) for L in Ls], [float(T) for T in Ts]
    if nbins < 2 or bin_sweeps < 1:
        raise ValueError("need at least two bins of at least one sweep")
    flat_L = [L for L in Ls for _ in Ts]
    flat_b = [1.0 / T for _ in Ls for T in Ts]
    own = runner is None
    if own:
        runner = Replicas(flat_L, flat_b, model=model, precision=precision, start="random", seed=seed)
    shape = (len(Ls), len(Ts), nbins)
    m2, m4, e = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    t0 = time.perf_counter()
    try:
        if eq_sweeps > 0:
            runner.sweep(eq_sweeps)
        for b in range(nbins):
            runner.reset_stats()
            runner.sweep(bin_sweeps)
            for r, L in enumerate(flat_L):
                s = runner.stats(r)
                n = s["count"]
                if n != bin_sweeps:
                    raise RuntimeError(f"replica {r}: {n} measurements in a bin of {bin_sweeps} sweeps")
                i, j = divmod(r, len(Ts))
                m2[i, j, b] = s["sum_m2"] / n
                m4[i, j, b] = s["sum_m4"] / n
                e[i, j, b] = s["sum_E"] / n / (16 * L ** 3)
    finally:
        if own:
            runner.close()
    return BinnedRun(Ls, Ts, model, m2, m4, e, bin_sweeps, time.perf_counter() - t0,
                     dict(eq_sweeps=eq_sweeps, nbins=nbins, seed=seed, precision=precision))


def jackknife(f, *bins):
    """f applied to the bin means, its jackknife error, and the leave-one-out
    values.  Every array holds the bins along its last axis; f must work
    elementwise (it is called with the means, and with the leave-one-out
    means along a last axis of length nbins)."""
    n = bins[0].shape[-1]
    full = f(*[b.mean(-1) for b in bins])
    loo = [(b.sum(-1, keepdims=True) - b) / (n - 1) for b in bins]
    vals = f(*loo)
    err = np.sqrt((n - 1) / n * ((vals - vals.mean(-1, keepdims=True)) ** 2).sum(-1))
    return full, err, vals


def moment_ratio(run: BinnedRun):
    """U = <m^4>/<m^2>^2 (Eq. 2) per (L, T): value, error, leave-one-out values."""
    return jackknife(lambda a, b: b / (a * a), run.m2, run.m4)


def crossing_temperature(Ts, Ua, Ub) -> float:
    """Temperature where Ua(T) - Ub(T) first changes sign on the grid Ts
    (ascending), by linear interpolation; NaN if it does not."""
    Ts = np.asarray(Ts, dtype=np.float64)
    d = np.asarray(Ua, dtype=np.float64) - np.asarray(Ub, dtype=np.float64)
    for i in range(len(Ts) - 1):
        if d[i] == 0.0:
            return float(Ts[i])
        if d[i] * d[i + 1] < 0.0:
            return float(Ts[i] - d[i] * (Ts[i + 1] - Ts[i]) / (d[i + 1] - d[i]))
    return float(Ts[-1]) if d[-1] == 0.0 else float("nan")


def crossings(run: BinnedRun) -> list:
    """Crossing temperature of U(T) for each pair of successive sizes, with
    its jackknife error."""
    U, _, Uj = moment_ratio(run)
    out = []
    for a in range(len(run.Ls) - 1):
        Tx = crossing_temperature(run.Ts, U[a], U[a + 1])
        samples = np.array([crossing_temperature(run.Ts, Uj[a, :, k], Uj[a + 1, :, k])
                            for k in range(Uj.shape[-1])])
        n = len(samples)
        ok = np.isfinite(samples)
        err = float(np.sqrt((n - 1) / n * ((samples - samples.mean()) ** 2).sum())) if ok.all() else float("nan")
        out.append(dict(L=[run.Ls[a], run.Ls[a + 1]], T=Tx, err=err))
    return out


def _interpolate(xb, yb, sb, x):
    """Values and variances of the curve (xb ascending, yb, errors sb) at the
    points x inside its range: Lagrange interpolation through the three grid
    points nearest to each x (two if the curve has only two), variances
    propagated through the squared weights."""
    n = len(xb)
    k = np.clip(np.searchsorted(xb, x, side="right") - 1, 0, n - 2)
    if n < 3:
        w = (x - xb[k]) / (xb[k + 1] - xb[k])
        return (1 - w) * yb[k] + w * yb[k + 1], (1 - w) ** 2 * sb[k] ** 2 + w ** 2 * sb[k + 1] ** 2
    # triple k-1, k, k+1 or k, k+1, k+2: the one centred nearer to x
    right = (k == 0) | ((k + 2 < n) & (x - xb[k] > xb[k + 1] - x))
    i0 = np.where(right, k, k - 1)
    i0 = np.clip(i0, 0, n - 3)
    x0, x1, x2 = xb[i0], xb[i0 + 1], xb[i0 + 2]
    w0 = (x - x1) * (x - x2) / ((x0 - x1) * (x0 - x2))
    w1 = (x - x0) * (x - x2) / ((x1 - x0) * (x1 - x2))
    w2 = (x - x0) * (x - x1) / ((x2 - x0) * (x2 - x1))
    y = w0 * yb[i0] + w1 * yb[i0 + 1] + w2 * yb[i0 + 2]
    v = w0 ** 2 * sb[i0] ** 2 + w1 ** 2 * sb[i0 + 1] ** 2 + w2 ** 2 * sb[i0 + 2] ** 2
    return y, v


def collapse_quality(xs, ys, ss) -> float:
    """Mean of (y_i - y_j(x_i))^2 / (s_i^2 + s_j(x_i)^2) over every point i of
    every size and every other size j whose curve spans x_i; y_j and s_j^2
    interpolate size j's points (quadratically, through the three nearest).
    Infinite if no point is spanned by another size's curve."""
    terms = []
    for a in range(len(xs)):
        for b in range(len(xs)):
            if a == b:
                continue
            order = np.argsort(xs[b])
            xb, yb, sb = xs[b][order], ys[b][order], ss[b][order]
            inside = (xs[a] >= xb[0]) & (xs[a] <= xb[-1])
            if not inside.any():
                continue
            y, v = _interpolate(xb, yb, sb, xs[a][inside])
            terms.append((ys[a][inside] - y) ** 2 / (ss[a][inside] ** 2 + v))
    if not terms:
        return float("inf")
    return float(np.concatenate(terms).mean())


def _u_collapse(Ls, Ts, U, Uerr, Tc, nu):
    Ts = np.asarray(Ts, dtype=np.float64)
    xs = [(Ts - Tc) / Tc * linear_size(L) ** (1.0 / nu) for L in Ls]
    return collapse_quality(xs, list(U), list(Uerr))


def _m2_collapse(Ls, Ts, M2, M2err, Tc, nu, bnu):
    Ts = np.asarray(Ts, dtype=np.float64)
    xs, ys, ss = [], [], []
    for i, L in enumerate(Ls):
        scale = linear_size(L) ** (2.0 * bnu)
        xs.append((Ts - Tc) / Tc * linear_size(L) ** (1.0 / nu))
        ys.append(M2[i] * scale)
        ss.append(M2err[i] * scale)
    return collapse_quality(xs, ys, ss)


def _fit_tc_nu(Ls, Ts, U, Uerr, Tc0, nu0):
    from scipy.optimize import minimize
    res = minimize(lambda p: _u_collapse(Ls, Ts, U, Uerr, p[0], p[1]) if p[1] > 0.05 else np.inf,
                   x0=[Tc0, nu0], method="Nelder-Mead",
                   options=dict(xatol=1e-7, fatol=1e-9, maxiter=4000, initial_simplex=[
                       [Tc0, nu0], [Tc0 * (1 + 2e-3), nu0], [Tc0, nu0 * 1.1]]))
    return float(res.x[0]), float(res.x[1]), float(res.fun)


def _fit_bnu(Ls, Ts, M2, M2err, Tc, nu, lo=0.2, hi=1.0):
    from scipy.optimize import minimize_scalar
    res = minimize_scalar(lambda b: _m2_collapse(Ls, Ts, M2, M2err, Tc, nu, b), bounds=(lo, hi),
                          method="bounded", options=dict(xatol=1e-7))
    return float(res.x), float(res.fun)


def fit_collapse(run: BinnedRun, Tc0: float, nu0: float = 0.65) -> dict:
    """T_c and nu minimising the collapse criterion of U (Eq. 3), then beta/nu
    minimising that of <m^2> (Eq. 4) at those T_c and nu.  Errors: jackknife
    over the bins (each leave-one-out sample refitted with the full-sample
    error bars)."""
    U, Uerr, Uj = moment_ratio(run)
    M2, M2err, M2j = jackknife(lambda a: a, run.m2)
    Tc, nu, S = _fit_tc_nu(run.Ls, run.Ts, U, Uerr, Tc0, nu0)
    bnu, Sm = _fit_bnu(run.Ls, run.Ts, M2, M2err, Tc, nu)
    n = Uj.shape[-1]
    samples = []
    for k in range(n):
        t, v, _ = _fit_tc_nu(run.Ls, run.Ts, Uj[..., k], Uerr, Tc, nu)
        b, _ = _fit_bnu(run.Ls, run.Ts, M2j[..., k], M2err, t, v)
        samples.append((t, v, b))
    samples = np.array(samples)
    err = np.sqrt((n - 1) / n * ((samples - samples.mean(0)) ** 2).sum(0))
    return dict(Tc=Tc, Tc_err=float(err[0]), nu=nu, nu_err=float(err[1]), beta_over_nu=bnu,
                beta_over_nu_err=float(err[2]), S_U=S, S_m2=Sm)


def analyse(run: BinnedRun, Tc0: float, nu0: float = 0.65) -> dict:
    """U and <m^2> tables, crossings and collapse fits of one run."""
    U, Uerr, _ = moment_ratio(run)
    M2, M2err, _ = jackknife(lambda a: a, run.m2)
    E, Eerr, _ = jackknife(lambda a: a, run.e)
    table = [dict(L=L, T=T, U=float(U[i, j]), U_err=float(Uerr[i, j]), m2=float(M2[i, j]),
                  m2_err=float(M2err[i, j]), e=float(E[i, j]), e_err=float(Eerr[i, j]))
             for i, L in enumerate(run.Ls) for j, T in enumerate(run.Ts)]
    return dict(model=run.model, Ls=run.Ls, Ts=run.Ts, bins=int(run.m2.shape[-1]), bin_sweeps=run.bin_sweeps,
                table=table, crossings=crossings(run), collapse=fit_collapse(run, Tc0, nu0),
                seconds=run.seconds, **run.meta)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--model", type=int, default=1, choices=[1, 2, 3])
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1], help="0 FP32 spins, 1 FP64 (n-vector)")
    ap.add_argument("--L", type=int, nargs="+", required=True)
    ap.add_argument("--T", type=float, nargs="+", required=True)
    ap.add_argument("--eq", type=int, default=2000)
    ap.add_argument("--bins", type=int, default=40)
    ap.add_argument("--bin-sweeps", type=int, default=500)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--tc0", type=float, default=None, help="starting T_c of the fit (default: middle of --T)")
    ap.add_argument("--nu0", type=float, default=0.65)
    a = ap.parse_args(argv)
    Ts = sorted(a.T)
    run = run_bins(sorted(a.L), Ts, a.model, a.precision, a.eq, a.bins, a.bin_sweeps, a.seed)
    out = analyse(run, a.tc0 if a.tc0 is not None else Ts[len(Ts) // 2], a.nu0)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
