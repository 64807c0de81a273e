"""Pins of the oracle's time correlation <delta_i(t + l K) delta_i(t)> (the
exercise on <dT_i^{n+m} dT_i^n> of Sec. 6; delta = T - T_ref, lags in whole
sampling intervals, sample pairs within one run, pooled over realizations).

* The accumulator equals its definition on stored trajectories, and lag 0 is
  the pooled second moment.
* The conditional mean of one step is affine in the state (forward Euler:
  the noise has mean zero; the heat predictor-corrector step: by
  quadrature), so E[T^{t+j} (T^t)^T] = M^j E[T^t (T^t)^T] + c_j E[T^t]^T
  exactly; the oracle's pooled correlations lie within a few batch standard
  errors of it.
* At equilibrium on a periodic grid every Fourier mode decays by
  lambda_k = 1 - r mu_k per step, so the cell-averaged correlation is
  (1/N^2) sum_k lambda_k^{l K} S_k; a larger conductivity (larger r)
  decorrelates faster, the exercise's question.
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she, theory


def _td(p):
    r, eps = she.dimensionless(p)
    return {"dim": p["dim"], "n": p["n"], "bc": p["bc"], "r": r, "eps": eps,
            "wall_lo": p["wall_lo"], "wall_hi": p["wall_hi"],
            "equation": p["equation"], "perturb_ic": p["perturb_ic"],
            "scheme": p.get("scheme", "fe")}


def test_accumulator_matches_definition():
    p = W.oracle_rod(n=(5, 1, 1), bc="periodic", wall_lo=1.5, wall_hi=1.5, kB=0.01, stats_interval=2,
                     relax_steps=1, tc_lags=3)
    R, nsteps = 2, 11
    o = she.run(p, R, nsteps)
    tref = she.reference_profile(p)
    ref = np.zeros((3, 5))
    for rho in range(R):
        T = she.run(p, 1, 0, stream0=rho)["state"][0]
        snaps = []
        for n in range(nsteps):
            T = she.step(p, T, n, rho)
            m = n + 1
            if m % 2 == 0 and m > 1:
                snaps.append(T - tref)
        for s in range(len(snaps)):
            for l in range(min(3, s + 1)):
                ref[l] += snaps[s] * snaps[s - l]
    assert np.allclose(o["sum_tc"], ref, rtol=1e-12, atol=1e-15)
    assert np.array_equal(o["sum_tc"][0], o["sum_d2"])
    ns = o["n_samples_per_realization"]
    assert list(o["n_tc"]) == [R * max(0, ns - l) for l in range(3)]


@pytest.mark.parametrize("maker", [
    lambda: W.oracle_rod(n=(4, 1, 1), wall_lo=1.0, wall_hi=3.0, kB=0.02),
    lambda: W.oracle_rod(n=(5, 1, 1), bc="periodic", wall_lo=2.0, wall_hi=2.0, kB=0.01),
    lambda: W.oracle_rod(n=(4, 1, 1), equation="species", n0=50.0, D=1.0, dt=0.2, wall_lo=1.0, wall_hi=2.0),
    lambda: W.oracle_rod(n=(4, 1, 1), wall_lo=1.0, wall_hi=3.0, kB=0.02, scheme="pc")])
def test_time_corr_matches_exact_recursion(maker):
    L, K, relax, nsteps, R, B = 6, 2, 10, 60, 2000, 16
    p = dict(maker(), stats_interval=K, relax_steps=relax, tc_lags=L)
    ex, cnt = theory.lagged_expectation(_td(p), nsteps, K, relax, L)
    vals = []
    for b in range(B):
        o = she.run(p, R, nsteps, stream0=b * R)
        assert list(o["n_tc"]) == list((cnt * R).astype(int))
        vals.append(she.finalize(p, o)["time_corr"])
    vals = np.array(vals)
    z = (vals.mean(axis=0) - ex) / (vals.std(axis=0, ddof=1) / np.sqrt(B))
    assert np.max(np.abs(z)) < 4.5, z
    assert np.mean(z * z) < 2.5, z
    # the correlation decays with the lag
    assert np.all(np.abs(ex[-1]) < np.abs(ex[0]))


def _equilibrium_corr(kappa, L):
    N, B, R = 16, 12, 64
    p = W.oracle_rod(n=(N, 1, 1), bc="periodic", kB=1e-4, kappa=kappa, stats_interval=1, relax_steps=400,
                     tc_lags=L)
    r, eps = she.dimensionless(p)
    vals = []
    for b in range(B):
        o = she.run(p, R, 1400, stream0=b * R)
        vals.append(she.finalize(p, o)["time_corr"].mean(axis=1))    # averaged over the cells
    vals = np.array(vals)
    k = np.arange(N)
    mu = 4.0 * np.sin(np.pi * k / N) ** 2
    Sk = theory.structure_factor((N,), r, eps * 1.0)
    ex = np.array([np.sum((1.0 - r * mu) ** l * Sk) / N ** 2 for l in range(L)])
    return vals, ex


def test_time_corr_decay_closed_form_and_conductivity():
    L = 8
    v1, e1 = _equilibrium_corr(1.0, L)       # r = 0.2
    v2, e2 = _equilibrium_corr(0.5, L)       # r = 0.1
    for vals, ex in ((v1, e1), (v2, e2)):
        z = (vals.mean(axis=0) - ex) / (vals.std(axis=0, ddof=1) / np.sqrt(len(vals)))
        assert np.max(np.abs(z)) < 4.5, z
    # higher conductivity, faster decorrelation
    assert e1[L - 1] / e1[0] < 0.8 * e2[L - 1] / e2[0]
    assert v1.mean(axis=0)[L - 1] / v1.mean(axis=0)[0] < v2.mean(axis=0)[L - 1] / v2.mean(axis=0)[0]
