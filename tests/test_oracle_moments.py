"""Statistical pins of the oracle against the exact moment recursion.

The face noise is independent of the state at the start of each step, so the
first two moments of the discrete scheme obey an exact closed recursion
(oracle/theory.py; heat noise ~ T_face, Eq. (2.12); species ~ sqrt(c_face),
Eq. (4.7)).  The oracle's sample statistics, pooled over realizations and
sampling times exactly as it accumulates them (Eq. (3.9)), must agree with
the recursion's expectations within a few standard errors taken over
independent realization batches.  A dropped sqrt(2) at a wall, a wrong noise
amplitude, a noise on the wrong face or with the wrong sign, or a wrong wall
stencil each moves some entry by many standard errors.
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she, theory


def _theory_dict(p):
    r, eps = she.dimensionless(p)
    return {"dim": p["dim"], "n": p["n"], "bc": p["bc"], "r": r, "eps": eps,
            "wall_lo": p["wall_lo"], "wall_hi": p["wall_hi"],
            "equation": p["equation"], "perturb_ic": p["perturb_ic"]}


def _batched(p, R, B, nsteps, want_cov=1):
    """Run B batches of R realizations (distinct streams); return per-batch
    mean-delta vectors and second-moment matrices."""
    m1, m2 = [], []
    for b in range(B):
        o = she.run(p, R, nsteps, stream0=b * R, want_cov=want_cov)
        n = o["n_samples"]
        m1.append(o["sum_d"] / n)
        m2.append(o["sum_dd"] / n)
    return np.array(m1), np.array(m2)


def _check(p, R, B, nsteps, zmax=4.5):
    m1, m2 = _batched(p, R, B, nsteps)
    ex = theory.pooled_expectation(_theory_dict(p), nsteps, p["stats_interval"],
                                   p["relax_steps"])
    se1 = m1.std(axis=0, ddof=1) / np.sqrt(B)
    se2 = m2.std(axis=0, ddof=1) / np.sqrt(B)
    z1 = (m1.mean(axis=0) - ex["mean_delta"]) / np.maximum(se1, 1e-300)
    z2 = (m2.mean(axis=0) - ex["second"]) / np.maximum(se2, 1e-300)
    assert np.max(np.abs(z1)) < zmax, z1
    assert np.max(np.abs(z2)) < zmax, z2
    return ex, m2.mean(axis=0)


@pytest.mark.parametrize("walls", [(1.0, 1.0), (1.0, 3.0)])
def test_heat_dirichlet_4cells(walls):
    p = W.oracle_rod(n=(4, 1, 1), wall_lo=walls[0], wall_hi=walls[1], kB=0.02,
                     stats_interval=1, relax_steps=30)
    ex, got = _check(p, R=2000, B=16, nsteps=60)
    # the wall cells carry the sqrt(2) wall noise: dropping it would lower
    # their variance well outside the tolerance
    assert ex["second"][0, 0] > 0.0 and got[0, 0] > 0.0


def test_heat_periodic_5cells():
    p = W.oracle_rod(n=(5, 1, 1), bc="periodic", wall_lo=2.0, wall_hi=2.0, kB=0.01,
                     stats_interval=2, relax_steps=20)
    _check(p, R=2000, B=16, nsteps=60)


def test_species_dirichlet_4cells():
    p = W.oracle_rod(n=(4, 1, 1), equation="species", n0=50.0, D=1.0, dt=0.2,
                     wall_lo=1.0, wall_hi=2.0, stats_interval=1, relax_steps=30)
    _check(p, R=2000, B=16, nsteps=60)


def test_species_periodic_2d():
    p = W.species_2d(n=(3, 4, 1), n0=100.0, stats_interval=1, relax_steps=20)
    _check(p, R=1000, B=16, nsteps=40)


def test_heat_periodic_3d():
    p = W.cube_3d(n=(2, 3, 2), kB=0.01, perturb_ic=1, stats_interval=1, relax_steps=10)
    _check(p, R=1000, B=16, nsteps=30)


def test_first_step_mean_and_cov_from_fixed_state():
    # From one fixed state, one step: E[T'] = A T + b, Cov[T'] = Q(T).
    p = W.oracle_rod(n=(6, 1, 1), wall_lo=1.0, wall_hi=2.0, kB=0.05)
    td = _theory_dict(p)
    A, b, faces, tref, _ = theory.scheme(td)
    T0 = W.random_states(p, 1, seed=9)[0]
    R = 40000
    st = np.repeat(T0[None, :], R, axis=0)
    out = she.run(p, R, 1, state=st)["state"]
    mean_ex = A @ T0 + b
    cov_ex = theory.noise_cov(td, faces, T0, np.zeros((6, 6)))
    se = np.sqrt(np.diag(cov_ex) / R)
    assert np.max(np.abs(out.mean(axis=0) - mean_ex) / se) < 4.5
    cov = np.cov(out.T)
    se_c = np.sqrt((np.outer(np.diag(cov_ex), np.diag(cov_ex)) + cov_ex ** 2) / R)
    assert np.max(np.abs(cov - cov_ex) / se_c) < 4.5


def test_accumulators_match_state_definitions():
    # K = 1, one step: the pooled sums are the defining sums over the state
    p = W.oracle_rod(n=(8, 1, 1), bc="periodic", stats_interval=1, relax_steps=0,
                     want_cov=1, want_sk=1)
    o = she.run(p, 3, 1)
    d = o["state"] - she.reference_profile(p)[None, :]
    assert o["n_samples"] == 3
    assert np.allclose(o["sum_d"], d.sum(axis=0), rtol=0, atol=1e-15)
    assert np.allclose(o["sum_d2"], (d * d).sum(axis=0), rtol=0, atol=1e-15)
    assert np.allclose(o["sum_dd"], d.T @ d, rtol=0, atol=1e-15)
    sk = (np.abs(np.fft.fft(d, axis=1)) ** 2).sum(axis=0)
    assert np.allclose(o["sum_sk"], sk, rtol=1e-12, atol=1e-15)
    p3 = W.cube_3d(n=(4, 3, 2), perturb_ic=1, stats_interval=1, want_sk=2)
    o = she.run(p3, 2, 1, want_sk=2)
    d = (o["state"] - she.reference_profile(p3)[None, :]).reshape(2, 2, 3, 4)
    ska = []
    for ax, n in ((3, 4), (2, 3), (1, 2)):
        lines = d.size // (2 * n)
        ska.append((np.abs(np.fft.fft(d, axis=ax)) ** 2).sum(
            axis=tuple(i for i in range(4) if i != ax)) / lines)
    assert np.allclose(o["sum_sk_axes"], np.concatenate(ska), rtol=1e-12, atol=1e-15)
    p2 = W.species_2d(n=(4, 6, 1), stats_interval=1, relax_steps=0)
    o = she.run(p2, 2, 1, want_sk=1)
    d = (o["state"] - 1.0).reshape(2, 6, 4)
    sk = (np.abs(np.fft.fft2(d)) ** 2).sum(axis=0).ravel()
    assert np.allclose(o["sum_sk"], sk, rtol=1e-12, atol=1e-15)


def test_sampling_schedule_matches_paper_program():
    # Paper's program: 10 inner steps per outer iteration, sample after
    # outer iterations with index > M/(10*10); with relax = M/10 + K the
    # first sample is at step M/10 + 2K and there are M/K - M/(10K) - 1.
    M, K = 10_000, 10
    p = W.oracle_rod(n=(4, 1, 1), relax_steps=M // 10 + K, stats_interval=K)
    o = she.run(p, 1, M)
    assert o["n_samples"] == M // K - M // (10 * K) - 1
