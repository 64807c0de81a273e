"""Pins of the oracle's predictor-corrector scheme (Sec. 3).

The scheme is the forward-Euler step as predictor T*, then the corrector
(T + T* + D(T*) + div G(T*)) / 2 with the face values and the stencil taken
on T* and the same face normals (noise constant over the step).  Pins that do
not run the oracle's code path:

* the deterministic limit: every sine (Dirichlet) or Fourier (periodic) mode
  is multiplied per step by Heun's factor 1 - x + x^2/2, x = r mu, and the
  linear profile is a fixed point;
* conservation of the total on periodic grids with the noise on;
* the exact first and second moments of the heat equation, propagated by
  Gauss-Hermite quadrature over the face normals (theory.py explains why
  that is exact); the quadrature itself reproduces the closed forward-Euler
  recursion to rounding;
* one step from a fixed state (heat exactly, species by a converged rule);
* the periodic structure factor against the closed form of the scheme,
  whose deviation from the flat value is O(x^2) where forward Euler's is
  O(x) (the error orders of the paper's exercises, Sec. 6).
A corrector that used fresh noise, the old state's face values, a missing
factor 1/2, or the wrong stage's stencil moves at least one of these.
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


@pytest.mark.parametrize("maker", [
    lambda: W.oracle_rod(n=(4, 1, 1), wall_lo=1.0, wall_hi=3.0, kB=0.02, stats_interval=1, relax_steps=30),
    lambda: W.oracle_rod(n=(5, 1, 1), bc="periodic", wall_lo=2.0, wall_hi=2.0, kB=0.01, stats_interval=2)])
def test_quadrature_reproduces_closed_fe_recursion(maker):
    td = _td(maker())
    a = theory.pooled_expectation(td, 60, td.get("K", 2), 20)
    b = theory.pooled_expectation_quadrature(td, 60, td.get("K", 2), 20)
    assert np.max(np.abs(a["second"] - b["second"])) < 1e-11 * np.max(np.abs(a["second"]))
    assert np.max(np.abs(a["mean_delta"] - b["mean_delta"])) < 1e-12


@pytest.mark.parametrize("N,walls", [(2, (1.0, 1.0)), (3, (1.0, 3.0)), (32, (1.0, 2.0))])
def test_pc_sine_modes_exact(N, walls):
    p = W.oracle_rod(n=(N, 1, 1), stochastic=0, perturb_ic=0, wall_lo=walls[0], wall_hi=walls[1],
                     scheme="pc")
    r, _ = she.dimensionless(p)
    T0 = W.random_states(p, 1, seed=N)[0]
    for nsteps in (1, 7, 300):
        got = she.run(p, 1, nsteps, state=T0[None, :])["state"][0]
        ex = theory.sine_mode_solution(N, r, walls[0], walls[1], T0, nsteps, scheme="pc")
        assert np.max(np.abs(got - ex)) < 1e-12 * max(1.0, np.max(np.abs(ex)))
        fe = theory.sine_mode_solution(N, r, walls[0], walls[1], T0, nsteps)
        if N > 2 and nsteps == 7:
            assert np.max(np.abs(got - fe)) > 1e-6       # not the forward-Euler map


@pytest.mark.parametrize("N", [2, 5, 16])
def test_pc_fourier_modes_exact(N):
    p = W.oracle_rod(n=(N, 1, 1), bc="periodic", stochastic=0, perturb_ic=0, dt=0.23, scheme="pc")
    r, _ = she.dimensionless(p)
    T0 = W.random_states(p, 1, seed=100 + N)[0]
    got = she.run(p, 1, 50, state=T0[None, :])["state"][0]
    ex = theory.fourier_mode_solution(N, r, T0, 50, scheme="pc")
    assert np.max(np.abs(got - ex)) < 1e-12


def test_pc_fourier_modes_2d_3d():
    p2 = W.species_2d(n=(6, 4, 1), stochastic=0, perturb_ic=0, scheme="pc")
    T0 = W.random_states(p2, 1, seed=5)[0]
    got = she.run(p2, 1, 20, state=T0[None, :])["state"][0]
    r, _ = she.dimensionless(p2)
    mu = (4 * np.sin(np.pi * np.arange(6) / 6)[None, :] ** 2
          + 4 * np.sin(np.pi * np.arange(4) / 4)[:, None] ** 2)
    ex = np.real(np.fft.ifft2(np.fft.fft2(T0.reshape(4, 6)) * theory.amplification(r * mu, "pc") ** 20)).ravel()
    assert np.max(np.abs(got - ex)) < 1e-12
    p3 = W.cube_3d(n=(4, 3, 5), stochastic=0, perturb_ic=0, scheme="pc")
    T0 = W.random_states(p3, 1, seed=6)[0]
    got = she.run(p3, 1, 10, state=T0[None, :])["state"][0]
    r, _ = she.dimensionless(p3)
    mu = (4 * np.sin(np.pi * np.arange(4) / 4)[None, None, :] ** 2
          + 4 * np.sin(np.pi * np.arange(3) / 3)[None, :, None] ** 2
          + 4 * np.sin(np.pi * np.arange(5) / 5)[:, None, None] ** 2)
    ex = np.real(np.fft.ifftn(np.fft.fftn(T0.reshape(5, 3, 4)) * theory.amplification(r * mu, "pc") ** 10)).ravel()
    assert np.max(np.abs(got - ex)) < 1e-12


def test_pc_linear_profile_is_steady():
    p = W.oracle_rod(n=(32, 1, 1), stochastic=0, perturb_ic=0, wall_lo=1.0, wall_hi=2.0, scheme="pc")
    T0 = she.reference_profile(p)
    got = she.run(p, 1, 100, state=T0[None, :])["state"][0]
    assert np.max(np.abs(got - T0)) < 1e-13


@pytest.mark.parametrize("maker", [lambda: W.oracle_rod(n=(9, 1, 1), bc="periodic", scheme="pc"),
                                   lambda: W.species_2d(n=(5, 4, 1), scheme="pc"),
                                   lambda: W.cube_3d(n=(3, 4, 2), perturb_ic=1, scheme="pc")])
def test_pc_periodic_total_conserved(maker):
    p = maker()
    st = she.run(p, 3, 0)["state"]
    tot0 = st.sum(axis=1)
    st2 = she.run(p, 3, 200, state=st)["state"]
    assert np.max(np.abs(st2.sum(axis=1) - tot0)) < 1e-11 * st.shape[1]


def _batched(p, R, B, nsteps):
    m1, m2 = [], []
    for b in range(B):
        o = she.run(p, R, nsteps, stream0=b * R, want_cov=1)
        n = o["n_samples"]
        m1.append(o["sum_d"] / n)
        m2.append(o["sum_dd"] / n)
    return np.array(m1), np.array(m2)


@pytest.mark.parametrize("maker", [
    lambda: W.oracle_rod(n=(4, 1, 1), wall_lo=1.0, wall_hi=1.0, kB=0.02, stats_interval=1, relax_steps=30),
    lambda: W.oracle_rod(n=(4, 1, 1), wall_lo=1.0, wall_hi=3.0, kB=0.02, stats_interval=1, relax_steps=30),
    lambda: W.oracle_rod(n=(5, 1, 1), bc="periodic", wall_lo=2.0, wall_hi=2.0, kB=0.01, stats_interval=2,
                         relax_steps=20)])
def test_pc_heat_moments_match_exact_recursion(maker):
    p = dict(maker(), scheme="pc")
    nsteps, R, B = 60, 2000, 16
    ex = theory.pooled_expectation_quadrature(_td(p), nsteps, p["stats_interval"], p["relax_steps"])
    m1, m2 = _batched(p, R, B, nsteps)
    se1 = m1.std(axis=0, ddof=1) / np.sqrt(B)
    se2 = m2.std(axis=0, ddof=1) / np.sqrt(B)
    z1 = (m1.mean(axis=0) - ex["mean_delta"]) / np.maximum(se1, 1e-300)
    z2 = (m2.mean(axis=0) - ex["second"]) / np.maximum(se2, 1e-300)
    assert np.max(np.abs(z1)) < 4.5, z1
    assert np.max(np.abs(z2)) < 4.5, z2
    # the scheme matters at this r: forward Euler's second moment is far off
    fe = theory.pooled_expectation(_td(dict(p, scheme="fe")), nsteps, p["stats_interval"], p["relax_steps"])
    zfe = (m2.mean(axis=0) - fe["second"]) / np.maximum(se2, 1e-300)
    assert np.max(np.abs(zfe)) > 10.0


@pytest.mark.parametrize("equation,npts", [("heat", 3), ("species", 6)])
def test_pc_first_step_from_fixed_state(equation, npts):
    kw = dict(equation="species", n0=50.0, D=1.0) if equation == "species" else dict(kB=0.05)
    p = W.oracle_rod(n=(4, 1, 1), wall_lo=1.0, wall_hi=2.0, scheme="pc", **kw)
    T0 = W.random_states(p, 1, seed=9)[0]
    mean_ex, cov_ex = theory.first_step_quadrature(_td(p), T0, npts)
    if equation == "species":
        # the rule has converged: one more node changes nothing visible
        m2, c2 = theory.first_step_quadrature(_td(p), T0, npts + 1)
        assert np.max(np.abs(c2 - cov_ex)) < 1e-6 * np.max(np.abs(cov_ex))
    R = 40000
    out = she.run(p, R, 1, state=np.repeat(T0[None, :], R, axis=0))["state"]
    se = np.sqrt(np.diag(cov_ex) / R)
    assert np.max(np.abs(out.mean(axis=0) - mean_ex) / se) < 4.5
    cov = np.cov(out.T)
    se_c = np.sqrt((np.outer(np.diag(cov_ex), np.diag(cov_ex)) + cov_ex ** 2) / R)
    assert np.max(np.abs(cov - cov_ex) / se_c) < 4.5


def test_pc_structure_factor_matches_closed_form():
    N, B, R = 16, 12, 64
    p = W.oracle_rod(n=(N, 1, 1), bc="periodic", kB=1e-4, stats_interval=5, relax_steps=400,
                     want_sk=1, scheme="pc")
    r, eps = she.dimensionless(p)
    vals = []
    for b in range(B):
        o = she.run(p, R, 3000, stream0=b * R)
        vals.append(she.finalize(p, o)["sk_fluct"])
    vals = np.array(vals)
    se = vals.std(axis=0, ddof=1) / np.sqrt(B)
    ex = theory.structure_factor((N,), r, eps * 1.0, scheme="pc")
    z = (vals.mean(axis=0)[1:] - ex[1:]) / se[1:]
    assert np.max(np.abs(z)) < 4.5, z
    # the two schemes' errors at the highest k: PC below the flat value by
    # O(x^2), FE above it by O(x); the measurement sits on the PC side
    flat = eps * N
    fe = theory.structure_factor((N,), r, eps * 1.0)
    k = N // 2
    assert ex[k] < flat < fe[k]
    assert abs(vals.mean(axis=0)[k] - ex[k]) < 0.2 * abs(fe[k] - ex[k])


def test_pc_heat_2d_moments_match_exact_recursion():
    # 2 x 2 periodic grid: 8 faces, 3^8 quadrature nodes; the quadrature
    # reproduces the closed forward-Euler recursion in 2D as well
    p = W.species_2d(n=(2, 2, 1), equation="heat", kB=0.01, wall_lo=1.0, wall_hi=1.0, stats_interval=1,
                     relax_steps=10, perturb_ic=1, scheme="pc")
    td = _td(p)
    fe = theory.pooled_expectation(dict(td, scheme="fe"), 30, 1, 10)
    feq = theory.pooled_expectation_quadrature(dict(td, scheme="fe"), 30, 1, 10)
    assert np.max(np.abs(fe["second"] - feq["second"])) < 1e-9 * np.max(np.abs(fe["second"]))
    ex = theory.pooled_expectation_quadrature(td, 30, 1, 10)
    m1, m2 = _batched(p, 2000, 16, 30)
    se1 = m1.std(axis=0, ddof=1) / np.sqrt(16)
    se2 = m2.std(axis=0, ddof=1) / np.sqrt(16)
    z1 = (m1.mean(axis=0) - ex["mean_delta"]) / np.maximum(se1, 1e-300)
    z2 = (m2.mean(axis=0) - ex["second"]) / np.maximum(se2, 1e-300)
    assert np.max(np.abs(z1)) < 4.5, z1
    assert np.max(np.abs(z2)) < 4.5, z2
    zfe = (m2.mean(axis=0) - fe["second"]) / np.maximum(se2, 1e-300)
    assert np.max(np.abs(zfe)) > 10.0
