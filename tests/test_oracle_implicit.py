"""Pins of the oracle's implicit schemes (the exercise on backward Euler and
Crank-Nicolson, Sec. 6): (I - theta r L) T' = T + (1 - theta) r L T + r b +
div G(T), theta = 1 (backward Euler) or 1/2 (Crank-Nicolson), the
stochastic flux explicit from the state at the start of the step.

* One step equals numpy's dense solve of that equation; the noise enters
  through the same explicit face fluxes as forward Euler's, M (T'_noisy -
  T'_deterministic) = T_FE,noisy - T_FE,deterministic.
* Deterministic limit: every sine (Dirichlet) or Fourier (periodic) mode is
  multiplied per step by (1 - (1 - theta) x) / (1 + theta x), also far
  beyond forward Euler's stability limit.
* Pooled sample moments of the oracle within 4.5 batch SE of the exact
  moment recursion of the theta scheme (heat and species, Dirichlet and
  periodic, r = 0.2 and r = 2).
* The stationary structure factor of the recursion equals the closed form
  eps c N / (1 + (theta - 1/2) r mu_k) (flat for Crank-Nicolson at every
  time step), and the sampled S(k) of a long oracle run matches it.
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O
from oracle import theory as T


def _lap(N, bc):
    return T.laplacian_1d(N, bc)


@pytest.mark.parametrize("bc,scheme,r", [("dirichlet", "be", 0.3), ("dirichlet", "cn", 4.0),
                                         ("periodic", "be", 7.0), ("periodic", "cn", 0.2)])
def test_one_step_is_the_dense_solve(bc, scheme, r):
    N = 11
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.5, 1.5)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, wall_lo=walls[0], wall_hi=walls[1], dt=r, scheme=scheme, kB=3e-3)
    theta = 1.0 if scheme == "be" else 0.5
    x = W.random_states(p, 1, seed=2)[0]
    L = _lap(N, bc)
    b = np.zeros(N)
    if bc == "dirichlet":
        b[0], b[-1] = 2.0 * walls[0], 2.0 * walls[1]
    M = np.eye(N) - theta * r * L
    det = np.linalg.solve(M, x + (1.0 - theta) * r * L @ x + r * b)
    got_det = O.step(dict(p, stochastic=0), x, 5, 3)
    assert np.max(np.abs(got_det - det)) < 1e-13
    # the noise part: the explicit face fluxes of forward Euler, then M^{-1}
    got = O.step(p, x, 5, 3)
    fe = dict(p, scheme="fe", dt=0.2)          # any stable r: the noise flux scales with sqrt(r)
    noise_fe = O.step(dict(fe, dt=r), x, 5, 3) - O.step(dict(fe, dt=r, stochastic=0), x, 5, 3)
    assert np.max(np.abs(M @ (got - got_det) - noise_fe)) < 1e-13


@pytest.mark.parametrize("scheme", ["be", "cn"])
@pytest.mark.parametrize("r", [0.1, 1.0, 25.0])
def test_deterministic_modes(scheme, r):
    N, steps = 24, 40
    p = W.oracle_rod(n=(N, 1, 1), wall_lo=1.0, wall_hi=2.0, dt=r, scheme=scheme, stochastic=0, perturb_ic=0)
    tlin = 1.0 + (np.arange(N) + 0.5) / N
    x0 = tlin + 0.3 * np.sin(3 * np.pi * (np.arange(N) + 0.5) / N) - 0.1 * np.sin(7 * np.pi * (np.arange(N) + 0.5) / N)
    got = O.run(p, 1, steps, state=x0[None, :])["state"][0]
    ref = T.sine_mode_solution(N, r, 1.0, 2.0, x0, steps, scheme=scheme)
    assert np.max(np.abs(got - ref)) < 1e-12
    q = dict(p, bc="periodic", wall_hi=1.0)
    y0 = 1.0 + 0.2 * np.cos(2 * np.pi * 3 * np.arange(N) / N)
    got = O.run(q, 1, steps, state=y0[None, :])["state"][0]
    ref = T.fourier_mode_solution(N, r, y0, steps, scheme=scheme)
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("bc,eq,scheme,r", [("dirichlet", "heat", "be", 0.2), ("dirichlet", "heat", "cn", 2.0),
                                            ("periodic", "species", "be", 2.0), ("periodic", "heat", "cn", 0.2)])
def test_pooled_moments_match_the_exact_recursion(bc, eq, scheme, r):
    N, K, relax, steps, B, per = 6, 2, 10, 60, 32, 500
    walls = (1.0, 1.8) if bc == "dirichlet" else (1.3, 1.3)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, equation=eq, wall_lo=walls[0], wall_hi=walls[1], dt=r, scheme=scheme,
                     kB=0.02, n0=50.0, stats_interval=K, relax_steps=relax, want_cov=1, want_sk=0)
    rr, eps = O.dimensionless(p)
    pl = dict(dim=1, n=(N,), bc=bc, r=rr, eps=eps, wall_lo=walls[0], wall_hi=walls[1], equation=eq,
              scheme=scheme, perturb_ic=1)
    ex = T.pooled_expectation(pl, steps, K, relax)
    m1, m2 = [], []
    for bb in range(B):
        o = O.run(p, per, steps, stream0=bb * per)
        m1.append(o["sum_d"] / o["n_samples"])
        m2.append(o["sum_dd"] / o["n_samples"])
    m1, m2 = np.array(m1), np.array(m2)
    z1 = (m1.mean(0) - ex["mean_delta"]) / (m1.std(0, ddof=1) / np.sqrt(B))
    z2 = (m2.mean(0) - ex["second"]) / (m2.std(0, ddof=1) / np.sqrt(B))
    assert np.max(np.abs(z1)) < 4.5 and np.max(np.abs(z2)) < 4.5


@pytest.mark.parametrize("scheme", ["be", "cn"])
def test_structure_factor_closed_form_and_sampled(scheme):
    N, r = 16, 1.5
    pl = dict(dim=1, n=(N,), bc="periodic", r=r, eps=0.01, wall_lo=1.2, wall_hi=1.2, equation="species",
              scheme=scheme)
    _, C = T.stationary(pl, iters=50)
    F = np.exp(-2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N)
    S_rec = np.real(np.einsum("kj,jl,kl->k", F, C, np.conj(F)))
    S_th = T.structure_factor((N,), r, 0.012, scheme)
    assert np.max(np.abs(S_rec[1:] - S_th[1:]) / S_th[1:]) < 1e-12
    if scheme == "cn":
        assert np.allclose(S_th[1:], 0.012 * N, rtol=1e-14)        # flat at any time step
    # a sampled run against it (species: the closed form is exact)
    p = W.oracle_rod(n=(N, 1, 1), bc="periodic", equation="species", wall_lo=1.2, wall_hi=1.2, dt=r, n0=100.0,
                     scheme=scheme, stats_interval=5, relax_steps=100, want_cov=1, want_sk=1)
    o = O.finalize(p, O.run(p, 400, 3000))
    rel = np.abs(o["sk_fluct"][1:] - S_th[1:]) / S_th[1:]
    assert np.max(rel) < 0.05 and np.mean(rel) < 0.02


def test_large_time_step_stays_bounded():
    # far beyond forward Euler's r <= 1/2: both implicit schemes stay bounded
    for scheme in ("be", "cn"):
        p = W.oracle_rod(n=(32, 1, 1), wall_lo=1.0, wall_hi=2.0, dt=50.0, scheme=scheme, kB=1e-3)
        o = O.run(p, 4, 2000)
        assert np.all(np.isfinite(o["state"]))
        assert np.max(np.abs(o["state"] - O.reference_profile(p))) < 1.0
