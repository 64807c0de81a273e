"""Pins of the oracle's rod of several materials (the iron / aluminium
exercise of Sec. 6): per-cell conductivity lambda_i and heat capacity
rho c_V,i in the conservation form of the SHE (Sec. 2), stepped as Eq. (3.3)
with the face conductance the harmonic mean of its two cells'.

* Uniform materials give the uniform scheme to rounding (the variable path
  reduces to r = kappa dt / dx^2, eps = k_B / (rho c_V dV)).
* The deterministic steady state is the series-resistance profile (piecewise
  linear, its slope inversely proportional to each material's
  conductivity), computed here from the resistances, a fixed point of the
  step, reached from a perturbed start.
* The pooled sample moments of the oracle match the exact moment recursion
  (theory.pooled_expectation on the variable scheme) within 4.5 batch SE, at
  equilibrium and in a gradient.
* The equilibrium covariance of the recursion equals the closed form
  k_B T^2 / dV (C + L/2)^{-1} derived in theory.variable_equilibrium_cov,
  whose r -> 0 limit is each material's own k_B T^2 / (rho c_V,i dV)
  (Eq. (3.10) per material).
* A periodic rod conserves the energy sum rho c_V,i T_i, and its seeded
  perturbation has zero energy sum.
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O
from oracle import theory as T


def _rod(N=16, walls=(1.0, 1.0), bc="dirichlet", split=0.5, lam=(1.0, 3.0), rcv=(1.0, 0.7), **kw):
    k = int(round(N * split))
    lam_c = np.r_[np.full(k, lam[0]), np.full(N - k, lam[1])]
    rcv_c = np.r_[np.full(k, rcv[0]), np.full(N - k, rcv[1])]
    kw.setdefault("kB", 1e-3)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, wall_lo=walls[0], wall_hi=walls[1], dt=0.1,
                     want_cov=0, want_sk=0, relax_steps=0, realizations=4, **kw)
    p["lambda_cells"] = lam_c
    p["rho_cv_cells"] = rcv_c
    return p


def _prob_like(p):
    cond, cap, kb_dv = O.material_arrays(p)
    return dict(dim=1, n=p["n"], bc=p["bc"], cond=cond, cap=cap, kB_dV=kb_dv, wall_lo=p["wall_lo"],
                wall_hi=p["wall_hi"], equation="heat", perturb_ic=p.get("perturb_ic", 1))


@pytest.mark.parametrize("bc,scheme", [("dirichlet", "fe"), ("periodic", "fe"), ("dirichlet", "pc"),
                                       ("periodic", "pc")])
def test_uniform_materials_reduce_to_the_uniform_scheme(bc, scheme):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.5, 1.5)
    p = W.oracle_rod(n=(20, 1, 1), bc=bc, wall_lo=walls[0], wall_hi=walls[1], kB=2e-3, kappa=0.7,
                     rho_cv=1.3, dt=0.2, relax_steps=0, want_cov=1, want_sk=0, scheme=scheme)
    q = dict(p, lambda_cells=np.full(20, 0.7 * 1.3), rho_cv_cells=np.full(20, 1.3))
    a = O.run(p, 3, 300)
    b = O.run(q, 3, 300)
    assert np.max(np.abs(a["state"] - b["state"]) / np.abs(a["state"])) < 1e-13
    assert np.allclose(a["sum_dd"], b["sum_dd"], rtol=1e-11, atol=1e-16)


def _series_profile(lam_c, walls, N):
    # conduction through half a cell at each wall and every interior face in
    # series; face conductivity of two half cells in series = harmonic mean
    lf = 2.0 * lam_c[:-1] * lam_c[1:] / (lam_c[:-1] + lam_c[1:])
    res = np.r_[0.5 / lam_c[0], 1.0 / lf, 0.5 / lam_c[-1]]
    q = (walls[1] - walls[0]) / res.sum()
    return walls[0] + q * np.cumsum(res)[:-1]


def test_steady_profile_is_the_series_resistance_profile():
    p = _rod(N=16, walls=(1.0, 2.0), stochastic=0, perturb_ic=0)
    prof = _series_profile(p["lambda_cells"], (1.0, 2.0), 16)
    assert np.allclose(O.reference_profile(p), prof, rtol=1e-14)
    # piecewise linear with slopes inversely proportional to the conductivity
    slope = np.diff(prof)
    assert np.allclose(slope[:7] / slope[8:], 3.0, rtol=1e-12)
    # a fixed point of the deterministic step, reached from a perturbed start
    assert np.allclose(O.step(p, prof, 0, 0), prof, rtol=1e-14)
    x0 = prof + 0.1 * np.sin(np.pi * (np.arange(16) + 0.5) / 16)
    out = O.run(p, 1, 20000, state=x0[None, :])["state"][0]
    assert np.max(np.abs(out - prof)) < 1e-10


@pytest.mark.parametrize("walls,bc", [((1.0, 1.0), "dirichlet"), ((1.0, 2.0), "dirichlet"),
                                      ((1.4, 1.4), "periodic")])
def test_pooled_moments_match_the_exact_recursion(walls, bc):
    p = _rod(N=8, walls=walls, bc=bc, stats_interval=3, kB=0.02)
    p["relax_steps"] = 30
    steps, B, per = 120, 32, 400
    ex = T.pooled_expectation(_prob_like(p), steps, 3, 30)
    tref = O.reference_profile(p)
    m1, m2 = [], []
    for b in range(B):
        r = O.run(p, per, steps, stream0=b * per, want_cov=1)
        n = r["n_samples"]
        m1.append(r["sum_d"] / n)
        m2.append(r["sum_dd"] / n)
    m1, m2 = np.array(m1), np.array(m2)
    exp1 = ex["mean_delta"]
    exp2 = ex["second"]
    assert np.allclose(ex["tref"], tref, rtol=1e-12)
    z1 = (m1.mean(0) - exp1) / (m1.std(0, ddof=1) / np.sqrt(B))
    z2 = (m2.mean(0) - exp2) / (m2.std(0, ddof=1) / np.sqrt(B))
    assert np.max(np.abs(z1)) < 4.5
    assert np.max(np.abs(z2)) < 4.5


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_equilibrium_covariance_closed_form(bc):
    N = 12
    cond = np.r_[np.full(6, 0.08), np.full(6, 0.25)]
    cap = np.r_[np.full(6, 1.0), np.full(6, 0.684)]
    pl = dict(dim=1, n=(N,), bc=bc, cond=cond, cap=cap, kB_dV=1e-10, wall_lo=1.2, wall_hi=1.2,
              equation="heat")
    _, C = T.stationary(pl, iters=100)
    S = T.variable_equilibrium_cov(cond, cap, 1e-10, bc, 1.2)
    assert np.max(np.abs(C - S)) < 1e-8 * np.max(np.abs(S))
    # r -> 0: each material's own variance k_B T^2 / (rho c_V dV), no correlation
    S0 = T.variable_equilibrium_cov(cond * 1e-5, cap, 1.0, "dirichlet", 1.2)
    assert np.allclose(np.diag(S0), 1.44 / cap, rtol=1e-4)
    assert np.max(np.abs(S0 - np.diag(np.diag(S0)))) < 1e-4 * np.max(S0)


def test_periodic_rod_conserves_energy():
    p = _rod(N=14, walls=(1.3, 1.3), bc="periodic", kB=5e-3)
    cap = p["rho_cv_cells"]
    x0 = O.initial_state(p, 5)
    assert abs(cap @ (x0 - 1.3)) < 1e-13 * cap.sum()
    out = O.run(p, 1, 500, stream0=5)["state"][0]
    assert abs(cap @ out - cap @ x0) < 1e-12 * (cap @ x0)
