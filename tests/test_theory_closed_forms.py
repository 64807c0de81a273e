"""Pins of the exact moment recursion against the paper's published results.

The recursion in oracle/theory.py is built from the matrix form of the
scheme; here it is tied to results the paper states independently:

* Eq. (3.10): at equilibrium with Dirichlet walls, <dT_i dT_j> =
  eps T^2 delta_ij -- reached by the scheme as r -> 0 (with the sqrt(2)
  wall noise; without it the wall cells would fall short).
* Sec. 3 periodic correction: variance eps T^2 (1 - 1/N), off-diagonal
  -eps T^2 / N.
* Eq. (3.12): flat S_k = eps T^2 N (with the cell volume restored, since the
  printed form omits dV while Eq. (3.10) and the program use it).
* Eq. (3.13): non-equilibrium long-range correlation
  eps dT^2 (i+1/2)(N-j-1/2)/N^3.
* Exercise 5: species equilibrium <dn_i dn_j> = delta_ij <n_i>/dV, i.e.
  var(c) = eps_c <c>.
* Supplement (SM1.6): the stationary covariance solves the
  fluctuation-dissipation (Lyapunov) relation; the forward-Euler version
  has the closed form eps T^2 (I + r L/2)^{-1}.
"""
import numpy as np
import pytest

from oracle import theory


def _td(N, bc, r, eps, lo, hi, eq="heat"):
    return {"dim": 1, "n": (N, 1, 1), "bc": bc, "r": r, "eps": eps, "wall_lo": lo,
            "wall_hi": hi, "equation": eq, "perturb_ic": 0}


@pytest.mark.parametrize("N", [4, 16, 32])
def test_dirichlet_equilibrium_variance_is_eps_T2(N):
    T, eps = 1.7, 1e-6        # tiny eps: the multiplicative correction vanishes
    C = theory.fe_equilibrium_cov(N, "dirichlet", 1e-4, eps, T)
    assert np.allclose(C, eps * T * T * np.eye(N), rtol=0, atol=1e-3 * eps * T * T)
    m, Cs = theory.stationary(_td(N, "dirichlet", 1e-4, eps, T, T))
    assert np.allclose(m, T, rtol=1e-12)
    assert np.allclose(Cs, eps * T * T * np.eye(N), rtol=0, atol=2e-3 * eps * T * T)


def test_without_wall_sqrt2_the_walls_fall_short():
    # the recursion with the wall weight set to 1 instead of 2 (squared)
    # misses Eq. (3.10) in the wall cells -- the pin is sensitive to it
    N, T, eps, r = 8, 1.0, 1e-6, 1e-4
    td = _td(N, "dirichlet", r, eps, T, T)
    A, b, faces, tref, _ = theory.scheme(td)
    faces = [(P, q, 1.0, d) for (P, q, w2, d) in faces]
    import scipy.linalg
    Q = theory.noise_cov(td, faces, np.full(N, T), np.zeros((N, N)))
    C = scipy.linalg.solve_discrete_lyapunov(A, Q)
    assert C[0, 0] < 0.8 * eps * T * T


def test_fe_closed_form_equals_recursion_fixed_point():
    N, T, eps, r = 12, 2.0, 1e-8, 0.2
    C = theory.fe_equilibrium_cov(N, "dirichlet", r, eps, T)
    m, Cs = theory.stationary(_td(N, "dirichlet", r, eps, T, T))
    assert np.allclose(Cs, C, rtol=1e-6, atol=1e-6 * eps * T * T)


@pytest.mark.parametrize("N", [8, 32])
def test_periodic_conservation_correction(N):
    T, eps = 1.0, 1e-6
    m, C = theory.stationary(_td(N, "periodic", 1e-4, eps, T, T))
    v = eps * T * T
    assert np.allclose(np.diag(C), v * (1 - 1.0 / N), rtol=2e-3)
    off = C[~np.eye(N, dtype=bool)]
    assert np.allclose(off, -v / N, rtol=2e-2, atol=2e-3 * v)
    # periodic variance closed form from S_k
    assert np.isclose(theory.periodic_variance(N, 1e-4, v), v * (1 - 1.0 / N), rtol=1e-3)


@pytest.mark.parametrize("r", [0.05, 0.2])
def test_periodic_structure_factor_closed_form(r):
    N, T, eps = 16, 1.0, 1e-9
    m, C = theory.stationary(_td(N, "periodic", r, eps, T, T))
    F = np.exp(-2j * np.pi * np.outer(np.arange(N), np.arange(N)) / N)
    S = np.real(np.einsum("ki,ij,kj->k", F, C, np.conj(F)))
    ex = theory.fe_structure_factor((N,), r, eps * T * T)
    assert np.allclose(S[1:], ex[1:], rtol=1e-6)
    # and the flat value of Eq. (3.12) as r -> 0
    flat = theory.fe_structure_factor((N,), 1e-7, eps * T * T)
    assert np.allclose(flat[1:], eps * T * T * N, rtol=1e-6)


def test_2d_species_structure_factor_exact():
    # species noise is linear in c: the closed form is exact, not linearised
    td = {"dim": 2, "n": (4, 3, 1), "bc": "periodic", "r": 0.1, "eps": 0.01,
          "wall_lo": 1.3, "wall_hi": 1.3, "equation": "species", "perturb_ic": 0}
    m, C = theory.stationary(td)
    nc = 12
    kx, ky = np.meshgrid(np.arange(4), np.arange(3), indexing="xy")
    jx, jy = np.meshgrid(np.arange(4), np.arange(3), indexing="xy")
    ph = (np.outer(kx.ravel(), jx.ravel()) / 4.0 + np.outer(ky.ravel(), jy.ravel()) / 3.0)
    F = np.exp(-2j * np.pi * ph)
    S = np.real(np.einsum("ki,ij,kj->k", F, C, np.conj(F)))
    ex = theory.fe_structure_factor((4, 3), 0.1, 0.01 * 1.3)
    assert np.allclose(S[1:], ex[1:], rtol=1e-9)
    assert np.isclose(np.mean(np.diag(C)), np.sum(ex) / nc ** 2, rtol=1e-9)


def test_species_equilibrium_variance_exercise5():
    # <dn_i dn_j> = delta_ij <n_i>/dV  <=>  var(c) = eps_c c as r -> 0
    N, c, eps = 10, 2.5, 1e-3
    m, C = theory.stationary(_td(N, "dirichlet", 1e-4, eps, c, c, eq="species"))
    assert np.allclose(np.diag(C), eps * c, rtol=2e-3)
    assert np.max(np.abs(C - np.diag(np.diag(C)))) < 2e-3 * eps * c


@pytest.mark.parametrize("N", [32, 64])
def test_nonequilibrium_long_range_correlation(N):
    # Eq. (3.13) is a continuum result: the discrete scheme adds a local
    # correction within a few cells of the diagonal and O(r) forward-Euler
    # terms, so compare at small r, away from the diagonal, and through the
    # projection amplitude onto the theoretical shape.
    lo, hi, eps = 1.0, 2.0, 1e-6
    m, C = theory.stationary(_td(N, "dirichlet", 1e-5, eps, lo, hi))
    x = (np.arange(N) + 0.5) / N
    tlin = lo + (hi - lo) * x
    assert np.allclose(m, tlin, rtol=1e-12)           # exact linear mean
    lr = theory.long_range_correlation(N, eps, hi - lo)
    scale = np.max(np.abs(lr))
    sep = np.abs(np.subtract.outer(np.arange(N), np.arange(N)))
    far = sep >= N // 4
    assert np.max(np.abs(C[far] - lr[far])) < 0.02 * scale
    off = sep > 0
    amp = np.sum(C[off] * lr[off]) / np.sum(lr[off] ** 2)
    assert abs(amp - 1.0) < 0.01
    # local equilibrium on the diagonal: eps <T_i>^2 (Eq. (3.13), first term)
    assert np.allclose(np.diag(C), eps * tlin ** 2, rtol=2e-2)
