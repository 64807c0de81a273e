"""Deterministic-limit pins of the oracle step (alpha = 0, Sec. 3).

With the noise switched off the forward-Euler scheme (Eq. (3.3)) with the
Dirichlet wall stencil (Eq. (3.8)) is diagonalised exactly by half-shifted
sine modes, and on periodic grids by Fourier modes; the oracle must follow
those solutions to rounding, and converge to the continuum sine-series
solution of the heat equation as dx, dt -> 0.  Periodic grids conserve the
total (Sec. 3, the conservation argument behind the (1 - 1/N) correction),
with the noise on as well.
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she, theory


@pytest.mark.parametrize("N,walls", [(2, (1.0, 1.0)), (3, (1.0, 3.0)), (32, (1.0, 2.0)),
                                     (33, (2.5, 0.5))])
def test_sine_modes_exact(N, walls):
    p = W.oracle_rod(n=(N, 1, 1), stochastic=0, perturb_ic=0,
                     wall_lo=walls[0], wall_hi=walls[1])
    r, _ = she.dimensionless(p)
    T0 = W.random_states(p, 1, seed=N)[0]
    for nsteps in (1, 7, 300):
        got = she.run(p, 1, nsteps, state=T0[None, :])["state"][0]
        ex = theory.sine_mode_solution(N, r, walls[0], walls[1], T0, nsteps)
        assert np.max(np.abs(got - ex)) < 1e-12 * max(1.0, np.max(np.abs(ex)))


@pytest.mark.parametrize("N", [2, 5, 16])
def test_fourier_modes_exact(N):
    p = W.oracle_rod(n=(N, 1, 1), bc="periodic", stochastic=0, perturb_ic=0, dt=0.23)
    r, _ = she.dimensionless(p)
    T0 = W.random_states(p, 1, seed=100 + N)[0]
    got = she.run(p, 1, 50, state=T0[None, :])["state"][0]
    ex = theory.fourier_mode_solution(N, r, T0, 50)
    assert np.max(np.abs(got - ex)) < 1e-12


def test_fourier_modes_2d_3d():
    p2 = W.species_2d(n=(6, 4, 1), stochastic=0, perturb_ic=0)
    T0 = W.random_states(p2, 1, seed=5)[0]
    got = she.run(p2, 1, 20, state=T0[None, :])["state"][0]
    r, _ = she.dimensionless(p2)
    lam = 1.0 - r * (4 * np.sin(np.pi * np.arange(6) / 6)[None, :] ** 2
                     + 4 * np.sin(np.pi * np.arange(4) / 4)[:, None] ** 2)
    ex = np.real(np.fft.ifft2(np.fft.fft2(T0.reshape(4, 6)) * lam ** 20)).ravel()
    assert np.max(np.abs(got - ex)) < 1e-12
    p3 = W.cube_3d(n=(4, 3, 5), stochastic=0, perturb_ic=0)
    T0 = W.random_states(p3, 1, seed=6)[0]
    got = she.run(p3, 1, 10, state=T0[None, :])["state"][0]
    r, _ = she.dimensionless(p3)
    mu = (4 * np.sin(np.pi * np.arange(4) / 4)[None, None, :] ** 2
          + 4 * np.sin(np.pi * np.arange(3) / 3)[None, :, None] ** 2
          + 4 * np.sin(np.pi * np.arange(5) / 5)[:, None, None] ** 2)
    ex = np.real(np.fft.ifftn(np.fft.fftn(T0.reshape(5, 3, 4)) * (1 - r * mu) ** 10)).ravel()
    assert np.max(np.abs(got - ex)) < 1e-12


def test_linear_profile_is_steady():
    p = W.oracle_rod(n=(32, 1, 1), stochastic=0, perturb_ic=0, wall_lo=1.0, wall_hi=2.0)
    T0 = she.reference_profile(p)
    got = she.run(p, 1, 100, state=T0[None, :])["state"][0]
    assert np.max(np.abs(got - T0)) < 1e-13


def test_converges_to_continuum_sine_series():
    # T(x,0) = T_lin + sin(pi x / l): continuum solution decays as
    # exp(-kappa pi^2 t / l^2); FE error must shrink ~ dx^2 at fixed r.
    errs = []
    t_end = 0.05
    for N in (16, 32, 64):
        dx = 1.0 / N
        r = 0.2
        dt = r * dx * dx
        nsteps = int(round(t_end / dt))
        p = W.oracle_rod(n=(N, 1, 1), dx=dx, kappa=1.0, dt=dt, stochastic=0, perturb_ic=0,
                         wall_lo=0.0, wall_hi=0.0)
        x = (np.arange(N) + 0.5) * dx
        T0 = np.sin(np.pi * x)
        got = she.run(p, 1, nsteps, state=T0[None, :])["state"][0]
        exact = np.exp(-np.pi ** 2 * nsteps * dt) * np.sin(np.pi * x)
        errs.append(np.max(np.abs(got - exact)))
    assert errs[1] < errs[0] / 3.0 and errs[2] < errs[1] / 3.0, errs


@pytest.mark.parametrize("maker", [lambda: W.oracle_rod(n=(9, 1, 1), bc="periodic"),
                                   lambda: W.species_2d(n=(5, 4, 1)),
                                   lambda: W.cube_3d(n=(3, 4, 2), perturb_ic=1)])
def test_periodic_total_conserved(maker):
    p = maker()
    st = she.run(p, 3, 0)["state"]
    tot0 = st.sum(axis=1)
    st2 = she.run(p, 3, 200, state=st)["state"]
    assert np.max(np.abs(st2.sum(axis=1) - tot0)) < 1e-11 * st.shape[1]
    # the periodic initial perturbation is projected to zero sum
    ref = she.reference_profile(p)
    assert np.max(np.abs(tot0 - ref.sum())) < 1e-11 * st.shape[1]
