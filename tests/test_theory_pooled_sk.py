"""Pins of the pooled structure-factor closed forms (oracle/theory.py) that
the GPU physics checks compare against, by the exact moment recursion
(theory.pooled_expectation: m' = A m + b, C' = A C A^T + sum_f E[g_f^2]
d_f d_f^T, iterated with dense matrices over every step of the run and
pooled over the sampling schedule of Sec. 3, Eq. (3.9)) on small grids.

* Species (Eq. (4.7)): the face-noise variance is linear in the state, so
  the pooled S_k of a periodic grid from the seeded perturbation is exact:
  equal to the recursion's DFT of the pooled second moment to rounding.
* Heat (Eq. (2.12)): the noise is proportional to the face temperature, so
  its strength carries the face variance v_a; the per-axis closed form takes
  v_a at its stationary value from the first step on.  Against the recursion
  it holds to the stated order of that approximation, and dropping v_a (the
  linearised equation) misses by about v_a / T0^2, so the pin resolves the
  multiplicative term.
"""
import numpy as np

from oracle import theory as T


def _dft_matrix(shape):
    # F[k, j] = exp(-2 pi i sum_a k_a j_a / n_a), cells with axis 0 fastest
    dims = list(shape)
    idx = np.array(np.unravel_index(np.arange(int(np.prod(dims))), tuple(reversed(dims)))[::-1]).T
    ph = np.zeros((len(idx), len(idx)))
    for a, n in enumerate(dims):
        ph += np.outer(idx[:, a], idx[:, a]) / n
    return np.exp(-2j * np.pi * ph)


def _per_axis_from_second_moment(shape, M2):
    # (1/lines) sum over lines along a of <|1D DFT along a|^2>
    dims = list(shape)
    n = int(np.prod(dims))
    idx = np.array(np.unravel_index(np.arange(n), tuple(reversed(dims)))[::-1]).T
    out = []
    for a, na in enumerate(dims):
        lines = {}
        for i in range(n):
            key = tuple(np.delete(idx[i], a))
            lines.setdefault(key, [None] * na)[idx[i, a]] = i
        F = np.exp(-2j * np.pi * np.outer(np.arange(na), np.arange(na)) / na)
        acc = np.zeros(na)
        for cells in lines.values():
            sub = M2[np.ix_(cells, cells)]
            acc += np.real(np.einsum("kj,jl,kl->k", F, sub, np.conj(F)))
        out.append(acc / len(lines))
    return np.concatenate(out)


def test_species_pooled_structure_factor_is_exact():
    shape = (6, 4)
    pl = dict(dim=2, n=shape, bc="periodic", r=0.1, eps=0.01, wall_lo=1.2, wall_hi=1.2,
              equation="species", perturb_ic=1)
    K, relax, nsteps = 3, 7, 60
    ex = T.pooled_expectation(pl, nsteps, K, relax)
    F = _dft_matrix(shape)
    S_exact = np.real(np.einsum("kj,jl,kl->k", F, ex["second"], np.conj(F)))
    cells = np.prod(shape)
    s0 = pl["eps"] * 1.2 * cells            # flat seeded perturbation, sigma^2 = eps c
    S = T.fe_structure_factor_pooled(shape, pl["r"], pl["eps"] * 1.2, s0, K, relax, nsteps)
    assert abs(S_exact[0]) < 1e-12
    assert np.max(np.abs(S[1:] - S_exact[1:]) / S_exact[1:]) < 1e-10
    # the transient matters: the stationary spectrum alone is off
    S_inf = T.fe_structure_factor(shape, pl["r"], pl["eps"] * 1.2)
    assert np.max(np.abs(S_inf[1:] - S_exact[1:]) / S_exact[1:]) > 5e-4


def test_species_pooled_structure_factor_late_window():
    # sampling that starts after step0 > 0 and a relaxation inside the run
    shape = (5, 3)
    pl = dict(dim=2, n=shape, bc="periodic", r=0.12, eps=0.02, wall_lo=0.9, wall_hi=0.9,
              equation="species", perturb_ic=1)
    ex = T.pooled_expectation(pl, 40, 4, 25, step0=10)
    F = _dft_matrix(shape)
    S_exact = np.real(np.einsum("kj,jl,kl->k", F, ex["second"], np.conj(F)))
    # the recursion starts from the seeded perturbation at step 10
    S = T.fe_structure_factor_pooled(shape, pl["r"], 0.02 * 0.9, 0.02 * 0.9 * 15, 4, 25, 40, step0=10)
    assert np.max(np.abs(S[1:] - S_exact[1:]) / S_exact[1:]) < 1e-10


def _heat_case(shape, T0, eps, r, K, nsteps):
    pl = dict(dim=len(shape), n=shape, bc="periodic", r=r, eps=eps, wall_lo=T0, wall_hi=T0,
              equation="heat", perturb_ic=0)
    ex = T.pooled_expectation(pl, nsteps, K, 0)
    exact = _per_axis_from_second_moment(shape, ex["second"])
    got = T.heat_axes_structure_factor_pooled(shape, r, eps, T0, K, 0, nsteps)
    v = T.heat_face_variance(shape, r, eps, T0)
    return exact, got, v


def test_heat_per_axis_pooled_3d():
    T0, eps = 1.3, 0.02
    exact, got, v = _heat_case((4, 4, 4), T0, eps, 0.1, 4, 1200)
    assert np.allclose(v, v[0])                      # cubic grid: one face variance
    rel = np.max(np.abs(got - exact) / exact)
    assert rel < 5e-4, rel
    # the linearised form (v = 0) misses by about v / T0^2
    lin = got / (1.0 + v[0] / (T0 * T0))
    assert np.max(np.abs(lin - exact) / exact) > 0.5 * v[0] / (T0 * T0) > 5e-3


def test_heat_per_axis_pooled_2d_unequal_axes():
    # a non-square grid has a different face variance per axis
    T0, eps = 1.1, 0.03
    exact, got, v = _heat_case((6, 4), T0, eps, 0.12, 5, 1500)
    assert abs(v[0] - v[1]) > 1e-4 * abs(v[0])
    assert np.max(np.abs(got - exact) / exact) < 5e-4


def test_heat_face_variance_matches_stationary_covariance():
    # v_a against the stationary covariance of the exact recursion (discrete
    # Lyapunov equation with the multiplicative term, theory.stationary)
    shape = (5, 4)
    pl = dict(dim=2, n=shape, bc="periodic", r=0.1, eps=0.02, wall_lo=1.4, wall_hi=1.4,
              equation="heat", perturb_ic=0)
    _, C = T.stationary(pl, iters=200)
    faces = T.faces_nd_periodic(shape)
    n = int(np.prod(shape))
    v_faces = [P @ C @ P for P, _, _, _ in faces]
    v0, v1 = np.mean(v_faces[:n]), np.mean(v_faces[n:])
    v = T.heat_face_variance(shape, 0.1, 0.02, 1.4)
    assert np.allclose([v0, v1], v, rtol=1e-9)
