"""Physics of the GPU statistics at the full benchmark configurations,
through the C ABI, against what the paper and the exact discrete scheme
predict.

Each configuration runs as independent realization shards: separate handles
whose noise streams are disjoint contiguous ranges (stream_offset), so the
union is exactly the full ensemble and each shard gives one independent
estimate.  Standard errors come from the scatter of the shards, so a
comparison is a Student t with (shards - 1) degrees of freedom.  Many
entries (cells, wavenumbers) are tested at once through the mean of t^2,
whose expectation is nu / (nu - 2) when the prediction is right and grows by
(bias / SE)^2 when it is not, plus a bound on the largest |t|.

* 1D rod in a gradient (256 cells, walls 1 and 2, 4096 realizations, FP32,
  10^6 steps, covariance on tcgen05): mean, variance and off-diagonal
  covariance against the exact stationary moments of the forward-Euler
  recursion with multiplicative noise (oracle/theory.py `stationary`), and
  the far-field (|i - j| >= N/4) covariance projected on the long-range
  shape, the non-equilibrium correlation of Sec. 3, Eq. (3.13).
* 2D species (256^2 periodic, 256 realizations, FP32, 10^5 steps, full S(k)
  on tcgen05): every k != 0 against the forward-Euler structure factor
  eps_c c N / (1 - r mu_k / 2) (Eq. (3.12) with the cell volume restored
  and the finite-r correction), pooled over the sampling schedule from the
  seeded flat initial spectrum.
* 3D heat (256^3 periodic, 8 realizations, FP32, 10^4 steps, per-axis S(k)
  on tcgen05): against the per-axis transient from a uniform start with the
  multiplicative face-noise strength (T0^2 + v_a).
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O
from oracle import theory as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402


def _shards(p, nshards, stats_kw):
    R = p["realizations"]
    per = R // nshards
    assert per * nshards == R
    out = []
    for b in range(nshards):
        with S.Simulation(p, realizations=per, stream_offset=b * per) as sim:
            sim.step(p["steps"])
            out.append(sim.stats(**stats_kw))
    return out


def _t(values, predicted):
    """Student t of the shard mean against the prediction, per entry."""
    v = np.asarray(values)
    B = v.shape[0]
    se = v.std(axis=0, ddof=1) / np.sqrt(B)
    return (v.mean(axis=0) - predicted) / se, se


def _mean_t2_ok(t, nu, n_eff, width=6.0):
    """mean t^2 within `width` standard deviations of its expectation for n_eff
    independent t_nu entries: E t^2 = nu/(nu-2), Var t^2 = E t^4 - (E t^2)^2
    with E t^4 = 3 nu^2 / ((nu - 2)(nu - 4))."""
    e2 = nu / (nu - 2.0)
    var = 3.0 * nu * nu / ((nu - 2.0) * (nu - 4.0)) - e2 * e2
    m = float(np.mean(t * t))
    return abs(m - e2) <= width * np.sqrt(var / n_eff), m, e2


def test_gradient_rod_moments_and_long_range_correlation():
    p = W.gradient_rod()
    N = p["n"][0]
    B = 16
    outs = _shards(p, B, dict(cov=True))
    assert all(o["n_samples"] == p["realizations"] // B * 90_000 for o in outs)
    r, eps = O.dimensionless(p)
    pl = dict(dim=1, n=p["n"], bc="dirichlet", r=r, eps=eps, wall_lo=p["wall_lo"],
              wall_hi=p["wall_hi"], equation="heat")
    m_ex, C_ex = T.stationary(pl, iters=100)

    # mean profile: the exact steady mean (linear, Sec. 3) per cell
    # (the mean's scatter is carried by the few slowest modes, so the
    # cells' t values move together: about 4 independent entries)
    t_mean, _ = _t([o["mean"] for o in outs], m_ex)
    ok, m2, e2 = _mean_t2_ok(t_mean, B - 1, 4.0)
    print("mean: mean t^2 %.3f (expected %.3f), max |t| %.2f" % (m2, e2, np.max(np.abs(t_mean))))
    assert ok and np.max(np.abs(t_mean)) < 8.0

    # variance: the exact diagonal (eps <T_i>^2 with the forward-Euler and
    # multiplicative corrections)
    t_var, se_var = _t([o["var"] for o in outs], np.diag(C_ex))
    ok, m2, e2 = _mean_t2_ok(t_var, B - 1, N / 4.0)
    print("var: mean t^2 %.3f (expected %.3f), max |t| %.2f, median SE/var %.2e"
          % (m2, e2, np.max(np.abs(t_var)), np.median(se_var / np.diag(C_ex))))
    assert ok and np.max(np.abs(t_var)) < 8.0

    # off-diagonal: projection amplitude on the exact off-diagonal shape
    # (the forward-Euler short-range part and the long-range part together)
    off = ~np.eye(N, dtype=bool)
    shape_off = C_ex[off]
    a_off = [float(o["cov"][off] @ shape_off / (shape_off @ shape_off)) for o in outs]
    t_off, se_off = _t(a_off, 1.0)
    print("off-diagonal amplitude %.4f +- %.4f (t %.2f)" % (np.mean(a_off), se_off, t_off))
    assert abs(t_off) < 4.0

    # far field |i - j| >= N/4: the exact covariance there is the long-range
    # correlation alone; amplitude against it, and against the continuum
    # form of Eq. (3.13) (within 2 % of its scale there)
    i, j = np.indices((N, N))
    far = np.abs(i - j) >= N // 4
    lr_ex = C_ex[far]
    a_far = [float(o["cov"][far] @ lr_ex / (lr_ex @ lr_ex)) for o in outs]
    t_far, se_far = _t(a_far, 1.0)
    lr_c = T.long_range_correlation(N, eps, p["wall_hi"] - p["wall_lo"])[far]
    a_c = [float(o["cov"][far] @ lr_c / (lr_c @ lr_c)) for o in outs]
    print("long-range amplitude (exact discrete) %.4f +- %.4f (t %.2f); vs Eq. (3.13) %.4f +- %.4f"
          % (np.mean(a_far), se_far, t_far, np.mean(a_c), np.std(a_c, ddof=1) / np.sqrt(B)))
    assert abs(t_far) < 4.0
    assert abs(np.mean(a_c) - 1.0) < 4.0 * np.std(a_c, ddof=1) / np.sqrt(B) + 0.02
    # the signal is resolved: the amplitude is many standard errors from zero
    assert np.mean(a_far) > 5.0 * se_far


def test_species_2d_structure_factor():
    p = W.species_2d()
    nx, ny = p["n"][0], p["n"][1]
    B = 16
    outs = _shards(p, B, dict(sk=True))
    r, eps_c = O.dimensionless(p)
    c = p["wall_lo"]
    cells = nx * ny
    pred = T.fe_structure_factor_pooled((nx, ny), r, eps_c * c, eps_c * abs(c) * cells, p["stats_interval"],
                                        p["relax_steps"], p["steps"])
    # one entry per pair (k, -k) of the real field, k != 0
    kx, ky = np.meshgrid(np.arange(nx), np.arange(ny))
    lin = (ky * nx + kx).ravel()
    mirror = (((ny - ky) % ny) * nx + (nx - kx) % nx).ravel()
    keep = (lin < mirror) | ((lin == mirror) & (lin != 0))
    vals = np.array([o["sk"] for o in outs])[:, lin[keep]]
    t, se = _t(vals, pred[lin[keep]])
    ok, m2, e2 = _mean_t2_ok(t, B - 1, keep.sum())
    print("S(k) 2D: %d wavenumbers, mean t^2 %.4f (expected %.4f), max |t| %.2f, median SE/S %.2e"
          % (keep.sum(), m2, e2, np.max(np.abs(t)), np.median(se / pred[lin[keep]])))
    assert ok and np.max(np.abs(t)) < 9.0
    # the finite-r correction is resolved: the flat value eps_c c N is off
    flat = eps_c * c * cells
    t_flat = (vals.mean(axis=0) - flat) / se
    assert np.mean(t_flat * t_flat) > 10.0 * e2


def test_cube_3d_per_axis_structure_factor():
    p = W.cube_3d()
    n = p["n"][0]
    B = 8
    outs = _shards(p, B, dict(sk_axes=True))
    r, eps = O.dimensionless(p)
    pred = T.heat_axes_structure_factor_pooled(tuple(p["n"]), r, eps, p["wall_lo"], p["stats_interval"],
                                               p["relax_steps"], p["steps"])
    # k and n - k coincide (real field): k = 0 .. n/2 on each axis
    idx = np.concatenate([a * n + np.arange(n // 2 + 1) for a in range(3)])
    vals = np.array([o["sk_axes"] for o in outs])[:, idx]
    t, se = _t(vals, pred[idx])
    ok, m2, e2 = _mean_t2_ok(t, B - 1, len(idx) / 3.0)
    print("S(k) per axis 3D: mean t^2 %.3f (expected %.3f), max |t| %.2f, median SE/S %.2e"
          % (m2, e2, np.max(np.abs(t)), np.median(se / pred[idx])))
    assert ok and np.max(np.abs(t)) < 12.0
    # the multiplicative term is resolved: the linearised prediction is off
    v = T.heat_face_variance(tuple(p["n"]), r, eps, p["wall_lo"])
    lin = pred[idx] / (1.0 + v[0] / p["wall_lo"] ** 2)
    t_lin = (vals.mean(axis=0) - lin) / se
    assert np.mean(t_lin * t_lin) > 4.0 * e2
