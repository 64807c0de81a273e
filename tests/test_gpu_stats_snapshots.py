"""Parity of the tensor-core statistics at the benchmark shapes, on the
kernels' own snapshots, with error bars derived from the arithmetic.

Comparing an FP32 run with the FP64 oracle mixes two errors: the statistics'
arithmetic, and the FP32 trajectory drifting from the FP64 one (a random
walk of single-precision roundings, about 1e-7 per step, filtered by the
contractive step).  Here the second is removed: every launch is one step
that takes one sample (K = 1), the state the kernel sampled is read back
after it, and the host forms the same statistic from those exact FP32
snapshots in FP64.  What is left is the arithmetic of the statistics path:

* delta = T - T_ref in FP32, T_ref = fma(dref, i + 1/2, wall) rounded once
  (|error| <= 2^-24 |T_ref| <= 6e-8 for walls in [1, 2));
* the bf16 hi/lo split: x = hi + lo + e, |lo| <= 2^-9 |x|, |e| <= 2^-18 |x|,
  products hi hi' + hi lo' + lo hi' exact in FP32 and missing lo lo' and the
  split remainders: at most 3 x 2^-18 |x x'| per product;
* FP32 accumulation in tensor memory: each accumulation step of the tensor
  core errs by up to one unit in the last place of the partial sum, and the
  errors are biased (the accumulation truncates), so sums of same-signed
  terms (a diagonal) take the worst case: steps x 2^-23 x the sum.

Covariance (1D, 256 cells x 4096 realizations): a worst-case bound per
element, sum over samples and realizations of
(3 x 2^-18 + 32 x 2^-24) |d_i d_j| + 6e-8 (|d_i| + |d_j|), divided by n
(one sample per launch: each entry is one MMA accumulation of up to 32
products per CTA, bounded here as 32 steps).

Structure factors (2D full, 256 x 256; 3D per axis, 256^3): a worst-case
bound is of order the sum of |terms| while the result is a sum with random
signs (sqrt(terms) smaller), so the bar is probabilistic: each rounding is an
independent error uniform within its bound (the model of probabilistic
rounding-error analysis), which makes the error of a transform coefficient
approximately normal with a standard deviation computed from the data below,
and the bar is 8 of those standard deviations.
"""
import numpy as np
import pytest

import she_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402

U_SPLIT = 3.0 * 2.0 ** -18      # one bf16x3 product, relative
U_ACC = 2.0 ** -23              # one FP32 accumulation step of the tensor core, relative to the
                                # partial sum: up to one unit in the last place (it truncates)


def _ref_profile(p):
    N = p["n"][0]
    if p.get("bc", "dirichlet") == "dirichlet" and p["dim"] == 1:
        return p["wall_lo"] + (p["wall_hi"] - p["wall_lo"]) * (np.arange(N) + 0.5) / N
    return np.full(int(np.prod(p["n"][: p["dim"]])), float(p["wall_lo"]))


def test_covariance_on_own_snapshots_at_bench_shape():
    M = 16                                   # samples, one per single-step launch
    relax = 3000
    p = W.gradient_rod(relax_steps=relax, stats_interval=1, steps=relax + M)
    N, R = p["n"][0], p["realizations"]
    ref = _ref_profile(p)
    S2 = np.zeros((N, N))
    A2 = np.zeros((N, N))
    A1 = np.zeros(N)
    s1 = np.zeros(N)
    with S.Simulation(p) as sim:
        sim.step(relax)                      # no sample yet
        for _ in range(M):
            sim.step(1)                      # one launch, one sample
            st, _ = sim.state()
            d = st.astype(np.float64) - ref
            S2 += d.T @ d
            a = np.abs(d)
            A2 += a.T @ a
            A1 += a.sum(axis=0)
            s1 += d.sum(axis=0)
        g = sim.stats(cov=True)
    n = R * M
    assert g["n_samples"] == n
    mu = s1 / n
    second_gpu = g["cov"] + np.outer(g["mean"] - ref, g["mean"] - ref)
    second = S2 / n
    bound = ((U_SPLIT + 32 * U_ACC) * A2 + 6e-8 * (A1[:, None] + A1[None, :])) / n
    err = np.abs(second_gpu - second)
    print("covariance: max |err| / bound %.3f, max |err| / max diag %.2e"
          % (np.max(err / bound), np.max(err) / np.max(np.diag(second))))
    assert np.all(err <= bound)
    # the mean (CUDA-core moments) from the same snapshots
    assert np.max(np.abs((g["mean"] - ref) - mu)) <= 7e-8


def test_full_structure_factor_2d_on_own_snapshots_at_bench_shape():
    # Two stages, K = 256 in MMAs of 16 (x 3 split terms): 48 FP32
    # accumulation roundings per output.  Per realization and sample, the
    # SD of one coefficient's error (real or imaginary part) is the root sum
    # of squares of: the row stage's split errors carried through the column
    # stage (U_SPLIT ||delta|| / sqrt(3)); the column stage's split errors
    # on the intermediate D1 (the same size by Parseval); the row stage's
    # accumulation roundings (each <= U_ACC x the row's sum of |terms|,
    # 48 of them: 4 U_ACC ||(row L1 norms)||_2); the column stage's
    # (4 U_ACC x the column's sum of |D1|, largest column).
    M = 4
    relax = 400
    R = 8
    p = W.species_2d(realizations=R, relax_steps=relax, stats_interval=1, steps=relax + M)
    nx, ny = p["n"][0], p["n"][1]
    acc = np.zeros((ny, nx))
    var = np.zeros((ny, nx))
    with S.Simulation(p) as sim:
        sim.step(relax)
        for _ in range(M):
            sim.step(1)
            st, _ = sim.state()
            d = st.astype(np.float64).reshape(R, ny, nx) - p["wall_lo"]
            Fx = np.fft.fft(d, axis=2)                  # the row stage, [R][y][kx]
            F = np.fft.fft(Fx, axis=1)                  # [R][ky][kx]
            P = np.abs(F) ** 2
            acc += P.sum(axis=0)
            for rr in range(R):
                n2 = np.sum(d[rr] ** 2)
                rows_l1 = np.sum(np.abs(d[rr]), axis=1)
                col_l1 = np.max(np.sum(np.abs(Fx[rr].real) + np.abs(Fx[rr].imag), axis=0))
                sd2 = (2.0 * U_SPLIT ** 2 / 3.0 * n2 + 16.0 * U_ACC ** 2 * np.sum(rows_l1 ** 2)
                       + 16.0 * U_ACC ** 2 * col_l1 ** 2)
                # |F + e|^2 - |F|^2 ~ 2 (Re F e_re + Im F e_im): variance 4 |F|^2 sd2
                var += 4.0 * P[rr] * sd2
        g = sim.stats(sk=True)
    n = R * M
    assert g["n_samples"] == n
    host = (acc / n).ravel()
    bar = 8.0 * np.sqrt(var).ravel() / n
    err = np.abs(g["sk"][1:] - host[1:])
    print("S(k) 2D: max |err| / bar %.3f, max |err| / S %.2e, max bar / S %.2e"
          % (np.max(err / bar[1:]), np.max(err / host[1:]), np.max(bar[1:] / host[1:])))
    assert np.all(err <= bar[1:])


def test_per_axis_structure_factor_3d_on_own_snapshots_at_bench_shape():
    # The line covariance G = sum over lines of delta_line delta_line^T in
    # tiles of 32 lines (2 MMAs x 3 split terms each), about 14 tiles per CTA
    # and axis for one realization, flushed to FP64 after every sample: at
    # most 6 x 14 = 84 FP32 accumulation steps per element.  S_a(k) =
    # sum_jl G_jl cos(.) / lines.  The diagonal G_jj sums positive terms, so
    # its biased accumulation errors add up: 84 U_ACC sum_j G_jj / lines, the
    # same for every k.  Off the diagonal the terms have both signs; there
    # each element's accumulation error (<= 84 U_ACC sum_lines |delta_j
    # delta_l|) and every product's split error are taken as independent
    # between elements, root sum of squares, 8 standard deviations.
    M = 3
    relax = 100
    m_acc = 84.0
    p = W.cube_3d(realizations=1, relax_steps=relax, stats_interval=1, steps=relax + M)
    n = p["n"][0]
    acc = np.zeros(3 * n)
    var = np.zeros(3 * n)
    diag = np.zeros(3 * n)
    off = ~np.eye(n, dtype=bool)
    with S.Simulation(p) as sim:
        sim.step(relax)
        for _ in range(M):
            sim.step(1)
            st, _ = sim.state()
            d = st.astype(np.float64).reshape(n, n, n) - p["wall_lo"]     # [z][y][x]
            for a, ax in enumerate((2, 1, 0)):                           # axes x, y, z
                D = np.ascontiguousarray(np.moveaxis(d, ax, -1).reshape(-1, n))   # [lines][n]
                lines = D.shape[0]
                P = np.abs(np.fft.fft(D, axis=1)) ** 2
                acc[a * n:(a + 1) * n] += P.mean(axis=0)
                l2 = np.sum(D * D, axis=1)
                Dabs = np.abs(D)
                gabs = Dabs.T @ Dabs
                diag[a * n:(a + 1) * n] += m_acc * U_ACC * np.trace(gabs) / lines
                sd2 = (U_SPLIT ** 2 * np.sum(l2 ** 2) / 3.0
                       + (m_acc * U_ACC) ** 2 / 3.0 * np.sum(gabs[off] ** 2)) / (lines * lines)
                var[a * n:(a + 1) * n] += sd2
        g = sim.stats(sk_axes=True)
    assert g["n_samples"] == M
    host = acc / M
    bar = (diag + 8.0 * np.sqrt(var)) / M
    err = np.abs(g["sk_axes"] - host)
    print("S(k) per axis 3D: max |err| / bar %.3f, max |err| / S %.2e, max bar / S %.2e, mean signed err / S %.2e"
          % (np.max(err / bar), np.max(err / host), np.max(bar / host), np.mean((g["sk_axes"] - host) / host)))
    assert np.all(err <= bar)
