"""GPU checks of the tensor-core covariance kernel (tcgen05, bf16 hi/lo
split, FP32 accumulation in tensor memory) against the FP64 product.

The split keeps ~16 significant bits per product: the error of one entry of
X^T X is bounded by about 2^-15 * sum_k |x_ki x_kj|; the tolerance below is
that bound with margin."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402


@pytest.mark.parametrize("N", [1, 16, 32, 100, 128, 129, 200, 256])
@pytest.mark.parametrize("K", [1, 27, 32])
def test_syrk_probe_matches_fp64(N, K):
    rng = np.random.default_rng(N * 100 + K)
    X = rng.normal(0.0, 0.03, size=(K, N)).astype(np.float32)
    X64 = X.astype(np.float64)
    ref = X64.T @ X64
    bound = np.abs(X64).T @ np.abs(X64)
    C = S.she_syrk_probe(X)
    assert np.all(np.abs(C - ref) <= 4.0 * 2.0 ** -16 * bound + 1e-30)


import she_workloads as W  # noqa: E402
from oracle import she as O  # noqa: E402


def _cov_case(N, R, steps, walls=(1.0, 2.0), bc="dirichlet", K=10, sk=True, relax=0, **kw):
    p = W.gradient_rod(n=(N, 1, 1), realizations=R, relax_steps=relax, stats_interval=K,
                       wall_lo=walls[0], wall_hi=walls[1], bc=bc, want_cov=1, want_sk=int(sk), **kw)
    with S.Simulation(p, **({"steps_per_launch": 37} if kw.get("precision") == "fp64" else {})) as sim:
        sim.step(steps)
        g = sim.stats(cov=True, sk=sk)
    o = O.finalize(p, O.run(p, R, steps, want_cov=1, want_sk=int(sk)))
    return p, g, o


@pytest.mark.parametrize("N,R,steps", [(16, 40, 200), (32, 400, 300), (100, 300, 200),
                                       (130, 300, 120), (200, 300, 120), (256, 200, 150), (32, 5000, 60)])
def test_fused_covariance_matches_oracle(N, R, steps):
    # small grids, several realizations per CTA, ragged rows, one or two
    # 128-cell halves, and (R = 5000 > 32 x SMs) two realization waves
    p, g, o = _cov_case(N, R, steps)
    assert g["n_samples"] == o["n"]
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * scale
    # diagonal of the tensor-core covariance vs the CUDA-core variance
    assert np.max(np.abs(np.diag(g["cov"]) - g["var"])) < 2e-4 * scale
    assert np.max(np.abs(g["sk_fluct"] - o["sk_fluct"])) < 2e-4 * np.max(o["sk_fluct"])
    assert np.allclose(g["sk"], o["sk"], rtol=1e-6, atol=2e-4 * np.max(o["sk_fluct"]))


@pytest.mark.parametrize("N,R,steps", [(300, 64, 120), (700, 24, 80)])
def test_fp32_long_rows_covariance_on_cuda_cores(N, R, steps):
    # FP32 rows above the tensor-core kernel's 256 cells: the fused row
    # kernel steps them and an FP64 SYRK on the CUDA cores takes each sample
    p, g, o = _cov_case(N, R, steps)
    assert g["n_samples"] == o["n"]
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * scale
    assert np.max(np.abs(np.diag(g["cov"]) - g["var"])) < 1e-5 * scale
    assert np.max(np.abs(g["sk_fluct"] - o["sk_fluct"])) < 2e-4 * np.max(o["sk_fluct"])


def test_fused_covariance_periodic():
    p, g, o = _cov_case(64, 300, 200, walls=(1.0, 1.0), bc="periodic")
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * scale
    assert np.max(np.abs(g["sk_fluct"] - o["sk_fluct"])) < 2e-4 * np.max(o["sk_fluct"])


def test_full_size_covariance_matches_oracle():
    # 256 cells x 4096 realizations, the benchmark's launch shape, 10 snapshots
    p, g, o = _cov_case(256, 4096, 100, sk=False)
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * scale


@pytest.mark.parametrize("N,R,kw", [(200, 4600, {}), (256, 3000, {"scheme": "pc"}), (256, 4096, {"var": True}),
                                   (160, 2300, {"tc_lags": 3}), (256, 1200, {"species": True})])
def test_covariance_warp_mix_matches_oracle(N, R, kw):
    """Above 128 cells (16 x 16) a CTA's realizations go to warps of two and
    warps of one (count - 15 warps of two, the others of one on 32 lanes of
    8 cells): R = 4600 fills a first wave with 30 per CTA (all warps of two)
    and leaves 40 for a second, 3000 gives 19-20 per CTA, 4096 26-27 (with
    the material table's second layout), 2300 15-16 (with the time
    correlation), 1200 7-8 (species, all warps of one)."""
    kw = dict(kw)
    var, species = kw.pop("var", False), kw.pop("species", False)
    base = dict(n=(N, 1, 1), realizations=R, relax_steps=0, stats_interval=10, want_cov=1, want_sk=0, **kw)
    if species:
        base.update(equation="species", wall_lo=1.0, wall_hi=1.5, n0=300.0)
    p = W.two_material_rod(cells=N, **base) if var else W.gradient_rod(**base)
    steps = 40
    with S.Simulation(p) as sim:
        sim.step(steps)
        g = sim.stats(cov=True, time_corr=bool(kw.get("tc_lags")))
    o = O.finalize(p, O.run(p, R, steps, want_cov=1))
    assert g["n_samples"] == o["n"]
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * scale
    assert np.max(np.abs(g["mean"] - o["mean"])) < 1e-5 * np.max(np.abs(o["mean"]))
    if kw.get("tc_lags"):
        assert np.max(np.abs(g["time_corr"] - o["time_corr"])) < 1e-3 * np.max(np.abs(o["time_corr"]))


@pytest.mark.parametrize("N,precision,status", [(300, "fp32", "SHE_ERR_UNSUPPORTED"),
                                               (2049, "fp64", "SHE_ERR_INVALID_ARG")])
def test_covariance_row_limits(N, precision, status):
    # the FP32 covariance runs on the fused kernels only; rows of at most
    # 2048 cells (the plain form)
    p = W.gradient_rod(n=(N, 1, 1), realizations=4, precision=precision, want_cov=1, want_sk=0, kernel="plain")
    with pytest.raises(S.SheError) as e:
        S.Simulation(p)
    assert e.value.status == getattr(S._abi, status)


def test_bounded_wait_times_out_and_context_survives():
    # a wait on a barrier nothing completes gives up and reports it
    assert S.lib().she_wait_probe(64) == S._abi.SHE_ERR_TIMEOUT
    # the context is still usable afterwards
    X = np.ones((4, 16), dtype=np.float32)
    assert np.allclose(S.she_syrk_probe(X), 4.0)


@pytest.mark.parametrize("N,R,steps,bc,kernel", [(16, 40, 203, "dirichlet", "auto"), (130, 70, 157, "dirichlet", "auto"),
                                                 (256, 33, 90, "periodic", "auto"), (48, 20, 95, "dirichlet", "plain"),
                                                 (600, 12, 41, "dirichlet", "auto"), (1100, 5, 30, "periodic", "plain")])
def test_fp64_covariance_matches_oracle_exactly(N, R, steps, bc, kernel):
    # FP64 state and FP64 covariance (CUDA cores): the same sample paths as
    # the oracle, so the pooled covariance and S(k) agree to rounding order
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.5, 1.5)
    p, g, o = _cov_case(N, R, steps, walls=walls, bc=bc, K=7, relax=23, precision="fp64", kernel=kernel)
    assert g["n_samples"] == o["n"]
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 1e-10 * scale
    assert np.max(np.abs(np.diag(g["cov"]) - g["var"])) < 1e-10 * scale
    assert np.max(np.abs(g["sk_fluct"] - o["sk_fluct"])) < 1e-10 * np.max(o["sk_fluct"])
