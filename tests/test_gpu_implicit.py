"""GPU parity of the implicit schemes (backward Euler and Crank-Nicolson,
the implicit exercise of Sec. 6) through the C ABI: the diffusion implicit
with weight theta, the stochastic flux explicit,
(I - theta r L) T' = T + (1 - theta) r L T + r b + div G(T), solved per
realization and step by the kernel's partitioned tridiagonal solve.

* FP64 trajectories within 1e-12 of the oracle (the Thomas algorithm, cyclic
  by Sherman-Morrison): both schemes, Dirichlet and periodic, heat and
  species, ragged rows, every implicit layout (4 x 4 ... 32 x 32 cells x
  lanes; 8 x 32, 16 x 16 and 32 x 8 for the same 256-cell row), time steps below and far above forward Euler's limit, several
  launch windows; moments, the FP64 covariance and the time correlation.
* FP32: one step from a shared state within 2e-5; with the covariance (the
  tensor-core kernel stepping the implicit scheme), the mean, the covariance
  and the time correlation of whole runs against the oracle.
* Deterministic limit at r = 30: every sine mode multiplied per step by
  (1 - (1 - theta) x) / (1 + theta x).
* About 10^6 realizations of 4- and 5-cell rods within 4.5 batch SE of the
  exact moment recursion of the theta scheme.
* Refusals: 2D, the plain form, a rod of several materials, 1D rows longer
  than 1024 cells on the fused kernels.
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


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


def _rod(N, bc, scheme, r, eq="heat", R=5, precision="fp64", **kw):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.3, 1.3)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, equation=eq, wall_lo=walls[0], wall_hi=walls[1], dt=r, scheme=scheme,
                     realizations=R, kB=2e-3, n0=300.0, relax_steps=0, stats_interval=4, want_cov=0, want_sk=0,
                     precision=precision)
    p.update(kw)
    return p


@pytest.mark.parametrize("N", [16, 13, 30, 64, 100, 256, 200, 512, 777])
@pytest.mark.parametrize("bc,scheme,r,eq,kB", [("dirichlet", "be", 0.3, "heat", 2e-3),
                                               ("periodic", "cn", 5.0, "heat", 2e-3),
                                               ("dirichlet", "cn", 40.0, "heat", 1e-4),
                                               ("periodic", "be", 2.0, "species", 2e-3)])
def test_fp64_trajectory_matches_oracle(N, bc, scheme, r, eq, kB):
    p = _rod(N, bc, scheme, r, eq, kB=kB)
    with S.Simulation(p, steps_per_launch=29) as sim:
        sim.step(90)
        x, _ = sim.state()
        g = sim.stats(raw=True)
    o = O.run(p, p["realizations"], 90)
    # relative to the value, or to 1 where a fluctuating value passes near 0
    assert np.max(np.abs(x - o["state"]) / np.maximum(np.abs(o["state"]), 1.0)) < 1e-12
    assert g["n_samples"] == o["n_samples"]
    assert np.allclose(g["sum_d2"], o["sum_d2"], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("layout", ["8,32", "16,16", "32,8"])
@pytest.mark.parametrize("N,bc,scheme,eq", [(256, "dirichlet", "cn", "heat"), (200, "periodic", "be", "heat"),
                                            (250, "dirichlet", "be", "species")])
def test_forced_layouts_match_oracle(monkeypatch, layout, N, bc, scheme, eq):
    """Every implicit layout of a 256-cell row (SHE_TUNE_1D picks it, as the
    autotuner does) keeps the trajectories within 1e-12."""
    monkeypatch.setenv("SHE_TUNE_1D", layout)
    p = _rod(N, bc, scheme, 3.0, eq, R=9)
    with S.Simulation(p, steps_per_launch=37) as sim:
        c, l = (int(v) for v in layout.split(","))
        assert int(sim.sizes().layout) == 100 * c + l
        sim.step(80)
        x, _ = sim.state()
    o = O.run(p, p["realizations"], 80)
    assert np.max(np.abs(x - o["state"]) / np.maximum(np.abs(o["state"]), 1.0)) < 1e-12


@pytest.mark.parametrize("scheme", ["be", "cn"])
def test_fp64_covariance_and_time_correlation(scheme):
    p = _rod(48, "dirichlet", scheme, 3.0, want_cov=1, tc_lags=3)
    with S.Simulation(p) as sim:
        sim.step(200)
        g = sim.stats(cov=True, time_corr=True)
    o = O.finalize(p, O.run(p, p["realizations"], 200, want_cov=1))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 1e-10 * np.max(np.diag(o["cov"]))
    assert np.allclose(g["time_corr"], o["time_corr"], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("N,bc,scheme", [(256, "dirichlet", "be"), (130, "periodic", "cn"), (1000, "dirichlet", "cn")])
def test_fp32_one_step_from_shared_state(N, bc, scheme):
    p = _rod(N, bc, scheme, 4.0, precision="fp32", R=16)
    x = W.random_states(p, 16, seed=N).astype(np.float32)
    with S.Simulation(p) as sim:
        sim.set_state(x, 321)
        sim.step(1)
        got, _ = sim.state()
    ref = np.array([O.step(p, x[i].astype(np.float64), 321, i) for i in range(16)])
    assert rel_err(got.astype(np.float64), ref) < 2e-5


@pytest.mark.parametrize("N,bc,scheme,eq,lags", [(256, "dirichlet", "cn", "heat", 0), (200, "periodic", "be", "heat", 4),
                                                 (100, "dirichlet", "be", "species", 0),
                                                 (30, "periodic", "cn", "heat", 3), (16, "dirichlet", "cn", "heat", 0),
                                                 (13, "periodic", "be", "species", 2), (64, "dirichlet", "be", "heat", 5)])
def test_fp32_covariance_on_the_tensor_cores(N, bc, scheme, eq, lags):
    """FP32 with the covariance: the fused tensor-core kernel steps the
    implicit scheme with the factor tables of its own layout (4 cells per lane
    up to 128 cells, 16 x 16 above); whole runs against the FP64 oracle, the
    covariance within the bar of the explicit FP32 covariance tests."""
    R, steps = 64, 240
    p = _rod(N, bc, scheme, 2.5, eq, R=R, precision="fp32", want_cov=1, tc_lags=lags, stats_interval=6)
    with S.Simulation(p, steps_per_launch=70) as sim:
        sim.step(steps)
        g = sim.stats(cov=True, time_corr=lags > 0)
    o = O.finalize(p, O.run(p, R, steps, want_cov=1))
    tref = O.reference_profile(p)
    assert np.max(np.abs(g["mean"] - o["mean"])) < 1e-5 * np.max(np.abs(o["mean"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["var"] - np.diag(o["cov"]))) < 2e-4 * np.max(np.diag(o["cov"]))
    if lags:
        assert np.max(np.abs(g["time_corr"] - o["time_corr"])) < 1e-3 * np.max(np.abs(o["time_corr"]))
        assert np.allclose(g["time_corr"][0], g["var"] + (g["mean"] - tref) ** 2, rtol=1e-4)


@pytest.mark.parametrize("scheme", ["be", "cn"])
def test_deterministic_modes_at_large_time_step(scheme):
    N, r, steps = 100, 30.0, 25
    p = _rod(N, "dirichlet", scheme, r, stochastic=0, perturb_ic=0, R=2)
    xs = (np.arange(N) + 0.5) / N
    x0 = 1.0 + xs + 0.2 * np.sin(2 * np.pi * xs) + 0.05 * np.sin(9 * np.pi * xs)
    with S.Simulation(p) as sim:
        sim.set_state(np.vstack([x0, x0]), 0)
        sim.step(steps)
        got, _ = sim.state()
    ref = T.sine_mode_solution(N, r, 1.0, 2.0, x0, steps, scheme=scheme)
    assert np.max(np.abs(got[0] - ref)) < 1e-12


BATCHES, PER_BATCH = 32, 32768


@pytest.mark.parametrize("N,bc,eq,scheme,r,precision", [(4, "dirichlet", "heat", "be", 2.0, "fp32"),
                                                        (5, "periodic", "species", "cn", 0.8, "fp64"),
                                                        (4, "periodic", "heat", "cn", 6.0, "fp32")])
def test_moments_match_exact_recursion(N, bc, eq, scheme, r, precision):
    K, relax, steps = 3, 12, 60
    walls = (1.0, 1.6) if bc == "dirichlet" else (1.2, 1.2)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, equation=eq, wall_lo=walls[0], wall_hi=walls[1], dt=r, scheme=scheme,
                     kB=0.02, n0=50.0, stats_interval=K, relax_steps=relax, want_cov=0, want_sk=0,
                     precision=precision)
    rr, eps = O.dimensionless(p)
    pl = dict(dim=1, n=(N,), bc=bc, r=rr, eps=eps, wall_lo=walls[0], wall_hi=walls[1], equation=eq,
              scheme=scheme, perturb_ic=1)
    ex = T.pooled_expectation(pl, steps, K, relax)
    tref = O.reference_profile(p)
    m1, m2 = [], []
    for b in range(BATCHES):
        with S.Simulation(dict(p, realizations=PER_BATCH, seed=7919 + 104729 * b)) as sim:
            sim.step(steps)
            g = sim.stats()
        mu = g["mean"] - tref
        m1.append(mu)
        m2.append(g["var"] + mu * mu)
    m1, m2 = np.array(m1), np.array(m2)
    z1 = (m1.mean(0) - ex["mean_delta"]) / (m1.std(0, ddof=1) / np.sqrt(BATCHES))
    z2 = (m2.mean(0) - np.diag(ex["second"])) / (m2.std(0, ddof=1) / np.sqrt(BATCHES))
    assert np.max(np.abs(z1)) < 4.5 and np.max(np.abs(z2)) < 4.5


@pytest.mark.parametrize("kw,status", [
    (dict(kernel="plain"), "SHE_ERR_UNSUPPORTED"),
    (dict(n=(1025, 1, 1)), "SHE_ERR_UNSUPPORTED"),
])
def test_implicit_refusals(kw, status):
    p = _rod(32, "dirichlet", "cn", 2.0, **kw)
    with pytest.raises(S.SheError) as e:
        S.Simulation(p)
    assert e.value.status == getattr(S._abi, status)


def test_implicit_2d_and_materials_refused():
    with pytest.raises(S.SheError) as e:
        S.Simulation(W.species_2d(n=(16, 8, 1), scheme="be", want_sk=0))
    assert e.value.status == S._abi.SHE_ERR_UNSUPPORTED
    with pytest.raises(S.SheError) as e:
        S.Simulation(W.two_material_rod(cells=32, scheme="cn", want_cov=0, precision="fp64"))
    assert e.value.status == S._abi.SHE_ERR_UNSUPPORTED


def test_fused_rows_longer_than_1024_refused_for_every_scheme():
    with pytest.raises(S.SheError) as e:
        S.Simulation(W.oracle_rod(n=(1100, 1, 1), want_cov=0, want_sk=0))
    assert e.value.status == S._abi.SHE_ERR_UNSUPPORTED
    # the plain form takes them
    with S.Simulation(W.oracle_rod(n=(1100, 1, 1), want_cov=0, want_sk=0, kernel="plain", realizations=2)) as sim:
        sim.step(3)
