"""GPU parity of the time correlation <delta_i(t + l K) delta_i(t)> (the
exercise on <dT_i^{n+m} dT_i^n>, Sec. 6) against the FP64 oracle, through the
C ABI: FP64 to 1e-9 relative across launch windows (forward Euler and
predictor-corrector, with and without the FP64 covariance), FP32 within the
single-precision trajectory error, also beside the tensor-core covariance,
the pairs restarting at she_reset_stats and at a state overwrite, and the
unsupported combinations refused."""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402


@pytest.mark.parametrize("N,bc,eq,scheme,cov", [(32, "dirichlet", "heat", "fe", 0),
                                                (33, "periodic", "species", "pc", 0),
                                                (130, "dirichlet", "heat", "pc", 0),
                                                (64, "dirichlet", "heat", "fe", 1)])
def test_fp64_time_corr_matches_oracle(N, bc, eq, scheme, cov):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.3, 1.3)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, equation=eq, wall_lo=walls[0], wall_hi=walls[1], n0=200.0, kB=5e-3,
                     realizations=5, stats_interval=3, relax_steps=10, tc_lags=5, want_cov=cov, want_sk=0,
                     scheme=scheme, precision="fp64")
    with S.Simulation(p, steps_per_launch=37) as sim:
        sim.step(200)
        g = sim.stats(time_corr=True, cov=bool(cov))
    o = O.finalize(p, O.run(p, 5, 200, want_cov=cov))
    assert g["time_corr"].shape == (5, N)
    assert np.allclose(g["time_corr"], o["time_corr"], rtol=1e-9, atol=1e-15)
    # lag 0 is the pooled second moment
    assert np.allclose(g["time_corr"][0], g["var"] + (g["mean"] - O.reference_profile(p)) ** 2, rtol=1e-9)


def test_fp32_time_corr_matches_oracle():
    p = W.gradient_rod(n=(256, 1, 1), realizations=64, relax_steps=0, stats_interval=10, want_cov=0,
                       tc_lags=8)
    with S.Simulation(p) as sim:
        sim.step(300)
        g = sim.stats(time_corr=True)
    o = O.finalize(p, O.run(p, 64, 300))
    scale = np.max(np.abs(o["time_corr"]))
    assert np.max(np.abs(g["time_corr"] - o["time_corr"])) < 1e-3 * scale


@pytest.mark.parametrize("N,scheme,var", [(256, "fe", False), (200, "pc", False), (256, "fe", True), (100, "fe", False)])
def test_fp32_time_corr_beside_the_tensor_core_covariance(N, scheme, var):
    """FP32 with the covariance: the fused tensor-core kernel takes the time
    correlation too (its lag sums in FP64 device memory); both statistics
    against the oracle, the time correlation within the FP32 bar above, the
    covariance within the bar of the covariance tests."""
    kw = dict(n=(N, 1, 1), realizations=64, relax_steps=0, stats_interval=10, want_cov=1, tc_lags=6,
              scheme=scheme)
    p = W.two_material_rod(cells=N, **kw) if var else W.gradient_rod(**kw)
    with S.Simulation(p) as sim:
        sim.step(300)
        g = sim.stats(time_corr=True, cov=True)
    o = O.finalize(p, O.run(p, 64, 300, want_cov=1))
    scale = np.max(np.abs(o["time_corr"]))
    assert np.max(np.abs(g["time_corr"] - o["time_corr"])) < 1e-3 * scale
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * np.max(np.diag(o["cov"]))
    assert np.allclose(g["time_corr"][0], g["var"] + (g["mean"] - O.reference_profile(p)) ** 2, rtol=1e-4)


def test_pairs_restart_at_reset():
    p = W.oracle_rod(n=(16, 1, 1), realizations=4, stats_interval=2, relax_steps=0, tc_lags=4, want_cov=0,
                     want_sk=0, precision="fp64")
    with S.Simulation(p) as sim:
        sim.step(50)
        st, step = sim.state()
        S.she_reset_stats(sim.h)
        sim.step(40)
        g = sim.stats(time_corr=True)
    o = O.finalize(p, O.run(p, 4, 40, step0=step, state=st))
    assert np.allclose(g["time_corr"], o["time_corr"], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("device", [False, True])
def test_pairs_restart_at_set_state(device):
    # the statistics span two trajectories: 60 steps from the initial
    # condition, then 44 steps from an overwritten state; the time
    # correlation pairs samples within each of them only, so it is the sum of
    # two oracle runs (each pairs within its own run) over their pair counts
    p = W.oracle_rod(n=(24, 1, 1), wall_lo=1.0, wall_hi=1.5, realizations=4, stats_interval=2,
                     relax_steps=0, tc_lags=5, want_cov=0, want_sk=0, precision="fp64")
    x = W.random_states(p, 4, seed=3)
    with S.Simulation(p, steps_per_launch=14) as sim:
        sim.step(60)
        if device:
            d = torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
            torch.cuda.synchronize()
            S.she_set_state_device(sim.h, d.data_ptr(), d.numel() * 8, 60)
        else:
            sim.set_state(x, 60)
        sim.step(44)
        g = sim.stats(time_corr=True)
    a = O.run(p, 4, 60)
    b = O.run(p, 4, 44, step0=60, state=x)
    tc = (a["sum_tc"] + b["sum_tc"]) / (a["n_tc"] + b["n_tc"])[:, None]
    assert np.allclose(g["time_corr"], tc, rtol=1e-9, atol=1e-15)
    # the moments pool both trajectories
    ref = O.reference_profile(p)
    n = a["n_samples"] + b["n_samples"]
    mu = (a["sum_d"] + b["sum_d"]) / n
    assert np.allclose(g["mean"], ref + mu, rtol=1e-12)


@pytest.mark.parametrize("kw,status", [(dict(kernel="plain"), "SHE_ERR_UNSUPPORTED"),
                                       (dict(tc_lags=65), "SHE_ERR_INVALID_ARG")])
def test_time_corr_outside_its_kernel_is_refused(kw, status):
    q = dict(dict(tc_lags=4, want_cov=0, want_sk=0), **kw)
    p = W.oracle_rod(**q)
    with pytest.raises(S.SheError) as e:
        S.Simulation(p)
    assert e.value.status == getattr(S._abi, status)


def test_time_corr_2d_is_refused():
    p = W.species_2d(n=(8, 6, 1), tc_lags=3, want_sk=0)
    with pytest.raises(S.SheError) as e:
        S.Simulation(p)
    assert e.value.status == S._abi.SHE_ERR_UNSUPPORTED
