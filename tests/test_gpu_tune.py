"""The autotuner of the fused 1D kernel (she_params.tune), through the C ABI:
the layout it picks (cells per lane x lanes per realization) is one of the
scheme's layouts that holds the row, keeps the FP64 trajectories within
1e-12 of the oracle, is written to the cache file keyed by GPU model,
library build and problem shape, and is read back (no timing runs) by the
next handle of the same shape; SHE_TUNE_1D still overrides.  The implicit
schemes (backward Euler, Crank-Nicolson) are tuned the same way, each
candidate with its own factor tables."""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402

FE = {404, 408, 416, 432, 832, 1616, 1632, 3208, 3232}
PC = {404, 408, 416, 432, 832, 1632}
THETA = {404, 804, 808, 832, 1608, 1616, 3208, 3216, 3232}


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("SHE_TUNE_CACHE", str(path))
    monkeypatch.delenv("SHE_TUNE_1D", raising=False)
    return path


@pytest.mark.parametrize("N,scheme,bc", [(130, "fe", "dirichlet"), (256, "fe", "periodic"), (64, "pc", "dirichlet"),
                                         (500, "pc", "periodic"), (256, "cn", "dirichlet"), (200, "be", "periodic")])
def test_tuned_layout_keeps_parity_and_is_cached(cache, N, scheme, bc):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.4, 1.4)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, wall_lo=walls[0], wall_hi=walls[1], realizations=96, relax_steps=20,
                     want_cov=0, want_sk=0, scheme=scheme, tune=1)
    with S.Simulation(p) as sim:
        layout = int(sim.sizes().layout)
        tuning_launches = sim.launches()
        sim.step(150)
        x, _ = sim.state()
    assert layout in (PC if scheme == "pc" else THETA if scheme in ("be", "cn") else FE)
    assert (layout // 100) * (layout % 100) >= N
    o = O.run(p, 96, 150)
    assert np.max(np.abs(x - o["state"]) / np.abs(o["state"])) < 1e-12
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].split("\t")[-1] == str(layout)
    # the next handle of the same shape takes the cached layout without timing
    with S.Simulation(p) as sim2:
        assert int(sim2.sizes().layout) == layout
        assert sim2.launches() < tuning_launches
    assert len(cache.read_text().splitlines()) == 1


def test_tuned_time_correlation_fp32(cache):
    p = W.gradient_rod(n=(256, 1, 1), realizations=512, relax_steps=0, want_cov=0, tc_lags=6, tune=1)
    with S.Simulation(p) as sim:
        layout = int(sim.sizes().layout)
        sim.step(200)
        g = sim.stats(time_corr=True)
    assert layout in FE
    o = O.finalize(p, O.run(p, 512, 200))
    assert np.max(np.abs(g["time_corr"] - o["time_corr"])) < 1e-3 * np.max(np.abs(o["time_corr"]))


def test_override_beats_the_tuner(cache, monkeypatch):
    monkeypatch.setenv("SHE_TUNE_1D", "16,16")
    p = W.oracle_rod(n=(256, 1, 1), realizations=8, want_cov=0, want_sk=0, tune=1)
    with S.Simulation(p) as sim:
        assert int(sim.sizes().layout) == 1616
    assert not cache.exists()


def test_no_fused_layout_for_other_kernels(cache):
    # the FP32 covariance kernel has its own layout; 2D has none
    with S.Simulation(W.gradient_rod(n=(64, 1, 1), realizations=8, tune=1)) as sim:
        assert int(sim.sizes().layout) == 0
    with S.Simulation(W.species_2d(n=(16, 8, 1), realizations=2, want_sk=0, tune=1)) as sim:
        assert int(sim.sizes().layout) == 0
