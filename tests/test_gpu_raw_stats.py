"""The raw accumulators and the host finalisation through the C ABI:
she_stats_raw followed by she_finalize gives exactly what she_stats gives
(1D with the covariance and the time correlation, 2D with the full S(k), 3D
with the per-axis S(k)), and the element-wise sum of two shards' raw blocks
(disjoint noise streams, stream_offset) finalises to the statistics of one
handle running the whole ensemble."""
import numpy as np
import pytest

import she_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402


CASES = [
    (W.gradient_rod(n=(64, 1, 1), realizations=96, relax_steps=100, steps=600, want_sk=1),
     dict(cov=True, sk=True), 600),
    (W.oracle_rod(n=(40, 1, 1), wall_lo=1.0, wall_hi=1.5, realizations=12, relax_steps=20, tc_lags=5,
                  want_cov=1, want_sk=0), dict(cov=True, time_corr=True), 400),
    (W.species_2d(n=(32, 24, 1), realizations=6, relax_steps=10, want_sk=3), dict(sk=True, sk_axes=True), 60),
    (W.cube_3d(n=(128, 8, 6), realizations=2, relax_steps=0), dict(sk_axes=True), 20),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_raw_then_finalize_equals_stats(case):
    p, kw, steps = CASES[case]
    with S.Simulation(p) as sim:
        sim.step(steps)
        g = sim.stats(**kw)
        raw = sim.stats_raw()
    f = S.she_finalize(sim.params, raw, **kw)
    assert f["n_samples"] == g["n_samples"]
    for k in g:
        if k != "n_samples":
            assert np.array_equal(np.asarray(f[k]), np.asarray(g[k]), equal_nan=True), k


def test_two_shards_sum_to_one_handle():
    p = W.oracle_rod(n=(48, 1, 1), wall_lo=1.0, wall_hi=2.0, realizations=64, relax_steps=30, tc_lags=3,
                     want_cov=1, want_sk=0)
    with S.Simulation(p) as sim:
        sim.step(300)
        one = sim.stats(cov=True, time_corr=True)
    raws = []
    for k in range(2):
        with S.Simulation(p, realizations=32, stream_offset=32 * k) as sim:
            sim.step(300)
            raws.append(sim.stats_raw())
    merged = {k: (raws[0][k] + raws[1][k]) if isinstance(raws[0][k], np.ndarray) else raws[0][k]
              for k in raws[0]}
    merged["n_samples"] = raws[0]["n_samples"] + raws[1]["n_samples"]
    f = S.she_finalize(S.params_from_problem(p), merged, cov=True, time_corr=True)
    assert f["n_samples"] == one["n_samples"]
    for k in ("mean", "var", "cov", "time_corr"):
        assert np.allclose(f[k], one[k], rtol=1e-11, atol=1e-16), k
