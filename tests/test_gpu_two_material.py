"""GPU parity of the rod of several materials (the iron / aluminium
exercise, Sec. 6) against the FP64 oracle, through the C ABI: per-cell
conductivity and heat capacity (she_params.lambda_cells / rho_cv_cells).

* FP64 trajectories element by element within 1e-12 relative: forward Euler
  and predictor-corrector, Dirichlet and periodic, ragged rows, several
  launch windows; moments, the FP64 covariance and the time correlation.
* FP32: one step from a shared state within 2e-5; the fused tensor-core
  covariance against the oracle's on the same seeds.
* A uniform rod given as arrays equals the uniform path.
* The equilibrium variance of each material is its own
  k_B T^2 / (rho c_V dV) with the forward-Euler correction: the exact
  stationary covariance of the recursion (close to the linearised
  (C + L/2)^{-1} k_B T^2 / dV), within batch SE.
* Refusals: a species rod, the plain form, a batch, one array without the
  other, non-positive entries, an unstable time step.
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


def _rod(N, bc="dirichlet", walls=(1.0, 2.0), precision="fp64", R=6, **kw):
    p = W.two_material_rod(cells=N, bc=bc, wall_lo=walls[0], wall_hi=walls[1], realizations=R,
                           precision=precision, want_cov=0, relax_steps=0, stats_interval=5, kB=2e-3)
    p.update(kw)
    return p


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.abs(b))


@pytest.mark.parametrize("N,bc,scheme", [(16, "dirichlet", "fe"), (37, "dirichlet", "fe"), (130, "periodic", "fe"),
                                         (256, "dirichlet", "fe"), (1000, "dirichlet", "fe"),
                                         (33, "dirichlet", "pc"), (130, "periodic", "pc"), (256, "dirichlet", "pc")])
def test_fp64_trajectory_matches_oracle(N, bc, scheme):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.4, 1.4)
    p = _rod(N, bc, walls, scheme=scheme)
    with S.Simulation(p, steps_per_launch=37) as sim:
        x0, _ = sim.state()
        sim.step(150)
        x1, _ = sim.state()
        g = sim.stats(raw=True)
    ref0 = np.array([O.initial_state(p, r) for r in range(p["realizations"])])
    assert rel_err(x0, ref0) < 1e-14
    o = O.run(p, p["realizations"], 150)
    assert rel_err(x1, o["state"]) < 1e-12
    assert g["n_samples"] == o["n_samples"]
    assert np.allclose(g["sum_d"], o["sum_d"], rtol=1e-9, atol=1e-13)
    assert np.allclose(g["sum_d2"], o["sum_d2"], rtol=1e-9, atol=1e-15)
    of = O.finalize(p, o)
    assert rel_err(g["mean"], of["mean"]) < 1e-12


def test_fp64_covariance_and_time_correlation():
    p = _rod(64, want_cov=1, tc_lags=4)
    with S.Simulation(p, steps_per_launch=23) as sim:
        sim.step(200)
        g = sim.stats(cov=True, time_corr=True)
    o = O.finalize(p, O.run(p, p["realizations"], 200, want_cov=1))
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 1e-10 * scale
    assert np.allclose(g["time_corr"], o["time_corr"], rtol=1e-9, atol=1e-15)


def test_uniform_arrays_equal_the_uniform_path():
    p = W.oracle_rod(n=(64, 1, 1), wall_lo=1.0, wall_hi=2.0, realizations=4, relax_steps=0, want_cov=0,
                     want_sk=0, kappa=0.8, rho_cv=1.25, dt=0.2)
    q = dict(p, lambda_cells=np.full(64, 0.8 * 1.25), rho_cv_cells=np.full(64, 1.25))
    with S.Simulation(p) as a, S.Simulation(q) as b:
        a.step(300)
        b.step(300)
        xa, _ = a.state()
        xb, _ = b.state()
    assert rel_err(xb, xa) < 1e-13


@pytest.mark.parametrize("N,bc", [(256, "dirichlet"), (100, "periodic"), (1024, "dirichlet")])
def test_fp32_one_step_from_shared_state(N, bc):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.4, 1.4)
    p = _rod(N, bc, walls, precision="fp32", R=16)
    x = W.random_states(p, 16, seed=N).astype(np.float32)
    with S.Simulation(p) as sim:
        sim.set_state(x, 777)
        sim.step(1)
        got, _ = sim.state()
    ref = np.array([O.step(p, x[r].astype(np.float64), 777, r) for r in range(16)])
    assert rel_err(got.astype(np.float64), ref) < 2e-5


def test_fp32_covariance_kernel_matches_oracle():
    p = _rod(256, precision="fp32", R=300, want_cov=1, stats_interval=10)
    with S.Simulation(p) as sim:
        sim.step(150)
        g = sim.stats(cov=True)
    o = O.finalize(p, O.run(p, 300, 150, want_cov=1))
    assert g["n_samples"] == o["n"]
    scale = np.max(np.diag(o["cov"]))
    # FP32 trajectories against FP64 ones (the same bar as the uniform rod's)
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * scale
    assert np.max(np.abs(np.diag(g["cov"]) - g["var"])) < 2e-4 * scale


def test_equilibrium_variance_per_material():
    # walls equal: each material's variance is its own k_B T^2 / (rho c_V dV)
    # with the forward-Euler correction, the exact (C + L/2)^{-1} k_B T^2 / dV
    N, B, per = 16, 16, 2048
    p = _rod(N, walls=(1.3, 1.3), precision="fp64", R=B * per, stats_interval=10, relax_steps=2000, kB=1e-3)
    vs = []
    for b in range(B):
        with S.Simulation(p, realizations=per, stream_offset=b * per) as sim:
            sim.step(12000)
            vs.append(sim.stats()["var"])
    vs = np.array(vs)
    cond, cap, kb_dv = O.material_arrays(p)
    # the exact stationary covariance of the recursion (with the O(eps)
    # multiplicative term the linearised closed form leaves out)
    _, S_ex = T.stationary(dict(dim=1, n=p["n"], bc="dirichlet", cond=cond, cap=cap, kB_dV=kb_dv,
                                wall_lo=1.3, wall_hi=1.3, equation="heat"), iters=100)
    assert np.allclose(S_ex, T.variable_equilibrium_cov(cond, cap, kb_dv, "dirichlet", 1.3), rtol=5e-3,
                       atol=5e-3 * np.max(S_ex))
    t = (vs.mean(0) - np.diag(S_ex)) / (vs.std(0, ddof=1) / np.sqrt(B))
    print("per-material variance: mean t^2 %.2f, iron %.4e aluminium %.4e (ratio %.3f, rho c_V ratio %.3f)"
          % (np.mean(t * t), vs.mean(0)[4], vs.mean(0)[12], vs.mean(0)[12] / vs.mean(0)[4], cap[0] / cap[-1]))
    assert np.mean(t * t) < 4.0 and np.max(np.abs(t)) < 6.0
    # the materials differ by their heat capacities (about 1/0.684 here)
    assert abs(vs.mean(0)[12] / vs.mean(0)[4] - S_ex[12, 12] / S_ex[4, 4]) < 0.05


@pytest.mark.parametrize("kw,status", [
    (dict(equation="species"), "SHE_ERR_UNSUPPORTED"),
    (dict(kernel="plain"), "SHE_ERR_UNSUPPORTED"),
    (dict(dt=0.5), "SHE_ERR_UNSTABLE"),
])
def test_material_rod_refusals(kw, status):
    p = _rod(32, **kw)
    with pytest.raises(S.SheError) as e:
        S.Simulation(p)
    assert e.value.status == getattr(S._abi, status)


def test_material_arrays_validated():
    p = _rod(32)
    bad = dict(p, lambda_cells=np.r_[np.full(31, 1.0), -1.0])
    with pytest.raises(S.SheError) as e:
        S.Simulation(bad)
    assert e.value.status == S._abi.SHE_ERR_INVALID_ARG
    params = S.params_from_problem(p)
    params.rho_cv_cells = None                   # one array without the other
    import ctypes
    h = ctypes.c_void_p()
    assert S.lib().she_init(ctypes.byref(params), ctypes.byref(h)) == S._abi.SHE_ERR_INVALID_ARG
    with pytest.raises(S.SheError):
        S.BatchSimulation([dict(_rod(32, precision="fp32", R=1))])
