"""GPU parity of the predictor-corrector scheme (Sec. 3) against the FP64
oracle, through the C ABI.

* FP64 trajectories at the same seed match the oracle to a relative 1e-12:
  every PC layout (4, 8 and 16 cells per lane), ragged tails, Dirichlet and
  periodic, heat and species, launch windows that split the run.
* FP32: one step from a shared state within 2e-5 relative.
* The fused tensor-core covariance under PC (its 16 x 16 layout at 256
  cells, the 4-cell layouts below 128) matches the oracle's covariance; the
  FP64 covariance matches it to rounding.
* About 10^6 realizations of 4-cell rods match the exact PC moment
  recursion (Gauss-Hermite quadrature over the face normals) within a few
  standard errors, independently of the oracle's sample paths.
* 2D (one pass: the predictor state carried one row ahead of the corrector,
  each normal drawn once) and 3D (a predictor pass and a corrector pass that
  draws the same normals again): FP64 trajectories to 1e-12 over several
  bands, tiles, ragged rows, a 2-row grid and row runs that cross
  realizations; FP32 one step within 2e-5, also at the full 256^2 x 256
  benchmark shape on sampled realizations; the full 2D S(k) on the
  corrector's output.
* Combinations outside the PC kernels are refused with SHE_ERR_UNSUPPORTED.
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O
from oracle import theory

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


CASES = [
    # (N, bc, equation, walls): layouts 4x4, 4x8, 4x32, 8x32 and 16x32, ragged or not
    (2, "dirichlet", "heat", (1.0, 1.0)),
    (5, "dirichlet", "species", (1.0, 2.0)),
    (16, "periodic", "heat", (1.5, 1.5)),
    (33, "periodic", "species", (1.0, 1.0)),
    (130, "dirichlet", "heat", (1.0, 3.0)),
    (256, "dirichlet", "heat", (1.0, 2.0)),
    (256, "periodic", "species", (1.2, 1.2)),
    (300, "dirichlet", "species", (2.0, 1.0)),
    (512, "periodic", "heat", (1.0, 1.0)),
]


def _prob(N, bc, eq, walls, **kw):
    kw.setdefault("realizations", 5)
    return W.oracle_rod(n=(N, 1, 1), bc=bc, equation=eq, wall_lo=walls[0], wall_hi=walls[1],
                        n0=200.0, kB=5e-3, want_cov=0, want_sk=0, scheme="pc", **kw)


@pytest.mark.parametrize("N,bc,eq,walls", CASES)
def test_pc_fp64_trajectory_parity(N, bc, eq, walls):
    p = _prob(N, bc, eq, walls, precision="fp64", stats_interval=7, relax_steps=50, steps_per_launch=64)
    nsteps = 300
    with S.Simulation(p) as sim:
        sim.step(nsteps)
        st, step = sim.state()
        stats = sim.stats(raw=True)
    assert step == nsteps
    ref = O.run(p, 5, nsteps)
    assert rel_err(st, ref["state"]) < 1e-12
    assert stats["n_samples"] == ref["n_samples"]
    assert np.allclose(stats["sum_d"], ref["sum_d"], rtol=1e-9, atol=1e-12)
    assert np.allclose(stats["sum_d2"], ref["sum_d2"], rtol=1e-9, atol=1e-15)
    # a forward-Euler run of the same seed is elsewhere
    fe = O.run(dict(p, scheme="fe"), 5, nsteps)["state"]
    assert rel_err(st, fe) > 1e-6


@pytest.mark.parametrize("N,bc,eq,walls", CASES)
def test_pc_fp32_one_step_parity(N, bc, eq, walls):
    p = _prob(N, bc, eq, walls, precision="fp32")
    R = 5
    x = W.random_states(p, R, seed=N).astype(np.float32)
    with S.Simulation(p) as sim:
        for step in (0, 1, 12345, 2**31 + 7):
            sim.set_state(x, step)
            sim.step(1)
            got, _ = sim.state()
            for rho in range(R):
                ref = O.step(p, x[rho].astype(np.float64), step, rho)
                assert rel_err(got[rho].astype(np.float64), ref) < 2e-5


@pytest.mark.parametrize("N,R,steps,bc", [(16, 40, 200, "dirichlet"), (100, 300, 200, "dirichlet"),
                                          (200, 300, 120, "dirichlet"), (256, 200, 150, "dirichlet"),
                                          (256, 100, 150, "periodic"), (64, 2000, 60, "dirichlet")])
def test_pc_fused_covariance_matches_oracle(N, R, steps, bc):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.0, 1.0)
    p = W.gradient_rod(n=(N, 1, 1), realizations=R, relax_steps=0, stats_interval=10, wall_lo=walls[0],
                       wall_hi=walls[1], bc=bc, want_cov=1, want_sk=1, scheme="pc")
    with S.Simulation(p) as sim:
        sim.step(steps)
        g = sim.stats(cov=True, sk=True)
    o = O.finalize(p, O.run(p, R, steps, want_cov=1, want_sk=1))
    assert g["n_samples"] == o["n"]
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 2e-4 * scale
    assert np.max(np.abs(np.diag(g["cov"]) - g["var"])) < 2e-4 * scale
    assert np.max(np.abs(g["sk_fluct"] - o["sk_fluct"])) < 2e-4 * np.max(o["sk_fluct"])


@pytest.mark.parametrize("N,R,steps,bc", [(16, 40, 203, "dirichlet"), (256, 33, 90, "periodic")])
def test_pc_fp64_covariance_matches_oracle_exactly(N, R, steps, bc):
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.5, 1.5)
    p = W.gradient_rod(n=(N, 1, 1), realizations=R, relax_steps=23, stats_interval=7, wall_lo=walls[0],
                       wall_hi=walls[1], bc=bc, want_cov=1, want_sk=1, precision="fp64", scheme="pc")
    with S.Simulation(p, steps_per_launch=37) as sim:
        sim.step(steps)
        g = sim.stats(cov=True, sk=True)
    o = O.finalize(p, O.run(p, R, steps, want_cov=1, want_sk=1))
    scale = np.max(np.diag(o["cov"]))
    assert np.max(np.abs(g["cov"] - o["cov"])) < 1e-10 * scale
    assert np.max(np.abs(g["sk_fluct"] - o["sk_fluct"])) < 1e-10 * np.max(o["sk_fluct"])


def _td(p):
    r, eps = O.dimensionless(p)
    return {"dim": p["dim"], "n": p["n"], "bc": p["bc"], "r": r, "eps": eps,
            "wall_lo": p["wall_lo"], "wall_hi": p["wall_hi"],
            "equation": p["equation"], "perturb_ic": p["perturb_ic"], "scheme": "pc"}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("bc,walls", [("dirichlet", (1.0, 3.0)), ("periodic", (2.0, 2.0))])
def test_pc_million_realizations_match_exact_recursion(precision, bc, walls):
    n = 4 if bc == "dirichlet" else 5
    p = W.oracle_rod(n=(n, 1, 1), bc=bc, wall_lo=walls[0], wall_hi=walls[1], kB=0.02, stats_interval=1,
                     relax_steps=30, precision=precision, scheme="pc")
    nsteps, B, Rb = 60, 32, 32768
    ex = theory.pooled_expectation_quadrature(_td(p), nsteps, 1, 30)
    m1, m2 = [], []
    for b in range(B):
        q = dict(p, realizations=Rb, seed=7919 + 104729 * b, want_cov=1)
        with S.Simulation(q) as sim:
            sim.step(nsteps)
            g = sim.stats(cov=True)
        assert g["n_samples"] == ex["count"] * Rb
        mu = g["mean"] - ex["tref"]
        m1.append(mu)
        m2.append(g["cov"] + np.outer(mu, mu))
    m1, m2 = np.array(m1), np.array(m2)
    z1 = (m1.mean(axis=0) - ex["mean_delta"]) / (m1.std(axis=0, ddof=1) / np.sqrt(B))
    z2 = ((m2.mean(axis=0) - ex["second"]) / (m2.std(axis=0, ddof=1) / np.sqrt(B)))[np.triu_indices(n)]
    z = np.concatenate([z1, z2])
    assert np.max(np.abs(z)) < 4.5, z
    assert np.mean(z * z) < 2.5, z


@pytest.mark.parametrize("kw", [dict(kernel="plain", precision="fp64"),
                                dict(n=(600, 1, 1))])
def test_pc_outside_its_kernels_is_refused(kw):
    p = W.oracle_rod(scheme="pc", want_cov=0, want_sk=0, **kw)
    with pytest.raises(S.SheError) as e:
        S.Simulation(p)
    assert e.value.status == S._abi.SHE_ERR_UNSUPPORTED


def _p2(nx, ny, eq, **kw):
    kw.setdefault("realizations", 3)
    kw.setdefault("stats_interval", 3)
    kw.setdefault("relax_steps", 10)
    kw.setdefault("want_sk", 0)
    return W.species_2d(n=(nx, ny, 1), equation=eq, n0=200.0, kB=3e-3, wall_lo=1.3, wall_hi=1.3,
                        scheme="pc", **kw)


def _p3(shape, eq, **kw):
    kw.setdefault("realizations", 2)
    kw.setdefault("stats_interval", 2)
    kw.setdefault("relax_steps", 3)
    kw.setdefault("want_sk", 0)
    return W.cube_3d(n=shape, equation=eq, n0=150.0, kB=4e-3, wall_lo=1.2, wall_hi=1.2, perturb_ic=1,
                     scheme="pc", **kw)


@pytest.mark.parametrize("nx,ny,R", [(8, 6, 3), (20, 33, 3), (64, 48, 3), (132, 7, 3), (256, 20, 3), (64, 2, 3),
                                      (256, 64, 20), (40, 3, 5)])
@pytest.mark.parametrize("eq", ["species", "heat"])
def test_pc_2d_fp64_trajectory_parity(nx, ny, R, eq):
    p = _p2(nx, ny, eq, precision="fp64", realizations=R)
    with S.Simulation(p) as sim:
        sim.step(25)
        st, _ = sim.state()
        g = sim.stats(raw=True)
    ref = O.run(p, R, 25)
    assert rel_err(st, ref["state"]) < 1e-12
    assert g["n_samples"] == ref["n_samples"]
    assert np.allclose(g["sum_d2"], ref["sum_d2"], rtol=1e-9, atol=1e-15)
    fe = O.run(dict(p, scheme="fe"), R, 25)["state"]
    assert rel_err(st, fe) > 1e-7


def test_pc_2d_fp32_one_step_full_size():
    """The benchmark shape (256 x 256 species, 256 realizations) in the
    launch configuration the bench times: one step from a shared state,
    sampled realizations against the oracle."""
    p = W.species_2d(scheme="pc", want_sk=0)
    R = p["realizations"]
    x = W.random_states(p, R, seed=5).astype(np.float32)
    with S.Simulation(p) as sim:
        sim.set_state(x, 777)
        sim.step(1)
        got, _ = sim.state()
    for rho in (0, 101, 255):
        ref = O.step(p, x[rho].astype(np.float64), 777, rho)
        assert rel_err(got[rho].astype(np.float64), ref) < 2e-5


@pytest.mark.parametrize("nx,ny", [(8, 6), (132, 7), (256, 20)])
def test_pc_2d_fp32_one_step_parity(nx, ny):
    p = _p2(nx, ny, "species", precision="fp32")
    x = W.random_states(p, 3, seed=nx * 7 + ny).astype(np.float32)
    with S.Simulation(p) as sim:
        for step in (0, 99, 123456):
            sim.set_state(x, step)
            sim.step(1)
            got, _ = sim.state()
            for rho in range(3):
                ref = O.step(p, x[rho].astype(np.float64), step, rho)
                assert rel_err(got[rho].astype(np.float64), ref) < 2e-5


def test_pc_2d_full_structure_factor():
    p = _p2(16, 12, "species", precision="fp32", want_sk=1, stats_interval=3, relax_steps=0, realizations=6)
    with S.Simulation(p) as sim:
        sim.step(12)
        g = sim.stats(sk=True)
    o = O.finalize(p, O.run(p, 6, 12, want_sk=1))
    assert g["n_samples"] == o["n"]
    scale = np.max(np.abs(o["sk_fluct"][1:]))
    assert np.max(np.abs(g["sk_fluct"] - o["sk_fluct"])) < 2e-4 * scale


@pytest.mark.parametrize("shape", [(128, 2, 2), (128, 9, 5), (128, 8, 40), (256, 16, 3)])
@pytest.mark.parametrize("eq", ["heat", "species"])
def test_pc_3d_fp64_trajectory_parity(shape, eq):
    p = _p3(shape, eq, precision="fp64")
    with S.Simulation(p) as sim:
        sim.step(6)
        st, _ = sim.state()
        g = sim.stats(raw=True)
    ref = O.run(p, 2, 6)
    assert rel_err(st, ref["state"]) < 1e-12
    assert g["n_samples"] == ref["n_samples"]
    assert np.allclose(g["sum_d2"], ref["sum_d2"], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("shape", [(128, 2, 2), (128, 9, 5)])
def test_pc_3d_fp32_one_step_parity(shape):
    p = _p3(shape, "heat", precision="fp32")
    x = W.random_states(p, 2, seed=sum(shape)).astype(np.float32)
    with S.Simulation(p) as sim:
        for step in (0, 77):
            sim.set_state(x, step)
            sim.step(1)
            got, _ = sim.state()
            for rho in range(2):
                ref = O.step(p, x[rho].astype(np.float64), step, rho)
                assert rel_err(got[rho].astype(np.float64), ref) < 2e-5
