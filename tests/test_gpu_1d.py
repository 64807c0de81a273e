"""GPU parity of the 1D step kernels against the FP64 oracle, through the C ABI.

* Noise generator: raw Philox words bit-exact, FP64 normals to 1e-13, FP32
  normals within the stated single-precision error.
* FP64 trajectories (fused kernel and plain form) at the same seed match the
  oracle to a relative 1e-12, over several tiles of cells per lane and
  ragged tails, Dirichlet and periodic, heat and species.
* FP32: one step from a shared state matches the oracle to 2e-5 relative;
  multi-step trajectories stay within 2e-4.
* Statistics (mean, var) at the same seeds match the oracle's.
* At the full 256-cell x 4096-realization size in the benchmark's launch
  configuration, sampled realizations match the oracle.
* Checkpoint/resume is bit-exact; invalid parameters return status codes.
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2406_12157_gb300 import build
    build.build()


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


# ------------------------------------------------------------------ noise --

def test_noise_bits_and_normals_match_oracle():
    count = 4096
    for (seed, c1, c2, c3) in [(0, 0, 0, 0), (123456789012345, 77, 4095, 0), (2**64 - 1, 2**32 - 1, 5, 2)]:
        bits, z64, z32 = S.she_noise_probe(seed, 1000, c1, c2, c3, count)
        for k in range(0, count, 97):
            ref = O.philox([1000 + k, c1, c2, c3], [seed & 0xFFFFFFFF, seed >> 32])
            assert list(bits[k]) == ref
            zr = O.normals4(seed, 1000 + k, c1, c2, c3)
            assert np.max(np.abs(z64[k] - zr)) < 1e-13
        zr_all = np.array([O.normals4(seed, 1000 + k, c1, c2, c3) for k in range(count)])
        d = np.abs(z32.astype(np.float64) - zr_all)
        assert d.max() < 5e-4
        assert np.quantile(d, 0.999) < 2e-5


def test_device_philox_known_answers():
    # the published Philox-4x32-10 known answers (Salmon et al., SC'11)
    kats = [((0, 0, 0, 0), (0, 0), [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
            ((0xffffffff,) * 4, (0xffffffff, 0xffffffff), [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
            ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
             [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1])]
    for ctr, key, out in kats:
        bits, _, _ = S.she_noise_probe(key[0] | (key[1] << 32), *ctr, 1)
        assert [int(x) for x in bits[0]] == out


# ------------------------------------------------------------ trajectories --

CASES = [
    # (N, bc, equation, walls)
    (2, "dirichlet", "heat", (1.0, 1.0)),
    (3, "periodic", "heat", (1.5, 1.5)),
    (5, "dirichlet", "species", (1.0, 2.0)),
    (32, "dirichlet", "heat", (1.0, 1.0)),
    (33, "periodic", "species", (1.0, 1.0)),
    (130, "dirichlet", "heat", (1.0, 3.0)),
    (256, "dirichlet", "heat", (1.0, 2.0)),
    (257, "periodic", "heat", (2.0, 2.0)),
    (600, "dirichlet", "species", (2.0, 1.0)),
    (1000, "periodic", "heat", (1.0, 1.0)),
]


def _prob(N, bc, eq, walls, **kw):
    kw.setdefault("realizations", 5)
    p = W.oracle_rod(n=(N, 1, 1), bc=bc, equation=eq, wall_lo=walls[0], wall_hi=walls[1],
                     n0=200.0, kB=5e-3, want_cov=0, want_sk=0, **kw)
    return p


@pytest.mark.parametrize("N,bc,eq,walls", CASES)
@pytest.mark.parametrize("kernel", ["auto", "plain"])
def test_fp64_trajectory_parity(N, bc, eq, walls, kernel):
    p = _prob(N, bc, eq, walls, precision="fp64", stats_interval=7, relax_steps=50,
              steps_per_launch=64)
    nsteps = 300
    with S.Simulation(p, kernel=kernel) as sim:
        st0, step0 = sim.state()
        ref0 = O.run(p, 5, 0)["state"]
        assert step0 == 0
        assert rel_err(st0, ref0) < 1e-13           # initial condition
        sim.step(nsteps)
        st, step = sim.state()
        assert step == nsteps
        ref = O.run(p, 5, nsteps)
        assert rel_err(st, ref["state"]) < 1e-12
        stats = sim.stats(raw=True)
        assert stats["n_samples"] == ref["n_samples"]
        assert np.allclose(stats["sum_d"], ref["sum_d"], rtol=1e-9, atol=1e-12)
        assert np.allclose(stats["sum_d2"], ref["sum_d2"], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("N,bc,eq,walls", CASES)
def test_fp32_one_step_parity(N, bc, eq, walls):
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


@pytest.mark.parametrize("N,bc,eq,walls", CASES[3:8])
def test_fp32_trajectory_stays_close(N, bc, eq, walls):
    p = _prob(N, bc, eq, walls, precision="fp32")
    with S.Simulation(p) as sim:
        sim.step(2000)
        got, _ = sim.state()
    ref = O.run(p, 5, 2000)["state"]
    assert rel_err(got.astype(np.float64), ref) < 2e-4


def test_fp32_statistics_match_oracle():
    p = W.oracle_rod(precision="fp32", realizations=16, want_cov=0, want_sk=0)
    with S.Simulation(p) as sim:
        sim.step(p["steps"])
        g = sim.stats()
    o = O.finalize(p, O.run(p, 16, p["steps"]))
    assert g["n_samples"] == o["n"]
    assert np.max(np.abs(g["mean"] - o["mean"])) < 1e-5
    assert rel_err(g["var"], o["var"]) < 2e-3
    assert np.all(np.isfinite(g["var_se"])) and np.all(g["var_se"] > 0)


def test_fp64_statistics_match_oracle_32_cells():
    p = W.oracle_rod(want_cov=0, want_sk=0)   # 32 cells, 16 realizations, FP64
    with S.Simulation(p) as sim:
        sim.step(p["steps"])
        g = sim.stats()
    o = O.finalize(p, O.run(p, 16, p["steps"]))
    assert g["n_samples"] == o["n"]
    assert rel_err(g["mean"], o["mean"]) < 1e-12
    assert rel_err(g["var"], o["var"]) < 1e-8


def test_full_size_sampled_realizations():
    # 256 cells x 4096 realizations, FP32, default launch shape
    p = W.gradient_rod(want_cov=0)
    steps = 1000
    with S.Simulation(p) as sim:
        sim.step(steps)
        got, _ = sim.state()
    for rho in (0, 1, 1234, 4095):
        ref = O.run(p, 1, steps, stream0=rho)["state"][0]
        assert rel_err(got[rho].astype(np.float64), ref) < 2e-4


def test_checkpoint_resume_bit_exact():
    p = _prob(256, "dirichlet", "heat", (1.0, 2.0), precision="fp32")
    with S.Simulation(p) as a, S.Simulation(p) as b:
        a.step(777)
        mid, step = a.state()
        a.step(500)
        b.set_state(mid, step)
        b.step(500)
        assert np.array_equal(a.state()[0], b.state()[0])


def test_deterministic_limit_on_gpu():
    # alpha = 0: exact sine-mode solution (Sec. 3, deterministic option)
    from oracle import theory
    p = _prob(64, "dirichlet", "heat", (1.0, 2.0), precision="fp64", stochastic=0, perturb_ic=0)
    x = W.random_states(p, 5, seed=3)
    with S.Simulation(p) as sim:
        sim.set_state(x, 0)
        sim.step(400)
        got, _ = sim.state()
    r, _ = O.dimensionless(p)
    for rho in range(5):
        ex = theory.sine_mode_solution(64, r, 1.0, 2.0, x[rho], 400)
        assert np.max(np.abs(got[rho] - ex)) < 1e-12


@pytest.mark.parametrize("bad,status", [
    (dict(dt=0.6), S._abi.SHE_ERR_UNSTABLE),
    (dict(n=(1, 1, 1)), S._abi.SHE_ERR_INVALID_ARG),
    (dict(bc="periodic", wall_lo=1.0, wall_hi=2.0), S._abi.SHE_ERR_INVALID_ARG),
    (dict(realizations=0), S._abi.SHE_ERR_INVALID_ARG),
    (dict(stats_interval=0), S._abi.SHE_ERR_INVALID_ARG),
    (dict(dx=-1.0), S._abi.SHE_ERR_INVALID_ARG),
])
def test_invalid_parameters_return_status(bad, status):
    p = W.oracle_rod(want_cov=0, want_sk=0)
    p.update(bad)
    with pytest.raises(S.SheError) as e:
        S.Simulation(p)
    assert e.value.status == status


def test_stats_before_any_sample_is_a_state_error():
    p = W.oracle_rod(want_cov=0, want_sk=0, relax_steps=10**6)
    with S.Simulation(p) as sim:
        sim.step(10)
        with pytest.raises(S.SheError) as e:
            sim.stats()
        assert e.value.status == S._abi.SHE_ERR_STATE


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_zero_steps_is_a_no_op(dim):
    if dim == 1:
        p = _prob(40, "dirichlet", "heat", (1.0, 2.0), precision="fp32")
    elif dim == 2:
        p = W.species_2d(n=(16, 8, 1), realizations=2, relax_steps=0, want_sk=0)
    else:
        p = W.cube_3d(n=(128, 8, 4), realizations=2, want_sk=0)
    with S.Simulation(p) as sim:
        x0, s0 = sim.state()
        n0 = sim.launches()
        sim.step(0)
        x1, s1 = sim.state()
        assert s1 == s0 == 0 and sim.launches() == n0
        assert np.array_equal(x0, x1)


def test_profile_times_step_kernels():
    p = _prob(256, "dirichlet", "heat", (1.0, 2.0), precision="fp32", realizations=64, relax_steps=0)
    with S.Simulation(p, steps_per_launch=500) as sim:
        sim.profile(True)
        sim.step(2000)
        pr = sim.profile_read()
        assert pr["step_launches"] == 4 and pr["step_ms"] > 0.0
        assert pr["stats_launches"] == 0
        assert sim.profile_read()["step_launches"] == 0      # read clears
        sim.profile(False)
        sim.step(500)
        assert sim.profile_read()["step_launches"] == 0
    p2 = W.species_2d(n=(64, 32, 1), realizations=2, relax_steps=0, stats_interval=5, want_sk=1)
    with S.Simulation(p2) as sim:
        sim.profile(True)
        sim.step(20)
        pr = sim.profile_read()
        assert pr["step_launches"] == 20 and pr["stats_launches"] == 4
        assert pr["step_ms"] > 0.0 and pr["stats_ms"] > 0.0


def test_nonfinite_state_is_reported():
    p = _prob(32, "dirichlet", "heat", (1.0, 1.0), precision="fp32")
    with S.Simulation(p) as sim:
        x, _ = sim.state()
        x[2, 5] = np.nan
        sim.set_state(x, 0)
        sim.step(20)
        with pytest.raises(S.SheError) as e:
            sim.stats()
        assert e.value.status == S._abi.SHE_ERR_NONFINITE


@pytest.mark.parametrize("layout,N", [("4,4", 13), ("4,8", 29), ("4,16", 64), ("4,32", 100),
                                      ("8,32", 256), ("8,32", 250), ("16,16", 256), ("16,16", 201),
                                      ("16,32", 512), ("32,8", 256), ("32,8", 255), ("32,32", 1024)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_every_layout_fp64_parity(layout, N, bc, monkeypatch):
    # each (cells per lane, lanes per realization) layout of the fused kernel,
    # full and ragged rows, against the oracle; R = 7 leaves idle segments
    monkeypatch.setenv("SHE_TUNE_1D", layout)
    walls = (1.0, 2.0) if bc == "dirichlet" else (1.0, 1.0)
    p = _prob(N, bc, "heat", walls, precision="fp64", realizations=7, stats_interval=3,
              relax_steps=5)
    with S.Simulation(p) as sim:
        sim.step(120)
        st, _ = sim.state()
        g = sim.stats(raw=True)
    ref = O.run(p, 7, 120)
    assert rel_err(st, ref["state"]) < 1e-12
    assert np.allclose(g["sum_d2"], ref["sum_d2"], rtol=1e-9, atol=1e-15)
