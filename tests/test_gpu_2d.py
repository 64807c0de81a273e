"""GPU parity of the 2D step kernel (periodic, heat and species) against the
FP64 oracle, through the C ABI: FP64 trajectories to 1e-12, FP32 one step to
2e-5, statistics, full 256 x 256 size on sampled realizations, conservation."""
import numpy as np
import pytest

import she_workloads as W
from oracle import she as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2406_12157_gb300 as S  # noqa: E402


def rel_err(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


GRIDS = [(8, 6), (12, 5), (16, 16), (20, 33), (64, 48), (132, 7), (256, 20), (264, 9)]


def _p(nx, ny, eq, **kw):
    kw.setdefault("realizations", 3)
    kw.setdefault("stats_interval", 3)
    kw.setdefault("relax_steps", 10)
    kw.setdefault("want_sk", 0)
    return W.species_2d(n=(nx, ny, 1), equation=eq, n0=200.0, kB=3e-3, wall_lo=1.3, wall_hi=1.3, **kw)


@pytest.mark.parametrize("nx,ny", GRIDS)
@pytest.mark.parametrize("eq", ["species", "heat"])
def test_fp64_trajectory_parity_2d(nx, ny, eq):
    p = _p(nx, ny, eq, precision="fp64")
    with S.Simulation(p) as sim:
        sim.step(40)
        st, _ = sim.state()
        g = sim.stats(raw=True)
    ref = O.run(p, 3, 40)
    assert rel_err(st, ref["state"]) < 1e-12
    assert g["n_samples"] == ref["n_samples"]
    assert np.allclose(g["sum_d2"], ref["sum_d2"], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("nx,ny", GRIDS)
def test_fp32_one_step_parity_2d(nx, ny):
    p = _p(nx, ny, "species", precision="fp32")
    x = W.random_states(p, 3, seed=nx * 7 + ny).astype(np.float32)
    with S.Simulation(p) as sim:
        for step in (0, 99, 123456):
            sim.set_state(x, step)
            sim.step(1)
            got, _ = sim.state()
            for rho in range(3):
                ref = O.step(p, x[rho].astype(np.float64), step, rho)
                assert rel_err(got[rho].astype(np.float64), ref) < 2e-5


def test_fp32_statistics_2d():
    p = _p(32, 24, "species", precision="fp32", realizations=8)
    with S.Simulation(p) as sim:
        sim.step(600)
        g = sim.stats(raw=True)
    ref = O.finalize(p, O.run(p, 8, 600))
    assert g["n_samples"] == ref["n"]
    assert rel_err(g["var"], ref["var"]) < 2e-3


def test_full_size_2d_sampled():
    p = W.species_2d(realizations=16, want_sk=0)
    with S.Simulation(p) as sim:
        sim.step(50)
        got, _ = sim.state()
    for rho in (0, 7, 15):
        ref = O.run(p, 1, 50, stream0=rho)["state"][0]
        assert rel_err(got[rho].astype(np.float64), ref) < 1e-4


def test_total_conserved_2d():
    p = _p(64, 64, "species", precision="fp64")
    with S.Simulation(p) as sim:
        x0, _ = sim.state()
        sim.step(100)
        x1, _ = sim.state()
    assert np.max(np.abs(x1.sum(axis=1) - x0.sum(axis=1))) < 1e-10 * x0.shape[1]


@pytest.mark.parametrize("nx,ny", [(16, 16), (132, 7), (256, 20), (64, 256)])
def test_per_axis_structure_factor_2d(nx, ny):
    p = _p(nx, ny, "species", precision="fp32", want_sk=2, stats_interval=2, relax_steps=0)
    with S.Simulation(p) as sim:
        sim.step(20)
        g = sim.stats(sk_axes=True)
    o = O.finalize(p, O.run(p, 3, 20, want_sk=2))
    assert g["n_samples"] == o["n"]
    ref = o["sk_axes"]
    assert np.max(np.abs(g["sk_axes"] - ref)) < 2e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("nx,ny,R", [(16, 12, 6), (64, 48, 4), (256, 16, 3), (132, 20, 3), (16, 256, 2), (32, 255, 2)])
def test_full_structure_factor_2d(nx, ny, R):
    # S(kx, ky) from the two-stage tcgen05 DFT vs the oracle's 2D DFT by its
    # definition (Eq. (3.11) along both axes) on the same trajectories
    p = _p(nx, ny, "species", precision="fp32", want_sk=1, stats_interval=3, relax_steps=0,
           realizations=R)
    with S.Simulation(p) as sim:
        sim.step(12)
        g = sim.stats(sk=True)
    o = O.finalize(p, O.run(p, R, 12, want_sk=1))
    assert g["n_samples"] == o["n"]
    scale = np.max(np.abs(o["sk_fluct"][1:]))
    assert np.max(np.abs(g["sk_fluct"] - o["sk_fluct"])) < 2e-4 * scale
    assert np.allclose(g["sk"][1:], o["sk"][1:], rtol=0, atol=2e-4 * scale)
    assert abs(g["sk"][0] - o["sk"][0]) < 1e-6 * abs(o["sk"][0])


@pytest.mark.parametrize("scheme", ["fe", "pc"])
@pytest.mark.parametrize("steps", [1, 7])
def test_nonfinite_state_is_reported_2d(scheme, steps):
    """A NaN in the state is reported (SHE_ERR_NONFINITE) after the step
    batch, whichever step of the batch checks it."""
    p = _p(32, 24, "species", precision="fp32", scheme=scheme, relax_steps=0, stats_interval=1)
    with S.Simulation(p) as sim:
        x, _ = sim.state()
        x[1, 100] = np.nan
        sim.set_state(x, 0)
        sim.step(steps)
        with pytest.raises(S.SheError) as e:
            sim.stats()
        assert e.value.status == S._abi.SHE_ERR_NONFINITE
