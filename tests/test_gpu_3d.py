"""GPU parity of the 3D step kernel (periodic, heat and species) against the
FP64 oracle, through the C ABI: FP64 trajectories to 1e-12 over several
y-tiles and z-bands (incl. partial ones), FP32 one step to 2e-5, statistics,
one full 256^3 realization for two steps, conservation."""
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


GRIDS = [(128, 2, 2), (128, 9, 5), (256, 16, 3), (128, 8, 40), (512, 3, 2)]


def _p(shape, eq, **kw):
    kw.setdefault("realizations", 2)
    kw.setdefault("stats_interval", 2)
    kw.setdefault("relax_steps", 3)
    kw.setdefault("want_sk", 0)
    return W.cube_3d(n=shape, equation=eq, n0=150.0, kB=4e-3, wall_lo=1.2, wall_hi=1.2,
                     perturb_ic=1, **kw)


@pytest.mark.parametrize("shape", GRIDS)
@pytest.mark.parametrize("eq", ["heat", "species"])
def test_fp64_trajectory_parity_3d(shape, eq):
    p = _p(shape, eq, precision="fp64")
    with S.Simulation(p) as sim:
        sim.step(6)
        st, _ = sim.state()
        g = sim.stats(raw=True)
    ref = O.run(p, 2, 6)
    assert rel_err(st, ref["state"]) < 1e-12
    assert g["n_samples"] == ref["n_samples"]
    assert np.allclose(g["sum_d2"], ref["sum_d2"], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("shape", GRIDS[:3])
def test_fp32_one_step_parity_3d(shape):
    p = _p(shape, "heat", precision="fp32")
    x = W.random_states(p, 2, seed=sum(shape)).astype(np.float32)
    with S.Simulation(p) as sim:
        for step in (0, 4321):
            sim.set_state(x, step)
            sim.step(1)
            got, _ = sim.state()
            for rho in range(2):
                ref = O.step(p, x[rho].astype(np.float64), step, rho)
                assert rel_err(got[rho].astype(np.float64), ref) < 2e-5


def test_fp32_statistics_3d():
    p = _p((128, 6, 5), "heat", precision="fp32", realizations=4)
    with S.Simulation(p) as sim:
        sim.step(60)
        g = sim.stats()
    ref = O.finalize(p, O.run(p, 4, 60))
    assert g["n_samples"] == ref["n"]
    assert rel_err(g["var"], ref["var"]) < 2e-3


def test_full_size_3d_one_realization():
    p = W.cube_3d(realizations=8, want_sk=0, perturb_ic=1)
    with S.Simulation(p) as sim:
        sim.step(2)
        got, _ = sim.state()
    ref = O.run(p, 1, 2, stream0=5)["state"][0]
    assert rel_err(got[5].astype(np.float64), ref) < 2e-5


def test_total_conserved_3d():
    p = _p((128, 8, 8), "heat", precision="fp64")
    with S.Simulation(p) as sim:
        x0, _ = sim.state()
        sim.step(30)
        x1, _ = sim.state()
    assert np.max(np.abs(x1.sum(axis=1) - x0.sum(axis=1))) < 1e-10 * x0.shape[1]


@pytest.mark.parametrize("shape", [(128, 8, 40), (256, 16, 3), (128, 3, 130)])
def test_per_axis_structure_factor_3d(shape):
    # S(k) along x, y and z from the tensor-core line covariance vs the
    # oracle's direct line DFTs (Eq. (3.11)) on the same trajectories
    p = _p(shape, "heat", precision="fp32", want_sk=2, stats_interval=3, relax_steps=0)
    with S.Simulation(p) as sim:
        sim.step(9)
        g = sim.stats(sk_axes=True)
    o = O.finalize(p, O.run(p, 2, 9, want_sk=2))
    assert g["n_samples"] == o["n"]
    ref = o["sk_axes"]
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(g["sk_axes"] - ref)) < 2e-4 * scale


@pytest.mark.parametrize("steps", [1, 5])
def test_nonfinite_state_is_reported_3d(steps):
    """A NaN in the state is reported (SHE_ERR_NONFINITE) after the step batch."""
    p = _p((128, 8, 4), "heat", precision="fp32", relax_steps=0, stats_interval=1)
    with S.Simulation(p) as sim:
        x, _ = sim.state()
        x[0, 1000] = np.inf
        sim.set_state(x, 0)
        sim.step(steps)
        with pytest.raises(S.SheError) as e:
            sim.stats()
        assert e.value.status == S._abi.SHE_ERR_NONFINITE
