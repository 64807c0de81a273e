"""Brute-force statistical check of the CUDA path on tiny grids against the
exact moment recursion, independently of the oracle's sample paths.

The face noise is independent of the state at the start of each step, so the
first two moments of the discrete scheme follow a closed recursion
(oracle/theory.py; heat noise ~ T_face, Eq. (2.12); species ~ sqrt(c_face),
Eq. (4.7)).  About 10^6 GPU realizations, split into independent batches by
the Philox key (Sec. 3), are pooled over the sampling schedule exactly as the
library accumulates them; each entry of the pooled mean and second moment
must lie within a few batch standard errors of the recursion's expectation,
and the z-scores together must look like unit-variance noise.  A dropped
sqrt(2) at a wall, a wrong noise amplitude, a noise on the wrong face or a
wrong wall stencil in the kernels each moves some entry by many standard
errors at this sample size.
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

BATCHES = 32
PER_BATCH = 32768          # 32 x 32768 = 1,048,576 realizations


def _theory_dict(p):
    r, eps = O.dimensionless(p)
    return {"dim": p["dim"], "n": p["n"], "bc": p["bc"], "r": r, "eps": eps,
            "wall_lo": p["wall_lo"], "wall_hi": p["wall_hi"],
            "equation": p["equation"], "perturb_ic": p["perturb_ic"]}


def _gpu_batches(p, nsteps, tref, cov):
    """Per-batch pooled mean delta and second moment (full matrix when the
    covariance is accumulated, else its diagonal)."""
    m1, m2 = [], []
    for b in range(BATCHES):
        q = dict(p, realizations=PER_BATCH, seed=7919 + 104729 * b, want_cov=int(cov))
        with S.Simulation(q) as sim:
            sim.step(nsteps)
            g = sim.stats(cov=cov)
        mu = g["mean"] - tref
        m1.append(mu)
        m2.append(g["cov"] + np.outer(mu, mu) if cov else g["var"] + mu * mu)
    return np.array(m1), np.array(m2), g["n_samples"]


def _z(batches, expect):
    se = batches.std(axis=0, ddof=1) / np.sqrt(len(batches))
    return (batches.mean(axis=0) - expect) / np.maximum(se, 1e-300)


def _check(p, nsteps, cov, zmax=4.5):
    ex = theory.pooled_expectation(_theory_dict(p), nsteps, p["stats_interval"], p["relax_steps"])
    m1, m2, count = _gpu_batches(p, nsteps, ex["tref"], cov)
    assert count == ex["count"] * PER_BATCH          # samples pooled over realizations
    second = ex["second"] if cov else np.diag(ex["second"])
    z2 = _z(m2, second)
    if cov:
        z2 = z2[np.triu_indices(len(second))]      # the distinct entries
    z = np.concatenate([_z(m1, ex["mean_delta"]), z2])
    assert np.max(np.abs(z)) < zmax, z
    # a bias below the per-entry tolerance but common to many entries shows
    # up as an excess of the mean squared z-score over 1
    assert np.mean(z * z) < 2.5, z
    return ex, m2.mean(axis=0)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("walls", [(1.0, 1.0), (1.0, 3.0)])
def test_heat_dirichlet_4cells_million_realizations(walls, precision):
    p = W.oracle_rod(n=(4, 1, 1), wall_lo=walls[0], wall_hi=walls[1], kB=0.02,
                     stats_interval=1, relax_steps=30, precision=precision)
    ex, got = _check(p, 60, cov=True)
    # the wall cells carry the sqrt(2) wall noise: without it their variance
    # would fall well below the recursion's
    assert got[0, 0] > 0.5 * ex["second"][0, 0]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_heat_periodic_5cells_million_realizations(precision):
    p = W.oracle_rod(n=(5, 1, 1), bc="periodic", wall_lo=2.0, wall_hi=2.0, kB=0.01,
                     stats_interval=2, relax_steps=20, precision=precision)
    _check(p, 60, cov=True)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_species_dirichlet_4cells_million_realizations(precision):
    p = W.oracle_rod(n=(4, 1, 1), equation="species", n0=50.0, D=1.0, dt=0.2,
                     wall_lo=1.0, wall_hi=2.0, stats_interval=1, relax_steps=30,
                     precision=precision)
    _check(p, 60, cov=True)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_species_periodic_2d_million_realizations(precision):
    p = W.species_2d(n=(4, 3, 1), n0=100.0, stats_interval=1, relax_steps=20,
                     precision=precision, want_sk=0)
    _check(p, 40, cov=False)
