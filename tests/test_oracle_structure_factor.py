"""The oracle's structure factor against the forward-Euler closed form.

S_k = <|hat T_k|^2> with the unnormalised DFT of Eq. (3.11).  At equilibrium
the scheme's stationary value is eps T^2 N / (1 - r mu_k/2) (heat,
linearised) or eps c N / (1 - r mu_k/2) (species, exact), which tends to the
flat Eq. (3.12) as r -> 0.  Statistical agreement within a few standard errors
over realization batches.
"""
import numpy as np
import pytest

import she_workloads as W
from oracle import she, theory


def test_sk_1d_periodic_heat():
    N, B, R = 16, 12, 64
    p = W.oracle_rod(n=(N, 1, 1), bc="periodic", kB=1e-4, stats_interval=5,
                     relax_steps=400, want_sk=1)
    r, eps = she.dimensionless(p)
    vals = []
    for b in range(B):
        o = she.run(p, R, 3000, stream0=b * R)
        vals.append(she.finalize(p, o)["sk_fluct"])
    vals = np.array(vals)
    se = vals.std(axis=0, ddof=1) / np.sqrt(B)
    ex = theory.fe_structure_factor((N,), r, eps * 1.0)
    z = (vals.mean(axis=0)[1:] - ex[1:]) / se[1:]
    assert np.max(np.abs(z)) < 4.5, z
    # FE is visibly off the flat Eq. (3.12) at high k (Sec. 3, Fig. 5 remark)
    assert ex[N // 2] > 1.3 * eps * N


def test_sk_2d_periodic_species():
    shape = (6, 4)
    B, R = 12, 32
    p = W.species_2d(n=(6, 4, 1), n0=500.0, stats_interval=4, relax_steps=200,
                     want_sk=1)
    r, eps = she.dimensionless(p)
    vals = []
    for b in range(B):
        o = she.run(p, R, 1500, stream0=b * R)
        vals.append(she.finalize(p, o)["sk_fluct"])
    vals = np.array(vals)
    se = vals.std(axis=0, ddof=1) / np.sqrt(B)
    ex = theory.fe_structure_factor(shape, r, eps * 1.0)
    z = (vals.mean(axis=0)[1:] - ex[1:]) / se[1:]
    assert np.max(np.abs(z)) < 4.5, z


@pytest.mark.parametrize("scheme", ["fe", "pc"])
@pytest.mark.parametrize("dt", [0.05, 0.1])
def test_sk_error_order_sweep(scheme, dt):
    # the error-order exercise (Sec. 6): at r = 0.05 and 0.1 the measured
    # S_k follows eps N / (1 - x/2) (forward Euler, O(x)) or
    # eps N (2 - x) / (2 - x + x^2/2) (predictor-corrector, O(x^2)), x = r mu_k
    N, B, R = 16, 12, 64
    p = W.oracle_rod(n=(N, 1, 1), bc="periodic", kB=1e-4, dt=dt, stats_interval=5, relax_steps=800,
                     want_sk=1, scheme=scheme)
    r, eps = she.dimensionless(p)
    vals = []
    for b in range(B):
        o = she.run(p, R, 3000, stream0=b * R)
        vals.append(she.finalize(p, o)["sk_fluct"])
    vals = np.array(vals)
    se = vals.std(axis=0, ddof=1) / np.sqrt(B)
    ex = theory.structure_factor((N,), r, eps * 1.0, scheme=scheme)
    z = (vals.mean(axis=0)[1:] - ex[1:]) / se[1:]
    assert np.max(np.abs(z)) < 4.5, z
    # the size of the deviation from the flat value at the highest k
    x = r * 4.0
    dev = ex[N // 2] / (eps * N) - 1.0
    if scheme == "fe":
        assert abs(dev - (0.5 * x / (1.0 - 0.5 * x))) < 1e-12
    else:
        assert abs(dev + (0.5 * x * x / (2.0 - x + 0.5 * x * x))) < 1e-12
