"""Seeded synthetic workloads shared by the tests, the bench and the oracle side.

This module holds parameters and seeded random inputs only -- none of the
method's arithmetic.  Problems are plain dicts in the paper's physical terms
(Sec. 3): grid, spacing dx, cross-section (1D) or thickness (2D), kappa,
rho*c_V and k_B for heat, D and n0 for species, wall values, dt, seed,
realizations, sampling interval K and relaxation steps.  All workloads are in
nondimensional units with dx = 1 and a unit cell volume, so k_B (heat) or
1/n0 (species) *is* the relative equilibrium variance eps, and kappa*dt (or
D*dt) *is* the diffusion number r.

Workloads (shaped like the paper's runs, Sec. 3, Figs. 2-6, and the
configurations this library is measured on):

* ``oracle_rod``     1D, 32 cells, Dirichlet walls T = 1, eps = 1e-3,
                     r = 0.2, 1e4 steps, 16 realizations, FP64, seed 0.
* ``gradient_rod``   1D, 256 cells, walls 1 and 2 (linear mean profile),
                     4096 realizations, FP32, 1e6 steps, statistics every
                     10 steps after 1e5, full 256 x 256 covariance.
* ``species_2d``     2D 256 x 256 periodic species diffusion with
                     multiplicative noise, D = 1, r = 0.1, eps_c = 1e-3,
                     c = 1 plus a seeded zero-sum perturbation,
                     256 realizations, FP32, 1e5 steps, S(k).
* ``batched_rods``   10,000 1D Dirichlet instances, N log-uniform in
                     [16, 2048], kappa uniform in [0.5, 2], walls uniform
                     in [1, 3], r = 0.2 each, per-instance seed, FP32.
* ``cube_3d``        3D 256^3 periodic heat, T0 = 1, r = 0.1, eps = 1e-3,
                     no perturbation, 8 realizations, FP32, 1e4 steps,
                     per-axis S(k).
* ``iron_rod``       the paper's own physical rod: iron, l = 20 nm,
                     A = 4 nm^2, 32 cells, a = 0.1 (r = 0.05), 300 K
                     equilibrium or 100 K / 500 K walls.
* ``two_material_rod`` the iron / aluminium rod of the exercise (Sec. 6) in
                     the units of ``gradient_rod``: 256 cells, iron (rho c_V
                     1, conductivity 1) on the left half, aluminium (rho c_V
                     0.684, conductivity 3.386: the ratios of aluminium's
                     2700 kg/m^3 x 897 J/(kg K) and 237 W/(m K) to the
                     paper's iron) on the right, walls 1 and 2, dt 0.08
                     (r = 0.08 in iron, 0.396 in aluminium), k_B = 1e-3,
                     4096 realizations, FP32, covariance.
* ``iron_aluminium_rod`` the paper's physical rod (l = 20 nm, A = 4 nm^2,
                     32 cells, the iron time step a = 0.1) with its right half
                     aluminium.
"""
import numpy as np


def _base(**kw):
    p = {
        "dim": 1, "n": (32, 1, 1), "dx": 1.0, "area": 1.0,
        "equation": "heat", "kappa": 1.0, "rho_cv": 1.0, "kB": 1e-3,
        "D": 1.0, "n0": 1000.0,
        "bc": "dirichlet", "wall_lo": 1.0, "wall_hi": 1.0,
        "dt": 0.2, "seed": 0, "realizations": 16,
        "stochastic": 1, "perturb_ic": 1, "stats_interval": 10,
        "relax_steps": 0, "want_cov": 0, "want_sk": 0,
        "precision": "fp64", "steps": 10_000, "scheme": "fe",
    }
    p.update(kw)
    return p


def oracle_rod(**kw):
    """32-cell rod at equilibrium, walls T = 1, eps = 1e-3, r = 0.2;
    sampling after M/10 + K steps as the paper's program does (Sec. 3)."""
    p = _base(n=(32, 1, 1), wall_lo=1.0, wall_hi=1.0, dt=0.2, realizations=16,
              steps=10_000, relax_steps=1_010, precision="fp64", want_cov=1, want_sk=1)
    p.update(kw)
    return p


def gradient_rod(**kw):
    """256-cell rod, walls 1 and 2, 4096 realizations, FP32, 1e6 steps."""
    p = _base(n=(256, 1, 1), wall_lo=1.0, wall_hi=2.0, dt=0.2, realizations=4096,
              steps=1_000_000, relax_steps=100_000, precision="fp32", want_cov=1)
    p.update(kw)
    return p


def species_2d(**kw):
    """2D periodic species diffusion, 256 x 256, r = 0.1, eps_c = 1e-3."""
    p = _base(dim=2, n=(256, 256, 1), equation="species", D=1.0, n0=1000.0, dt=0.1,
              bc="periodic", wall_lo=1.0, wall_hi=1.0, realizations=256,
              steps=100_000, relax_steps=10_000, precision="fp32", want_sk=1)
    p.update(kw)
    return p


def cube_3d(**kw):
    """3D periodic heat, 256^3, r = 0.1, eps = 1e-3, uniform start."""
    p = _base(dim=3, n=(256, 256, 256), dt=0.1, bc="periodic", wall_lo=1.0, wall_hi=1.0,
              realizations=8, perturb_ic=0, steps=10_000, relax_steps=0,
              precision="fp32", want_sk=2)
    p.update(kw)
    return p


def iron_rod(noneq=False, **kw):
    """The paper's iron rod (Sec. 3): l = 20 nm, A = 4 nm^2, 32 cells,
    rho = 7870 kg/m^3, c_V = 450 J/(kg K), lambda = 70 W/(m K),
    dt = 0.1 dx^2/(2 kappa)."""
    n = 32
    length = 2.0e-8
    dx = length / n
    rho, c_v, lam = 7870.0, 450.0, 70.0
    kappa = lam / (rho * c_v)
    walls = (100.0, 500.0) if noneq else (300.0, 300.0)
    p = _base(n=(n, 1, 1), dx=dx, area=(2.0e-9) ** 2, kappa=kappa, rho_cv=rho * c_v,
              kB=1.38e-23, wall_lo=walls[0], wall_hi=walls[1],
              dt=0.1 * dx * dx / (2.0 * kappa), realizations=16)
    p.update(kw)
    return p


def batched_rods(count=10_000, seed=0, r=0.2):
    """Uneven batch: N ~ log-uniform[16, 2048], kappa ~ U[0.5, 2], walls
    ~ U[1, 3] each, dt chosen so that every instance has diffusion number r,
    per-instance seed = seed + id.  Returns a list of problem dicts."""
    rng = np.random.default_rng(12345 + seed)
    logn = rng.uniform(np.log(16.0), np.log(2048.0), size=count)
    ns = np.clip(np.round(np.exp(logn)).astype(np.int64), 16, 2048)
    kap = rng.uniform(0.5, 2.0, size=count)
    tl = rng.uniform(1.0, 3.0, size=count)
    tr = rng.uniform(1.0, 3.0, size=count)
    out = []
    for i in range(count):
        out.append(_base(n=(int(ns[i]), 1, 1), kappa=float(kap[i]), dt=r / float(kap[i]),
                         wall_lo=float(tl[i]), wall_hi=float(tr[i]), seed=seed + i,
                         realizations=1, precision="fp32", steps=100_000,
                         relax_steps=10_000))
    return out


def random_states(prob, R, seed, spread=0.05):
    """Seeded random states near the wall values (for one-step parity
    checks from a shared state): [R, cells] float64, values in
    (lo*(1-spread), hi*(1+spread)) with lo/hi the wall range."""
    cells = 1
    for v in prob["n"][: prob["dim"]]:
        cells *= v
    rng = np.random.default_rng(seed)
    lo = min(prob["wall_lo"], prob["wall_hi"]) * (1.0 - spread)
    hi = max(prob["wall_lo"], prob["wall_hi"]) * (1.0 + spread)
    return rng.uniform(lo, hi, size=(R, cells))


# Material data: the paper's iron (Sec. 3) and aluminium (standard values).
IRON = dict(rho=7870.0, c_v=450.0, lam=70.0)
ALUMINIUM = dict(rho=2700.0, c_v=897.0, lam=237.0)


def two_material_rod(**kw):
    """Iron / aluminium rod (the exercise of Sec. 6) in nondimensional units:
    per-cell conductivity ``lambda_cells`` and heat capacity ``rho_cv_cells``,
    iron (1, 1) left of the middle, aluminium (the ratios to iron) right."""
    n = int(kw.pop("cells", 256))
    rcv_al = ALUMINIUM["rho"] * ALUMINIUM["c_v"] / (IRON["rho"] * IRON["c_v"])
    lam_al = ALUMINIUM["lam"] / IRON["lam"]
    half = n // 2
    p = _base(n=(n, 1, 1), wall_lo=1.0, wall_hi=2.0, dt=0.08, realizations=4096, steps=1_000_000,
              relax_steps=100_000, precision="fp32", want_cov=1, kB=1e-3)
    p["lambda_cells"] = np.r_[np.full(half, 1.0), np.full(n - half, lam_al)]
    p["rho_cv_cells"] = np.r_[np.full(half, 1.0), np.full(n - half, rcv_al)]
    p.update(kw)
    return p


def iron_aluminium_rod(noneq=False, **kw):
    """The paper's rod (l = 20 nm, A = 4 nm^2, 32 cells) with aluminium from
    l/2 to l, dt = 0.1 dx^2 / (2 kappa_iron) (the paper's a = 0.1 for iron)."""
    p = iron_rod(noneq=noneq, **kw)
    n = p["n"][0]
    p["lambda_cells"] = np.r_[np.full(n // 2, IRON["lam"]), np.full(n - n // 2, ALUMINIUM["lam"])]
    p["rho_cv_cells"] = np.r_[np.full(n // 2, IRON["rho"] * IRON["c_v"]),
                              np.full(n - n // 2, ALUMINIUM["rho"] * ALUMINIUM["c_v"])]
    return p
