"""ctypes binding of the FP64 C oracle ``she_oracle.c``.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A *problem* is a plain dict in the paper's physical terms (grid, dx, cross
section, kappa, rho*c_V, k_B or D, n0, walls, dt, seed, ...), as produced by
``she_workloads``.  This module converts it to the two dimensionless numbers
the explicit scheme depends on -- the diffusion number r = kappa*dt/dx^2 and
the relative variance eps = k_B/(rho c_V dV) (species: 1/(n0 dV)) -- with its
own arithmetic, following Sec. 3, Eq. (3.3) and Eq. (3.7) of the paper.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HEAT, SPECIES = 0, 1
PERIODIC, DIRICHLET = 0, 1
FE, PC, BE, CN = 0, 1, 2, 3


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("n", ctypes.c_int32 * 3),
        ("equation", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("r", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("wall_lo", ctypes.c_double),
        ("wall_hi", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("stochastic", ctypes.c_int32),
        ("perturb_ic", ctypes.c_int32),
        ("stats_interval", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
        ("relax_steps", ctypes.c_int64),
        ("want_cov", ctypes.c_int32),
        ("want_sk", ctypes.c_int32),
        ("tc_lags", ctypes.c_int32),
        ("pad1", ctypes.c_int32),
        ("cond", ctypes.POINTER(ctypes.c_double)),
        ("cap", ctypes.POINTER(ctypes.c_double)),
        ("kB_dV", ctypes.c_double),
    ]


_LIB = None


def lib():
    """Load (building if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_normals4.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 4 + [dp]
        L.orc_normals4.restype = None
        L.orc_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                 ctypes.c_uint32, ctypes.c_uint32]
        L.orc_normal.restype = ctypes.c_double
        L.orc_wall_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_wall_normal.restype = ctypes.c_double
        L.orc_reference_profile.argtypes = [ctypes.POINTER(OrcParams), dp]
        L.orc_reference_profile.restype = None
        L.orc_initial_state.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_uint32, dp]
        L.orc_initial_state.restype = None
        L.orc_step.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_uint32, ctypes.c_uint32,
                               dp, dp]
        L.orc_step.restype = ctypes.c_int
        L.orc_run.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int64, ctypes.c_uint32,
                              ctypes.c_uint32, ctypes.c_int64, dp, ctypes.c_int,
                              ctypes.POINTER(ctypes.c_int64), dp, dp, dp, dp, dp, dp]
        L.orc_run.restype = ctypes.c_int
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------- parameters --

def cell_volume(prob):
    """dV: 1D A*dx (Sec. 3, 'volume of a grid cell'); 2D dx^2*thickness
    (the ``area`` field holds the thickness); 3D dx^3."""
    dim = prob["dim"]
    dx = prob["dx"]
    if dim == 1:
        return prob["area"] * dx
    if dim == 2:
        return prob["area"] * dx * dx
    return dx ** 3


def dimensionless(prob):
    """(r, eps) of Eq. (3.3)/(3.7): r = kappa dt/dx^2 and
    eps = k_B/(rho c_V dV) for heat; r = D dt/dx^2, eps = 1/(n0 dV) for species."""
    dV = cell_volume(prob)
    dx2 = prob["dx"] ** 2
    if prob.get("equation", "heat") == "heat":
        return prob["kappa"] * prob["dt"] / dx2, prob["kB"] / (prob["rho_cv"] * dV)
    return prob["D"] * prob["dt"] / dx2, 1.0 / (prob["n0"] * dV)


def material_arrays(prob):
    """A rod of several materials (the iron / aluminium exercise, Sec. 6):
    per cell the conductance number a_i = lambda_i dt / dx^2 and the heat
    capacity per volume rho c_V,i, and k_B / dV; None for a uniform problem.
    The problem gives ``lambda_cells`` (thermal conductivity per cell) and
    ``rho_cv_cells``."""
    lam = prob.get("lambda_cells")
    if lam is None:
        return None
    lam = np.asarray(lam, dtype=np.float64)
    cap = np.ascontiguousarray(prob["rho_cv_cells"], dtype=np.float64)
    cond = np.ascontiguousarray(lam * prob["dt"] / prob["dx"] ** 2)
    return cond, cap, prob["kB"] / cell_volume(prob)


def to_params(prob):
    p = OrcParams()
    dim = prob["dim"]
    n = list(prob["n"]) + [1] * (3 - len(prob["n"]))
    p.dim = dim
    p.n[0], p.n[1], p.n[2] = n[0], n[1], n[2]
    p.equation = HEAT if prob.get("equation", "heat") == "heat" else SPECIES
    p.bc = DIRICHLET if prob.get("bc", "dirichlet") == "dirichlet" else PERIODIC
    r, eps = dimensionless(prob)
    p.r, p.eps = r, eps
    p.wall_lo, p.wall_hi = prob["wall_lo"], prob["wall_hi"]
    p.seed = prob.get("seed", 0)
    p.stochastic = int(prob.get("stochastic", 1))
    p.perturb_ic = int(prob.get("perturb_ic", 1))
    p.stats_interval = int(prob.get("stats_interval", 10))
    p.scheme = {"fe": FE, "pc": PC, "be": BE, "cn": CN}[prob.get("scheme", "fe")]
    p.relax_steps = int(prob.get("relax_steps", 0))
    p.want_cov = int(prob.get("want_cov", 0))
    p.want_sk = int(prob.get("want_sk", 0))
    p.tc_lags = int(prob.get("tc_lags", 0))
    mat = material_arrays(prob)
    if mat is not None:
        cond, cap, kb_dv = mat
        p._keep = (cond, cap)              # the struct holds pointers into these
        p.cond = _dp(cond)
        p.cap = _dp(cap)
        p.kB_dV = kb_dv
    return p


def cells(prob):
    c = 1
    for v in prob["n"][: prob["dim"]]:
        c *= v
    return c


# -------------------------------------------------------------------- RNG --

def philox(ctr, key):
    """Philox-4x32-10 block: 4 x uint32 counter, 2 x uint32 key -> 4 x uint32."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals4(seed, c0, c1, c2, c3):
    z = np.zeros(4)
    lib().orc_normals4(seed, c0, c1, c2, c3, _dp(z))
    return z


def normal(seed, g, step, stream, tag=0):
    return lib().orc_normal(seed, g, step, stream, tag)


def wall_normal(seed, step, stream):
    return lib().orc_wall_normal(seed, step, stream)


# ------------------------------------------------------------ simulation --

def reference_profile(prob):
    p = to_params(prob)
    out = np.zeros(cells(prob))
    lib().orc_reference_profile(ctypes.byref(p), _dp(out))
    return out


def initial_state(prob, stream):
    p = to_params(prob)
    out = np.zeros(cells(prob))
    lib().orc_initial_state(ctypes.byref(p), stream, _dp(out))
    return out


def step(prob, state, step_index, stream):
    """One step of one realization from `state`: forward Euler (Eq. (3.3)),
    the predictor-corrector scheme of Sec. 3 (``prob["scheme"] == "pc"``), or
    backward Euler / Crank-Nicolson ("be" / "cn", the implicit exercise of
    Sec. 6)."""
    p = to_params(prob)
    T = np.ascontiguousarray(state, dtype=np.float64)
    out = np.zeros_like(T)
    rc = lib().orc_step(ctypes.byref(p), step_index, stream, _dp(T), _dp(out))
    if rc != 0:
        raise RuntimeError("orc_step failed: %d" % rc)
    return out


def run(prob, R, nsteps, step0=0, stream0=0, state=None, want_cov=None, want_sk=None, tc_lags=None):
    """Run R realizations for nsteps steps; return the final states and the
    pooled accumulators of the sampling schedule (Eq. (3.9)).

    If ``state`` is None the initial condition is generated; otherwise the
    given [R, cells] array is the starting state at absolute step ``step0``.
    """
    p = to_params(prob)
    if want_cov is not None:
        p.want_cov = int(want_cov)
    if want_sk is not None:
        p.want_sk = int(want_sk)
    if tc_lags is not None:
        p.tc_lags = int(tc_lags)
    nc = cells(prob)
    if state is None:
        st = np.zeros((R, nc))
        init = 1
    else:
        st = np.array(state, dtype=np.float64, copy=True).reshape(R, nc)
        init = 0
    st = np.ascontiguousarray(st)
    ns = ctypes.c_int64(0)
    sum_d = np.zeros(nc)
    sum_d2 = np.zeros(nc)
    sum_dd = np.zeros(nc * nc) if p.want_cov else None
    sum_sk = np.zeros(nc) if (p.want_sk & 1) else None
    axes_len = sum(prob["n"][: prob["dim"]])
    sum_ska = np.zeros(axes_len) if (p.want_sk & 2) else None
    L = int(p.tc_lags)
    sum_tc = np.zeros(L * nc) if L > 0 else None
    rc = lib().orc_run(ctypes.byref(p), R, stream0, step0, nsteps, _dp(st), init,
                       ctypes.byref(ns), _dp(sum_d), _dp(sum_d2), _dp(sum_dd),
                       _dp(sum_sk), _dp(sum_ska), _dp(sum_tc))
    if rc != 0:
        raise RuntimeError("orc_run failed: %d" % rc)
    out = {
        "state": st,
        "n_samples_per_realization": ns.value,
        "n_samples": ns.value * R,
        "sum_d": sum_d,
        "sum_d2": sum_d2,
    }
    if sum_dd is not None:
        out["sum_dd"] = sum_dd.reshape(nc, nc)
    if sum_sk is not None:
        out["sum_sk"] = sum_sk
    if sum_ska is not None:
        out["sum_sk_axes"] = sum_ska
    if sum_tc is not None:
        # sample pairs l sampling intervals apart within this run, pooled over
        # the realizations
        out["sum_tc"] = sum_tc.reshape(L, nc)
        out["n_tc"] = np.array([R * max(0, ns.value - l) for l in range(L)], dtype=np.int64)
    return out


def finalize(prob, acc):
    """Turn pooled sums into the statistics the paper reports: mean and
    (biased, 1/n) variance per cell as in Sec. 3, the equal-time covariance,
    and S_k = <|hat T_k|^2> of Eq. (3.11) (plus its fluctuation part)."""
    n = acc["n_samples"]
    tref = reference_profile(prob)
    mu = acc["sum_d"] / n
    res = {"n": n, "mean": tref + mu, "var": acc["sum_d2"] / n - mu * mu}
    if "sum_dd" in acc:
        res["cov"] = acc["sum_dd"] / n - np.outer(mu, mu)
    if "sum_sk" in acc:
        shape = tuple(reversed(prob["n"][: prob["dim"]]))
        mu_hat = np.fft.fftn(mu.reshape(shape)).ravel()
        ref_hat = np.fft.fftn(tref.reshape(shape)).ravel()
        dd = acc["sum_sk"] / n
        res["sk_fluct"] = dd - np.abs(mu_hat) ** 2
        res["sk"] = np.abs(ref_hat) ** 2 + 2.0 * np.real(np.conj(ref_hat) * mu_hat) + dd
    if "sum_sk_axes" in acc:
        res["sk_axes"] = acc["sum_sk_axes"] / n
    if "sum_tc" in acc:
        # <delta_i(t + l K) delta_i(t)> per lag l and cell i (delta = T - T_ref)
        res["time_corr"] = acc["sum_tc"] / np.maximum(acc["n_tc"], 1)[:, None]
    return res


def num_threads():
    return lib().orc_num_threads()


def lib_path():
    return _build.LIB if os.path.exists(_build.LIB) else None
