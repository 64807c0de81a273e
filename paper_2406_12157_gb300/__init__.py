"""GB300-native stochastic heat / species diffusion library (Python binding).

Thin binding of the C ABI in ``include/she.h`` (``libshe.so``), with the same
names.  Argument marshalling only; every step runs in the library's CUDA
kernels for sm_103a.  If the library is not built, every call raises
``LibraryMissing`` -- there is no CPU fallback.

Method: Garcia et al., "An Introduction to Computational Fluctuating
Hydrodynamics" (2024), Sec. 3 (forward-Euler scheme, Eq. (3.3); Dirichlet
walls, Eq. (3.8); sampling, Eq. (3.9)) and Sec. 4 (species noise, Eq. (4.7)).
"""
import ctypes

import numpy as np

from . import _abi
from ._abi import (LibraryMissing, SHE_BE, SHE_CN, SHE_DIRICHLET, SHE_FE, SHE_PC, SHE_FP32, SHE_FP64,  # noqa: F401
                   SHE_HEAT,
                   SHE_KERNEL_AUTO, SHE_KERNEL_PLAIN, SHE_PERIODIC, SHE_SK_AXES, SHE_SK_FULL,
                   SHE_SPECIES)

__all__ = ["SheError", "LibraryMissing", "params_from_problem", "she_init", "she_init_batch",
           "she_step_n", "she_get_sizes", "she_stats", "she_reset_stats", "she_get_state",
           "she_set_state", "she_get_state_device", "she_set_state_device", "she_last_error",
           "she_free", "she_noise_probe", "she_launch_count", "she_syrk_probe", "she_profile",
           "she_profile_read", "she_stats_raw", "she_finalize", "Simulation", "BatchSimulation", "lib"]


class SheError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (_abi.STATUS_NAMES.get(status, status), msg))


def lib():
    return _abi.load()


def _check(status, h=None, what=""):
    if status != _abi.SHE_OK:
        msg = what
        if h is not None:
            m = lib().she_last_error(h)
            if m:
                msg = "%s: %s" % (what, m.decode(errors="replace"))
        raise SheError(status, msg)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    ptr = getattr(stream, "cuda_stream", None)     # torch.cuda.Stream
    if ptr is not None:
        return int(ptr)
    raise TypeError("stream must be None, an int cudaStream_t or a torch.cuda.Stream")


def params_from_problem(prob, stream=None, **overrides):
    """Build a ``she_params`` from a problem dict in the paper's physical
    terms (see she_workloads for the fields)."""
    q = dict(prob)
    q.update(overrides)
    p = _abi.she_params()
    p.dim = int(q["dim"])
    n = list(q["n"]) + [1] * (3 - len(q["n"]))
    for a in range(3):
        p.n[a] = int(n[a]) if a < p.dim else 1
    p.dx = float(q["dx"])
    p.area = float(q.get("area", 1.0))
    p.equation = SHE_HEAT if q.get("equation", "heat") in ("heat", SHE_HEAT) else SHE_SPECIES
    p.bc = SHE_DIRICHLET if q.get("bc", "dirichlet") in ("dirichlet", SHE_DIRICHLET) else SHE_PERIODIC
    p.kappa = float(q.get("kappa", 1.0))
    p.rho_cv = float(q.get("rho_cv", 1.0))
    p.kB = float(q.get("kB", 0.0))
    p.D = float(q.get("D", 1.0))
    p.n0 = float(q.get("n0", 1.0))
    p.wall_lo = float(q["wall_lo"])
    p.wall_hi = float(q["wall_hi"])
    p.dt = float(q["dt"])
    p.seed = int(q.get("seed", 0))
    p.realizations = int(q.get("realizations", 1))
    p.scheme = {"fe": SHE_FE, "pc": SHE_PC, "be": SHE_BE, "cn": SHE_CN, SHE_FE: SHE_FE, SHE_PC: SHE_PC,
                SHE_BE: SHE_BE, SHE_CN: SHE_CN}[q.get("scheme", "fe")]
    p.stochastic = int(q.get("stochastic", 1))
    p.perturb_ic = int(q.get("perturb_ic", 1))
    prec = q.get("precision", "fp32")
    p.precision = SHE_FP64 if prec in ("fp64", SHE_FP64) else SHE_FP32
    p.stats_interval = int(q.get("stats_interval", 10))
    p.want_cov = int(q.get("want_cov", 0))
    p.relax_steps = int(q.get("relax_steps", 0))
    p.want_sk = int(q.get("want_sk", 0))
    kern = q.get("kernel", "auto")
    p.kernel = SHE_KERNEL_PLAIN if kern in ("plain", SHE_KERNEL_PLAIN) else SHE_KERNEL_AUTO
    p.steps_per_launch = int(q.get("steps_per_launch", 0))
    p.stream_offset = int(q.get("stream_offset", 0))
    p.tc_lags = int(q.get("tc_lags", 0))
    p.tune = int(q.get("tune", 0))
    if q.get("lambda_cells") is not None:
        # a rod of several materials: the arrays are read during she_init only;
        # the struct keeps them alive as long as it lives
        lam = np.ascontiguousarray(q["lambda_cells"], dtype=np.float64)
        rcv = np.ascontiguousarray(q["rho_cv_cells"], dtype=np.float64)
        p._keep = (lam, rcv)
        p.lambda_cells = _ptr(lam)
        p.rho_cv_cells = _ptr(rcv)
    sp = _stream_ptr(stream)
    p.stream = sp
    return p


def she_init(params):
    h = ctypes.c_void_p()
    _check(lib().she_init(ctypes.byref(params), ctypes.byref(h)), None, "she_init")
    _HANDLE_FLAGS[h.value] = {"cov": bool(params.want_cov) or (int(params.dim) == 1 and bool(params.want_sk & 1))}
    return h


def she_init_batch(params_list):
    arr = (_abi.she_params * len(params_list))(*params_list)
    h = ctypes.c_void_p()
    _check(lib().she_init_batch(arr, len(params_list), ctypes.byref(h)), None, "she_init_batch")
    return h


def she_step_n(h, n):
    _check(lib().she_step_n(h, int(n)), h, "she_step_n")


def she_get_sizes(h):
    s = _abi.she_sizes()
    _check(lib().she_get_sizes(h, ctypes.byref(s)), h, "she_get_sizes")
    return s


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def she_stats(h, cov=False, sk=False, sk_axes=False, raw=False, time_corr=False):
    """Finalised statistics as numpy arrays (see she_stats_out in she.h)."""
    s = she_get_sizes(h)
    c = int(s.cells)
    out = {k: np.empty(c) for k in ("mean", "var", "var_se")}
    if cov:
        out["cov"] = np.empty(c * c)
    if sk:
        out["sk"] = np.empty(c)
        out["sk_fluct"] = np.empty(c)
    if sk_axes:
        out["sk_axes"] = np.empty(int(s.axes_len))
    if raw:
        out["sum_d"] = np.empty(c)
        out["sum_d2"] = np.empty(c)
    L = int(s.tc_lags)
    if time_corr and L > 0:
        out["time_corr"] = np.empty(L * c)
    st = _abi.she_stats_out()
    for k, v in out.items():
        setattr(st, k, _ptr(v))
    _check(lib().she_stats(h, ctypes.byref(st)), h, "she_stats")
    out["n_samples"] = int(st.n_samples)
    if cov:
        out["cov"] = out["cov"].reshape(c, c)
    if "time_corr" in out:
        out["time_corr"] = out["time_corr"].reshape(L, c)
    return out


_RAW_KEYS = ("batch_n", "batch_sum_d", "batch_sum_d2", "sum_dd", "sk_sum", "axes_sum", "tc_sum", "tc_pairs")


def _raw_struct(raw):
    st = _abi.she_raw()
    st.n_samples = int(raw["n_samples"])
    st.batches = int(raw["batches"])
    for k in _RAW_KEYS:
        v = raw.get(k)
        if v is None:
            continue
        if k in ("batch_n", "tc_pairs"):
            setattr(st, k, v.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        else:
            setattr(st, k, _ptr(v))
    return st


def she_stats_raw(h):
    """The raw FP64 accumulators (see she_raw in she.h) as numpy arrays:
    every entry a sum or a count, so replicas merge by addition."""
    s = she_get_sizes(h)
    c, B, L = int(s.cells), int(s.batches), int(s.tc_lags)
    out = {"batch_n": np.empty(B, dtype=np.int64), "batch_sum_d": np.empty(B * c),
           "batch_sum_d2": np.empty(B * c)}
    if _stats_flags(h)["cov"]:
        out["sum_dd"] = np.empty(c * c)
    if s.sk_raw_len:
        out["sk_sum"] = np.empty(int(s.sk_raw_len))
    if s.axes_raw_len:
        out["axes_sum"] = np.empty(int(s.axes_raw_len))
    if L:
        out["tc_sum"] = np.empty(L * c)
        out["tc_pairs"] = np.empty(L, dtype=np.int64)
    out["n_samples"] = 0
    out["batches"] = B
    st = _raw_struct(out)
    _check(lib().she_stats_raw(h, ctypes.byref(st)), h, "she_stats_raw")
    out["n_samples"] = int(st.n_samples)
    return out


def _stats_flags(h):
    # whether the handle accumulates the covariance: probe with a NULL-free
    # request is not possible, so the binding remembers it per handle
    return _HANDLE_FLAGS.get(h.value, {"cov": False})


_HANDLE_FLAGS = {}


def she_finalize(params, raw, cov=False, sk=False, sk_axes=False, time_corr=False):
    """Statistics (as she_stats) of the problem `params` from a raw block,
    e.g. the sum of several replicas' she_stats_raw blocks.  Host only."""
    p = params
    c = 1
    for a in range(int(p.dim)):
        c *= int(p.n[a])
    out = {k: np.empty(c) for k in ("mean", "var", "var_se", "sum_d", "sum_d2")}
    if cov:
        out["cov"] = np.empty(c * c)
    if sk:
        out["sk"] = np.empty(c)
        out["sk_fluct"] = np.empty(c)
    if sk_axes:
        out["sk_axes"] = np.empty(sum(int(p.n[a]) for a in range(int(p.dim))))
    L = int(p.tc_lags)
    if time_corr and L > 0:
        out["time_corr"] = np.empty(L * c)
    st = _abi.she_stats_out()
    for k, v in out.items():
        setattr(st, k, _ptr(v))
    rs = _raw_struct(raw)
    _check(lib().she_finalize(ctypes.byref(p), ctypes.byref(rs), ctypes.byref(st)), None, "she_finalize")
    out["n_samples"] = int(st.n_samples)
    if cov:
        out["cov"] = out["cov"].reshape(c, c)
    if "time_corr" in out:
        out["time_corr"] = out["time_corr"].reshape(L, c)
    return out


def she_reset_stats(h):
    _check(lib().she_reset_stats(h), h, "she_reset_stats")


def she_get_state(h):
    """Return (state [realizations, cells] as float32/float64, step)."""
    s = she_get_sizes(h)
    dt = np.float64 if s.elem_bytes == 8 else np.float32
    buf = np.empty((int(s.realizations), int(s.cells)), dtype=dt)
    step = ctypes.c_uint64()
    _check(lib().she_get_state(h, buf.ctypes.data, buf.nbytes, ctypes.byref(step)), h, "she_get_state")
    return buf, int(step.value)


def she_set_state(h, state, step):
    s = she_get_sizes(h)
    dt = np.float64 if s.elem_bytes == 8 else np.float32
    buf = np.ascontiguousarray(state, dtype=dt)
    _check(lib().she_set_state(h, buf.ctypes.data, buf.nbytes, int(step)), h, "she_set_state")


def she_get_state_device(h, dev_ptr, nbytes):
    _check(lib().she_get_state_device(h, int(dev_ptr), int(nbytes)), h, "she_get_state_device")


def she_set_state_device(h, dev_ptr, nbytes, step):
    _check(lib().she_set_state_device(h, int(dev_ptr), int(nbytes), int(step)), h,
           "she_set_state_device")


def she_last_error(h):
    m = lib().she_last_error(h)
    return m.decode(errors="replace") if m else ""


def she_free(h):
    if h is not None and h.value:
        _HANDLE_FLAGS.pop(h.value, None)
        lib().she_free(h)
        h.value = None


def she_launch_count(h):
    return int(lib().she_launch_count(h))


def she_profile(h, enable):
    _check(lib().she_profile(h, 1 if enable else 0), h, "she_profile")


def she_profile_read(h):
    """Device time (ms) and launch counts of the step and statistics kernels
    timed since profiling started or was last read."""
    sm, sn = ctypes.c_double(), ctypes.c_int64()
    tm, tn = ctypes.c_double(), ctypes.c_int64()
    _check(lib().she_profile_read(h, ctypes.byref(sm), ctypes.byref(sn), ctypes.byref(tm), ctypes.byref(tn)),
           h, "she_profile_read")
    return {"step_ms": sm.value, "step_launches": int(sn.value), "stats_ms": tm.value,
            "stats_launches": int(tn.value)}


def she_noise_probe(seed, c0, c1, c2, c3, count):
    """Raw Philox words and Box-Muller normals (FP64 and FP32) from the
    device generator for counters (c0 + k, c1, c2, c3), k < count."""
    bits = np.empty(4 * count, dtype=np.uint32)
    z64 = np.empty(4 * count, dtype=np.float64)
    z32 = np.empty(4 * count, dtype=np.float32)
    _check(lib().she_noise_probe(seed, c0, c1, c2, c3, count, bits.ctypes.data, z64.ctypes.data,
                                 z32.ctypes.data), None, "she_noise_probe")
    return bits.reshape(count, 4), z64.reshape(count, 4), z32.reshape(count, 4)


def she_syrk_probe(X):
    """C = X^T X (FP64 result) for X [K <= 32, N <= 256] via the library's
    tcgen05 covariance kernel (bf16 hi/lo split, FP32 accumulation)."""
    Xf = np.ascontiguousarray(X, dtype=np.float32)
    K, N = Xf.shape
    C = np.empty((N, N), dtype=np.float64)
    _check(lib().she_syrk_probe(Xf.ctypes.data, K, N, C.ctypes.data), None, "she_syrk_probe")
    return C


class BatchSimulation:
    """Owning wrapper of a batch handle of uneven 1D instances
    (``she_init_batch``): ``with BatchSimulation(problems) as b: ...``.
    The state and per-cell statistics are the instances back to back."""

    def __init__(self, problems, stream=None, **overrides):
        self.params = [params_from_problem(q, stream=stream, **overrides) for q in problems]
        self.offsets = []
        off = 0
        for q in problems:
            self.offsets.append(off)
            off += int(q["n"][0])
        self.h = she_init_batch(self.params)

    def step(self, n):
        she_step_n(self.h, n)

    def stats(self, **kw):
        return she_stats(self.h, **kw)

    def state(self):
        st, step = she_get_state(self.h)
        return st.reshape(-1), step

    def set_state(self, state, step):
        she_set_state(self.h, np.asarray(state).reshape(1, -1), step)

    def launches(self):
        return she_launch_count(self.h)

    def profile(self, enable=True):
        she_profile(self.h, enable)

    def profile_read(self):
        return she_profile_read(self.h)

    def close(self):
        she_free(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """Owning wrapper of one handle: ``with Simulation(problem) as sim: ...``."""

    def __init__(self, prob, stream=None, **overrides):
        self.params = params_from_problem(prob, stream=stream, **overrides)
        self.h = she_init(self.params)

    def step(self, n):
        she_step_n(self.h, n)

    def stats(self, **kw):
        return she_stats(self.h, **kw)

    def stats_raw(self):
        return she_stats_raw(self.h)

    def state(self):
        return she_get_state(self.h)

    def set_state(self, state, step):
        she_set_state(self.h, state, step)

    def sizes(self):
        return she_get_sizes(self.h)

    def launches(self):
        return she_launch_count(self.h)

    def profile(self, enable=True):
        she_profile(self.h, enable)

    def profile_read(self):
        return she_profile_read(self.h)

    def close(self):
        she_free(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
