"""ctypes declarations of the C ABI in ``include/she.h``.

Argument marshalling only: every step of the hot path runs in libshe's CUDA
kernels.  Loading fails loudly (``LibraryMissing``) when the library has not
been built -- there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libshe.so")

SHE_OK = 0
SHE_ERR_INVALID_ARG = 1
SHE_ERR_UNSTABLE = 2
SHE_ERR_OOM = 3
SHE_ERR_CUDA = 4
SHE_ERR_NONFINITE = 5
SHE_ERR_TIMEOUT = 6
SHE_ERR_STATE = 7
SHE_ERR_UNSUPPORTED = 8
STATUS_NAMES = {0: "SHE_OK", 1: "SHE_ERR_INVALID_ARG", 2: "SHE_ERR_UNSTABLE", 3: "SHE_ERR_OOM",
                4: "SHE_ERR_CUDA", 5: "SHE_ERR_NONFINITE", 6: "SHE_ERR_TIMEOUT",
                7: "SHE_ERR_STATE", 8: "SHE_ERR_UNSUPPORTED"}

SHE_HEAT, SHE_SPECIES = 0, 1
SHE_PERIODIC, SHE_DIRICHLET = 0, 1
SHE_FP32, SHE_FP64 = 0, 1
SHE_FE = 0
SHE_PC = 1
SHE_BE = 2
SHE_CN = 3
SHE_SK_FULL, SHE_SK_AXES = 1, 2
SHE_KERNEL_AUTO, SHE_KERNEL_PLAIN = 0, 1
# face fluxes the fixed scratch array of she_step_plain_noalloc holds
SHE_NOALLOC_MAX_FACES = 1 << 20

# Every symbol include/she.h declares (checked by the CPU test suite).
EXPORTS = ["she_init", "she_init_batch", "she_step_n", "she_get_sizes", "she_stats",
           "she_reset_stats", "she_get_state", "she_set_state", "she_get_state_device",
           "she_set_state_device", "she_last_error", "she_free", "she_noise_probe",
           "she_launch_count", "she_syrk_probe", "she_step_plain_noalloc", "she_wait_probe",
           "she_profile", "she_profile_read", "she_stats_raw", "she_finalize"]


class she_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("n", ctypes.c_int32 * 3),
        ("dx", ctypes.c_double),
        ("area", ctypes.c_double),
        ("equation", ctypes.c_int32),
        ("bc", ctypes.c_int32),
        ("kappa", ctypes.c_double),
        ("rho_cv", ctypes.c_double),
        ("kB", ctypes.c_double),
        ("D", ctypes.c_double),
        ("n0", ctypes.c_double),
        ("wall_lo", ctypes.c_double),
        ("wall_hi", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("realizations", ctypes.c_int64),
        ("scheme", ctypes.c_int32),
        ("stochastic", ctypes.c_int32),
        ("perturb_ic", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("stats_interval", ctypes.c_int32),
        ("want_cov", ctypes.c_int32),
        ("relax_steps", ctypes.c_int64),
        ("want_sk", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("steps_per_launch", ctypes.c_int32),
        ("stream_offset", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("tc_lags", ctypes.c_int32),
        ("lambda_cells", ctypes.POINTER(ctypes.c_double)),
        ("rho_cv_cells", ctypes.POINTER(ctypes.c_double)),
        ("tune", ctypes.c_int32),
    ]


_dp = ctypes.POINTER(ctypes.c_double)


class she_stats_out(ctypes.Structure):
    _fields_ = [
        ("n_samples", ctypes.c_int64),
        ("mean", _dp),
        ("var", _dp),
        ("var_se", _dp),
        ("cov", _dp),
        ("sk", _dp),
        ("sk_fluct", _dp),
        ("sk_axes", _dp),
        ("sum_d", _dp),
        ("sum_d2", _dp),
        ("time_corr", _dp),
    ]


class she_sizes(ctypes.Structure):
    _fields_ = [
        ("cells", ctypes.c_int64),
        ("realizations", ctypes.c_int64),
        ("instances", ctypes.c_int64),
        ("state_bytes", ctypes.c_int64),
        ("elem_bytes", ctypes.c_int64),
        ("axes_len", ctypes.c_int64),
        ("step", ctypes.c_uint64),
        ("tc_lags", ctypes.c_int64),
        ("batches", ctypes.c_int64),
        ("sk_raw_len", ctypes.c_int64),
        ("axes_raw_len", ctypes.c_int64),
        ("layout", ctypes.c_int64),
    ]


_i64p = ctypes.POINTER(ctypes.c_int64)


class she_raw(ctypes.Structure):
    _fields_ = [
        ("n_samples", ctypes.c_int64),
        ("batches", ctypes.c_int64),
        ("batch_n", _i64p),
        ("batch_sum_d", _dp),
        ("batch_sum_d2", _dp),
        ("sum_dd", _dp),
        ("sk_sum", _dp),
        ("axes_sum", _dp),
        ("tc_sum", _dp),
        ("tc_pairs", _i64p),
    ]


class LibraryMissing(RuntimeError):
    """libshe.so has not been built (run ``python -m paper_2406_12157_gb300.build``)."""


_LIB = None


def load(path=None):
    """Load libshe.so and declare its signatures.  Raises LibraryMissing if
    the library file does not exist."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise LibraryMissing("libshe.so not found at %s; build it with "
                             "paper_2406_12157_gb300.build.build()" % p)
    L = ctypes.CDLL(p)
    H = ctypes.c_void_p
    L.she_init.argtypes = [ctypes.POINTER(she_params), ctypes.POINTER(H)]
    L.she_init.restype = ctypes.c_int
    L.she_init_batch.argtypes = [ctypes.POINTER(she_params), ctypes.c_int64, ctypes.POINTER(H)]
    L.she_init_batch.restype = ctypes.c_int
    L.she_step_n.argtypes = [H, ctypes.c_uint64]
    L.she_step_n.restype = ctypes.c_int
    L.she_get_sizes.argtypes = [H, ctypes.POINTER(she_sizes)]
    L.she_get_sizes.restype = ctypes.c_int
    L.she_stats.argtypes = [H, ctypes.POINTER(she_stats_out)]
    L.she_stats.restype = ctypes.c_int
    L.she_reset_stats.argtypes = [H]
    L.she_reset_stats.restype = ctypes.c_int
    L.she_get_state.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_uint64)]
    L.she_get_state.restype = ctypes.c_int
    L.she_set_state.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64]
    L.she_set_state.restype = ctypes.c_int
    L.she_get_state_device.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t]
    L.she_get_state_device.restype = ctypes.c_int
    L.she_set_state_device.argtypes = [H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64]
    L.she_set_state_device.restype = ctypes.c_int
    L.she_last_error.argtypes = [H]
    L.she_last_error.restype = ctypes.c_char_p
    L.she_free.argtypes = [H]
    L.she_free.restype = None
    L.she_noise_probe.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]
    L.she_noise_probe.restype = ctypes.c_int
    L.she_syrk_probe.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    L.she_syrk_probe.restype = ctypes.c_int
    L.she_step_plain_noalloc.argtypes = [ctypes.POINTER(she_params), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_uint64]
    L.she_step_plain_noalloc.restype = ctypes.c_int
    L.she_wait_probe.argtypes = [ctypes.c_uint32]
    L.she_wait_probe.restype = ctypes.c_int
    L.she_launch_count.argtypes = [H]
    L.she_launch_count.restype = ctypes.c_int64
    L.she_profile.argtypes = [H, ctypes.c_int]
    L.she_profile.restype = ctypes.c_int
    L.she_profile_read.argtypes = [H, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    L.she_profile_read.restype = ctypes.c_int
    L.she_stats_raw.argtypes = [H, ctypes.POINTER(she_raw)]
    L.she_stats_raw.restype = ctypes.c_int
    L.she_finalize.argtypes = [ctypes.POINTER(she_params), ctypes.POINTER(she_raw), ctypes.POINTER(she_stats_out)]
    L.she_finalize.restype = ctypes.c_int
    if path is None:
        _LIB = L
    return L
