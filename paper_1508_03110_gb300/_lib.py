"""ctypes declarations of the C ABI in include/als.h (argument marshalling only).

Loading fails loudly if the CUDA library has not been built: there is no CPU
fallback for any entry point.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libals.so")

ALS_OK, ALS_EINVAL, ALS_ENOMEM, ALS_EBUDGET, ALS_ECUDA, ALS_ENOTSPD, ALS_ELINESEARCH, \
    ALS_ETIMEOUT, ALS_EBUSY, ALS_ENOTSUP = range(10)
STATUS_NAMES = {0: "ALS_OK", 1: "ALS_EINVAL", 2: "ALS_ENOMEM", 3: "ALS_EBUDGET", 4: "ALS_ECUDA",
                5: "ALS_ENOTSPD", 6: "ALS_ELINESEARCH", 7: "ALS_ETIMEOUT", 8: "ALS_EBUSY",
                9: "ALS_ENOTSUP"}
ALS_FP64, ALS_MIXED = 0, 1
ALS_LS_BACKTRACK, ALS_LS_EXACT, ALS_LS_MORE_THUENTE = 0, 1, 2
ALS_BETA_PR, ALS_BETA_FR, ALS_BETA_HS, ALS_BETA_PR_PLUS = 0, 1, 2, 3
ALS_PRECOND_ALS, ALS_PRECOND_NONE = 0, 1
ALS_DT_F64, ALS_DT_F32 = 0, 1
ALS_GRAM_AUTO, ALS_GRAM_FMA, ALS_GRAM_TC = 0, 1, 2

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Config(ctypes.Structure):
    _fields_ = [
        ("n_f", ctypes.c_int32), ("lam", ctypes.c_double), ("precision", ctypes.c_int32),
        ("ls_mode", ctypes.c_int32), ("ls_alpha0", ctypes.c_double), ("ls_tau", ctypes.c_double),
        ("ls_c", ctypes.c_double), ("ls_max_shrinks", ctypes.c_int32),
        ("refine_steps", ctypes.c_int32), ("gram_path", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_size_t), ("alloc", ALLOC_FN), ("free", FREE_FN),
        ("alloc_user", ctypes.c_void_p), ("beta_form", ctypes.c_int32), ("preconditioner", ctypes.c_int32),
        ("ls_c2", ctypes.c_double),
    ]


class IterInfo(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int64), ("f", ctypes.c_double), ("gnorm", ctypes.c_double),
        ("gnorm0", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
        ("c", ctypes.c_double * 5), ("shrinks", ctypes.c_int32), ("fallback", ctypes.c_int32),
        ("fallbacks", ctypes.c_int64), ("notspd", ctypes.c_int64), ("kernels", ctypes.c_int64),
    ]


class Launch(ctypes.Structure):
    _fields_ = [
        ("heavy_min", ctypes.c_int32), ("grid_mult", ctypes.c_int32), ("sweep_bin_min", ctypes.c_int32),
        ("split_min", ctypes.c_int32), ("seg_len", ctypes.c_int32), ("gram_path", ctypes.c_int32),
        ("dual_max", ctypes.c_int32), ("gather_tma", ctypes.c_int32), ("tc_chunk", ctypes.c_int32),
        ("chol_tc", ctypes.c_int32), ("dual_warp", ctypes.c_int32),
    ]


class TuneReport(ctypes.Structure):
    _fields_ = [
        ("chosen", Launch), ("candidates", ctypes.c_int32),
        ("pass_ms_default", ctypes.c_double), ("pass_ms_tuned", ctypes.c_double),
        ("sweep_ms_default", ctypes.c_double), ("sweep_ms_tuned", ctypes.c_double),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [
        ("max_batch", ctypes.c_int32), ("max_batch_ratings", ctypes.c_int64), ("slots", ctypes.c_int32),
        ("max_jobs", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_size_t),
    ]


class SweepTiming(ctypes.Structure):
    _fields_ = [
        ("sweep_ms", ctypes.c_double), ("ms", ctypes.c_double * 6), ("rows", ctypes.c_int64 * 6),
        ("ratings", ctypes.c_int64 * 6), ("launches", ctypes.c_int32 * 6),
    ]


SWEEP_CLASSES = ("k_sweep_tc_pf", "k_sweep_tc", "k_sweep_dual", "k_sweep_fma", "split", "k_sweep_tc_seg")

# name -> (restype, argtypes); the full list of symbols include/als.h declares
_vp, _i32, _i64, _dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "als_config_default": (None, [ctypes.POINTER(Config)]),
    "als_create": (_i32, [ctypes.POINTER(Config), _i64, _i64, _i64, _vp, _vp, _vp, _vp, _i32, _vp,
                          ctypes.POINTER(_vp)]),
    "als_create_batched": (_i32, [ctypes.POINTER(Config), _i32, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp,
                                  ctypes.POINTER(_vp)]),
    "als_batch_info": (_i32, [_vp, _i32, ctypes.POINTER(IterInfo)]),
    "als_batch_grad_norms": (_i32, [_vp, _i32, ctypes.POINTER(_dbl)]),
    "als_get_ratings": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "als_set_factors": (_i32, [_vp, _vp, _vp, _i32, _i32]),
    "als_get_factors": (_i32, [_vp, _vp, _vp, _i32, _i32]),
    "als_get_state": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_dbl), _i32, _i32]),
    "als_set_state": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_dbl), _i32, _i32]),
    "als_sweep": (_i32, [_vp, _i32]),
    "alsncg_step": (_i32, [_vp, ctypes.POINTER(IterInfo)]),
    "alsncg_run": (_i32, [_vp, _i32, _dbl, _i32, ctypes.POINTER(IterInfo), ctypes.POINTER(_i32)]),
    "als_loss": (_i32, [_vp, ctypes.POINTER(_dbl)]),
    "als_grad": (_i32, [_vp, _vp, _i32, _i32, ctypes.POINTER(_dbl)]),
    "als_linesearch_coeffs": (_i32, [_vp, _vp, _i32, _i32, ctypes.POINTER(_dbl)]),
    "als_linesearch_coeffs_static": (_i32, [_i64, _i64, _i32, _i32, _dbl, _vp, _vp, _vp, _vp, _vp, _vp,
                                            _i32, _vp, _vp]),
    "als_foldin": (_i32, [_vp, _i64, _vp, _vp, _vp, _i32, _vp, _i32, _i32]),
    "als_server_config_default": (None, [ctypes.POINTER(ServerConfig)]),
    "als_server_create": (_i32, [_vp, ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)]),
    "als_server_submit_foldin": (_i32, [_vp, _i64, _vp, _vp, ctypes.POINTER(_i64)]),
    "als_server_replay": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_dbl)]),
    "als_server_submit_job": (_i32, [_vp, ctypes.POINTER(Config), _i64, _i64, _i64, _vp, _vp, _vp, _vp, _i32,
                                     ctypes.POINTER(_i64)]),
    "als_server_wait": (_i32, [_vp, _i64, _dbl, _vp, ctypes.POINTER(_dbl)]),
    "als_server_stats": (_i32, [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), ctypes.POINTER(_i64),
                                ctypes.POINTER(_dbl)]),
    "als_server_destroy": (None, [_vp]),
    "als_get_launch": (_i32, [_vp, ctypes.POINTER(Launch)]),
    "als_set_launch": (_i32, [_vp, ctypes.POINTER(Launch)]),
    "als_autotune": (_i32, [_vp, _i32, ctypes.POINTER(TuneReport)]),
    "als_group_run": (_i32, [ctypes.POINTER(_vp), _i32, _i32, _dbl, _i32, ctypes.POINTER(IterInfo),
                             ctypes.POINTER(_i32)]),
    "als_selftest_wait_expiry": (_i32, [_vp, _dbl, ctypes.POINTER(_i64)]),
    "als_rank_topt": (_i32, [_vp, _i32, _vp, _i32]),
    "als_rank_accuracy": (_i32, [_vp, _i32, _vp, _i32, ctypes.POINTER(_dbl), _vp]),
    "als_time_sweep": (_i32, [_vp, _i32, ctypes.POINTER(SweepTiming)]),
    "als_probe_alu_peaks": (_i32, [ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]),
    "als_sync": (_i32, [_vp]),
    "als_destroy": (None, [_vp]),
    "als_last_error": (ctypes.c_char_p, []),
    "als_version": (ctypes.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libals.so and declare every entry point.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"the CUDA library {path} is not built; run `python -c \"import __graft_entry__ as g; "
            f"g.build()\"` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class ALSError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.als_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, where):
    if status != ALS_OK:
        raise ALSError(status, where)
