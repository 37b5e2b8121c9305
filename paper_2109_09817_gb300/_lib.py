"""ctypes view of libgp's C ABI (include/gp.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgp.so")

GP_OK, GP_EINVAL, GP_ENOMEM, GP_ENOTCONV, GP_EBREAKDOWN, GP_ENONPD, GP_ETIMEOUT, GP_ECUDA = range(8)
ERROR_NAMES = {0: "GP_OK", 1: "GP_EINVAL", 2: "GP_ENOMEM", 3: "GP_ENOTCONV",
               4: "GP_EBREAKDOWN", 5: "GP_ENONPD", 6: "GP_ETIMEOUT", 7: "GP_ECUDA"}
GP_FP32_PLAIN, GP_FP32_SPLIT_TF32, GP_FP32_SPLIT_F16, GP_TF32 = range(4)
GP_VAR_NONE, GP_VAR_EXACT, GP_VAR_CACHED = 0, 1, 2
GP_VAR_CACHE_MAX_RANK = 128
GP_PC_SIGMA, GP_PC_RESID = 0, 1
GP_STOP_RECURRENCE, GP_STOP_TRUE = 0, 1
GP_OPT_SYMMETRIC_KMV = 1
GP_HOST = 0x100

# Every symbol include/gp.h declares.
EXPORTS = (
    "gp_create", "gp_destroy", "gp_set_stream", "gp_sync", "gp_last_error",
    "gp_launch_count", "gp_set_option", "gp_profile", "gp_profile_read", "gp_kmatmul", "gp_kcross_matmul", "gp_pivchol", "gp_mbcg",
    "gp_lanczos_logquad",
    "gp_mbcg_refine", "gp_bcg", "gp_logml_and_grad", "gp_model_fit", "gp_model_free", "gp_predict",
    "gp_model_variance_cache", "gp_predict_sum", "gp_subset_indices", "gp_hyperopt", "gp_train",
    "gp_kmatmul_noalloc", "gp_server_create", "gp_server_add_model", "gp_server_predict", "gp_server_molecule",
    "gp_server_solve", "gp_server_wait", "gp_server_stats", "gp_server_last_error",
    "gp_server_destroy",
)


class GpTheta(ctypes.Structure):
    _fields_ = [("lengthscale", ctypes.POINTER(ctypes.c_double)),
                ("outputscale", ctypes.c_double),
                ("sigma2", ctypes.c_double)]


class GpStats(ctypes.Structure):
    _fields_ = [("iters_max", ctypes.c_int), ("iters_y", ctypes.c_int),
                ("rank", ctypes.c_int), ("n_kmatmul", ctypes.c_int),
                ("relres_y", ctypes.c_double), ("relres_max", ctypes.c_double),
                ("logdet_P", ctypes.c_double), ("yKinvy", ctypes.c_double),
                ("true_relres_y", ctypes.c_double), ("true_checks", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libgp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"libgp.so not found at {path}: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` "
            "(no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    vp, i64, c_int, c_dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    th = ctypes.POINTER(GpTheta)
    st = ctypes.POINTER(GpStats)
    ip = ctypes.POINTER(ctypes.c_int)
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "gp_create": (c_int, [ctypes.POINTER(vp), c_int, vp]),
        "gp_destroy": (None, [vp]),
        "gp_set_stream": (c_int, [vp, vp]),
        "gp_sync": (c_int, [vp]),
        "gp_last_error": (ctypes.c_char_p, [vp]),
        "gp_launch_count": (i64, [vp]),
        "gp_set_option": (c_int, [vp, c_int, c_int]),
        "gp_profile": (c_int, [vp, c_int]),
        "gp_profile_read": (c_int, [vp, ctypes.POINTER(i64), dp, dp, dp]),
        "gp_kmatmul": (c_int, [vp, vp, i64, c_int, th, vp, c_int, vp, c_int]),
        "gp_kcross_matmul": (c_int, [vp, vp, i64, vp, i64, c_int, th, vp, c_int, vp, c_int]),
        "gp_pivchol": (c_int, [vp, vp, i64, c_int, th, c_int, vp, vp, ip, vp]),
        "gp_mbcg": (c_int, [vp, vp, i64, c_int, th, vp, c_int, vp, vp, c_int, c_dbl, c_int,
                            c_int, c_int, vp, vp, vp, ip, dp]),
        "gp_lanczos_logquad": (c_int, [vp, vp, vp, c_int, c_int, ip, dp]),
        "gp_bcg": (c_int, [vp, vp, i64, c_int, th, vp, c_int, vp, vp, c_int, c_dbl, c_int, c_int,
                           vp, ip, dp]),
        "gp_mbcg_refine": (c_int, [vp, vp, i64, c_int, th, vp, c_int, vp, vp, c_int, c_dbl,
                                   c_dbl, c_int, c_int, c_int, c_int, vp, ip, ip, dp]),
        "gp_logml_and_grad": (c_int, [vp, vp, i64, c_int, th, vp, c_int, ctypes.c_uint64,
                                      c_int, c_int, c_dbl, c_int, c_int, c_int, dp, dp, dp, dp, st]),
        "gp_model_fit": (c_int, [vp, vp, i64, c_int, th, vp, c_int, c_int, c_int, c_dbl, c_int,
                                 c_int, c_int, ctypes.POINTER(vp), st]),
        "gp_model_free": (None, [vp]),
        "gp_predict": (c_int, [vp, vp, vp, i64, vp, vp, c_int]),
        "gp_model_variance_cache": (c_int, [vp, vp, vp, c_int, ip]),
        "gp_predict_sum": (c_int, [vp, vp, vp, i64, dp, dp, c_int]),
        "gp_subset_indices": (c_int, [i64, i64, ctypes.c_uint64, ctypes.POINTER(i64)]),
        "gp_hyperopt": (c_int, [vp, vp, i64, c_int, vp, i64, ctypes.c_uint64, c_int, c_dbl, c_int, c_int,
                                c_int, c_dbl, c_int, c_int, dp, dp, dp, dp, dp]),
        "gp_train": (c_int, [vp, vp, i64, c_int, vp, i64, ctypes.c_uint64, c_int, c_dbl, c_int, c_int,
                             c_int, c_dbl, c_int, c_int, c_dbl, dp, dp, dp, dp, ctypes.POINTER(vp)]),
        "gp_kmatmul_noalloc": (c_int, [vp, i64, c_int, th, vp, c_int, vp, vp]),
        "gp_server_create": (c_int, [ctypes.POINTER(vp), c_int, i64, c_dbl]),
        "gp_server_add_model": (c_int, [vp, vp, i64, c_int, th, vp, c_int, c_int, c_dbl, c_int,
                                        c_int, c_int, ip]),
        "gp_server_predict": (c_int, [vp, c_int, vp, i64, vp, vp, ctypes.POINTER(ctypes.c_uint64)]),
        "gp_server_molecule": (c_int, [vp, c_int, vp, i64, c_int, vp, i64, dp,
                                       ctypes.POINTER(ctypes.c_uint64)]),
        "gp_server_solve": (c_int, [vp, vp, i64, c_int, th, vp, c_int, c_dbl, c_int, vp,
                                    ctypes.POINTER(ctypes.c_uint64)]),
        "gp_server_wait": (c_int, [vp, ctypes.c_uint64, c_dbl, dp]),
        "gp_server_stats": (c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "gp_server_last_error": (ctypes.c_char_p, [vp]),
        "gp_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
