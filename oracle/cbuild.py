"""Build and load the C part of the oracle (test infrastructure only)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmv_oracle.c")
_LIB = os.path.join(_HERE, "_kmv_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile kmv_oracle.c into a shared object next to it."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def load_c():
    """Load the compiled oracle, building it first if needed."""
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    lp = ctypes.POINTER(ctypes.c_int64)
    i64 = ctypes.c_int64
    lib.oracle_khat_rows.argtypes = [fp, i64, ctypes.c_int, dp, ctypes.c_double,
                                     ctypes.c_double, dp, ctypes.c_int, lp, i64,
                                     dp]
    lib.oracle_khat_rows.restype = None
    lib.oracle_kcross_rows.argtypes = [fp, i64, fp, i64, ctypes.c_int, dp,
                                       ctypes.c_double, dp, ctypes.c_int, dp]
    lib.oracle_kcross_rows.restype = None
    lib.oracle_kernel_block.argtypes = [fp, i64, fp, i64, ctypes.c_int, dp,
                                        ctypes.c_double, dp]
    lib.oracle_kernel_block.restype = None
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def c_khat_rows(X, lengthscale, s, sigma2, V, rows):
    """(K(X,X)+sigma2 I)[rows, :] @ V in FP64, streamed (never stores K)."""
    lib = load_c()
    X = np.ascontiguousarray(X, dtype=np.float32)
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    ell = np.ascontiguousarray(lengthscale, dtype=np.float64)
    N, d = X.shape
    t = V.shape[1]
    out = np.zeros((rows.shape[0], t), dtype=np.float64)
    lib.oracle_khat_rows(_p(X, ctypes.c_float), N, d, _p(ell, ctypes.c_double),
                         float(s), float(sigma2), _p(V, ctypes.c_double), t,
                         _p(rows, ctypes.c_int64), rows.shape[0],
                         _p(out, ctypes.c_double))
    return out


def c_kcross(Xp, X, lengthscale, s, V):
    """K(X', X) @ V in FP64, streamed."""
    lib = load_c()
    Xp = np.ascontiguousarray(Xp, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    V = np.ascontiguousarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    ell = np.ascontiguousarray(lengthscale, dtype=np.float64)
    M, d = Xp.shape
    N = X.shape[0]
    t = V.shape[1]
    out = np.zeros((M, t), dtype=np.float64)
    lib.oracle_kcross_rows(_p(Xp, ctypes.c_float), M, _p(X, ctypes.c_float), N,
                           d, _p(ell, ctypes.c_double), float(s),
                           _p(V, ctypes.c_double), t, _p(out, ctypes.c_double))
    return out


def c_kernel_block(X1, X2, lengthscale, s):
    """Dense K(X1, X2) in FP64 by direct differences."""
    lib = load_c()
    X1 = np.ascontiguousarray(X1, dtype=np.float32)
    X2 = np.ascontiguousarray(X2, dtype=np.float32)
    ell = np.ascontiguousarray(lengthscale, dtype=np.float64)
    n1, d = X1.shape
    n2 = X2.shape[0]
    out = np.zeros((n1, n2), dtype=np.float64)
    lib.oracle_kernel_block(_p(X1, ctypes.c_float), n1, _p(X2, ctypes.c_float),
                            n2, d, _p(ell, ctypes.c_double), float(s),
                            _p(out, ctypes.c_double))
    return out


def c_threads() -> int:
    return int(load_c().oracle_num_threads())
