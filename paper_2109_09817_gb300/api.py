"""Python binding of libgp with the C ABI's names (argument marshalling only).

Every step of the path runs in libgp's CUDA kernels; this module only turns
torch device tensors into pointers and sizes and raises on error codes.
PyTorch supplies device memory and the stream.

Layouts (as in include/gp.h): features X are (N, d) float32 row-major; a
block of t vectors of length N is a (t, N) float32 tensor (row c = vector c).
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import (GP_FP32_SPLIT_F16, GP_FP32_PLAIN, GP_FP32_SPLIT_TF32,  # noqa: F401
                   GP_TF32, GP_VAR_EXACT, GP_VAR_NONE, GP_VAR_CACHED, GP_OK, GP_ENOTCONV,
                   GP_EBREAKDOWN, GP_EINVAL, GP_PC_SIGMA, GP_PC_RESID, ERROR_NAMES,
                   GP_STOP_RECURRENCE, GP_STOP_TRUE)

PRECISIONS = {"fp32": GP_FP32_PLAIN, "split_tf32": GP_FP32_SPLIT_TF32,
              "split_f16": GP_FP32_SPLIT_F16, "tf32": GP_TF32}


class GPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


@dataclasses.dataclass
class Theta:
    """Hyperparameters (natural, positive): lengthscale (d,), s, sigma^2."""
    lengthscale: np.ndarray
    outputscale: float = 1.0
    sigma2: float = 1e-4

    def as_c(self):
        ell = np.ascontiguousarray(self.lengthscale, dtype=np.float64)
        th = _lib.GpTheta(ell.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                          float(self.outputscale), float(self.sigma2))
        return th, ell  # keep `ell` alive for the call


class Context:
    """A libgp context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        self.lib = _lib.load()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        rc = self.lib.gp_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if rc != GP_OK:
            raise GPError(rc, "gp_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def check(self, rc: int, allow=()):
        if rc != GP_OK and rc not in allow:
            raise GPError(rc, self.lib.gp_last_error(self.h).decode())
        return rc

    @property
    def launches(self) -> int:
        return int(self.lib.gp_launch_count(self.h))

    def sync(self):
        self.check(self.lib.gp_sync(self.h))

    def set_option(self, option: int, value: int):
        """gp_set_option (e.g. _lib.GP_OPT_SYMMETRIC_KMV, 0 or 1)."""
        self.check(self.lib.gp_set_option(self.h, option, value))


def _p(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dev(ctx: Context, t: torch.Tensor, dtype, name: str):
    if not (t.is_cuda and t.device.index == ctx.device):
        raise ValueError(f"{name} must be on cuda:{ctx.device}")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _block(ctx, V, N, name):
    if V.dim() == 1:
        V = V.view(1, -1)
    _dev(ctx, V, torch.float32, name)
    if V.shape[1] != N:
        raise ValueError(f"{name} must be (t, {N})")
    return V


def gp_kmatmul(ctx: Context, X: torch.Tensor, theta: Theta, V: torch.Tensor,
               precision: int = GP_FP32_PLAIN, out: Optional[torch.Tensor] = None):
    """(K(X,X) + sigma^2 I) V; V and the result are (t, N)."""
    _dev(ctx, X, torch.float32, "X")
    N, d = X.shape
    V = _block(ctx, V, N, "V")
    out = torch.empty_like(V) if out is None else out
    th, keep = theta.as_c()
    ctx.check(ctx.lib.gp_kmatmul(ctx.h, _p(X), N, d, ctypes.byref(th), _p(V), V.shape[0],
                                 _p(out), precision))
    return out


def _host(a, name):
    """A host array argument (numpy, or a CPU torch tensor, e.g. pinned):
    float32, C-contiguous; returns (pointer, keep-alive)."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 host tensor")
        return ctypes.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a.ctypes.data_as(ctypes.c_void_p), a


def gp_kmatmul_host(ctx: Context, X, theta: Theta, V, precision: int = GP_FP32_PLAIN):
    """gp_kmatmul with GP_HOST: X (N, d) and V (t, N) in host memory; returns
    the (t, N) result as a numpy array (the call synchronises)."""
    xp, xk = _host(X, "X")
    N, d = xk.shape
    V = V.reshape(1, -1) if V.ndim == 1 else V
    vp, vk = _host(V, "V")
    t = vk.shape[0]
    out = np.empty((t, N), dtype=np.float32)
    th, keep = theta.as_c()
    ctx.check(ctx.lib.gp_kmatmul(ctx.h, xp, N, d, ctypes.byref(th), vp, t,
                                 out.ctypes.data_as(ctypes.c_void_p), precision | _lib.GP_HOST))
    return out


def gp_kcross_matmul(ctx: Context, Xp: torch.Tensor, X: torch.Tensor, theta: Theta,
                     V: torch.Tensor, precision: int = GP_FP32_PLAIN):
    """K(X', X) V; V is (t, N), the result (t, M)."""
    _dev(ctx, X, torch.float32, "X")
    _dev(ctx, Xp, torch.float32, "Xp")
    N, d = X.shape
    M = Xp.shape[0]
    V = _block(ctx, V, N, "V")
    out = torch.empty((V.shape[0], M), dtype=torch.float32, device=X.device)
    th, keep = theta.as_c()
    ctx.check(ctx.lib.gp_kcross_matmul(ctx.h, _p(Xp), M, _p(X), N, d, ctypes.byref(th),
                                       _p(V), V.shape[0], _p(out), precision))
    return out


def gp_pivchol(ctx: Context, X: torch.Tensor, theta: Theta, k: int, want_resid: bool = False):
    """Rank-k pivoted Cholesky (FP64).  Returns (L (k, N) float64, piv (k,),
    rank), plus the residual diagonal (N,) float64 when ``want_resid``."""
    _dev(ctx, X, torch.float32, "X")
    N, d = X.shape
    L = torch.empty((max(k, 1), N), dtype=torch.float64, device=X.device)
    piv = torch.empty(max(k, 1), dtype=torch.int64, device=X.device)
    res = torch.empty(N, dtype=torch.float64, device=X.device) if want_resid else None
    rank = ctypes.c_int(0)
    th, keep = theta.as_c()
    ctx.check(ctx.lib.gp_pivchol(ctx.h, _p(X), N, d, ctypes.byref(th), k, _p(L), _p(piv),
                                 ctypes.byref(rank), _p(res)))
    if want_resid:
        return L[:k], piv[:k], rank.value, res
    return L[:k], piv[:k], rank.value


def gp_mbcg(ctx: Context, X: torch.Tensor, theta: Theta, L: Optional[torch.Tensor],
            B: torch.Tensor, tol: float = 1e-6, max_iter: int = 1000,
            precision: int = GP_FP32_PLAIN, allow_notconv: bool = True,
            resid: Optional[torch.Tensor] = None, stop: int = GP_STOP_RECURRENCE):
    """Batched PCG on K-hat Omega = B; returns dict(Omega, alpha, beta, iters,
    relres, rc).  L: (k, N) float64 from gp_pivchol or None; resid: its
    residual diagonal for the GP_PC_RESID form, or None for P = L L^T + sigma^2 I.
    stop: GP_STOP_RECURRENCE or GP_STOP_TRUE (relres then holds the measured
    true residuals)."""
    _dev(ctx, X, torch.float32, "X")
    N, d = X.shape
    B = _block(ctx, B, N, "B")
    t = B.shape[0]
    k = 0 if L is None else L.shape[0]
    if L is not None:
        _dev(ctx, L, torch.float64, "L")
    Om = torch.empty_like(B)
    ah = torch.zeros((max_iter, t), dtype=torch.float64, device=X.device)
    bh = torch.zeros((max_iter, t), dtype=torch.float64, device=X.device)
    iters = (ctypes.c_int * t)()
    rr = (ctypes.c_double * t)()
    th, keep = theta.as_c()
    allow = (GP_ENOTCONV,) if allow_notconv else ()
    if resid is not None:
        _dev(ctx, resid, torch.float64, "resid")
    rc = ctx.check(ctx.lib.gp_mbcg(ctx.h, _p(X), N, d, ctypes.byref(th), _p(L), k, _p(resid), _p(B), t,
                                   tol, max_iter, stop, precision, _p(Om), _p(ah), _p(bh), iters, rr),
                   allow=allow)
    return dict(Omega=Om, alpha=ah, beta=bh, iters=np.array(iters[:]),
                relres=np.array(rr[:]), rc=rc)


def gp_lanczos_logquad(ctx: Context, alpha: torch.Tensor, beta: torch.Tensor, iters) -> np.ndarray:
    """e1^T log(T_c) e1 for each column c of mBCG's coefficient histories
    (alpha, beta: (max_iter, t) float64 on the device, as gp_mbcg returns
    them; iters: t step counts).  Returns a float64 array of t."""
    _dev(ctx, alpha, torch.float64, "alpha")
    _dev(ctx, beta, torch.float64, "beta")
    if alpha.shape != beta.shape or alpha.dim() != 2:
        raise ValueError("alpha and beta must be (max_iter, t) arrays of one shape")
    max_iter, t = alpha.shape
    it = np.asarray(iters, dtype=np.int64).reshape(-1)
    if it.shape[0] != t:
        raise ValueError("iters must hold one count per column")
    ci = (ctypes.c_int * t)(*[int(v) for v in it])
    q = (ctypes.c_double * t)()
    ctx.check(ctx.lib.gp_lanczos_logquad(ctx.h, _p(alpha), _p(beta), t, max_iter, ci, q))
    return np.array(q[:])


def gp_bcg(ctx: Context, X: torch.Tensor, theta: Theta, L: Optional[torch.Tensor],
           B: torch.Tensor, tol: float = 1e-4, max_iter: int = 1000,
           precision: int = GP_FP32_SPLIT_TF32, resid: Optional[torch.Tensor] = None,
           allow_notconv: bool = False):
    """AltBBMM block CG on S^T K-hat S (t <= 32 right-hand sides); returns
    dict(Omega, iters, relres, rc)."""
    _dev(ctx, X, torch.float32, "X")
    N, d = X.shape
    B = _block(ctx, B, N, "B")
    t = B.shape[0]
    k = 0 if L is None else L.shape[0]
    if L is not None:
        _dev(ctx, L, torch.float64, "L")
    if resid is not None:
        _dev(ctx, resid, torch.float64, "resid")
    Om = torch.empty_like(B)
    it = ctypes.c_int(0)
    rr = (ctypes.c_double * t)()
    th, keep = theta.as_c()
    allow = (GP_ENOTCONV,) if allow_notconv else ()
    rc = ctx.check(ctx.lib.gp_bcg(ctx.h, _p(X), N, d, ctypes.byref(th), _p(L), k, _p(resid), _p(B), t,
                                  tol, max_iter, precision, _p(Om), ctypes.byref(it), rr), allow=allow)
    return dict(Omega=Om, iters=it.value, relres=np.array(rr[:]), rc=rc)


def gp_mbcg_refine(ctx: Context, X: torch.Tensor, theta: Theta, L: Optional[torch.Tensor],
                   B: torch.Tensor, tol: float = 1e-4, inner_tol: float = 1e-2,
                   max_outer: int = 10, max_iter: int = 1000,
                   inner_precision: int = GP_TF32, outer_precision: int = GP_FP32_SPLIT_TF32,
                   resid: Optional[torch.Tensor] = None, allow_notconv: bool = False):
    """Mixed-precision iterative refinement of K-hat Omega = B; returns
    dict(Omega, outer, inner, relres, rc)."""
    _dev(ctx, X, torch.float32, "X")
    N, d = X.shape
    B = _block(ctx, B, N, "B")
    t = B.shape[0]
    k = 0 if L is None else L.shape[0]
    if L is not None:
        _dev(ctx, L, torch.float64, "L")
    if resid is not None:
        _dev(ctx, resid, torch.float64, "resid")
    Om = torch.empty_like(B)
    outer = ctypes.c_int(0)
    inner = ctypes.c_int(0)
    rr = (ctypes.c_double * t)()
    th, keep = theta.as_c()
    allow = (GP_ENOTCONV,) if allow_notconv else ()
    rc = ctx.check(ctx.lib.gp_mbcg_refine(ctx.h, _p(X), N, d, ctypes.byref(th), _p(L), k, _p(resid),
                                          _p(B), t, tol, inner_tol, max_outer, max_iter,
                                          inner_precision, outer_precision, _p(Om),
                                          ctypes.byref(outer), ctypes.byref(inner), rr),
                   allow=allow)
    return dict(Omega=Om, outer=outer.value, inner=inner.value, relres=np.array(rr[:]), rc=rc)


def gp_logml_and_grad(ctx: Context, X: torch.Tensor, theta: Theta, y: torch.Tensor,
                      n_probes: int = 15, seed: int = 0, k: int = 32, tol: float = 1e-6,
                      max_iter: int = 1000, precision: int = GP_FP32_PLAIN,
                      want_grad: bool = True, allow_notconv: bool = False,
                      precond: int = GP_PC_SIGMA, stop: int = GP_STOP_RECURRENCE):
    """Eq. (ll) and its gradient (natural parameters l_1..l_d, s, sigma^2).
    stop applies to y's column (GP_STOP_TRUE: its true residual is verified)."""
    _dev(ctx, X, torch.float32, "X")
    _dev(ctx, y, torch.float32, "y")
    N, d = X.shape
    logml = ctypes.c_double()
    logdet = ctypes.c_double()
    se = ctypes.c_double()
    grad = (ctypes.c_double * (d + 2))()
    stats = _lib.GpStats()
    th, keep = theta.as_c()
    allow = (GP_ENOTCONV,) if allow_notconv else ()
    rc = ctx.check(ctx.lib.gp_logml_and_grad(
        ctx.h, _p(X), N, d, ctypes.byref(th), _p(y), n_probes, ctypes.c_uint64(seed), k, precond, tol,
        max_iter, stop, precision, ctypes.byref(logml), ctypes.byref(logdet),
        grad if want_grad else None, ctypes.byref(se), ctypes.byref(stats)), allow=allow)
    return dict(logml=logml.value, logdet=logdet.value, logdet_stderr=se.value,
                grad=np.array(grad[:]) if want_grad else None, stats=stats.as_dict(), rc=rc)


def gp_logml_and_grad_host(ctx: Context, X, theta: Theta, y, n_probes: int = 15, seed: int = 0,
                           k: int = 32, tol: float = 1e-6, max_iter: int = 1000,
                           precision: int = GP_FP32_PLAIN, want_grad: bool = True,
                           allow_notconv: bool = False, precond: int = GP_PC_SIGMA,
                           stop: int = GP_STOP_RECURRENCE):
    """gp_logml_and_grad with GP_HOST: X (N, d) and y (N,) in host memory."""
    xp, xk = _host(X, "X")
    yp, yk = _host(y, "y")
    N, d = xk.shape
    logml = ctypes.c_double()
    logdet = ctypes.c_double()
    se = ctypes.c_double()
    grad = (ctypes.c_double * (d + 2))()
    stats = _lib.GpStats()
    th, keep = theta.as_c()
    allow = (GP_ENOTCONV,) if allow_notconv else ()
    rc = ctx.check(ctx.lib.gp_logml_and_grad(
        ctx.h, xp, N, d, ctypes.byref(th), yp, n_probes, ctypes.c_uint64(seed), k, precond, tol,
        max_iter, stop, precision | _lib.GP_HOST, ctypes.byref(logml), ctypes.byref(logdet),
        grad if want_grad else None, ctypes.byref(se), ctypes.byref(stats)), allow=allow)
    return dict(logml=logml.value, logdet=logdet.value, logdet_stderr=se.value,
                grad=np.array(grad[:]) if want_grad else None, stats=stats.as_dict(), rc=rc)


class Model:
    """A fitted model resident on the device (gp_model_fit / gp_predict)."""

    def __init__(self, ctx: Context, X: torch.Tensor, theta: Theta, y: torch.Tensor,
                 k: int = 32, tol: float = 1e-6, max_iter: int = 1000,
                 precision: int = GP_FP32_PLAIN, precond: int = GP_PC_SIGMA, block: int = 1,
                 stop: int = GP_STOP_RECURRENCE):
        _dev(ctx, X, torch.float32, "X")
        _dev(ctx, y, torch.float32, "y")
        self.ctx = ctx
        N, d = X.shape
        self.N, self.d = N, d
        h = ctypes.c_void_p()
        stats = _lib.GpStats()
        th, keep = theta.as_c()
        ctx.check(ctx.lib.gp_model_fit(ctx.h, _p(X), N, d, ctypes.byref(th), _p(y), k, precond, block, tol,
                                       max_iter, stop, precision, ctypes.byref(h), ctypes.byref(stats)))
        self.h = h
        self.stats = stats.as_dict()

    @classmethod
    def _from_handle(cls, ctx: Context, h, N: int, d: int):
        m = cls.__new__(cls)
        m.ctx, m.h, m.N, m.d, m.stats = ctx, h, N, d, None
        return m

    def free(self):
        if getattr(self, "h", None):
            self.ctx.lib.gp_model_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def gp_model_fit(ctx: Context, X, theta, y, k=32, tol=1e-6, max_iter=1000,
                 precision=GP_FP32_PLAIN, precond=GP_PC_SIGMA, block=1,
                 stop=GP_STOP_RECURRENCE) -> Model:
    return Model(ctx, X, theta, y, k, tol, max_iter, precision, precond, block, stop)


def gp_predict(ctx: Context, model: Model, Xp: torch.Tensor, var_mode: int = GP_VAR_NONE):
    """Predictive mean (and latent variance with GP_VAR_EXACT or
    GP_VAR_CACHED), Eq. (pred)."""
    _dev(ctx, Xp, torch.float32, "Xp")
    M = Xp.shape[0]
    mean = torch.empty(M, dtype=torch.float32, device=Xp.device)
    var = torch.empty(M, dtype=torch.float32, device=Xp.device) if var_mode else None
    ctx.check(ctx.lib.gp_predict(ctx.h, model.h, _p(Xp), M, _p(mean), _p(var), var_mode))
    return mean, var


def gp_model_variance_cache(ctx: Context, model: Model, rank: int,
                            b: Optional[torch.Tensor] = None) -> int:
    """Build the model's rank-`rank` Lanczos variance cache from the start
    vector b (device, N floats; None = K-hat a); returns the steps taken."""
    if b is not None:
        _dev(ctx, b, torch.float32, "b")
    out = ctypes.c_int(0)
    ctx.check(ctx.lib.gp_model_variance_cache(ctx.h, model.h, _p(b), rank, ctypes.byref(out)))
    return out.value


def gp_predict_sum(ctx: Context, model: Model, Xp: torch.Tensor, var_mode: int = GP_VAR_NONE):
    """(sum of the predictive means over the rows of Xp, variance of that sum
    or None), Sec. 2.1's per-molecule energy."""
    _dev(ctx, Xp, torch.float32, "Xp")
    ms = ctypes.c_double()
    vs = ctypes.c_double()
    ctx.check(ctx.lib.gp_predict_sum(ctx.h, model.h, _p(Xp), Xp.shape[0], ctypes.byref(ms),
                                     ctypes.byref(vs) if var_mode else None, var_mode))
    return ms.value, (vs.value if var_mode else None)


def gp_subset_indices(N: int, M: int, seed: int) -> np.ndarray:
    """M distinct sorted row indices of 0..N-1 (seeded partial shuffle)."""
    lib = _lib.load()
    idx = np.empty(M, dtype=np.int64)
    rc = lib.gp_subset_indices(N, M, ctypes.c_uint64(seed),
                               idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != GP_OK:
        raise GPError(rc, "gp_subset_indices: bad arguments")
    return idx


def _hyper_args(theta: Theta, d: int):
    ell = np.ascontiguousarray(theta.lengthscale, dtype=np.float64).copy()
    if ell.shape != (d,):
        raise ValueError(f"lengthscale must have {d} entries")
    return ell, ctypes.c_double(theta.outputscale), ctypes.c_double(theta.sigma2)


def gp_hyperopt(ctx: Context, X: torch.Tensor, y: torch.Tensor, theta0: Theta, subset: int,
                seed: int = 0, steps: int = 10, lr: float = 0.05, n_probes: int = 15, k: int = 32,
                precond: int = GP_PC_RESID, tol: float = 1e-4, max_iter: int = 1000,
                precision: int = GP_FP32_SPLIT_F16):
    """Adam on log theta over a seeded random subset (Sec. 4); returns
    (theta, logml history of steps + 1 values, gradient at theta)."""
    _dev(ctx, X, torch.float32, "X")
    _dev(ctx, y, torch.float32, "y")
    N, d = X.shape
    ell, s, s2 = _hyper_args(theta0, d)
    hist = np.zeros(steps + 1)
    grad = np.zeros(d + 2)
    dp = ctypes.POINTER(ctypes.c_double)
    ctx.check(ctx.lib.gp_hyperopt(ctx.h, _p(X), N, d, _p(y), subset, ctypes.c_uint64(seed), steps, lr,
                                  n_probes, k, precond, tol, max_iter, precision, ell.ctypes.data_as(dp),
                                  ctypes.byref(s), ctypes.byref(s2), hist.ctypes.data_as(dp),
                                  grad.ctypes.data_as(dp)))
    return Theta(ell, s.value, s2.value), hist, grad


def gp_train(ctx: Context, X: torch.Tensor, y: torch.Tensor, theta0: Theta, subset: int,
             seed: int = 0, steps: int = 10, lr: float = 0.05, n_probes: int = 15, k: int = 32,
             precond: int = GP_PC_RESID, tol: float = 1e-4, max_iter: int = 1000,
             precision: int = GP_FP32_SPLIT_F16, sigma2_add: float = 1e-5):
    """gp_hyperopt, then the full fit with sigma^2 + sigma2_add; returns
    (Model, optimised theta, logml history)."""
    _dev(ctx, X, torch.float32, "X")
    _dev(ctx, y, torch.float32, "y")
    N, d = X.shape
    ell, s, s2 = _hyper_args(theta0, d)
    hist = np.zeros(steps + 1)
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    ctx.check(ctx.lib.gp_train(ctx.h, _p(X), N, d, _p(y), subset, ctypes.c_uint64(seed), steps, lr,
                               n_probes, k, precond, tol, max_iter, precision, sigma2_add,
                               ell.ctypes.data_as(dp), ctypes.byref(s), ctypes.byref(s2),
                               hist.ctypes.data_as(dp), ctypes.byref(h)))
    return Model._from_handle(ctx, h, N, d), Theta(ell, s.value, s2.value), hist


class Server:
    """Continuous-batching request loop over resident models (gp_server_*).

    predict()/solve() take host numpy arrays and return a ticket; wait()
    returns (status, latency_ms).  The arrays are kept alive here until their
    request has been waited for."""

    def __init__(self, device: int = 0, max_batch_rows: int = 65536, reserve_bytes: float = 0.0):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        rc = self.lib.gp_server_create(ctypes.byref(h), device, max_batch_rows, reserve_bytes)
        if rc != GP_OK:
            raise GPError(rc, "gp_server_create failed")
        self.h = h
        self.device = device
        self._keep = {}

    def check(self, rc: int):
        if rc != GP_OK:
            raise GPError(rc, self.lib.gp_server_last_error(self.h).decode())
        return rc

    def add_model(self, X: torch.Tensor, theta: Theta, y: torch.Tensor, k: int = 32,
                  precond: int = GP_PC_RESID, tol: float = 1e-4, max_iter: int = 1000,
                  precision: int = GP_FP32_SPLIT_TF32, var_rank: int = 0) -> int:
        if not (X.is_cuda and y.is_cuda):
            raise ValueError("add_model takes device tensors")
        N, d = X.shape
        mid = ctypes.c_int(-1)
        th, keep = theta.as_c()
        self.check(self.lib.gp_server_add_model(self.h, _p(X), N, d, ctypes.byref(th), _p(y), k,
                                                precond, tol, max_iter, precision, var_rank,
                                                ctypes.byref(mid)))
        return mid.value

    def predict(self, model_id: int, Xp: np.ndarray, want_var: bool = False):
        """Queue a predict request; wait() returns the means, or (means,
        variances) with want_var."""
        Xp = np.ascontiguousarray(Xp, dtype=np.float32)
        mean = np.empty(Xp.shape[0], dtype=np.float32)
        var = np.empty(Xp.shape[0], dtype=np.float32) if want_var else None
        tk = ctypes.c_uint64()
        self.check(self.lib.gp_server_predict(self.h, model_id, Xp.ctypes.data_as(ctypes.c_void_p),
                                              Xp.shape[0], mean.ctypes.data_as(ctypes.c_void_p),
                                              var.ctypes.data_as(ctypes.c_void_p) if want_var else None,
                                              ctypes.byref(tk)))
        self._keep[tk.value] = (Xp, (mean, var) if want_var else mean)
        return tk.value

    def molecule(self, diag_id: int, Xd: np.ndarray, off_id: int, Xo: np.ndarray):
        """Queue a molecule request; wait() returns (E_corr mean, variance)."""
        Xd = np.ascontiguousarray(Xd, dtype=np.float32)
        Xo = np.ascontiguousarray(Xo, dtype=np.float32)
        energy = np.zeros(2, dtype=np.float64)
        tk = ctypes.c_uint64()
        self.check(self.lib.gp_server_molecule(
            self.h, diag_id, Xd.ctypes.data_as(ctypes.c_void_p), Xd.shape[0], off_id,
            Xo.ctypes.data_as(ctypes.c_void_p) if Xo.shape[0] else None, Xo.shape[0],
            energy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(tk)))
        self._keep[tk.value] = (Xd, energy, Xo)
        return tk.value

    def solve(self, X: np.ndarray, theta: Theta, y: np.ndarray, k: int = 32, tol: float = 1e-4,
              max_iter: int = 1000):
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        alpha = np.empty(X.shape[0], dtype=np.float32)
        th, ell = theta.as_c()
        tk = ctypes.c_uint64()
        self.check(self.lib.gp_server_solve(self.h, X.ctypes.data_as(ctypes.c_void_p), X.shape[0],
                                            X.shape[1], ctypes.byref(th),
                                            y.ctypes.data_as(ctypes.c_void_p), k, tol, max_iter,
                                            alpha.ctypes.data_as(ctypes.c_void_p),
                                            ctypes.byref(tk)))
        self._keep[tk.value] = (X, y, alpha, ell)
        return tk.value

    def wait(self, ticket: int, timeout_s: float = 600.0):
        """Returns (status, latency_ms, result array)."""
        lat = ctypes.c_double(0.0)
        rc = self.lib.gp_server_wait(self.h, ctypes.c_uint64(ticket), timeout_s, ctypes.byref(lat))
        if rc == _lib.GP_ETIMEOUT:
            return rc, None, None
        kept = self._keep.pop(ticket, None)
        out = None if kept is None else kept[1] if len(kept) <= 3 else kept[2]
        if isinstance(out, np.ndarray) and out.dtype == np.float64 and out.shape == (2,):
            out = (float(out[0]), float(out[1]))
        return rc, lat.value, out

    def stats(self):
        b, p = ctypes.c_int64(), ctypes.c_int64()
        self.check(self.lib.gp_server_stats(self.h, ctypes.byref(b), ctypes.byref(p)))
        return {"batches": b.value, "predicted": p.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.gp_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
