"""gp_kmatmul_noalloc against the FP64 oracle and against gp_kmatmul,
through the C ABI (GPU).

gp_kmatmul_noalloc serves callers that may not allocate device memory (a
process whose memory belongs to another framework's pool, a real-time loop
that may not call cudaMalloc/cudaFree): its scratch lives in a fixed device
array inside the library.  This file is collected last so that a run which
stops at the first failure has already run every other test; it passes both
alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


def test_noalloc_matches_kmatmul_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_09817_gb300 as gp
    from paper_2109_09817_gb300 import _lib
    from synth import make_workload
    from _parity import check_kmv, khat_ref

    lib = _lib.load()
    ctx = gp.Context(0)
    stream = torch.cuda.current_stream()
    cases = [make_workload("gp2k", N=3000, d=32, seed=21), make_workload("gp2k", N=1500, d=20, seed=22)]
    for w, t in zip(cases, (17, 5)):   # two calls in a row, different shapes
        X = torch.from_numpy(w.X).cuda()
        V = torch.randn(t, w.N, device="cuda", generator=torch.Generator("cuda").manual_seed(t))
        theta = gp.Theta(w.lengthscale, 0.9, 1e-3)
        ref = gp.gp_kmatmul(ctx, X, theta, V).cpu().numpy()
        Vh = V.cpu().numpy().T.astype(np.float64)
        oref, aref = khat_ref(w.X, Vh, w.lengthscale, 0.9, 1e-3)
        out = torch.full_like(V, float("nan"))
        th, keep = theta.as_c()
        rc = lib.gp_kmatmul_noalloc(ctypes.c_void_p(X.data_ptr()), w.N, w.d, ctypes.byref(th),
                                    ctypes.c_void_p(V.data_ptr()), t, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        # the oracle's FP64 product: the FP32 form's tolerance, column by
        # column and entry by entry
        check_kmv(got.T, oref, aref, 1e-5, "fp32")
        assert _relerr(got, ref) <= 1e-5
    # sizes beyond the fixed scratch are rejected before any work
    big = torch.zeros((70000, 4), device="cuda")
    Vb = torch.zeros((1, 70000), device="cuda")
    th, keep = gp.Theta(np.ones(4)).as_c()
    rc = lib.gp_kmatmul_noalloc(ctypes.c_void_p(big.data_ptr()), 70000, 4, ctypes.byref(th),
                                ctypes.c_void_p(Vb.data_ptr()), 1, ctypes.c_void_p(Vb.data_ptr() + 0),
                                ctypes.c_void_p(stream.cuda_stream))
    assert rc == _lib.GP_EINVAL
    ctx.close()
