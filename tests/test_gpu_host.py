"""GP_HOST: the product and training-pass calls with host arrays, through
the C ABI (GPU).  The results match the device-array calls on the same
inputs (the same kernels run on the staged copies; their atomics add in a
varying order, so to FP32 rounding, not bitwise) and the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gp_oracle as go  # noqa: E402
from synth import make_workload  # noqa: E402
from _parity import check_kmv, khat_ref  # noqa: E402


@pytest.fixture(scope="module")
def gp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_09817_gb300 as gp_
    return gp_


@pytest.fixture(scope="module")
def ctx(gp):
    c = gp.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", ["fp32", "split_f16"])
def test_kmatmul_host_arrays(gp, ctx, prec):
    w = make_workload("gp2k", N=1800, d=24)
    V = np.random.default_rng(1).standard_normal((9, w.N)).astype(np.float32)
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    got = gp.gp_kmatmul_host(ctx, w.X, th, V, gp.PRECISIONS[prec])
    dev = gp.gp_kmatmul(ctx, torch.from_numpy(w.X).cuda(), th, torch.from_numpy(V).cuda(),
                        gp.PRECISIONS[prec]).cpu().numpy()
    assert np.max(np.abs(got - dev)) <= 1e-6 * np.max(np.abs(dev))
    ref, aref = khat_ref(w.X, V.T, w.lengthscale, 1.0, w.sigma2)
    check_kmv(got.T, ref, aref, 1e-5 if prec == "fp32" else 2e-5, prec)
    # pinned torch tensors go through the same call
    got2 = gp.gp_kmatmul_host(ctx, torch.from_numpy(w.X).pin_memory(), th,
                              torch.from_numpy(V).pin_memory(), gp.PRECISIONS[prec])
    assert np.max(np.abs(got2 - dev)) <= 1e-6 * np.max(np.abs(dev))


def test_logml_and_grad_host_arrays(gp, ctx):
    w = make_workload("gp2k", N=1000, d=8)
    th = gp.Theta(w.lengthscale, 1.0, w.sigma2)
    kw = dict(n_probes=8, seed=3, k=16, tol=1e-6, max_iter=1000, allow_notconv=True,
              precision=gp.GP_FP32_SPLIT_F16)
    a = gp.gp_logml_and_grad_host(ctx, w.X, th, w.y, **kw)
    b = gp.gp_logml_and_grad(ctx, torch.from_numpy(w.X).cuda(), th, torch.from_numpy(w.y).cuda(), **kw)
    assert abs(a["logml"] - b["logml"]) <= 1e-6 * abs(b["logml"])
    assert np.max(np.abs(a["grad"] - b["grad"])) <= 1e-4 * np.max(np.abs(b["grad"]))


def test_host_flag_only_where_documented(gp, ctx):
    from paper_2109_09817_gb300 import _lib
    w = make_workload("gp2k", N=100, d=4)
    X = torch.from_numpy(w.X).cuda()
    B = torch.from_numpy(w.y[None, :].copy()).cuda()
    with pytest.raises(gp.GPError) as e:
        gp.gp_mbcg(ctx, X, gp.Theta(w.lengthscale), None, B, precision=gp.GP_FP32_PLAIN | _lib.GP_HOST)
    assert e.value.code == gp.GP_EINVAL
