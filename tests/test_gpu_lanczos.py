"""Lanczos quadrature on the device (gp_lanczos_logquad) against the oracle.

Sec. 3.2: the log-determinant term of Eq. ll is estimated from mBCG's
coefficients through e1^T log(T_c) e1 of each column's Lanczos tridiagonal.
The device evaluates it by a trapezoid rule on an integral representation;
the oracle (oracle.gp_oracle.quadrature_log) by the eigendecomposition of the
same T_c.  Parity is per column, to 1e-10 absolute (or relative above 1).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import gp_oracle as go  # noqa: E402
from synth import make_workload  # noqa: E402

TOL = 1e-10


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


def _ref(al, be, iters):
    out = []
    for c, m in enumerate(iters):
        m = int(m)
        out.append(go.quadrature_log(*go.lanczos_tridiagonal(al[:m, c], be[:m, c], m)) if m > 0 else 0.0)
    return np.array(out)


def _check(q, ref):
    err = np.abs(q - ref)
    bound = TOL * np.maximum(1.0, np.abs(ref))
    assert np.all(err <= bound), (err.max(), q, ref)


def test_random_histories_match_oracle(gp, ctx):
    # any positive alpha and non-negative beta give a positive definite T;
    # lengths from the empty and 1 x 1 cases to several thousand steps
    rng = np.random.default_rng(41)
    max_iter = 3000
    iters = np.array([0, 1, 2, 17, 64, 500, 1499, 3000])
    t = len(iters)
    al = np.exp(rng.uniform(-4.0, 3.0, (max_iter, t)))
    be = np.exp(rng.uniform(-6.0, 0.5, (max_iter, t)))
    q = gp.gp_lanczos_logquad(ctx, torch.from_numpy(al).cuda(), torch.from_numpy(be).cuda(), iters)
    assert q[0] == 0.0
    assert abs(q[1] - np.log(1.0 / al[0, 1])) < TOL * max(1.0, abs(np.log(al[0, 1])))
    _check(q, _ref(al, be, iters))


def test_wide_spectrum_matches_oracle(gp, ctx):
    # eigenvalues over ten decades
    rng = np.random.default_rng(42)
    max_iter = 1200
    iters = np.array([1200, 900, 300])
    al = np.exp(rng.uniform(-12.0, 8.0, (max_iter, 3)))
    be = np.exp(rng.uniform(-10.0, 2.0, (max_iter, 3)))
    q = gp.gp_lanczos_logquad(ctx, torch.from_numpy(al).cuda(), torch.from_numpy(be).cuda(), iters)
    _check(q, _ref(al, be, iters))


def test_mbcg_coefficients_match_oracle(gp, ctx):
    # the coefficients a preconditioned solve actually produces
    w = make_workload("gp2k", N=1024, d=8)
    theta = gp.Theta(w.lengthscale, w.outputscale, w.sigma2)
    X = torch.from_numpy(w.X).cuda()
    rng = np.random.default_rng(5)
    Z = torch.from_numpy(rng.choice([-1.0, 1.0], (6, w.N)).astype(np.float32)).cuda()
    L, piv, _ = gp.gp_pivchol(ctx, X, theta, 16)
    r = gp.gp_mbcg(ctx, X, theta, L, Z, tol=1e-8, max_iter=800)
    q = gp.gp_lanczos_logquad(ctx, r["alpha"], r["beta"], r["iters"])
    _check(q, _ref(r["alpha"].cpu().numpy(), r["beta"].cpu().numpy(), r["iters"]))


def test_indefinite_tridiagonal_is_reported(gp, ctx):
    # a negative alpha makes T_00 negative: GP_EBREAKDOWN, not a value
    al = np.ones((8, 2))
    be = np.full((8, 2), 0.25)
    al[0, 1] = -1.0
    with pytest.raises(gp.GPError) as e:
        gp.gp_lanczos_logquad(ctx, torch.from_numpy(al).cuda(), torch.from_numpy(be).cuda(), [8, 8])
    assert e.value.code == gp.api.GP_EBREAKDOWN
    # bad step counts are rejected before any work
    with pytest.raises(gp.GPError) as e:
        gp.gp_lanczos_logquad(ctx, torch.from_numpy(al).cuda(), torch.from_numpy(be).cuda(), [9, 8])
    assert e.value.code == gp.GP_EINVAL
