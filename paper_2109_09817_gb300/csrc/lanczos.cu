// Lanczos quadrature of the log-determinant (A8), FP64.
//
// arXiv 2109.09817 Sec. 3.2: mBCG's coefficients estimate the marginal
// likelihood (Eq. ll) through Lanczos tridiagonals.  For column c with
// coefficients alpha_j, beta_j over its first m steps, the PCG/Lanczos
// relation gives T (m x m):
//   T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T_{j,j+1} = sqrt(beta_j)/alpha_j,
// and e1^T log(T) e1 = sum_i q_{0i}^2 log(lambda_i) over T's eigenpairs.
// The eigenpairs come from the implicit symmetric tridiagonal QR iteration
// with Wilkinson shifts (Golub & Van Loan, "Matrix Computations", Sec. 8.3),
// carrying only the first row q_0 of the eigenvector matrix.  One block per
// column; T and q_0 live in shared memory.
#include <cmath>

#include "gp_internal.cuh"

namespace gp {
namespace {

// One implicit QR sweep with a Wilkinson shift on the unreduced block
// [lo, hi] of (a, b); q is the first eigenvector row, updated as Q <- Q G^T.
__device__ void qr_sweep(double* a, double* b, double* q, int lo, int hi) {
  const double bl = b[hi - 1];
  const double del = 0.5 * (a[hi - 1] - a[hi]);
  const double sgn = del >= 0.0 ? 1.0 : -1.0;
  const double mu = a[hi] - bl * bl / (del + sgn * hypot(del, bl));
  double x = a[lo] - mu;
  double z = b[lo];
  for (int k = lo; k < hi; ++k) {
    // rotation G = [[c, s], [-s, c]] on rows/cols (k, k+1) zeroing z
    const double r = hypot(x, z);
    double c = 1.0, s = 0.0;
    if (r > 0.0) {
      c = x / r;
      s = z / r;
    }
    if (k > lo) b[k - 1] = r;   // the entry that held the bulge partner
    const double ak = a[k], ak1 = a[k + 1], bk = b[k];
    a[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
    a[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
    b[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
    if (k + 1 < hi) {
      z = s * b[k + 1];         // new bulge at (k, k+2)
      b[k + 1] = c * b[k + 1];
      x = b[k];
    }
    const double q0 = q[k], q1 = q[k + 1];
    q[k] = c * q0 + s * q1;
    q[k + 1] = -s * q0 + c * q1;
  }
}

// One block per column; the tridiagonal and q_0 live in shared memory (the
// sweeps are sequential, so one thread runs them after a parallel fill).
__global__ void lanczos_quad_kernel(const double* __restrict__ ah,
                                    const double* __restrict__ bh, int t,
                                    int c0, int nc, const int* __restrict__ iters,
                                    int max_iter, double* __restrict__ quad,
                                    int* bad) {
  extern __shared__ double sm[];
  const int i = blockIdx.x;
  if (i >= nc) return;
  const int c = c0 + i;
  const int m = min(iters[c], max_iter);
  double* a = sm;
  double* b = a + m + 1;
  double* q = b + m + 1;
  if (m <= 0) {
    if (threadIdx.x == 0) quad[i] = 0.0;
    return;
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double al = ah[(int64_t)j * t + c];
    double dj = 1.0 / al;
    if (j > 0) dj += bh[(int64_t)(j - 1) * t + c] / ah[(int64_t)(j - 1) * t + c];
    a[j] = dj;
    b[j] = (j < m - 1) ? sqrt(bh[(int64_t)j * t + c]) / al : 0.0;
    q[j] = (j == 0) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double eps = 2.220446049250313e-16;
  int hi = m - 1;
  int guard = 0;
  while (hi > 0) {
    if (fabs(b[hi - 1]) <= eps * (fabs(a[hi - 1]) + fabs(a[hi]))) {
      b[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && fabs(b[lo - 1]) > eps * (fabs(a[lo - 1]) + fabs(a[lo]))) --lo;
    if (lo > 0) b[lo - 1] = 0.0;
    qr_sweep(a, b, q, lo, hi);
    if (++guard > 50 * m) {
      atomicOr(bad, 2);
      break;
    }
  }
  double s = 0.0;
  for (int j = 0; j < m; ++j) {
    if (!(a[j] > 0.0)) {
      atomicOr(bad, 1);
      continue;
    }
    s += q[j] * q[j] * log(a[j]);
  }
  quad[i] = s;
}

}  // namespace

int lanczos_quadrature(gp_ctx* ctx, const double* alpha_hist,
                       const double* beta_hist, int t, int c0, int nc,
                       const int* iters_dev, int max_iter, double* quad_dev,
                       int* bad_dev) {
  const size_t shm = sizeof(double) * 3 * ((size_t)max_iter + 1);
  if (shm > 220 * 1024)
    return set_err(ctx, GP_EINVAL, "Lanczos quadrature: max_iter %d too large", max_iter);
  if (shm > 48 * 1024)
    GP_CUDA(ctx, cudaFuncSetAttribute(lanczos_quad_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  lanczos_quad_kernel<<<(unsigned)std::max(nc, 1), 64, shm, ctx->stream>>>(
      alpha_hist, beta_hist, t, c0, nc, iters_dev, max_iter, quad_dev, bad_dev);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

}  // namespace gp
