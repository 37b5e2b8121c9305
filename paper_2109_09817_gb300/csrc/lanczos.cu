// Lanczos quadrature of the log-determinant (A8), FP64.
//
// arXiv 2109.09817 Sec. 3.2: mBCG's coefficients estimate the marginal
// likelihood (Eq. ll) through Lanczos tridiagonals.  For column c with
// coefficients alpha_j, beta_j over its first m steps, the PCG/Lanczos
// relation gives T (m x m):
//   T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T_{j,j+1} = sqrt(beta_j)/alpha_j,
// and the quadrature Q = e1^T log(T) e1 = sum_i w_i log(lambda_i) over T's
// eigenpairs, w_i = q_{0i}^2 (sum_i w_i = 1).
//
// Q is evaluated without the eigenpairs.  For lambda > 0,
//   log(lambda) = int_R [sig(u) - sig(u - log lambda)] du,  sig(u) = 1/(1 + e^-u)
// (a logistic step shifted by log lambda), and
//   sum_i w_i sig(u - log lambda_i) = e^u e1^T (T + e^u I)^{-1} e1 = e^u g(e^u),
// so Q = int_R [sig(u) - e^u g(e^u)] du.  For T positive definite and s >= 0,
// g(s) is the continued fraction of the bottom-up factorisation of T + s I:
//   d_{m-1} = T_{m-1,m-1} + s,  d_j = T_jj + s - T_{j,j+1}^2 / d_{j+1},
//   g(s) = 1 / d_0,
// every pivot d_j positive (the s = 0 pivots test T's definiteness).
// The integrand is analytic in the strip |Im u| < pi (the poles of sig) and
// decays exponentially both ways, so the trapezoid rule with step h errs by
// about 4 pi exp(-2 pi^2 / h) (1e-33 at h = 0.25).  The truncated tails are
// bounded exactly: below u_lo by e^{u_lo} (1 + g(0)), above u_hi by
// e^{-u_hi} (1 + T_00) (sum_i w_i lambda_i = T_00, sum_i w_i / lambda_i =
// g(0)); both are set to 1e-16.  Every node is an independent O(m)
// recurrence, so a block's threads share the nodes of one column, instead
// of one thread running O(m^2) sequential QR sweeps.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr double kQuadStep = 0.25;     // trapezoid step in u = log s
constexpr int kQuadMaxNodes = 8192;    // the step widens beyond this many nodes
constexpr double kTailTol = 1e-16;     // bound on each truncated tail
constexpr int kQuadThreads = 256;

// One block per column: T's diagonal and squared off-diagonal in shared
// memory, then the trapezoid nodes spread over the block's threads.
__global__ void __launch_bounds__(kQuadThreads) lanczos_quad_kernel(
    const double* __restrict__ ah, const double* __restrict__ bh, int t, int c0, int nc,
    const int* __restrict__ iters, int max_iter, double* __restrict__ quad, int* bad) {
  extern __shared__ double sm[];
  __shared__ double red[kQuadThreads / 32];
  __shared__ double s_ulo, s_h;
  __shared__ int s_nodes, s_ok;
  const int i = blockIdx.x;
  if (i >= nc) return;
  const int c = c0 + i;
  const int m = min(iters[c], max_iter);
  if (m <= 0) {
    if (threadIdx.x == 0) quad[i] = 0.0;
    return;
  }
  double* a = sm;             // T_jj
  double* b2 = a + m;         // T_{j,j+1}^2 = beta_j / alpha_j^2
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double al = ah[(int64_t)j * t + c];
    double dj = 1.0 / al;
    if (j > 0) dj += bh[(int64_t)(j - 1) * t + c] / ah[(int64_t)(j - 1) * t + c];
    a[j] = dj;
    b2[j] = (j < m - 1) ? bh[(int64_t)j * t + c] / (al * al) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // s = 0: the pivots of T; all positive iff T is positive definite
    double d = a[m - 1];
    bool ok = d > 0.0;
    for (int j = m - 2; j >= 0; --j) {
      d = a[j] - b2[j] / d;
      ok = ok && d > 0.0;
    }
    ok = ok && isfinite(d) && isfinite(a[0]);
    const double g0 = ok ? 1.0 / d : 0.0;
    const double ulo = log(kTailTol / (1.0 + g0));
    const double uhi = log((1.0 + a[0]) / kTailTol);
    double h = kQuadStep;
    if ((uhi - ulo) / h + 1.0 > kQuadMaxNodes) h = (uhi - ulo) / (kQuadMaxNodes - 1);
    s_ok = ok ? 1 : 0;
    s_ulo = ulo;
    s_h = h;
    s_nodes = ok ? (int)ceil((uhi - ulo) / h) + 1 : 0;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) {
      atomicOr(bad, 1);
      quad[i] = 0.0;
    }
    return;
  }
  const double ulo = s_ulo, h = s_h;
  double acc = 0.0;
  for (int k = threadIdx.x; k < s_nodes; k += blockDim.x) {
    const double u = ulo + k * h;
    const double s = exp(u);
    double d = a[m - 1] + s;
    for (int j = m - 2; j >= 0; --j) d = a[j] + s - b2[j] / d;
    acc += 1.0 / (1.0 + exp(-u)) - s / d;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    quad[i] = h * sum;
  }
}

}  // namespace

int lanczos_quadrature(gp_ctx* ctx, const double* alpha_hist,
                       const double* beta_hist, int t, int c0, int nc,
                       const int* iters_dev, int max_iter, double* quad_dev,
                       int* bad_dev) {
  const size_t shm = sizeof(double) * 2 * (size_t)std::max(max_iter, 1);
  if (shm > 200 * 1024)
    return set_err(ctx, GP_EINVAL, "Lanczos quadrature: max_iter %d too large", max_iter);
  if (shm > 48 * 1024)
    GP_CUDA(ctx, cudaFuncSetAttribute(lanczos_quad_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  lanczos_quad_kernel<<<(unsigned)std::max(nc, 1), kQuadThreads, shm, ctx->stream>>>(
      alpha_hist, beta_hist, t, c0, nc, iters_dev, max_iter, quad_dev, bad_dev);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

}  // namespace gp

using namespace gp;

extern "C" int gp_lanczos_logquad(gp_ctx* ctx, const double* alpha_hist, const double* beta_hist, int t,
                                  int max_iter, const int* iters, double* quad) {
  if (!ctx) return GP_EINVAL;
  if (!alpha_hist || !beta_hist || !iters || !quad || t < 1 || t > 256 || max_iter < 1)
    return set_err(ctx, GP_EINVAL, "gp_lanczos_logquad: bad arguments");
  for (int c = 0; c < t; ++c)
    if (iters[c] < 0 || iters[c] > max_iter)
      return set_err(ctx, GP_EINVAL, "gp_lanczos_logquad: iters[%d] = %d outside [0, %d]", c, iters[c], max_iter);
  GP_CUDA(ctx, cudaSetDevice(ctx->device));
  // device scratch: iters (t ints), the failure flag, then t doubles, each
  // part 16-byte aligned
  const size_t ioff = 0, boff = (sizeof(int) * (size_t)t + 15) / 16 * 16, qoff = boff + 16;
  char* scr = static_cast<char*>(ws_get(ctx, WS_LZ_SCR, qoff + sizeof(double) * (size_t)t));
  char* h = static_cast<char*>(pinned_get(ctx, qoff + sizeof(double) * (size_t)t));
  if (!scr || !h) return set_err(ctx, GP_ENOMEM, "workspace (Lanczos quadrature)");
  int* iters_dev = reinterpret_cast<int*>(scr + ioff);
  int* bad_dev = reinterpret_cast<int*>(scr + boff);
  double* quad_dev = reinterpret_cast<double*>(scr + qoff);
  std::memcpy(h, iters, sizeof(int) * (size_t)t);
  GP_CUDA(ctx, cudaMemcpyAsync(iters_dev, h, sizeof(int) * (size_t)t, cudaMemcpyHostToDevice, ctx->stream));
  GP_CUDA(ctx, cudaMemsetAsync(bad_dev, 0, sizeof(int), ctx->stream));
  GP_TRY(lanczos_quadrature(ctx, alpha_hist, beta_hist, t, 0, t, iters_dev, max_iter, quad_dev, bad_dev));
  GP_CUDA(ctx, cudaMemcpyAsync(h + qoff, quad_dev, sizeof(double) * (size_t)t, cudaMemcpyDeviceToHost,
                               ctx->stream));
  GP_CUDA(ctx, cudaMemcpyAsync(h + boff, bad_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::memcpy(quad, h + qoff, sizeof(double) * (size_t)t);
  if (*reinterpret_cast<const int*>(h + boff))
    return set_err(ctx, GP_EBREAKDOWN, "Lanczos tridiagonal not positive definite");
  return GP_OK;
}
