// Hyperparameter optimisation on a random subset, then the full fit.
//
// arXiv 2109.09817 Sec. 4 (computational details): the hyperparameters are
// optimised on a random subset of the training pairs, and the full model is
// then fitted with sigma^2_add added to the optimised noise.  The paper does
// not name the optimiser; this one is Adam (Kingma & Ba, 2015) on log theta,
// ascending the log marginal likelihood of Eq. (ll) with the gradient of
// gp_logml_and_grad (stochastic traces, Sec. 3.2).  The probe seed is the
// same at every step, so the objective seen by the optimiser is one smooth
// function of theta (common random numbers), not a fresh estimate per step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "gp_internal.cuh"

namespace gp {
namespace {

// rows[i] of X (n x d, row-major) and y -> Xs, ys (device gather)
__global__ void gather_rows_kernel(const float* __restrict__ X, const float* __restrict__ y, int d,
                                   const int64_t* __restrict__ idx, int64_t m, float* __restrict__ Xs,
                                   float* __restrict__ ys) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * d; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d, j = e % d;
    Xs[e] = X[idx[i] * d + j];
    if (j == 0) ys[i] = y[idx[i]];
  }
}

// SplitMix64 (Steele, Lea & Flood 2014): the subset's random stream
uint64_t splitmix64(uint64_t& state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace
}  // namespace gp

using namespace gp;

extern "C" {

int gp_subset_indices(int64_t N, int64_t M, uint64_t seed, int64_t* idx) {
  if (N < 1 || M < 1 || M > N || !idx) return GP_EINVAL;
  // the first M draws of a Fisher-Yates shuffle of 0..N-1; only the touched
  // positions are stored (memory O(M)); returned sorted
  std::unordered_map<int64_t, int64_t> moved;
  moved.reserve((size_t)M * 2);
  auto at = [&](int64_t pos) {
    auto it = moved.find(pos);
    return it == moved.end() ? pos : it->second;
  };
  uint64_t st = seed;
  for (int64_t i = 0; i < M; ++i) {
    const uint64_t r = splitmix64(st);
    const int64_t j = i + (int64_t)(r % (uint64_t)(N - i));   // uniform on [i, N) up to 2^-64 bias
    const int64_t vi = at(i), vj = at(j);
    moved[j] = vi;
    moved[i] = vj;
    idx[i] = vj;
  }
  std::sort(idx, idx + M);
  return GP_OK;
}

int gp_hyperopt(gp_ctx* ctx, const float* X, int64_t N, int d, const float* y, int64_t subset, uint64_t seed,
                int steps, double lr, int n_probes, int k, int precond, double tol, int max_iter, int precision,
                double* lengthscale, double* outputscale, double* sigma2, double* logml_hist,
                double* grad_out) {
  if (!ctx || !X || !y || N < 1 || d < 1 || d > 256 || subset < 1 || subset > N || steps < 0 || !(lr > 0.0) ||
      n_probes < 1 || k < 0 || k > subset || !lengthscale || !outputscale || !sigma2 ||
      !(*outputscale > 0.0) || !(*sigma2 > 0.0))
    return set_err(ctx, GP_EINVAL, "gp_hyperopt: bad arguments");
  for (int j = 0; j < d; ++j)
    if (!(lengthscale[j] > 0.0)) return set_err(ctx, GP_EINVAL, "gp_hyperopt: lengthscale[%d] <= 0", j);
  GP_CUDA(ctx, cudaSetDevice(ctx->device));
  // the subset rows on the device
  std::vector<int64_t> idx((size_t)subset);
  GP_TRY(gp_subset_indices(N, subset, seed, idx.data()));
  int64_t* didx = static_cast<int64_t*>(ws_get(ctx, WS_HO_IDX, sizeof(int64_t) * (size_t)subset));
  float* Xs = ws<float>(ctx, WS_HO_X, (size_t)subset * d);
  float* ys = ws<float>(ctx, WS_HO_Y, (size_t)subset);
  if (!didx || !Xs || !ys) return set_err(ctx, GP_ENOMEM, "workspace (subset)");
  GP_CUDA(ctx, cudaMemcpyAsync(didx, idx.data(), sizeof(int64_t) * (size_t)subset, cudaMemcpyHostToDevice,
                               ctx->stream));
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(subset * d, 256), 8LL * ctx->num_sms));
  gather_rows_kernel<<<g, 256, 0, ctx->stream>>>(X, y, d, didx, subset, Xs, ys);
  GP_LAUNCHED(ctx);
  // Adam on the log parameters p = (log l_1..log l_d, log s, log sigma^2)
  const int np = d + 2;
  std::vector<double> p(np), m1(np, 0.0), m2(np, 0.0), grad(np), ell(d);
  for (int j = 0; j < d; ++j) p[j] = std::log(lengthscale[j]);
  p[d] = std::log(*outputscale);
  p[d + 1] = std::log(*sigma2);
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int it = 0; it <= steps; ++it) {
    for (int j = 0; j < d; ++j) ell[j] = std::exp(p[j]);
    gp_theta th{ell.data(), std::exp(p[d]), std::exp(p[d + 1])};
    double logml = 0.0, logdet = 0.0;
    const int rc = gp_logml_and_grad(ctx, Xs, subset, d, &th, ys, n_probes, seed ^ 0x5eedULL, k, precond, tol,
                                     max_iter, GP_STOP_RECURRENCE, precision, &logml, &logdet, grad.data(),
                                     nullptr, nullptr);
    if (rc != GP_OK && rc != GP_ENOTCONV) return rc;
    if (logml_hist) logml_hist[it] = logml;
    if (it == steps) {
      if (grad_out) std::memcpy(grad_out, grad.data(), sizeof(double) * np);
      break;
    }
    // ascent on log theta: dL/dlog(theta) = theta dL/dtheta
    const double c1 = 1.0 - std::pow(b1, it + 1), c2 = 1.0 - std::pow(b2, it + 1);
    for (int i = 0; i < np; ++i) {
      const double gi = std::exp(p[i]) * grad[i];
      m1[i] = b1 * m1[i] + (1.0 - b1) * gi;
      m2[i] = b2 * m2[i] + (1.0 - b2) * gi * gi;
      p[i] += lr * (m1[i] / c1) / (std::sqrt(m2[i] / c2) + eps);
    }
  }
  for (int j = 0; j < d; ++j) lengthscale[j] = std::exp(p[j]);
  *outputscale = std::exp(p[d]);
  *sigma2 = std::exp(p[d + 1]);
  return GP_OK;
}

int gp_train(gp_ctx* ctx, const float* X, int64_t N, int d, const float* y, int64_t subset, uint64_t seed,
             int steps, double lr, int n_probes, int k, int precond, double tol, int max_iter, int precision,
             double sigma2_add, double* lengthscale, double* outputscale, double* sigma2, double* logml_hist,
             gp_model** out) {
  if (!out || !(sigma2_add >= 0.0)) return set_err(ctx, GP_EINVAL, "gp_train: bad arguments");
  *out = nullptr;
  GP_TRY(gp_hyperopt(ctx, X, N, d, y, subset, seed, steps, lr, n_probes, k, precond, tol, max_iter, precision,
                     lengthscale, outputscale, sigma2, logml_hist, nullptr));
  gp_theta th{lengthscale, *outputscale, *sigma2 + sigma2_add};
  return gp_model_fit(ctx, X, N, d, &th, y, std::min<int64_t>(k, N), precond, 1, tol, max_iter,
                      GP_STOP_RECURRENCE, precision, out, nullptr);
}

}  // extern "C"
