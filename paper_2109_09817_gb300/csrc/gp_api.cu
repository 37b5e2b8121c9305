// C ABI of libgp (declared in include/gp.h): contexts, workspace, and the
// drivers of the exact-GP path of arXiv 2109.09817.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <vector>

#include "gp_internal.cuh"


namespace gp {

int set_err(gp_ctx* ctx, int code, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

int check_cuda(gp_ctx* ctx, cudaError_t e, const char* what) {
  // clear a non-sticky error so that it is not reported again by the next
  // launch check (a sticky one stays, and every later call reports it)
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation)
    return set_err(ctx, GP_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return set_err(ctx, GP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* ws_get(gp_ctx* ctx, int slot, size_t bytes) {
  DevBuf& b = ctx->ws[slot];
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return b.p;
  if (b.p) {
    // kernels queued earlier may still read the old buffer
    cudaStreamSynchronize(ctx->stream);
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  const size_t want = (bytes + 255) / 256 * 256;
  if (cudaMalloc(&b.p, want) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return nullptr;
  }
  b.bytes = want;
  return b.p;
}

void* pinned_get(gp_ctx* ctx, size_t bytes) {
  if (ctx->pinned_bytes >= bytes) return ctx->pinned;
  if (ctx->pinned) {
    cudaStreamSynchronize(ctx->stream);
    cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_bytes = 0;
  }
  const size_t want = std::max<size_t>(bytes, 4096);
  if (cudaMallocHost(&ctx->pinned, want) != cudaSuccess) {
    cudaGetLastError();
    ctx->pinned = nullptr;
    return nullptr;
  }
  ctx->pinned_bytes = want;
  return ctx->pinned;
}

namespace {

__global__ void var_from_dots_kernel(const double* __restrict__ dots, int64_t m,
                                     double s, float* __restrict__ var) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    var[i] = (float)(s - dots[i]);
}

// out[i * ldo + a] = s * k(x_a, x'_i) for a < n (cross covariance columns),
// from prepared features (same scaling and centring on both sides).
__global__ void kcols_kernel(const float* __restrict__ xr, const float* __restrict__ nr,
                             int64_t n, const float* __restrict__ xq,
                             const float* __restrict__ nq, int64_t m, int d_pad,
                             float s, float* __restrict__ out, int64_t ldo) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (a >= n || i >= m) return;
  float dot = 0.f;
  const float* xa = xr + a * d_pad;
  const float* xi = xq + i * d_pad;
  for (int j = 0; j < d_pad; ++j) dot = fmaf(xa[j], xi[j], dot);
  const float u2 = fmaxf(nr[a] + nq[i] - 2.f * dot, 0.f);
  float u, e;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(u) : "f"(u2));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-u));
  out[i * ldo + a] = s * fmaf(u2, kC2, fmaf(u, kC1, 1.f)) * e;
}

int check_common(gp_ctx* ctx, const float* X, int64_t N, int d,
                 const gp_theta* theta) {
  if (!ctx) return GP_EINVAL;
  if (!X || N <= 0 || d <= 0 || !theta || !theta->lengthscale)
    return set_err(ctx, GP_EINVAL, "null pointer or non-positive size (N=%lld, d=%d)", (long long)N, d);
  if (d > 256) return set_err(ctx, GP_EINVAL, "d = %d > 256", d);
  if (!(theta->outputscale > 0.0) || !(theta->sigma2 > 0.0))
    return set_err(ctx, GP_EINVAL, "outputscale and sigma2 must be > 0");
  for (int j = 0; j < d; ++j)
    if (!(theta->lengthscale[j] > 0.0) || !std::isfinite(theta->lengthscale[j]))
      return set_err(ctx, GP_EINVAL, "lengthscale[%d] must be finite and > 0", j);
  GP_CUDA(ctx, cudaSetDevice(ctx->device));
  return GP_OK;
}

int prep_train(gp_ctx* ctx, const float* X, int64_t N, int d,
               const gp_theta* theta, int precision, Prep* p) {
  double* mu = ws<double>(ctx, WS_MU, (size_t)d);
  if (!mu) return set_err(ctx, GP_ENOMEM, "workspace (mean)");
  GP_TRY(feature_mean(ctx, X, N, d, mu));
  return prepare_features(ctx, X, N, d, mu, theta->lengthscale, precision, WS_XT, p);
}

bool valid_precision(int p) { return p >= GP_FP32_PLAIN && p <= GP_TF32; }
bool valid_stop(int r) { return r == GP_STOP_RECURRENCE || r == GP_STOP_TRUE; }

// host array -> device workspace slot (asynchronous on the context stream
// for pinned memory; the runtime stages pageable memory itself)
const float* stage_in(gp_ctx* ctx, int slot, const float* src, size_t bytes) {
  float* dst = static_cast<float*>(ws_get(ctx, slot, bytes));
  if (!dst) return nullptr;
  if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return dst;
}

int stage_out(gp_ctx* ctx, float* dst, const float* src, size_t bytes) {
  GP_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

__global__ void fill_one_kernel(float* __restrict__ v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 1.f;
}

int fill_one(gp_ctx* ctx, float* v, int64_t n) {
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), 1024));
  fill_one_kernel<<<g, 256, 0, ctx->stream>>>(v, n);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

// the model's preconditioner P = L L^T + D (FP32 factor copy and D^{-1/2})
Precond model_precond(const gp_model* m) {
  Precond pc;
  pc.k = m->k;
  pc.n = m->n;
  pc.L = m->L;
  pc.L32 = m->L32;
  pc.ld32 = m->n_pad;
  pc.cfac = m->cfac;
  pc.cinv = m->cfac ? m->cfac + (size_t)m->k * m->k : nullptr;
  pc.dh = m->dh;
  pc.logdet = m->pc_logdet;
  pc.sigma2 = m->sigma2;
  return pc;
}

}  // namespace
}  // namespace gp

using namespace gp;

extern "C" {

int gp_create(gp_ctx** out, int device, void* stream) {
  if (!out) return GP_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GP_ECUDA;
  }
  gp_ctx* ctx = new gp_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
    ctx->num_sms = sms;
  *out = ctx;
  return GP_OK;
}

void gp_destroy(gp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& e : ctx->ev) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  for (auto& b : ctx->ws)
    if (b.p) cudaFree(b.p);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->status_host) cudaFreeHost(ctx->status_host);
  delete ctx;
}

int gp_set_stream(gp_ctx* ctx, void* stream) {
  if (!ctx) return GP_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  ctx->stream = static_cast<cudaStream_t>(stream);
  return GP_OK;
}

int gp_sync(gp_ctx* ctx) {
  if (!ctx) return GP_EINVAL;
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

const char* gp_last_error(const gp_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

int64_t gp_launch_count(const gp_ctx* ctx) { return ctx ? ctx->launches : 0; }

int gp_set_option(gp_ctx* ctx, int option, int value) {
  if (!ctx) return GP_EINVAL;
  switch (option) {
    case GP_OPT_SYMMETRIC_KMV:
      if (value != 0 && value != 1) return set_err(ctx, GP_EINVAL, "gp_set_option: value must be 0 or 1");
      ctx->sym_kmv = value != 0;
      return GP_OK;
    default:
      return set_err(ctx, GP_EINVAL, "gp_set_option: unknown option %d", option);
  }
}

int gp_profile(gp_ctx* ctx, int enable) {
  if (!ctx) return GP_EINVAL;
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->prof = enable != 0;
  ctx->ev_used = 0;
  ctx->prof_flops = 0.0;
  ctx->prof_elems = 0.0;
  return GP_OK;
}

int gp_profile_read(gp_ctx* ctx, int64_t* products, double* ms, double* flops,
                    double* entries) {
  if (!ctx) return GP_EINVAL;
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double tot = 0.0;
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float e = 0.f;
    GP_CUDA(ctx, cudaEventElapsedTime(&e, ctx->ev[i].first, ctx->ev[i].second));
    tot += e;
  }
  if (products) *products = (int64_t)ctx->ev_used;
  if (ms) *ms = tot;
  if (flops) *flops = ctx->prof_flops;
  if (entries) *entries = ctx->prof_elems;
  return GP_OK;
}

int gp_kmatmul(gp_ctx* ctx, const float* X, int64_t N, int d,
               const gp_theta* theta, const float* V, int t, float* out,
               int precision) {
  if (ctx && (precision & GP_HOST)) {
    // host arrays: stage X and V on the device, run, copy out back
    GP_TRY(check_common(ctx, X, N, d, theta));
    if (!V || !out || t < 1 || t > kMaxT) return set_err(ctx, GP_EINVAL, "gp_kmatmul: bad V/out/t");
    const float* Xd = stage_in(ctx, WS_HS_X, X, sizeof(float) * (size_t)N * d);
    const float* Vd = stage_in(ctx, WS_HS_V, V, sizeof(float) * (size_t)N * t);
    float* Od = ws<float>(ctx, WS_HS_O, (size_t)N * t);
    if (!Xd || !Vd || !Od) return set_err(ctx, GP_ENOMEM, "workspace (host arrays)");
    GP_TRY(gp_kmatmul(ctx, Xd, N, d, theta, Vd, t, Od, precision & ~GP_HOST));
    return stage_out(ctx, out, Od, sizeof(float) * (size_t)N * t);
  }
  GP_TRY(check_common(ctx, X, N, d, theta));
  if (!V || !out || t < 1 || t > kMaxT || !valid_precision(precision))
    return set_err(ctx, GP_EINVAL, "gp_kmatmul: bad V/out/t/precision");
  if (V == out) return set_err(ctx, GP_EINVAL, "gp_kmatmul: out aliases V");
  Prep p;
  GP_TRY(prep_train(ctx, X, N, d, theta, precision, &p));
  return kmv(ctx, p, p, V, N, t, out, N, theta->outputscale, theta->sigma2, true, precision);
}

int gp_kcross_matmul(gp_ctx* ctx, const float* Xp, int64_t M, const float* X,
                     int64_t N, int d, const gp_theta* theta, const float* V,
                     int t, float* out, int precision) {
  if (ctx && (precision & GP_HOST)) {
    GP_TRY(check_common(ctx, X, N, d, theta));
    if (!Xp || M <= 0 || !V || !out || t < 1 || t > kMaxT)
      return set_err(ctx, GP_EINVAL, "gp_kcross_matmul: bad arguments");
    const float* Xd = stage_in(ctx, WS_HS_X, X, sizeof(float) * (size_t)N * d);
    const float* Xpd = stage_in(ctx, WS_HS_XP, Xp, sizeof(float) * (size_t)M * d);
    const float* Vd = stage_in(ctx, WS_HS_V, V, sizeof(float) * (size_t)N * t);
    float* Od = ws<float>(ctx, WS_HS_O, (size_t)M * t);
    if (!Xd || !Xpd || !Vd || !Od) return set_err(ctx, GP_ENOMEM, "workspace (host arrays)");
    GP_TRY(gp_kcross_matmul(ctx, Xpd, M, Xd, N, d, theta, Vd, t, Od, precision & ~GP_HOST));
    return stage_out(ctx, out, Od, sizeof(float) * (size_t)M * t);
  }
  GP_TRY(check_common(ctx, X, N, d, theta));
  if (!Xp || M <= 0 || !V || !out || t < 1 || t > kMaxT || !valid_precision(precision))
    return set_err(ctx, GP_EINVAL, "gp_kcross_matmul: bad arguments");
  Prep p, q;
  GP_TRY(prep_train(ctx, X, N, d, theta, precision, &p));
  GP_TRY(prepare_features(ctx, Xp, M, d, ws<double>(ctx, WS_MU, d), theta->lengthscale,
                          precision, WS_XT2, &q));
  return kmv(ctx, q, p, V, N, t, out, M, theta->outputscale, 0.0, false, precision);
}

int gp_pivchol(gp_ctx* ctx, const float* X, int64_t N, int d,
               const gp_theta* theta, int k, double* L, int64_t* piv,
               int* rank_out, double* resid_diag) {
  GP_TRY(check_common(ctx, X, N, d, theta));
  if (k < 0 || k > N || (k > 0 && (!L || !piv)) || !rank_out)
    return set_err(ctx, GP_EINVAL, "gp_pivchol: bad k/L/piv/rank_out");
  *rank_out = 0;
  if (k == 0) return GP_OK;
  return pivchol_run(ctx, X, N, d, theta->lengthscale, theta->outputscale, k, L, piv, rank_out,
                     resid_diag);
}

int gp_mbcg(gp_ctx* ctx, const float* X, int64_t N, int d,
            const gp_theta* theta, const double* L, int k,
            const double* resid_diag, const float* B,
            int t, double tol, int max_iter, int stop_rule, int precision, float* Omega,
            double* alpha_hist, double* beta_hist, int* iters,
            double* rel_resid) {
  GP_TRY(check_common(ctx, X, N, d, theta));
  if (!B || !Omega || t < 1 || t > kMaxT || max_iter < 1 || !(tol >= 0.0) ||
      k < 0 || (k > 0 && !L) || !valid_precision(precision) || !valid_stop(stop_rule))
    return set_err(ctx, GP_EINVAL, "gp_mbcg: bad arguments");
  Prep p;
  GP_TRY(prep_train(ctx, X, N, d, theta, precision, &p));
  Precond pc;
  GP_TRY(precond_setup(ctx, L, N, k, k, theta->sigma2, resid_diag, &pc));
  double* ah = alpha_hist ? alpha_hist : ws<double>(ctx, WS_CG_AH, (size_t)max_iter * t);
  double* bh = beta_hist ? beta_hist : ws<double>(ctx, WS_CG_BH, (size_t)max_iter * t);
  int* iters_dev = static_cast<int*>(ws_get(ctx, WS_GR_ACC, sizeof(int) * t + sizeof(double) * t + 64));
  if (!ah || !bh || !iters_dev) return set_err(ctx, GP_ENOMEM, "workspace (mbcg records)");
  double* rr_dev = reinterpret_cast<double*>(iters_dev + ((t + 1) & ~1));
  CgArgs a;
  a.prep = &p;
  a.s = theta->outputscale;
  a.sigma2 = theta->sigma2;
  a.pc = &pc;
  a.B = B;
  a.ldb = N;
  a.t = t;
  a.tol = tol;
  a.max_iter = max_iter;
  a.precision = precision;
  a.U = Omega;
  a.ldu = N;
  a.alpha_hist = ah;
  a.beta_hist = bh;
  a.iters_dev = iters_dev;
  a.relres_dev = rr_dev;
  a.true_cols = stop_rule == GP_STOP_TRUE ? t : 0;
  a.true_dev = rr_dev;   // rel_resid reports the verified true residuals
  CgResult res;
  GP_TRY(mbcg_run(ctx, a, &res));
  if (iters || rel_resid) {
    char* h = static_cast<char*>(pinned_get(ctx, (sizeof(int) + sizeof(double)) * t + 64));
    if (!h) return set_err(ctx, GP_ENOMEM, "pinned staging");
    GP_CUDA(ctx, cudaMemcpyAsync(h, iters_dev, sizeof(int) * t, cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(ctx, cudaMemcpyAsync(h + sizeof(int) * ((t + 1) & ~1), rr_dev, sizeof(double) * t,
                                 cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (iters) std::memcpy(iters, h, sizeof(int) * t);
    if (rel_resid) std::memcpy(rel_resid, h + sizeof(int) * ((t + 1) & ~1), sizeof(double) * t);
  }
  if (res.breakdown) return set_err(ctx, GP_EBREAKDOWN, "mBCG breakdown (loss of definiteness)");
  if (!res.converged)
    return set_err(ctx, GP_ENOTCONV,
                   res.true_checks > 0 && !res.true_ok
                       ? "mBCG: true residual above tol after %d verifications"
                       : "mBCG: max_iter=%d reached",
                   res.true_checks > 0 && !res.true_ok ? res.true_checks : max_iter);
  return GP_OK;
}

int gp_bcg(gp_ctx* ctx, const float* X, int64_t N, int d, const gp_theta* theta, const double* L, int k,
           const double* resid_diag, const float* B, int t, double tol, int max_iter, int precision,
           float* Omega, int* iters, double* rel_resid) {
  GP_TRY(check_common(ctx, X, N, d, theta));
  if (!B || !Omega || t < 1 || t > 32 || max_iter < 1 || !(tol > 0.0) || k < 0 || (k > 0 && !L) ||
      !valid_precision(precision))
    return set_err(ctx, GP_EINVAL, "gp_bcg: bad arguments");
  Prep p;
  GP_TRY(prep_train(ctx, X, N, d, theta, precision, &p));
  Precond pc;
  GP_TRY(precond_setup(ctx, L, N, k, k, theta->sigma2, resid_diag, &pc));
  return bcg_run(ctx, p, theta->outputscale, theta->sigma2, pc, B, N, t, tol, max_iter, precision, Omega, N,
                 iters, rel_resid, -1);
}

int gp_mbcg_refine(gp_ctx* ctx, const float* X, int64_t N, int d,
                   const gp_theta* theta, const double* L, int k,
                   const double* resid_diag, const float* B, int t, double tol,
                   double inner_tol, int max_outer, int max_iter,
                   int inner_precision, int outer_precision, float* Omega,
                   int* outer_steps, int* inner_steps, double* rel_resid) {
  GP_TRY(check_common(ctx, X, N, d, theta));
  if (!B || !Omega || t < 1 || t > kMaxT || max_iter < 1 || max_outer < 1 || !(tol > 0.0) ||
      !(inner_tol > 0.0) || k < 0 || (k > 0 && !L) || !valid_precision(inner_precision) ||
      (outer_precision != GP_FP32_PLAIN && outer_precision != GP_FP32_SPLIT_TF32 &&
       outer_precision != GP_FP32_SPLIT_F16))
    return set_err(ctx, GP_EINVAL, "gp_mbcg_refine: bad arguments");
  cudaStream_t st = ctx->stream;
  // outer products on the accurate features, inner ones on a second family
  Prep po, pi;
  GP_TRY(prep_train(ctx, X, N, d, theta, outer_precision, &po));
  const double* mu = static_cast<const double*>(ctx->ws[WS_MU].p);
  GP_TRY(prepare_features(ctx, X, N, d, mu, theta->lengthscale, inner_precision, WS_XT2, &pi));
  Precond pc;
  GP_TRY(precond_setup(ctx, L, N, k, k, theta->sigma2, resid_diag, &pc));
  const size_t nv = (size_t)t * N;
  float* R = ws<float>(ctx, WS_RF_R, nv);
  float* Dl = ws<float>(ctx, WS_RF_D, nv);
  float* W = ws<float>(ctx, WS_RF_W, nv);
  double* ah = ws<double>(ctx, WS_CG_AH, (size_t)max_iter * t);
  double* bh = ws<double>(ctx, WS_CG_BH, (size_t)max_iter * t);
  double* sm = ws<double>(ctx, WS_RF_S, (size_t)4 * t + 16);
  if (!R || !Dl || !W || !ah || !bh || !sm) return set_err(ctx, GP_ENOMEM, "workspace (refinement)");
  double* bb = sm;              // ||B_c||^2
  double* rr = sm + t;          // ||R_c||^2
  double* rr_dev = sm + 2 * t;  // inner relres (unused)
  int* it_dev = reinterpret_cast<int*>(sm + 3 * t);
  double* h = static_cast<double*>(pinned_get(ctx, sizeof(double) * 2 * t));
  if (!h) return set_err(ctx, GP_ENOMEM, "pinned staging");
  GP_TRY(dot_columns(ctx, B, B, N, N, t, bb));
  GP_CUDA(ctx, cudaMemsetAsync(Omega, 0, sizeof(float) * nv, st));
  GP_TRY(copy_vectors(ctx, B, N, R, N, N, t, 1.f));
  std::vector<double> bnorm(t), rel(t, 1.0);
  std::vector<char> done(t, 0);
  int outer = 0, inner = 0;
  bool all = false;
  for (int c = 0; c < t; ++c) rel[c] = 1.0;
  GP_CUDA(ctx, cudaMemcpyAsync(h, bb, sizeof(double) * t, cudaMemcpyDeviceToHost, st));
  GP_CUDA(ctx, cudaStreamSynchronize(st));
  for (int c = 0; c < t; ++c) {
    bnorm[c] = std::sqrt(h[c]);
    if (bnorm[c] == 0.0) {   // zero right-hand side: Omega_c = 0 is exact
      done[c] = 1;
      rel[c] = 0.0;
    }
  }
  while (outer < max_outer) {
    all = true;
    for (int c = 0; c < t; ++c) all = all && done[c];
    if (all) break;
    // inner solve K-hat delta = R in the inner precision
    CgArgs a;
    a.prep = &pi;
    a.s = theta->outputscale;
    a.sigma2 = theta->sigma2;
    a.pc = &pc;
    a.B = R;
    a.ldb = N;
    a.t = t;
    a.tol = inner_tol;
    a.max_iter = max_iter;
    a.precision = inner_precision;
    a.U = Dl;
    a.ldu = N;
    a.alpha_hist = ah;
    a.beta_hist = bh;
    a.iters_dev = it_dev;
    a.relres_dev = rr_dev;
    CgResult res;
    GP_TRY(mbcg_run(ctx, a, &res));
    // an inner breakdown (the inner operator lost definiteness) leaves the
    // iterate reached so far in delta; it is used, and the round must then
    // still reduce some residual
    const bool broke = res.breakdown;
    inner += res.iters_max;
    ++outer;
    // Omega += delta; R = B - K-hat Omega in the outer precision
    GP_TRY(axpby_vectors(ctx, 1.f, Omega, 1.f, Dl, Omega, N, N, t));
    GP_TRY(kmv(ctx, po, po, Omega, N, t, W, N, theta->outputscale, theta->sigma2, true, outer_precision));
    GP_TRY(axpby_vectors(ctx, 1.f, B, -1.f, W, R, N, N, t));
    GP_TRY(dot_columns(ctx, R, R, N, N, t, rr));
    GP_CUDA(ctx, cudaMemcpyAsync(h, rr, sizeof(double) * t, cudaMemcpyDeviceToHost, st));
    GP_CUDA(ctx, cudaStreamSynchronize(st));
    GP_TRY(check_status(ctx));
    bool progress = false;
    for (int c = 0; c < t; ++c) {
      if (done[c]) continue;
      const double prev = rel[c];
      rel[c] = std::sqrt(h[c]) / bnorm[c];
      if (rel[c] < 0.9 * prev) progress = true;
      // the measured residual carries the outer product's own error: a
      // column passes below 0.8 tol, the margin of GP_STOP_TRUE
      if (rel[c] < 0.8 * tol) {
        done[c] = 1;
        // a stopped column's residual is not refined further
        GP_CUDA(ctx, cudaMemsetAsync(R + (size_t)c * N, 0, sizeof(float) * N, st));
      }
    }
    if (broke && !progress) {
      if (outer_steps) *outer_steps = outer;
      if (inner_steps) *inner_steps = inner;
      if (rel_resid) std::memcpy(rel_resid, rel.data(), sizeof(double) * t);
      return set_err(ctx, GP_EBREAKDOWN, "refinement: inner mBCG breakdown without progress");
    }
  }
  all = true;
  for (int c = 0; c < t; ++c) all = all && done[c];
  if (outer_steps) *outer_steps = outer;
  if (inner_steps) *inner_steps = inner;
  if (rel_resid) std::memcpy(rel_resid, rel.data(), sizeof(double) * t);
  if (!all) return set_err(ctx, GP_ENOTCONV, "refinement: tol not reached after %d rounds", outer);
  return GP_OK;
}

int gp_logml_and_grad(gp_ctx* ctx, const float* X, int64_t N, int d,
                      const gp_theta* theta, const float* y, int n_probes,
                      uint64_t seed, int k, int precond, double tol, int max_iter,
                      int stop_rule, int precision, double* logml, double* logdet,
                      double* grad, double* logdet_stderr, gp_stats* stats) {
  if (ctx && (precision & GP_HOST)) {
    GP_TRY(check_common(ctx, X, N, d, theta));
    if (!y) return set_err(ctx, GP_EINVAL, "gp_logml_and_grad: null y");
    const float* Xd = stage_in(ctx, WS_HS_X, X, sizeof(float) * (size_t)N * d);
    const float* yd = stage_in(ctx, WS_HS_V, y, sizeof(float) * (size_t)N);
    if (!Xd || !yd) return set_err(ctx, GP_ENOMEM, "workspace (host arrays)");
    return gp_logml_and_grad(ctx, Xd, N, d, theta, yd, n_probes, seed, k, precond, tol, max_iter, stop_rule,
                             precision & ~GP_HOST, logml, logdet, grad, logdet_stderr, stats);
  }
  GP_TRY(check_common(ctx, X, N, d, theta));
  if (!y || n_probes < 1 || n_probes > 255 || k < 0 || k > N || max_iter < 1 ||
      !(tol >= 0.0) || !logml || !logdet || !valid_precision(precision) || !valid_stop(stop_rule) ||
      (precond != GP_PC_SIGMA && precond != GP_PC_RESID))
    return set_err(ctx, GP_EINVAL, "gp_logml_and_grad: bad arguments");
  const double s = theta->outputscale, sig2 = theta->sigma2;
  Prep p;
  GP_TRY(prep_train(ctx, X, N, d, theta, precision, &p));
  const int64_t ld = p.n_pad;
  const int T1 = 1 + n_probes;
  // 1. preconditioner
  double* L = ws<double>(ctx, WS_PC_L, (size_t)N * std::max(k, 1));
  int64_t* piv = static_cast<int64_t*>(ws_get(ctx, WS_PC_PIV, sizeof(int64_t) * std::max(k, 1)));
  if (!L || !piv) return set_err(ctx, GP_ENOMEM, "workspace (factor)");
  int rank = 0;
  double* resid = nullptr;
  if (k > 0 && precond == GP_PC_RESID) {
    resid = ws<double>(ctx, WS_PC_RES, (size_t)N);
    if (!resid) return set_err(ctx, GP_ENOMEM, "workspace (residual diagonal)");
  }
  if (k > 0) GP_TRY(pivchol_run(ctx, X, N, d, theta->lengthscale, s, k, L, piv, &rank, resid));
  Precond pc;
  GP_TRY(precond_setup(ctx, L, N, k, rank, sig2, resid, &pc));
  // 2. right-hand sides [y | z_1..z_t]
  float* B = ws<float>(ctx, WS_CG_B, (size_t)ld * T1);
  float* U = ws<float>(ctx, WS_CG_U, (size_t)ld * T1);
  float* Z0 = ws<float>(ctx, WS_CG_Z0, (size_t)ld * T1);
  double* ah = ws<double>(ctx, WS_CG_AH, (size_t)max_iter * T1);
  double* bh = ws<double>(ctx, WS_CG_BH, (size_t)max_iter * T1);
  char* rec = static_cast<char*>(ws_get(ctx, WS_GR_ACC, 64 * 1024));
  if (!B || !U || !Z0 || !ah || !bh || !rec) return set_err(ctx, GP_ENOMEM, "workspace (rhs)");
  double* rz0 = reinterpret_cast<double*>(rec);            // T1
  double* relres = rz0 + 256;                              // T1
  double* quad = relres + 256;                             // T1
  double* Gacc = quad + 256;                               // d_pad + 1
  double* dots = Gacc + 512;                               // T1 + 1
  int* iters = reinterpret_cast<int*>(dots + 512);         // T1
  int* bad = iters + 256;
  double* truer = reinterpret_cast<double*>(iters + 512);  // 1: y's true residual
  GP_CUDA(ctx, cudaMemsetAsync(B, 0, sizeof(float) * ld * T1, ctx->stream));
  GP_CUDA(ctx, cudaMemsetAsync(U, 0, sizeof(float) * ld * T1, ctx->stream));
  GP_CUDA(ctx, cudaMemsetAsync(Z0, 0, sizeof(float) * ld * T1, ctx->stream));
  GP_CUDA(ctx, cudaMemsetAsync(rec, 0, 64 * 1024, ctx->stream));
  GP_TRY(copy_vectors(ctx, y, N, B, ld, N, 1, 1.f));
  GP_TRY(probe_vectors(ctx, L, N, rank, sig2, resid, seed, n_probes, B + ld, ld));
  // 3. mBCG
  CgArgs a;
  a.prep = &p;
  a.s = s;
  a.sigma2 = sig2;
  a.pc = &pc;
  a.B = B;
  a.ldb = ld;
  a.t = T1;
  a.tol = tol;
  a.max_iter = max_iter;
  a.precision = precision;
  a.U = U;
  a.ldu = ld;
  a.alpha_hist = ah;
  a.beta_hist = bh;
  a.Z0 = Z0;
  a.rz0 = rz0;
  a.iters_dev = iters;
  a.relres_dev = relres;
  a.true_cols = stop_rule == GP_STOP_TRUE ? 1 : 0;   // y's column: the solve a = K-hat^{-1} y
  a.true_dev = truer;
  CgResult res;
  GP_TRY(mbcg_run(ctx, a, &res));
  if (res.breakdown) return set_err(ctx, GP_EBREAKDOWN, "mBCG breakdown (loss of definiteness)");
  // 4. Lanczos quadrature over the probe columns
  GP_TRY(lanczos_quadrature(ctx, ah, bh, T1, 1, n_probes, iters, max_iter, quad, bad));
  // 5. y^T a
  GP_TRY(dot_columns(ctx, B, U, ld, N, 1, dots));
  // 6. gradient
  float* Wg = nullptr;
  if (grad) {
    Wg = ws<float>(ctx, WS_GR_W, (size_t)ld * T1);
    if (!Wg) return set_err(ctx, GP_ENOMEM, "workspace (grad)");
    GP_CUDA(ctx, cudaMemsetAsync(Wg, 0, sizeof(float) * ld * T1, ctx->stream));
    GP_TRY(copy_vectors(ctx, U, ld, Wg, ld, N, 1, 0.5f));
    GP_TRY(copy_vectors(ctx, Z0 + ld, ld, Wg + ld, ld, N, n_probes, (float)(-0.5 / n_probes)));
    GP_TRY(grad_tiles(ctx, p, U, Wg, T1, Gacc, nullptr, precision));
    GP_TRY(dot_columns(ctx, U, Wg, ld, N, T1, dots + 1));
  }
  // 7. host assembly
  const size_t nrec = 64 * 1024;
  char* h = static_cast<char*>(pinned_get(ctx, nrec));
  if (!h) return set_err(ctx, GP_ENOMEM, "pinned staging");
  GP_CUDA(ctx, cudaMemcpyAsync(h, rec, nrec, cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const double* h_rz0 = reinterpret_cast<const double*>(h);
  const double* h_relres = h_rz0 + 256;
  const double* h_quad = h_relres + 256;
  const double* h_G = h_quad + 256;
  const double* h_dots = h_G + 512;
  const int* h_iters = reinterpret_cast<const int*>(h_dots + 512);
  const int h_bad = h_iters[256];
  const double h_true = *reinterpret_cast<const double*>(h_iters + 512);
  if (h_bad) return set_err(ctx, GP_EBREAKDOWN, "Lanczos tridiagonal not positive definite (%d)", h_bad);
  double acc = 0.0, acc2 = 0.0;
  for (int c = 1; c <= n_probes; ++c) {
    const double v = h_rz0[c] * h_quad[c - 1];
    acc += v;
    acc2 += v * v;
  }
  const double mean = acc / n_probes;
  const double var = n_probes > 1 ? (acc2 - n_probes * mean * mean) / (n_probes - 1) : 0.0;
  *logdet = pc.logdet + mean;
  if (logdet_stderr) *logdet_stderr = std::sqrt(std::max(var, 0.0) / n_probes);
  const double yKy = h_dots[0];
  *logml = -0.5 * yKy - 0.5 * (*logdet) - 0.5 * (double)N * std::log(2.0 * M_PI);
  if (grad) {
    const double c2 = kFeatScale * kFeatScale;
    for (int j = 0; j < d; ++j) grad[j] = 2.0 * s / (c2 * theta->lengthscale[j]) * h_G[j];
    grad[d] = h_G[p.d_pad];
    double gsig = 0.0;
    for (int q = 0; q < T1; ++q) gsig += h_dots[1 + q];
    grad[d + 1] = gsig;
  }
  if (stats) {
    int im = 0;
    double rm = 0.0;
    for (int c = 0; c < T1; ++c) {
      im = std::max(im, h_iters[c]);
      rm = std::max(rm, h_relres[c]);
    }
    stats->iters_max = im;
    stats->iters_y = h_iters[0];
    stats->rank = rank;
    stats->n_kmatmul = res.n_kmv;
    stats->relres_y = h_relres[0];
    stats->relres_max = rm;
    stats->logdet_P = pc.logdet;
    stats->yKinvy = yKy;
    stats->true_relres_y = res.true_checks > 0 ? h_true : -1.0;
    stats->true_checks = res.true_checks;
  }
  if (!res.converged)
    return set_err(ctx, GP_ENOTCONV,
                   res.true_checks > 0 && !res.true_ok ? "mBCG: y's true residual above tol after %d verifications"
                                                        : "mBCG: max_iter=%d reached",
                   res.true_checks > 0 && !res.true_ok ? res.true_checks : max_iter);
  return GP_OK;
}

int gp_model_fit(gp_ctx* ctx, const float* X, int64_t N, int d,
                 const gp_theta* theta, const float* y, int k, int precond, int block, double tol,
                 int max_iter, int stop_rule, int precision, gp_model** out, gp_stats* stats) {
  GP_TRY(check_common(ctx, X, N, d, theta));
  if (!y || !out || k < 0 || k > N || max_iter < 1 || !valid_precision(precision) || !valid_stop(stop_rule) ||
      (precond != GP_PC_SIGMA && precond != GP_PC_RESID) || block < 1 || block > 32)
    return set_err(ctx, GP_EINVAL, "gp_model_fit: bad arguments");
  *out = nullptr;
  Prep p;
  GP_TRY(prep_train(ctx, X, N, d, theta, precision, &p));
  gp_model* m = new gp_model();
  auto fail = [&](int rc) {
    gp_model_free(m);
    return rc;
  };
  m->device = ctx->device;
  m->n = N;
  m->n_pad = p.n_pad;
  m->d = d;
  m->d_pad = p.d_pad;
  m->precision = precision;
  m->ell.assign(theta->lengthscale, theta->lengthscale + d);
  m->s = theta->outputscale;
  m->sigma2 = theta->sigma2;
  m->tol = tol;
  m->max_iter = max_iter;
  const size_t ne = (size_t)p.n_pad * p.d_pad;
  if (cudaMalloc(&m->mu, sizeof(double) * d) != cudaSuccess ||
      cudaMalloc(&m->xt, sizeof(float) * ne) != cudaSuccess ||
      cudaMalloc(&m->norm, sizeof(float) * p.n_pad) != cudaSuccess ||
      cudaMalloc(&m->alpha, sizeof(float) * p.n_pad) != cudaSuccess) {
    cudaGetLastError();
    return fail(set_err(ctx, GP_ENOMEM, "model allocation"));
  }
  cudaStream_t st = ctx->stream;
  GP_CUDA(ctx, cudaMemcpyAsync(m->mu, ws<double>(ctx, WS_MU, d), sizeof(double) * d, cudaMemcpyDeviceToDevice, st));
  GP_CUDA(ctx, cudaMemcpyAsync(m->xt, p.xt, sizeof(float) * ne, cudaMemcpyDeviceToDevice, st));
  GP_CUDA(ctx, cudaMemcpyAsync(m->norm, p.norm, sizeof(float) * p.n_pad, cudaMemcpyDeviceToDevice, st));
  if (p.xt_hi) {
    if (cudaMalloc(&m->xt_hi, sizeof(float) * ne) != cudaSuccess ||
        cudaMalloc(&m->xt_lo, sizeof(float) * ne) != cudaSuccess)
      return fail(set_err(ctx, GP_ENOMEM, "model allocation"));
    GP_CUDA(ctx, cudaMemcpyAsync(m->xt_hi, p.xt_hi, sizeof(float) * ne, cudaMemcpyDeviceToDevice, st));
    GP_CUDA(ctx, cudaMemcpyAsync(m->xt_lo, p.xt_lo, sizeof(float) * ne, cudaMemcpyDeviceToDevice, st));
  }
  if (p.xh_hi) {
    const size_t nh = (size_t)p.n_pad * kHalfCols;
    if (cudaMalloc(&m->xh_hi, sizeof(__half) * nh) != cudaSuccess ||
        cudaMalloc(&m->xh_lo, sizeof(__half) * nh) != cudaSuccess ||
        cudaMalloc(&m->norm_h, sizeof(float) * p.n_pad) != cudaSuccess ||
        cudaMalloc(&m->xh_scale, sizeof(float)) != cudaSuccess)
      return fail(set_err(ctx, GP_ENOMEM, "model allocation"));
    GP_CUDA(ctx, cudaMemcpyAsync(m->xh_hi, p.xh_hi, sizeof(__half) * nh, cudaMemcpyDeviceToDevice, st));
    GP_CUDA(ctx, cudaMemcpyAsync(m->xh_lo, p.xh_lo, sizeof(__half) * nh, cudaMemcpyDeviceToDevice, st));
    GP_CUDA(ctx, cudaMemcpyAsync(m->norm_h, p.norm_h, sizeof(float) * p.n_pad, cudaMemcpyDeviceToDevice, st));
    GP_CUDA(ctx, cudaMemcpyAsync(m->xh_scale, p.xh_scale, sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  Prep mp = p;
  mp.xt = m->xt;
  mp.norm = m->norm;
  mp.xt_hi = m->xt_hi;
  mp.xt_lo = m->xt_lo;
  mp.xh_hi = m->xh_hi;
  mp.xh_lo = m->xh_lo;
  mp.norm_h = m->norm_h;
  mp.xh_scale = m->xh_scale;
  // preconditioner
  int rank = 0;
  double* resid = nullptr;
  if (k > 0) {
    if (cudaMalloc(&m->L, sizeof(double) * (size_t)N * k) != cudaSuccess)
      return fail(set_err(ctx, GP_ENOMEM, "model allocation"));
    int64_t* piv = static_cast<int64_t*>(ws_get(ctx, WS_PC_PIV, sizeof(int64_t) * k));
    if (!piv) return fail(set_err(ctx, GP_ENOMEM, "workspace"));
    if (precond == GP_PC_RESID) {
      resid = ws<double>(ctx, WS_PC_RES, (size_t)N);
      if (!resid) return fail(set_err(ctx, GP_ENOMEM, "workspace"));
    }
    int rc = pivchol_run(ctx, X, N, d, theta->lengthscale, m->s, k, m->L, piv, &rank, resid);
    if (rc != GP_OK) return fail(rc);
  }
  Precond pc;
  {
    int rc = precond_setup(ctx, m->L, N, k, rank, m->sigma2, resid, &pc);
    if (rc != GP_OK) return fail(rc);
  }
  if (cudaMalloc(&m->dh, sizeof(float) * pc.ld32) != cudaSuccess)
    return fail(set_err(ctx, GP_ENOMEM, "model allocation"));
  GP_CUDA(ctx, cudaMemcpyAsync(m->dh, pc.dh, sizeof(float) * pc.ld32, cudaMemcpyDeviceToDevice, st));
  m->k = rank;
  m->pc_logdet = pc.logdet;
  if (rank > 0) {
    if (cudaMalloc(&m->L32, sizeof(float) * (size_t)rank * pc.ld32) != cudaSuccess ||
        cudaMalloc(&m->cfac, sizeof(double) * (size_t)2 * rank * rank) != cudaSuccess)
      return fail(set_err(ctx, GP_ENOMEM, "model allocation"));
    GP_CUDA(ctx, cudaMemcpyAsync(m->L32, pc.L32, sizeof(float) * (size_t)rank * pc.ld32, cudaMemcpyDeviceToDevice, st));
    GP_CUDA(ctx, cudaMemcpyAsync(m->cfac, pc.cfac, sizeof(double) * (size_t)rank * rank, cudaMemcpyDeviceToDevice, st));
    GP_CUDA(ctx, cudaMemcpyAsync(m->cfac + (size_t)rank * rank, pc.cinv, sizeof(double) * (size_t)rank * rank,
                                 cudaMemcpyDeviceToDevice, st));
  }
  // a = K-hat^{-1} y
  GP_CUDA(ctx, cudaMemsetAsync(m->alpha, 0, sizeof(float) * p.n_pad, st));
  if (block > 1) {
    // AltBBMM (Sec. 3.1-3.2): y and block - 1 random right-hand sides share
    // one block Krylov space, which contains y's own; a = column 0
    const int64_t ldb = p.n_pad;
    float* Bb = ws<float>(ctx, WS_RF_R, (size_t)block * ldb);
    float* Ob = ws<float>(ctx, WS_RF_D, (size_t)block * ldb);
    if (!Bb || !Ob) return fail(set_err(ctx, GP_ENOMEM, "workspace (block fit)"));
    if (cudaMemsetAsync(Bb, 0, sizeof(float) * (size_t)block * ldb, st) != cudaSuccess)
      return fail(check_cuda(ctx, cudaGetLastError(), "cudaMemsetAsync"));
    int rc = copy_vectors(ctx, y, N, Bb, ldb, N, 1, 1.f);
    if (rc == GP_OK) rc = probe_vectors(ctx, m->L, N, rank, m->sigma2, resid, 0x5eedULL, block - 1, Bb + ldb, ldb);
    if (rc != GP_OK) return fail(rc);
    int iters = 0;
    std::vector<double> rel(block, 0.0);
    rc = bcg_run(ctx, mp, m->s, m->sigma2, pc, Bb, ldb, block, tol, max_iter, precision, Ob, ldb, &iters,
                 rel.data(), 0);
    if (rc != GP_OK) return fail(rc);
    rc = copy_vectors(ctx, Ob, ldb, m->alpha, p.n_pad, N, 1, 1.f);
    if (rc != GP_OK) return fail(rc);
    if (stats) {
      std::memset(stats, 0, sizeof(*stats));
      stats->iters_max = stats->iters_y = iters;
      stats->rank = rank;
      stats->n_kmatmul = iters;
      stats->relres_y = rel[0];
      stats->relres_max = *std::max_element(rel.begin(), rel.end());
      stats->logdet_P = pc.logdet;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(check_cuda(ctx, cudaGetLastError(), "sync"));
    *out = m;
    return GP_OK;
  }
  double* ah = ws<double>(ctx, WS_CG_AH, (size_t)max_iter);
  double* bh = ws<double>(ctx, WS_CG_BH, (size_t)max_iter);
  int* rec = static_cast<int*>(ws_get(ctx, WS_GR_ACC, 256));
  if (!ah || !bh || !rec) return fail(set_err(ctx, GP_ENOMEM, "workspace"));
  CgArgs a;
  a.prep = &mp;
  a.s = m->s;
  a.sigma2 = m->sigma2;
  a.pc = &pc;
  a.B = y;
  a.ldb = N;
  a.t = 1;
  a.tol = tol;
  a.max_iter = max_iter;
  a.precision = precision;
  a.U = m->alpha;
  a.ldu = p.n_pad;
  a.alpha_hist = ah;
  a.beta_hist = bh;
  a.iters_dev = rec;
  a.relres_dev = reinterpret_cast<double*>(rec + 2);
  a.true_cols = stop_rule == GP_STOP_TRUE ? 1 : 0;
  a.true_dev = reinterpret_cast<double*>(rec + 4);
  CgResult res;
  {
    int rc = mbcg_run(ctx, a, &res);
    if (rc != GP_OK) return fail(rc);
  }
  if (stats) {
    int* h = static_cast<int*>(pinned_get(ctx, 64));
    GP_CUDA(ctx, cudaMemcpyAsync(h, rec, 24, cudaMemcpyDeviceToHost, st));
    GP_CUDA(ctx, cudaStreamSynchronize(st));
    std::memset(stats, 0, sizeof(*stats));
    stats->iters_max = stats->iters_y = h[0];
    double rr, tr;
    std::memcpy(&rr, h + 2, sizeof(double));
    std::memcpy(&tr, h + 4, sizeof(double));
    stats->relres_y = stats->relres_max = rr;
    stats->true_relres_y = res.true_checks > 0 ? tr : -1.0;
    stats->true_checks = res.true_checks;
    stats->rank = rank;
    stats->n_kmatmul = res.n_kmv;
    stats->logdet_P = pc.logdet;
  }
  GP_CUDA(ctx, cudaStreamSynchronize(st));
  if (res.breakdown) return fail(set_err(ctx, GP_EBREAKDOWN, "mBCG breakdown"));
  if (!res.converged)
    return fail(set_err(ctx, GP_ENOTCONV,
                        res.true_checks > 0 && !res.true_ok ? "mBCG: y's true residual above tol after %d verifications"
                                                             : "mBCG: max_iter=%d reached",
                        res.true_checks > 0 && !res.true_ok ? res.true_checks : max_iter));
  *out = m;
  return GP_OK;
}

void gp_model_free(gp_model* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  for (void* q : {(void*)m->mu, (void*)m->xt, (void*)m->norm, (void*)m->xt_hi,
                  (void*)m->xt_lo, (void*)m->xh_hi, (void*)m->xh_lo, (void*)m->norm_h,
                  (void*)m->xh_scale, (void*)m->alpha,
                  (void*)m->L, (void*)m->L32, (void*)m->cfac, (void*)m->dh, (void*)m->love_R})
    if (q) cudaFree(q);
  delete m;
}

int gp_predict(gp_ctx* ctx, const gp_model* m, const float* Xp, int64_t M,
               float* mean, float* var, int var_mode) {
  if (!ctx || !m || !Xp || M <= 0 || !mean) return set_err(ctx, GP_EINVAL, "gp_predict: bad arguments");
  if (m->device != ctx->device) return set_err(ctx, GP_EINVAL, "gp_predict: model on another device");
  GP_CUDA(ctx, cudaSetDevice(ctx->device));
  Prep mp;
  mp.n = m->n;
  mp.n_pad = m->n_pad;
  mp.d = m->d;
  mp.d_pad = m->d_pad;
  mp.xt = m->xt;
  mp.norm = m->norm;
  mp.xt_hi = m->xt_hi;
  mp.xt_lo = m->xt_lo;
  mp.xh_hi = m->xh_hi;
  mp.xh_lo = m->xh_lo;
  mp.norm_h = m->norm_h;
  mp.xh_scale = m->xh_scale;
  Prep q;
  GP_TRY(prepare_features(ctx, Xp, M, m->d, m->mu, m->ell.data(), m->precision, WS_XT2, &q));
  GP_TRY(kmv(ctx, q, mp, m->alpha, m->n_pad, 1, mean, M, m->s, 0.0, false, m->precision));
  if (!var || var_mode == GP_VAR_NONE) return GP_OK;
  if (var_mode == GP_VAR_CACHED) {
    if (!m->love_R) return set_err(ctx, GP_EINVAL, "gp_predict: the model has no variance cache");
    return cached_variance(ctx, m, mp, q, var);
  }
  if (var_mode != GP_VAR_EXACT) return set_err(ctx, GP_EINVAL, "gp_predict: unknown var_mode");
  // exact latent variance: k(x',x') - k*^T K-hat^{-1} k*, in chunks of RHS
  Precond pc = model_precond(m);
  const int CH = 64;
  const int64_t ld = m->n_pad;
  float* Kc = ws<float>(ctx, WS_PR_K, (size_t)ld * CH);
  float* Om = ws<float>(ctx, WS_PR_O, (size_t)ld * CH);
  double* ah = ws<double>(ctx, WS_CG_AH, (size_t)m->max_iter * CH);
  double* bh = ws<double>(ctx, WS_CG_BH, (size_t)m->max_iter * CH);
  char* rec = static_cast<char*>(ws_get(ctx, WS_GR_ACC, 8192));
  if (!Kc || !Om || !ah || !bh || !rec) return set_err(ctx, GP_ENOMEM, "workspace (variance)");
  int* itd = reinterpret_cast<int*>(rec);
  double* rrd = reinterpret_cast<double*>(rec + 1024);
  double* dots = reinterpret_cast<double*>(rec + 4096);
  bool notconv = false;
  for (int64_t i0 = 0; i0 < M; i0 += CH) {
    const int nc = (int)std::min<int64_t>(CH, M - i0);
    GP_CUDA(ctx, cudaMemsetAsync(Kc, 0, sizeof(float) * ld * nc, ctx->stream));
    dim3 grid((unsigned)ceil_div(m->n, 256), (unsigned)nc);
    kcols_kernel<<<grid, 256, 0, ctx->stream>>>(mp.xt, mp.norm, m->n, q.xt + i0 * q.d_pad,
                                               q.norm + i0, nc, m->d_pad, (float)m->s, Kc, ld);
    GP_LAUNCHED(ctx);
    CgArgs a;
    a.prep = &mp;
    a.s = m->s;
    a.sigma2 = m->sigma2;
    a.pc = &pc;
    a.B = Kc;
    a.ldb = ld;
    a.t = nc;
    a.tol = m->tol;
    a.max_iter = m->max_iter;
    a.precision = m->precision;
    a.U = Om;
    a.ldu = ld;
    a.alpha_hist = ah;
    a.beta_hist = bh;
    a.iters_dev = itd;
    a.relres_dev = rrd;
    CgResult res;
    GP_TRY(mbcg_run(ctx, a, &res));
    if (res.breakdown) return set_err(ctx, GP_EBREAKDOWN, "mBCG breakdown (variance)");
    notconv |= !res.converged;
    GP_TRY(dot_columns(ctx, Kc, Om, ld, m->n, nc, dots));
    var_from_dots_kernel<<<1, 256, 0, ctx->stream>>>(dots, nc, m->s, var + i0);
    GP_LAUNCHED(ctx);
  }
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (notconv) return set_err(ctx, GP_ENOTCONV, "variance solves reached max_iter");
  return GP_OK;
}

int gp_model_variance_cache(gp_ctx* ctx, gp_model* m, const float* b, int rank, int* rank_out) {
  if (!ctx || !m || rank < 1 || rank > GP_VAR_CACHE_MAX_RANK || rank > m->n || !rank_out)
    return set_err(ctx, GP_EINVAL, "gp_model_variance_cache: bad arguments (1 <= rank <= %d)",
                   GP_VAR_CACHE_MAX_RANK);
  if (m->device != ctx->device) return set_err(ctx, GP_EINVAL, "gp_model_variance_cache: model on another device");
  GP_CUDA(ctx, cudaSetDevice(ctx->device));
  const Prep mp = model_prep_of(m);
  const float* start = b;
  if (!start) {
    // start at K-hat a, which is y up to the fit's tolerance
    float* kb = ws<float>(ctx, WS_LV_C, (size_t)m->n_pad);
    if (!kb) return set_err(ctx, GP_ENOMEM, "workspace (variance cache)");
    GP_TRY(kmv(ctx, mp, mp, m->alpha, m->n_pad, 1, kb, m->n_pad, m->s, m->sigma2, true, m->precision));
    start = kb;
  }
  float* R = nullptr;
  if (cudaMalloc(&R, sizeof(float) * (size_t)m->n_pad * rank) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, GP_ENOMEM, "variance cache allocation");
  }
  int k = 0;
  const int rc = lanczos_cache_build(ctx, mp, m->s, m->sigma2, m->precision, start, rank, R, &k);
  if (rc != GP_OK) {
    cudaFree(R);
    return rc;
  }
  if (m->love_R) cudaFree(m->love_R);
  m->love_R = R;
  m->love_m = k;
  *rank_out = k;
  return GP_OK;
}

int gp_predict_sum(gp_ctx* ctx, const gp_model* m, const float* Xp, int64_t M, double* mean_sum,
                   double* var_sum, int var_mode) {
  if (!ctx || !m || !Xp || M <= 0 || !mean_sum ||
      (var_sum && var_mode != GP_VAR_EXACT && var_mode != GP_VAR_CACHED))
    return set_err(ctx, GP_EINVAL, "gp_predict_sum: bad arguments");
  if (m->device != ctx->device) return set_err(ctx, GP_EINVAL, "gp_predict_sum: model on another device");
  if (var_sum && var_mode == GP_VAR_CACHED && !m->love_R)
    return set_err(ctx, GP_EINVAL, "gp_predict_sum: the model has no variance cache");
  GP_CUDA(ctx, cudaSetDevice(ctx->device));
  const Prep mp = model_prep_of(m);
  Prep q;
  GP_TRY(prepare_features(ctx, Xp, M, m->d, m->mu, m->ell.data(), m->precision, WS_XT2, &q));
  const int kc = var_mode == GP_VAR_CACHED ? m->love_m : 0;
  // sums: [0] the means, [1] 1^T K(X',X') 1, [2] c^T K-hat^{-1} c, [3..] R^T c
  double* sums = ws<double>(ctx, WS_LV_P, (size_t)4 + kc);
  float* mb = ws<float>(ctx, WS_LV_M, (size_t)std::max<int64_t>(M, 1));
  if (!sums || !mb) return set_err(ctx, GP_ENOMEM, "workspace (predict sum)");
  GP_CUDA(ctx, cudaMemsetAsync(sums, 0, sizeof(double) * (4 + kc), ctx->stream));
  GP_TRY(kmv(ctx, q, mp, m->alpha, m->n_pad, 1, mb, M, m->s, 0.0, false, m->precision));
  GP_TRY(row_sums(ctx, mb, M, 1, M, sums));
  if (var_sum) {
    GP_TRY(block_ksum(ctx, q, m->s, sums + 1));
    if (var_mode == GP_VAR_CACHED) {
      float* KR = ws<float>(ctx, WS_LV_K, (size_t)kc * M);
      if (!KR) return set_err(ctx, GP_ENOMEM, "workspace (predict sum)");
      GP_TRY(kmv(ctx, q, mp, m->love_R, m->n_pad, kc, KR, M, m->s, 0.0, false, m->precision));
      GP_TRY(row_sums(ctx, KR, M, kc, M, sums + 4));
    } else {
      // c = K(X, X') 1, then c^T K-hat^{-1} c by preconditioned CG
      const int64_t ld = m->n_pad;
      float* ones = mb;
      float* cv = ws<float>(ctx, WS_LV_C, (size_t)ld);
      float* wv = ws<float>(ctx, WS_LV_W, (size_t)ld);
      double* ah = ws<double>(ctx, WS_CG_AH, (size_t)m->max_iter);
      double* bh = ws<double>(ctx, WS_CG_BH, (size_t)m->max_iter);
      char* rec = static_cast<char*>(ws_get(ctx, WS_GR_ACC, 256));
      if (!cv || !wv || !ah || !bh || !rec) return set_err(ctx, GP_ENOMEM, "workspace (predict sum)");
      GP_TRY(fill_one(ctx, ones, M));
      GP_CUDA(ctx, cudaMemsetAsync(cv, 0, sizeof(float) * ld, ctx->stream));
      GP_TRY(kmv(ctx, mp, q, ones, M, 1, cv, ld, m->s, 0.0, false, m->precision));
      Precond pc = model_precond(m);
      CgArgs a;
      a.prep = &mp;
      a.s = m->s;
      a.sigma2 = m->sigma2;
      a.pc = &pc;
      a.B = cv;
      a.ldb = ld;
      a.t = 1;
      a.tol = m->tol;
      a.max_iter = m->max_iter;
      a.precision = m->precision;
      a.U = wv;
      a.ldu = ld;
      a.alpha_hist = ah;
      a.beta_hist = bh;
      a.iters_dev = reinterpret_cast<int*>(rec);
      a.relres_dev = reinterpret_cast<double*>(rec + 16);
      CgResult res;
      GP_TRY(mbcg_run(ctx, a, &res));
      if (res.breakdown) return set_err(ctx, GP_EBREAKDOWN, "mBCG breakdown (predict sum)");
      if (!res.converged) return set_err(ctx, GP_ENOTCONV, "predict sum: the solve reached max_iter");
      GP_TRY(dot_columns(ctx, cv, wv, ld, m->n, 1, sums + 2));
    }
  }
  double* h = static_cast<double*>(pinned_get(ctx, sizeof(double) * (4 + kc)));
  if (!h) return set_err(ctx, GP_ENOMEM, "pinned staging");
  GP_CUDA(ctx, cudaMemcpyAsync(h, sums, sizeof(double) * (4 + kc), cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  GP_TRY(check_status(ctx));
  *mean_sum = h[0];
  if (var_sum) {
    double quad = h[2];
    if (var_mode == GP_VAR_CACHED) {
      quad = 0.0;
      for (int j = 0; j < kc; ++j) quad += h[4 + j] * h[4 + j];
    }
    *var_sum = h[1] - quad;
  }
  return GP_OK;
}

}  // extern "C"
