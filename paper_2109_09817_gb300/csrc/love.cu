// Serving variances: the Lanczos variance cache and per-molecule sums.
//
// Eq. (pred) gives the latent posterior variance k(x',x') - k*^T K-hat^{-1}
// k*; one solve per test row is out of reach at N = 2^20, so serving reads
// K-hat^{-1} from a rank-m Lanczos cache (the low-rank cache of Pleiss et
// al., 2018): m steps of Lanczos on K-hat from a start vector b with full
// reorthogonalisation give K-hat Q ~ Q T with Q^T Q = I, and
//   K-hat^{-1} ~ Q T^{-1} Q^T = R R^T,  R = Q C^{-T},  T = C C^T,
// so that var(x') ~ k(x',x') - |R^T k*|^2, where R^T k* for a batch of test
// rows is ONE cross product K(X', X) R with the m columns of R as vectors.
//
// A molecule's correlation energy is the sum of its pair energies (Sec. 2.1);
// the variance of that sum over the rows of X' is
//   1^T K(X',X') 1 - c^T K-hat^{-1} c,  c = K(X, X') 1,
// read with the cache as 1^T K(X',X') 1 - |R^T c|^2, where R^T c = the row
// sums of K(X', X) R over the molecule's rows.
//
// Storage: Q (and R, which overwrites it) in FP32, m vectors of length n_pad
// (zero padded); every dot product, the Lanczos coefficients, the Cholesky
// factor of T and the sums of the molecule in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr int kBlk = 256;
constexpr int kPartBlocks = 304;   // row chunks of the two-stage reductions

__device__ __forceinline__ double block_sum64(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;
}

// part[b * k + i] = sum over the rows of chunk b of Q_i . w, i < k (FP64)
__global__ void qtw_partial_kernel(const float* __restrict__ Q, int64_t ld, int k, const float* __restrict__ w,
                                   int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  const int nb = gridDim.x;
  const int64_t chunk = (n + nb - 1) / nb;
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  for (int i = 0; i < k; ++i) {
    const float* q = Q + (int64_t)i * ld;
    double acc = 0.0;
    for (int64_t a = r0 + threadIdx.x; a < r1; a += blockDim.x) acc += (double)q[a] * (double)w[a];
    const double s = block_sum64(acc, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * k + i] = s;
  }
}

// c[i] = sum_b part[b * k + i]
__global__ void reduce_parts_kernel(const double* __restrict__ part, int nb, int k, double* __restrict__ c) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * k + i];
    c[i] = s;
  }
}

// w -= sum_{i<k} c_i Q_i (c in FP64, the sum per row in FP64)
__global__ void w_minus_qc_kernel(const float* __restrict__ Q, int64_t ld, int k, const double* __restrict__ c,
                                  float* __restrict__ w, int64_t n) {
  extern __shared__ double cs[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = c[i];
  __syncthreads();
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x) {
    double acc = (double)w[a];
    for (int i = 0; i < k; ++i) acc -= cs[i] * (double)Q[(int64_t)i * ld + a];
    w[a] = (float)acc;
  }
}

// dst = src * scale (FP64 scale), n rows; rows [n, n_pad) of dst set to 0
__global__ void scale_vec_kernel(const float* __restrict__ src, double scale, float* __restrict__ dst, int64_t n,
                                 int64_t npad) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < npad; a += (int64_t)gridDim.x * blockDim.x)
    dst[a] = a < n ? (float)((double)src[a] * scale) : 0.f;
}

// R = Q W in place, W (k x k, upper triangular, FP32) = C^{-T}: a block of
// 128 rows loads its Q rows into shared memory, then writes R rows.
__global__ void r_from_q_kernel(float* __restrict__ Q, int64_t ld, int k, const float* __restrict__ W,
                                int64_t npad) {
  extern __shared__ float sm[];
  float* sW = sm;                 // k x k
  float* sQ = sm + k * k;         // k x 128
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) sW[i] = W[i];
  const int64_t a0 = (int64_t)blockIdx.x * 128;
  for (int idx = threadIdx.x; idx < k * 128; idx += blockDim.x) {
    const int i = idx / 128, r = idx % 128;
    sQ[idx] = (a0 + r < npad) ? Q[(int64_t)i * ld + a0 + r] : 0.f;
  }
  __syncthreads();
  const int r = threadIdx.x;      // 128 threads: one row each
  if (a0 + r >= npad) return;
  for (int j = 0; j < k; ++j) {
    float acc = 0.f;
    for (int i = 0; i <= j; ++i) acc = fmaf(sQ[i * 128 + r], sW[i * k + j], acc);
    Q[(int64_t)j * ld + a0 + r] = acc;
  }
}

// var[i] = s - sum_j KR[j][i]^2 (KR: k vectors of length M, ld M)
__global__ void var_from_cache_kernel(const float* __restrict__ KR, int k, int64_t M, double s,
                                      float* __restrict__ var) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) {
      const double v = KR[(int64_t)j * M + i];
      acc += v * v;
    }
    var[i] = (float)(s - acc);
  }
}

// out[j] += sum_{i in this block's rows} A[j * lda + i] for j < k (FP64)
__global__ void row_sums_kernel(const float* __restrict__ A, int64_t lda, int k, int64_t M, double* __restrict__ out) {
  __shared__ double sh[32];
  const int j = blockIdx.y;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)A[(int64_t)j * lda + i];
  const double s = block_sum64(acc, sh);
  if (threadIdx.x == 0) atomicAdd(out + j, s);
}

// out[0] += sum_{a, b < M} k(x'_a, x'_b) over the prepared rows (x~ = c (x -
// mu) / l, so u = |x~_a - x~_b| and k / s = (1 + ln2 u + (ln2 u)^2 / 3) 2^-u),
// with u^2 by direct differences (no cancellation for close rows), k in
// FP32 and the sum in FP64.  One thread per row a, columns in chunks.
__global__ void block_ksum_kernel(const float* __restrict__ xt, int dp, int64_t M, double s, double* __restrict__ out) {
  __shared__ double sh[32];
  extern __shared__ float sx[];   // 64 columns x dp features
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  for (int64_t b0 = 0; b0 < M; b0 += 64) {
    __syncthreads();
    const int nb = (int)(M - b0 < 64 ? M - b0 : 64);
    for (int idx = threadIdx.x; idx < 64 * dp; idx += blockDim.x) {
      const int bb = idx / dp, j = idx % dp;
      sx[idx] = bb < nb ? xt[(b0 + bb) * dp + j] : 0.f;
    }
    __syncthreads();
    if (a < M) {
      const float* xa = xt + a * dp;
      for (int bb = 0; bb < nb; ++bb) {
        float u2 = 0.f;
        for (int j = 0; j < dp; ++j) {
          const float df = xa[j] - sx[bb * dp + j];
          u2 = fmaf(df, df, u2);
        }
        const float u = sqrtf(u2);
        const float kv = (b0 + bb == a) ? 1.f : fmaf(u2, kC2, fmaf(u, kC1, 1.f)) * exp2f(-u);
        acc += (double)kv;
      }
    }
  }
  const double sum = block_sum64(acc, sh);
  if (threadIdx.x == 0) atomicAdd(out, s * sum);
}

// sums[i * stride + off + j] = sum over the rows [seg[2i], seg[2i+1]) of
// A[j * lda + row] (FP64), grid (blocks, k, nseg)
__global__ void seg_row_sums_kernel(const float* __restrict__ A, int64_t lda, const int64_t* __restrict__ seg,
                                    int stride, int off, double* __restrict__ sums) {
  __shared__ double sh[32];
  const int j = blockIdx.y, i = blockIdx.z;
  const int64_t r0 = seg[2 * i], r1 = seg[2 * i + 1];
  double acc = 0.0;
  for (int64_t r = r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < r1; r += (int64_t)gridDim.x * blockDim.x)
    acc += (double)A[(int64_t)j * lda + r];
  const double v = block_sum64(acc, sh);
  if (threadIdx.x == 0 && v != 0.0) atomicAdd(sums + (int64_t)i * stride + off + j, v);
}

// sums[i * stride] += s sum_{a, b in part i} k(x'_a, x'_b), the part's rows
// [seg[2i], seg[2i+1]) of the prepared features; grid (blocks, nseg)
__global__ void seg_ksum_kernel(const float* __restrict__ xt, int dp, const int64_t* __restrict__ seg, int stride,
                                double s, double* __restrict__ sums) {
  __shared__ double sh[32];
  extern __shared__ float sx[];   // 64 columns x dp features
  const int i = blockIdx.y;
  const int64_t r0 = seg[2 * i], r1 = seg[2 * i + 1];
  double acc = 0.0;
  for (int64_t a0 = r0 + (int64_t)blockIdx.x * blockDim.x; a0 < r1; a0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = a0 + threadIdx.x;
    for (int64_t b0 = r0; b0 < r1; b0 += 64) {
      __syncthreads();
      const int nb = (int)(r1 - b0 < 64 ? r1 - b0 : 64);
      for (int idx = threadIdx.x; idx < 64 * dp; idx += blockDim.x) {
        const int bb = idx / dp, j = idx % dp;
        sx[idx] = bb < nb ? xt[(b0 + bb) * dp + j] : 0.f;
      }
      __syncthreads();
      if (a < r1) {
        const float* xa = xt + a * dp;
        for (int bb = 0; bb < nb; ++bb) {
          float u2 = 0.f;
          for (int j = 0; j < dp; ++j) {
            const float df = xa[j] - sx[bb * dp + j];
            u2 = fmaf(df, df, u2);
          }
          const float u = sqrtf(u2);
          acc += (b0 + bb == a) ? 1.0 : (double)(fmaf(u2, kC2, fmaf(u, kC1, 1.f)) * exp2f(-u));
        }
      }
    }
  }
  const double v = block_sum64(acc, sh);
  if (threadIdx.x == 0 && v != 0.0) atomicAdd(sums + (int64_t)i * stride, s * v);
}

Prep model_prep(const gp_model* m) {
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
  return mp;
}

// c (device, k doubles) = Q[:, :k]^T w; two stages
int qtw(gp_ctx* ctx, const float* Q, int64_t ld, int k, const float* w, int64_t n, double* part, double* c) {
  qtw_partial_kernel<<<kPartBlocks, kBlk, 0, ctx->stream>>>(Q, ld, k, w, n, part);
  GP_LAUNCHED(ctx);
  reduce_parts_kernel<<<1, 256, 0, ctx->stream>>>(part, kPartBlocks, k, c);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

int w_minus_qc(gp_ctx* ctx, const float* Q, int64_t ld, int k, const double* c, float* w, int64_t n) {
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kBlk), 8LL * ctx->num_sms));
  w_minus_qc_kernel<<<g, kBlk, sizeof(double) * (size_t)std::max(k, 1), ctx->stream>>>(Q, ld, k, c, w, n);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

}  // namespace

// m steps of Lanczos on K-hat from b (device, n floats) with full
// reorthogonalisation; R = Q C^{-T} written over Q (m vectors, ld n_pad).
// *m_out = the steps taken (fewer when b's Krylov space is exhausted).
int lanczos_cache_build(gp_ctx* ctx, const Prep& p, double s, double sigma2, int precision, const float* b,
                        int m, float* Q, int* m_out) {
  const int64_t n = p.n, ld = p.n_pad;
  float* w = ws<float>(ctx, WS_LV_W, (size_t)ld);
  double* part = ws<double>(ctx, WS_LV_P, (size_t)kPartBlocks * m + 2 * (size_t)m + 16);
  double* h = static_cast<double*>(pinned_get(ctx, sizeof(double) * (m + 8)));
  if (!w || !part || !h) return set_err(ctx, GP_ENOMEM, "workspace (variance cache)");
  double* c = part + (size_t)kPartBlocks * m;
  GP_CUDA(ctx, cudaMemsetAsync(Q, 0, sizeof(float) * (size_t)ld * m, ctx->stream));
  GP_CUDA(ctx, cudaMemsetAsync(w, 0, sizeof(float) * (size_t)ld, ctx->stream));
  // q_0 = b / |b|
  GP_TRY(dot_columns(ctx, b, b, n, n, 1, c));
  GP_CUDA(ctx, cudaMemcpyAsync(h, c, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (!(h[0] > 0.0) || !std::isfinite(h[0])) return set_err(ctx, GP_EINVAL, "variance cache: zero start vector");
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ld, kBlk), 8LL * ctx->num_sms));
  scale_vec_kernel<<<g, kBlk, 0, ctx->stream>>>(b, 1.0 / std::sqrt(h[0]), Q, n, ld);
  GP_LAUNCHED(ctx);
  std::vector<double> alpha(m, 0.0), beta(m, 0.0);
  int steps = 0;
  for (int j = 0; j < m; ++j) {
    float* q = Q + (size_t)j * ld;
    // w = K-hat q_j - beta_{j-1} q_{j-1}
    GP_TRY(kmv(ctx, p, p, q, ld, 1, w, ld, s, sigma2, true, precision));
    if (j > 0) GP_TRY(axpby_vectors(ctx, 1.f, w, (float)-beta[j - 1], Q + (size_t)(j - 1) * ld, w, ld, n, 1));
    // alpha_j = q_j . w;  w -= alpha_j q_j
    GP_TRY(dot_columns(ctx, q, w, ld, n, 1, c));
    GP_CUDA(ctx, cudaMemcpyAsync(h, c, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    GP_TRY(check_status(ctx));
    alpha[j] = h[0];
    GP_TRY(w_minus_qc(ctx, q, ld, 1, c, w, n));
    // full reorthogonalisation against q_0..q_j, twice
    for (int pass = 0; pass < 2; ++pass) {
      GP_TRY(qtw(ctx, Q, ld, j + 1, w, n, part, c));
      GP_TRY(w_minus_qc(ctx, Q, ld, j + 1, c, w, n));
    }
    steps = j + 1;
    GP_TRY(dot_columns(ctx, w, w, ld, n, 1, c));
    GP_CUDA(ctx, cudaMemcpyAsync(h, c, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    beta[j] = std::sqrt(std::max(h[0], 0.0));
    if (j + 1 == m || beta[j] <= 1e-12 * std::fabs(alpha[0])) break;
    scale_vec_kernel<<<g, kBlk, 0, ctx->stream>>>(w, 1.0 / beta[j], Q + (size_t)(j + 1) * ld, n, ld);
    GP_LAUNCHED(ctx);
  }
  // T = C C^T (FP64 Cholesky of the tridiagonal), W = C^{-T}
  const int k = steps;
  std::vector<double> C((size_t)k * k, 0.0), Wd((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) {
    double dsum = alpha[i];
    if (i > 0) dsum -= C[(size_t)i * k + i - 1] * C[(size_t)i * k + i - 1];
    if (!(dsum > 0.0)) return set_err(ctx, GP_EBREAKDOWN, "variance cache: Lanczos tridiagonal not positive definite");
    C[(size_t)i * k + i] = std::sqrt(dsum);
    if (i + 1 < k) C[(size_t)(i + 1) * k + i] = beta[i] / C[(size_t)i * k + i];
  }
  // W = C^{-T}: solve C^T W = I column by column (C lower bidiagonal)
  for (int col = 0; col < k; ++col) {
    // C^T is upper bidiagonal: row i has C[i][i] and C[i+1][i]
    for (int i = k - 1; i >= 0; --i) {
      double v = (i == col) ? 1.0 : 0.0;
      if (i + 1 < k) v -= C[(size_t)(i + 1) * k + i] * Wd[(size_t)(i + 1) * k + col];
      Wd[(size_t)i * k + col] = v / C[(size_t)i * k + i];
    }
  }
  float* Wf = ws<float>(ctx, WS_LV_T, (size_t)k * k);
  float* hw = static_cast<float*>(pinned_get(ctx, sizeof(float) * (size_t)k * k));
  if (!Wf || !hw) return set_err(ctx, GP_ENOMEM, "workspace (variance cache)");
  for (size_t i = 0; i < (size_t)k * k; ++i) hw[i] = (float)Wd[i];
  GP_CUDA(ctx, cudaMemcpyAsync(Wf, hw, sizeof(float) * (size_t)k * k, cudaMemcpyHostToDevice, ctx->stream));
  const size_t shm = sizeof(float) * ((size_t)k * k + (size_t)k * 128);
  GP_CUDA(ctx, cudaFuncSetAttribute(r_from_q_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  r_from_q_kernel<<<(unsigned)ceil_div(ld, 128), 128, shm, ctx->stream>>>(Q, ld, k, Wf, ld);
  GP_LAUNCHED(ctx);
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *m_out = k;
  return GP_OK;
}

// var (device, M) = s - |R^T k*|^2 for the prepared test rows q
int cached_variance(gp_ctx* ctx, const gp_model* m, const Prep& mp, const Prep& q, float* var) {
  float* KR = ws<float>(ctx, WS_LV_K, (size_t)m->love_m * q.n);
  if (!KR) return set_err(ctx, GP_ENOMEM, "workspace (cached variance)");
  GP_TRY(kmv(ctx, q, mp, m->love_R, m->n_pad, m->love_m, KR, q.n, m->s, 0.0, false, m->precision));
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(q.n, kBlk), 8LL * ctx->num_sms));
  var_from_cache_kernel<<<g, kBlk, 0, ctx->stream>>>(KR, m->love_m, q.n, m->s, var);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

// sums[0] += sum_{a,b} k(x'_a, x'_b) over the prepared test rows q (FP32 features)
int block_ksum(gp_ctx* ctx, const Prep& q, double s, double* sums) {
  const size_t shm = sizeof(float) * 64 * (size_t)q.d_pad;
  if (shm > 48 * 1024)
    GP_CUDA(ctx, cudaFuncSetAttribute(block_ksum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  block_ksum_kernel<<<(unsigned)ceil_div(q.n, kBlk), kBlk, shm, ctx->stream>>>(q.xt, q.d_pad, q.n, s, sums);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

// sums[j] += sum over the M columns of A (k vectors, ld lda)
int row_sums(gp_ctx* ctx, const float* A, int64_t lda, int k, int64_t M, double* sums) {
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(M, kBlk), 64));
  row_sums_kernel<<<dim3(gx, (unsigned)k), kBlk, 0, ctx->stream>>>(A, lda, k, M, sums);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

Prep model_prep_of(const gp_model* m) { return model_prep(m); }

// One serving batch of `rows` feature rows (device, rows x d) against a
// resident model: mean (device, rows) = K(X', X) a; var (device, nullable)
// from the cache; for each of nseg molecule parts (rows [seg[2i],
// seg[2i+1]) of the batch; seg device) sums[i (1 + kc)] = 1^T K 1 over
// the part and sums[i (1 + kc) + 1 + j] = the part's sum of K(X', X) R_j.
int serve_batch(gp_ctx* ctx, const gp_model* m, const float* Xp, int64_t rows, float* mean, float* var, int nseg,
                const int64_t* seg, double* sums, int64_t max_part_rows) {
  const Prep mp = model_prep(m);
  Prep q;
  GP_TRY(prepare_features(ctx, Xp, rows, m->d, m->mu, m->ell.data(), m->precision, WS_XT2, &q));
  GP_TRY(kmv(ctx, q, mp, m->alpha, m->n_pad, 1, mean, rows, m->s, 0.0, false, m->precision));
  if (!var && nseg == 0) return GP_OK;
  if (!m->love_R) return set_err(ctx, GP_EINVAL, "serving variances need the model's variance cache");
  const int kc = m->love_m;
  float* KR = ws<float>(ctx, WS_LV_K, (size_t)kc * rows);
  if (!KR) return set_err(ctx, GP_ENOMEM, "workspace (serving variances)");
  GP_TRY(kmv(ctx, q, mp, m->love_R, m->n_pad, kc, KR, rows, m->s, 0.0, false, m->precision));
  if (var) {
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, kBlk), 8LL * ctx->num_sms));
    var_from_cache_kernel<<<g, kBlk, 0, ctx->stream>>>(KR, kc, rows, m->s, var);
    GP_LAUNCHED(ctx);
  }
  if (nseg > 0) {
    const int stride = 1 + kc;
    GP_CUDA(ctx, cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)nseg * stride, ctx->stream));
    const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(max_part_rows, kBlk), 16));
    seg_row_sums_kernel<<<dim3(bx, (unsigned)kc, (unsigned)nseg), kBlk, 0, ctx->stream>>>(KR, rows, seg, stride, 1,
                                                                                          sums);
    GP_LAUNCHED(ctx);
    const size_t shm = sizeof(float) * 64 * (size_t)q.d_pad;
    if (shm > 48 * 1024)
      GP_CUDA(ctx, cudaFuncSetAttribute(seg_ksum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    seg_ksum_kernel<<<dim3(bx, (unsigned)nseg), kBlk, shm, ctx->stream>>>(q.xt, q.d_pad, seg, stride, m->s, sums);
    GP_LAUNCHED(ctx);
  }
  return GP_OK;
}

}  // namespace gp
