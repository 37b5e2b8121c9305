// Pivoted Cholesky preconditioner in FP64 (A7).
//
// arXiv 2109.09817 Sec. 3.2: BBMM preconditions CG with a pivoted Cholesky
// factor (refs. bach2013sharp, harbrecht2012low).  Greedy rank-k factor
// K ~ L L^T: at step j pick p = argmax of the residual diagonal
// d = diag(K - L L^T) (lowest index on ties), form the kernel column
// K(X, x_p) in FP64 by direct differences, subtract L_{:,<j} L_{p,<j}^T,
// divide by sqrt(d_p), update d -= l_j^2 and take p out (d_p = 0).
// Stops early when max d <= 1e-12 s.  The preconditioner is P = L L^T + D
// with D = sigma^2 I (the form of Sec. 3.2) or D = diag(K - L L^T) + sigma^2 I
// (diagonal-corrected: the residual diagonal d of the same factorisation).
// P is applied by the Woodbury identity with L~ = D^{-1/2} L and the k x k
// FP64 matrix C = I + L~^T L~:  P^{-1} = D^{-1/2} (I - L~ C^{-1} L~^T) D^{-1/2},
// log|P| = sum_a log D_a + log|C|.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gp_internal.cuh"

namespace gp {
namespace {

struct PcState {
  double dtop;
  int piv;
  int rank;
  int stop;
  int bad;
};

constexpr int kArgBlocks = 512;

__device__ __forceinline__ void better(double& v, int64_t& i, double v2, int64_t i2) {
  // larger value wins; equal values: lower index wins; NaN loses
  if (v2 > v || (v2 == v && i2 < i) || (v != v && v2 == v2)) {
    v = v2;
    i = i2;
  }
}

__global__ void pc_init_kernel(double* dres, int64_t n, double s, PcState* st) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x)
    dres[a] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->dtop = 0.0;
    st->piv = -1;
    st->rank = 0;
    st->stop = 0;
    st->bad = 0;
  }
}

__global__ void pc_argmax_partial(const double* __restrict__ dres, int64_t n,
                                  double* __restrict__ pv, int64_t* __restrict__ pi,
                                  const PcState* st) {
  if (st->stop) return;
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  double v = -1.0;
  int64_t idx = INT64_MAX;
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x)
    better(v, idx, dres[a], a);
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      double v2 = sv[threadIdx.x + off];
      int64_t i2 = si[threadIdx.x + off];
      double v1 = sv[threadIdx.x];
      int64_t i1 = si[threadIdx.x];
      better(v1, i1, v2, i2);
      sv[threadIdx.x] = v1;
      si[threadIdx.x] = i1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}

__global__ void pc_argmax_final(const double* __restrict__ pv,
                                const int64_t* __restrict__ pi, int nparts,
                                double thresh, int j, int64_t* __restrict__ piv,
                                PcState* st) {
  if (st->stop) return;
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  double v = -1.0;
  int64_t idx = INT64_MAX;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) better(v, idx, pv[b], pi[b]);
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      double v1 = sv[threadIdx.x];
      int64_t i1 = si[threadIdx.x];
      better(v1, i1, sv[threadIdx.x + off], si[threadIdx.x + off]);
      sv[threadIdx.x] = v1;
      si[threadIdx.x] = i1;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double top = sv[0];
    if (!(top == top) || isinf(top)) {
      st->bad = 1;
      st->stop = 1;
      return;
    }
    if (top <= thresh) {
      st->stop = 1;
      return;
    }
    st->dtop = top;
    st->piv = (int)si[0];
    piv[j] = si[0];
    st->rank = j + 1;
  }
}

// Column j of L and the residual-diagonal update; one thread per row.
__global__ void pc_column_kernel(const float* __restrict__ X, int64_t n, int d,
                                 const double* __restrict__ inv_l, double s,
                                 double* __restrict__ L, double* __restrict__ dres,
                                 int j, const PcState* __restrict__ st) {
  extern __shared__ double shp[];   // d pivot features, then j pivot-row L entries
  if (st->stop) return;
  const int p = st->piv;
  double* xp = shp;
  double* lp = shp + d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) xp[i] = (double)X[(int64_t)p * d + i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) lp[i] = L[(int64_t)i * n + p];
  __syncthreads();
  const double inv_sq = 1.0 / sqrt(st->dtop);
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    double r2 = 0.0;
    const float* xa = X + a * d;
    for (int i = 0; i < d; ++i) {
      const double u = ((double)xa[i] - xp[i]) * inv_l[i];
      r2 += u * u;
    }
    const double r = sqrt(r2);
    const double sr = kSqrt5 * r;
    double col = s * (1.0 + sr + (5.0 / 3.0) * r2) * exp(-sr);
    for (int i = 0; i < j; ++i) col -= L[(int64_t)i * n + a] * lp[i];
    const double l = col * inv_sq;
    L[(int64_t)j * n + a] = l;
    // the residual diagonal of a PSD Schur complement is >= 0 and exactly 0
    // at a pivot: a pivot (and a row whose residual has reached 0) stays 0,
    // rounding below 0 is clamped
    const double dr = dres[a];
    dres[a] = (a == p || dr == 0.0) ? 0.0 : fmax(dr - l * l, 0.0);
  }
}

__global__ void pc_rank_kernel(const PcState* st, int* rank, int* bad) {
  *rank = st->rank;
  *bad = st->bad;
}

// Gram matrix G = L^T L (rank x rank, FP64), partial sums over row chunks.
// grid = (row chunks, pair chunks of 8*256); each thread owns up to 8 pairs
// (i, jj), i >= jj, of the packed lower triangle.
__device__ __forceinline__ void unrank_pair(int pidx, int& i, int& jj) {
  i = (int)((sqrt(8.0 * pidx + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > pidx) --i;
  while ((i + 1) * (i + 2) / 2 <= pidx) ++i;
  jj = pidx - i * (i + 1) / 2;
}

__global__ void pc_gram_partial(const double* __restrict__ L, int64_t n, int k,
                                int64_t rows_per_blk, const double* __restrict__ Dg,
                                double* __restrict__ part) {
  extern __shared__ double sl[];   // 32 rows x k
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
  const int64_t r1 = min(n, r0 + rows_per_blk);
  const int npairs = k * (k + 1) / 2;
  const int pbase = blockIdx.y * 8 * blockDim.x;
  double acc[8];
  int pi_[8], pj_[8];
  for (int q = 0; q < 8; ++q) {
    acc[q] = 0.0;
    const int pidx = pbase + threadIdx.x + q * blockDim.x;
    pi_[q] = -1;
    pj_[q] = 0;
    if (pidx < npairs) unrank_pair(pidx, pi_[q], pj_[q]);
  }
  for (int64_t rb = r0; rb < r1; rb += 32) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * k; idx += blockDim.x) {
      const int rr = idx % 32, c = idx / 32;
      const int64_t row = rb + rr;
      sl[rr * k + c] = row < r1 ? L[(int64_t)c * n + row] / sqrt(Dg[row]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (pi_[q] < 0) continue;
      double a = acc[q];
      for (int rr = 0; rr < 32; ++rr) a += sl[rr * k + pi_[q]] * sl[rr * k + pj_[q]];
      acc[q] = a;
    }
  }
  for (int q = 0; q < 8; ++q) {
    const int pidx = pbase + threadIdx.x + q * blockDim.x;
    if (pidx < npairs) part[(int64_t)blockIdx.x * npairs + pidx] = acc[q];
  }
}

// C = I + G; in-place lower Cholesky (one block); logdet of C.
__global__ void pc_small_chol(const double* __restrict__ part, int nparts, int k,
                              double diag_add, double* __restrict__ C,
                              double* __restrict__ logdet_out, int* bad) {
  const int npairs = k * (k + 1) / 2;
  for (int pidx = threadIdx.x; pidx < npairs; pidx += blockDim.x) {
    int i, jj;
    unrank_pair(pidx, i, jj);
    double g = 0.0;
    for (int b = 0; b < nparts; ++b) g += part[(int64_t)b * npairs + pidx];
    if (i == jj) g += diag_add;
    C[i * k + jj] = g;
    C[jj * k + i] = (i == jj) ? g : 0.0;   // upper part cleared below
  }
  __syncthreads();
  // right-looking Cholesky on the lower triangle
  for (int c = 0; c < k; ++c) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const double dg = C[c * k + c];
      if (!(dg > 0.0)) *bad = 1;
      C[c * k + c] = sqrt(fmax(dg, 1e-300));
    }
    __syncthreads();
    const double piv = C[c * k + c];
    for (int r = c + 1 + threadIdx.x; r < k; r += blockDim.x) C[r * k + c] /= piv;
    __syncthreads();
    for (int idx = threadIdx.x; idx < (k - c - 1) * (k - c - 1); idx += blockDim.x) {
      const int r = c + 1 + idx / (k - c - 1);
      const int q = c + 1 + idx % (k - c - 1);
      if (q <= r) C[r * k + q] -= C[r * k + c] * C[q * k + c];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ld = 0.0;
    for (int c = 0; c < k; ++c) ld += 2.0 * log(C[c * k + c]);
    *logdet_out = ld;
  }
}

// Cinv = (F F^T)^{-1} from the lower factor F (k x k): column q of the
// inverse solves F F^T x = e_q; one thread per column.
__global__ void pc_small_inverse(const double* __restrict__ F, int k,
                                 double* __restrict__ Cinv) {
  for (int q = threadIdx.x; q < k; q += blockDim.x) {
    double* x = Cinv + (int64_t)q * k;   // column q (symmetric result)
    for (int j = 0; j < k; ++j) {
      double s = (j == q) ? 1.0 : 0.0;
      for (int i = 0; i < j; ++i) s -= F[j * k + i] * x[i];
      x[j] = s / F[j * k + j];
    }
    for (int j = k - 1; j >= 0; --j) {
      double s = x[j];
      for (int i = j + 1; i < k; ++i) s -= F[i * k + j] * x[i];
      x[j] = s / F[j * k + j];
    }
  }
}

// D_a = (resid_a or 0) + sigma2 (FP64), dh_a = D_a^{-1/2} (FP32, 0 on padding)
// L (FP64, row j contiguous, ld n) as FP32 pairs: Lff[j ld32 + a] = hi =
// fl32(L), Lff[(rank + j) ld32 + a] = fl32(L - hi); 0 on the padding rows
__global__ void pc_split_ff_kernel(const double* __restrict__ L, int64_t n, int rank, int64_t ld32,
                                   float* __restrict__ Lff) {
  const int64_t total = (int64_t)rank * ld32;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx / ld32, a = idx % ld32;
    const double v = a < n ? L[j * n + a] : 0.0;
    const float vh = (float)v;
    Lff[idx] = vh;
    Lff[total + idx] = (float)(v - (double)vh);
  }
}

__global__ void pc_diag_kernel(const double* __restrict__ resid, double sigma2, int64_t n,
                               int64_t ld32, double* __restrict__ Dg, float* __restrict__ dh,
                               float* __restrict__ d2ff) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < ld32;
       a += (int64_t)gridDim.x * blockDim.x) {
    if (a < n) {
      const double D = (resid ? resid[a] : 0.0) + sigma2;
      Dg[a] = D;
      dh[a] = (float)(1.0 / sqrt(D));
      // D^{-1} as an FP32 pair hi + lo (the Woodbury apply's float-float)
      const double q = 1.0 / D;
      const float qh = (float)q;
      d2ff[a] = qh;
      d2ff[ld32 + a] = (float)(q - (double)qh);
    } else {
      dh[a] = 0.f;
      d2ff[a] = 0.f;
      d2ff[ld32 + a] = 0.f;
    }
  }
}

// sum_a log D_a (FP64), fixed-order two-stage
__global__ void pc_logd_partial(const double* __restrict__ Dg, int64_t n, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x)
    acc += log(Dg[a]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// L~ = D^{-1/2} L in FP32, k_used x ld32 (zero on padding)
__global__ void to_f32_kernel(const double* __restrict__ L, int64_t n, int k,
                              const double* __restrict__ Dg, float* __restrict__ L32,
                              int64_t ld32) {
  const int64_t total = (int64_t)k * ld32;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / ld32, a = i % ld32;
    L32[i] = a < n ? (float)(L[c * n + a] / sqrt(Dg[a])) : 0.f;
  }
}

}  // namespace

int pivchol_run(gp_ctx* ctx, const float* X, int64_t n, int d,
                const double* lengthscale_host, double s, int k, double* L,
                int64_t* piv, int* rank_out, double* resid_out) {
  double* dres = ws<double>(ctx, WS_PC_D, (size_t)n);
  PcState* st = static_cast<PcState*>(ws_get(ctx, WS_PC_STATE, sizeof(PcState) + 64));
  double* pv = ws<double>(ctx, WS_PC_GRAM, 2 * kArgBlocks);
  double* inv_l = ws<double>(ctx, WS_SCALE, (size_t)d);
  double* hst = static_cast<double*>(pinned_get(ctx, sizeof(double) * (size_t)(d + 2)));
  if (!dres || !st || !pv || !inv_l || !hst) return set_err(ctx, GP_ENOMEM, "workspace (pivchol)");
  int64_t* pi = reinterpret_cast<int64_t*>(pv + kArgBlocks);
  for (int i = 0; i < d; ++i) hst[i] = 1.0 / lengthscale_host[i];
  GP_CUDA(ctx, cudaMemcpyAsync(inv_l, hst, sizeof(double) * d, cudaMemcpyHostToDevice, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  GP_CUDA(ctx, cudaMemsetAsync(L, 0, sizeof(double) * (size_t)n * k, ctx->stream));
  GP_CUDA(ctx, cudaMemsetAsync(piv, 0xff, sizeof(int64_t) * (size_t)k, ctx->stream));
  const unsigned eg = (unsigned)std::min<int64_t>(ceil_div(n, 256), 8LL * ctx->num_sms);
  pc_init_kernel<<<std::max(1u, eg), 256, 0, ctx->stream>>>(dres, n, s, st);
  GP_LAUNCHED(ctx);
  const int nparts = (int)std::min<int64_t>(kArgBlocks, std::max<int64_t>(1, ceil_div(n, 2048)));
  const double thresh = 1e-12 * s;
  for (int j = 0; j < k; ++j) {
    pc_argmax_partial<<<nparts, 256, 0, ctx->stream>>>(dres, n, pv, pi, st);
    GP_LAUNCHED(ctx);
    pc_argmax_final<<<1, 256, 0, ctx->stream>>>(pv, pi, nparts, thresh, j, piv, st);
    GP_LAUNCHED(ctx);
    const size_t shm = sizeof(double) * (size_t)(d + j + 1);
    pc_column_kernel<<<std::max(1u, eg), 256, shm, ctx->stream>>>(X, n, d, inv_l, s, L, dres, j, st);
    GP_LAUNCHED(ctx);
  }
  int* hr = static_cast<int*>(pinned_get(ctx, 2 * sizeof(int)));
  int* dr = reinterpret_cast<int*>(reinterpret_cast<char*>(st) + sizeof(PcState));
  pc_rank_kernel<<<1, 1, 0, ctx->stream>>>(st, dr, dr + 1);
  GP_LAUNCHED(ctx);
  GP_CUDA(ctx, cudaMemcpyAsync(hr, dr, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *rank_out = hr[0];
  if (hr[1]) return set_err(ctx, GP_ENONPD, "pivoted Cholesky: non-finite residual diagonal at step %d", hr[0]);
  if (resid_out)
    GP_CUDA(ctx, cudaMemcpyAsync(resid_out, dres, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
  return GP_OK;
}

int precond_setup(gp_ctx* ctx, const double* L, int64_t n, int k_alloc,
                  int rank, double sigma2, const double* resid, Precond* out) {
  Precond pc;
  pc.n = n;
  pc.k = rank;
  pc.L = L;
  pc.sigma2 = sigma2;
  pc.resid = resid;
  pc.ld32 = round_up(std::max<int64_t>(n, 1), kRowPad);
  (void)k_alloc;
  double* Dg = ws<double>(ctx, WS_PC_DG, (size_t)pc.ld32 + 512);
  float* dh = ws<float>(ctx, WS_PC_DH, (size_t)pc.ld32);
  float* d2ff = ws<float>(ctx, WS_PC_D2FF, (size_t)2 * pc.ld32);
  if (!Dg || !dh || !d2ff) return set_err(ctx, GP_ENOMEM, "workspace (preconditioner diagonal)");
  double* lpart = Dg + pc.ld32;   // 256 partial sums of log D
  const unsigned eg0 = (unsigned)std::min<int64_t>(ceil_div(pc.ld32, 256), 16LL * ctx->num_sms);
  pc_diag_kernel<<<eg0, 256, 0, ctx->stream>>>(resid, sigma2, n, pc.ld32, Dg, dh, d2ff);
  GP_LAUNCHED(ctx);
  pc_logd_partial<<<256, 256, 0, ctx->stream>>>(Dg, n, lpart);
  GP_LAUNCHED(ctx);
  pc.dh = dh;
  pc.d2ff = d2ff;
  double* cf = ws<double>(ctx, WS_PC_CF, (size_t)2 * std::max(rank, 1) * std::max(rank, 1) + 8);
  if (!cf) return set_err(ctx, GP_ENOMEM, "workspace (preconditioner)");
  double* cinv = cf + (size_t)rank * rank;
  double* ld_dev = cinv + (size_t)rank * rank;
  int* bad_dev = reinterpret_cast<int*>(ld_dev + 1);
  GP_CUDA(ctx, cudaMemsetAsync(ld_dev, 0, 2 * sizeof(double), ctx->stream));
  if (rank > 0) {
    float* L32 = ws<float>(ctx, WS_PC_L32, (size_t)rank * pc.ld32);
    float* Lff = ws<float>(ctx, WS_PC_LFF, (size_t)2 * rank * pc.ld32);
    if (!Lff) return set_err(ctx, GP_ENOMEM, "workspace (preconditioner factor pairs)");
    const unsigned egs = (unsigned)std::min<int64_t>(ceil_div((int64_t)rank * pc.ld32, 256), 16LL * ctx->num_sms);
    pc_split_ff_kernel<<<egs, 256, 0, ctx->stream>>>(L, n, rank, pc.ld32, Lff);
    GP_LAUNCHED(ctx);
    pc.Lff = Lff;
    const int npairs = rank * (rank + 1) / 2;
    const int nblk = (int)std::min<int64_t>(std::max<int64_t>(1, ceil_div(n, 4096)), 2 * ctx->num_sms);
    const int64_t rows_per_blk = ceil_div(n, nblk);
    double* part = ws<double>(ctx, WS_PC_GRAM, (size_t)nblk * npairs + 2 * kArgBlocks);
    if (!L32 || !part) return set_err(ctx, GP_ENOMEM, "workspace (preconditioner)");
    const unsigned eg = (unsigned)std::min<int64_t>(ceil_div((int64_t)rank * pc.ld32, 256), 16LL * ctx->num_sms);
    to_f32_kernel<<<eg, 256, 0, ctx->stream>>>(L, n, rank, Dg, L32, pc.ld32);
    GP_LAUNCHED(ctx);
    const size_t shm = sizeof(double) * 32 * rank;
    if (shm > 48 * 1024) {
      GP_CUDA(ctx, cudaFuncSetAttribute(pc_gram_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    }
    dim3 ggrid(nblk, (unsigned)ceil_div(npairs, 8 * 256));
    pc_gram_partial<<<ggrid, 256, shm, ctx->stream>>>(L, n, rank, rows_per_blk, Dg, part);
    GP_LAUNCHED(ctx);
    pc_small_chol<<<1, 256, 0, ctx->stream>>>(part, nblk, rank, 1.0, cf, ld_dev, bad_dev);
    GP_LAUNCHED(ctx);
    pc_small_inverse<<<1, 128, 0, ctx->stream>>>(cf, rank, cinv);
    GP_LAUNCHED(ctx);
    pc.L32 = L32;
    pc.cfac = cf;
    pc.cinv = cinv;
  }
  double* hb = static_cast<double*>(pinned_get(ctx, 260 * sizeof(double)));
  if (!hb) return set_err(ctx, GP_ENOMEM, "pinned staging");
  GP_CUDA(ctx, cudaMemcpyAsync(hb, ld_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaMemcpyAsync(hb + 2, lpart, 256 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int bad = 0;
  std::memcpy(&bad, hb + 1, sizeof(int));
  if (bad) return set_err(ctx, GP_ENONPD, "I + L~^T L~ is not positive definite");
  double sumlogd = 0.0;
  for (int i = 0; i < 256; ++i) sumlogd += hb[2 + i];
  pc.logdet = sumlogd + hb[0];
  *out = pc;
  return GP_OK;
}

}  // namespace gp
