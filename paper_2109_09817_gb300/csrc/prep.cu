// Feature preparation (A1): column means, scaled/centred features, row
// norms and the split (hi + lo) copies the tensor-core product reads.
//
// Kernel definition (arXiv 2109.09817, Sec. 4 "Matern 5/2"; ARD reading):
// r^2 = sum_j ((x_j - x'_j)/l_j)^2 is translation invariant, so the features
// are centred by their mean before the norm expansion
// r^2 = |x_a|^2 + |x_b|^2 - 2 x_a.x_b, which keeps the cancellation error of
// that expansion proportional to the (smaller) centred norms.
#include "gp_internal.cuh"

namespace gp {
namespace {

__device__ __forceinline__ float to_tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Partial column sums over a block of rows; grid (nblk, ceil(d/32)),
// block (32, 8).
__global__ void mean_partial_kernel(const float* __restrict__ X, int64_t n,
                                    int d, int64_t rows_per_blk,
                                    double* __restrict__ part) {
  __shared__ double sh[8][33];
  const int j = blockIdx.y * 32 + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
  const int64_t r1 = min(n, r0 + rows_per_blk);
  double acc = 0.0;
  if (j < d)
    for (int64_t r = r0 + threadIdx.y; r < r1; r += 8) acc += (double)X[r * d + j];
  sh[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && j < d) {
    double s = 0.0;
    for (int y = 0; y < 8; ++y) s += sh[y][threadIdx.x];
    part[(int64_t)blockIdx.x * d + j] = s;
  }
}

__global__ void mean_final_kernel(const double* __restrict__ part, int nblk,
                                  int d, int64_t n, double* __restrict__ mu) {
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * d + j];
    mu[j] = s / (double)n;
  }
}

// One warp per (padded) row.  norm_mode: 0 = |x~|^2, 1 = |hi+lo|^2 (split),
// 2 = |hi_tf32|^2, 3 = |hi_bf16|^2, 4 = |hi+lo|^2 with bf16 parts.
__global__ void prep_kernel(const float* __restrict__ X, int64_t n, int d,
                            int64_t n_pad, int d_pad,
                            const double* __restrict__ mu,
                            const double* __restrict__ scale,
                            float* __restrict__ xt, float* __restrict__ norm,
                            float* __restrict__ xhi, float* __restrict__ xlo,
                            __nv_bfloat16* __restrict__ bhi,
                            __nv_bfloat16* __restrict__ blo, int norm_mode) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n_pad) return;
  double nrm = 0.0;
  for (int j = lane; j < d_pad; j += 32) {
    float v = 0.f;
    if (row < n && j < d)
      v = (float)(((double)X[row * d + j] - mu[j]) * scale[j]);
    const int64_t o = row * d_pad + j;
    xt[o] = v;
    double e = (double)v;
    if (xhi) {
      const float h = to_tf32_rna(v);
      const float l = to_tf32_rna(v - h);
      xhi[o] = h;
      xlo[o] = l;
      if (norm_mode == 1) e = (double)h + (double)l;
      if (norm_mode == 2) e = (double)h;
    }
    if (bhi) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
      bhi[o] = h;
      blo[o] = l;
      if (norm_mode == 3) e = (double)__bfloat162float(h);
      if (norm_mode == 4) e = (double)__bfloat162float(h) + (double)__bfloat162float(l);
    }
    nrm += e * e;
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
  if (lane == 0) norm[row] = (float)nrm;
}

}  // namespace

int feature_mean(gp_ctx* ctx, const float* X, int64_t n, int d, double* mu) {
  const int nblk = (int)std::min<int64_t>(ceil_div(n, 512), 2 * ctx->num_sms);
  const int64_t rows_per_blk = ceil_div(n, nblk);
  double* part = ws<double>(ctx, WS_PART, (size_t)nblk * d);
  if (!part) return set_err(ctx, GP_ENOMEM, "workspace (mean partials)");
  dim3 grid(nblk, (unsigned)ceil_div(d, 32));
  mean_partial_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(X, n, d, rows_per_blk, part);
  GP_LAUNCHED(ctx);
  mean_final_kernel<<<1, 256, 0, ctx->stream>>>(part, nblk, d, n, mu);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

int prepare_features(gp_ctx* ctx, const float* X, int64_t n, int d,
                     const double* mu_dev, const double* lengthscale_host,
                     int precision, int slot_xt, Prep* out) {
  Prep p;
  p.n = n;
  p.d = d;
  p.n_pad = round_up(std::max<int64_t>(n, 1), kRowPad);
  p.d_pad = (int)round_up(d, kColPad);
  const size_t ne = (size_t)p.n_pad * p.d_pad;
  const int off = slot_xt - WS_XT;  // WS_XT or WS_XT2 families share layout
  float* xt = ws<float>(ctx, WS_XT + off, ne);
  float* nrm = ws<float>(ctx, WS_NORM + off, (size_t)p.n_pad);
  if (!xt || !nrm) return set_err(ctx, GP_ENOMEM, "workspace (features)");
  float *xhi = nullptr, *xlo = nullptr;
  __nv_bfloat16 *bhi = nullptr, *blo = nullptr;
  int norm_mode = 0;
  if (precision == GP_FP32_SPLIT_TF32 || precision == GP_TF32) {
    xhi = ws<float>(ctx, WS_XT_HI + off, ne);
    xlo = ws<float>(ctx, WS_XT_LO + off, ne);
    if (!xhi || !xlo) return set_err(ctx, GP_ENOMEM, "workspace (tf32 split)");
    norm_mode = precision == GP_TF32 ? 2 : 1;
  } else if (precision == GP_BF16_SPLIT || precision == GP_BF16) {
    bhi = ws<__nv_bfloat16>(ctx, WS_XB_HI + off, ne);
    blo = ws<__nv_bfloat16>(ctx, WS_XB_LO + off, ne);
    if (!bhi || !blo) return set_err(ctx, GP_ENOMEM, "workspace (bf16 split)");
    norm_mode = precision == GP_BF16 ? 3 : 4;
  }
  // scale_j = sqrt5 log2e / l_j, staged through the pinned buffer
  // WS_SCALE is shared by both feature families; every use is stream-ordered
  double* scale_dev = ws<double>(ctx, WS_SCALE, (size_t)d);
  double* hst = static_cast<double*>(pinned_get(ctx, sizeof(double) * (size_t)d));
  if (!scale_dev || !hst) return set_err(ctx, GP_ENOMEM, "workspace (scale)");
  for (int j = 0; j < d; ++j) {
    if (!(lengthscale_host[j] > 0.0)) return set_err(ctx, GP_EINVAL, "lengthscale[%d] <= 0", j);
    hst[j] = kFeatScale / lengthscale_host[j];
  }
  GP_CUDA(ctx, cudaMemcpyAsync(scale_dev, hst, sizeof(double) * d, cudaMemcpyHostToDevice, ctx->stream));
  // the pinned staging buffer is reused by later calls: wait for the copy
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int rows_per_block = 8;
  const unsigned grid = (unsigned)ceil_div(p.n_pad, rows_per_block);
  prep_kernel<<<grid, 32 * rows_per_block, 0, ctx->stream>>>(
      X, n, d, p.n_pad, p.d_pad, mu_dev, scale_dev, xt, nrm, xhi, xlo, bhi, blo, norm_mode);
  GP_LAUNCHED(ctx);
  p.xt = xt;
  p.norm = nrm;
  p.xt_hi = xhi;
  p.xt_lo = xlo;
  p.xb_hi = bhi;
  p.xb_lo = blo;
  *out = p;
  return GP_OK;
}

}  // namespace gp
