// Feature preparation (A1): column means, scaled/centred features, row
// norms and the split (hi + lo) copies the tensor-core products read.
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
// 2 = |hi_tf32|^2.  amax (nullable): running max |x~| over the matrix, as
// the bits of a non-negative float (their integer order is the float order).
__global__ void prep_kernel(const float* __restrict__ X, int64_t n, int d,
                            int64_t n_pad, int d_pad,
                            const double* __restrict__ mu,
                            const double* __restrict__ scale,
                            float* __restrict__ xt, float* __restrict__ norm,
                            float* __restrict__ xhi, float* __restrict__ xlo,
                            unsigned* __restrict__ amax, int norm_mode) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n_pad) return;
  double nrm = 0.0;
  float vmax = 0.f;
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
    vmax = fmaxf(vmax, fabsf(v));
    nrm += e * e;
  }
  for (int off = 16; off > 0; off >>= 1) {
    nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
  }
  if (lane == 0) {
    norm[row] = (float)nrm;
    if (amax && vmax > 0.f) atomicMax(amax, __float_as_uint(vmax));
  }
}

// 2^e with e chosen so that m 2^e lies in [2^14, 2^15) (1 for m = 0).
__device__ __forceinline__ int half_exponent(float m) {
  if (!(m > 0.f)) return 0;
  int ex;
  frexpf(m, &ex);            // m = f 2^ex, f in [0.5, 1)
  return kHalfTop - ex;
}

// FP16 split of the prepared features (GP_FP32_SPLIT_F16): one warp per
// padded row, two of the kHalfCols columns per lane.  v' = 2^e x~ (exact),
// hi = fp16(v'), lo = fp16(v' - hi), so hi + lo = v' to 2^-22 relative (the
// same 22 bits as the TF32 split).  norm_h = |hi + lo|^2 2^-2e in FP64, so
// that u^2 = n_a + n_b - 2 x~_a.x~_b vanishes for a row against itself.
__global__ void split_h_kernel(const float* __restrict__ xt, int64_t n_pad, int d_pad,
                               const unsigned* __restrict__ amax, __half* __restrict__ hhi,
                               __half* __restrict__ hlo, float* __restrict__ norm_h,
                               float* __restrict__ xh_scale) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  const int e = half_exponent(__uint_as_float(*amax));
  if (row == 0 && lane == 0) xh_scale[0] = ldexpf(1.f, -e);
  if (row >= n_pad) return;
  double nrm = 0.0;
  for (int j = lane; j < kHalfCols; j += 32) {
    const float v = j < d_pad ? ldexpf(xt[row * d_pad + j], e) : 0.f;
    const __half h = __float2half_rn(v);
    const __half l = __float2half_rn(v - __half2float(h));
    hhi[row * kHalfCols + j] = h;
    hlo[row * kHalfCols + j] = l;
    const double r = ldexp((double)__half2float(h) + (double)__half2float(l), -e);
    nrm += r * r;
  }
  for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
  if (lane == 0) norm_h[row] = (float)nrm;
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
  int norm_mode = 0;
  // the FP16 split form keeps the TF32 split too: the backward kernel of the
  // training pass reads it
  const bool half = precision == GP_FP32_SPLIT_F16;
  if (precision == GP_FP32_SPLIT_TF32 || precision == GP_TF32 || half) {
    xhi = ws<float>(ctx, WS_XT_HI + off, ne);
    xlo = ws<float>(ctx, WS_XT_LO + off, ne);
    if (!xhi || !xlo) return set_err(ctx, GP_ENOMEM, "workspace (tf32 split)");
    norm_mode = precision == GP_TF32 ? 2 : 1;
  }
  __half *hhi = nullptr, *hlo = nullptr;
  float *nrm_h = nullptr, *hsc = nullptr;
  unsigned* amax = nullptr;
  if (half) {
    if (p.d_pad > kHalfCols) return set_err(ctx, GP_EINVAL, "split FP16 form needs d <= %d", kHalfCols);
    const size_t nh = (size_t)p.n_pad * kHalfCols;
    hhi = ws<__half>(ctx, WS_XH_HI + off, nh);
    hlo = ws<__half>(ctx, WS_XH_LO + off, nh);
    nrm_h = ws<float>(ctx, WS_NORMH + off, (size_t)p.n_pad);
    hsc = ws<float>(ctx, WS_XH_SC + off, 64);   // [0] 2^-e, [16] max |x~| bits
    if (!hhi || !hlo || !nrm_h || !hsc) return set_err(ctx, GP_ENOMEM, "workspace (fp16 split)");
    amax = reinterpret_cast<unsigned*>(hsc + 16);
    GP_CUDA(ctx, cudaMemsetAsync(amax, 0, sizeof(unsigned), ctx->stream));
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
      X, n, d, p.n_pad, p.d_pad, mu_dev, scale_dev, xt, nrm, xhi, xlo, amax, norm_mode);
  GP_LAUNCHED(ctx);
  if (half) {
    split_h_kernel<<<grid, 32 * rows_per_block, 0, ctx->stream>>>(xt, p.n_pad, p.d_pad, amax, hhi, hlo,
                                                                    nrm_h, hsc);
    GP_LAUNCHED(ctx);
  }
  p.xt = xt;
  p.norm = nrm;
  p.xt_hi = xhi;
  p.xt_lo = xlo;
  p.xh_hi = hhi;
  p.xh_lo = hlo;
  p.norm_h = nrm_h;
  p.xh_scale = hsc;
  *out = p;
  return GP_OK;
}

}  // namespace gp
