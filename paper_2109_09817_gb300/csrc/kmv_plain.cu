// K-hat V on the FP32 pipe only (precision GP_FP32_PLAIN): the plain form the
// tensor-core product is measured against.
//
// arXiv 2109.09817 Sec. 3.1: CG needs only products with K-hat; Sec. 3.2:
// O(N) memory, so K is formed tile by tile and never stored; Sec. 4: the
// kernel work is done in tiles.  Per CTA: a 128-row tile I of the output and
// a range of 64-column tiles J.  For each J:
//   S   = X~_I X~_J^T                      (FFMA, d-chunks of 32 staged in smem)
//   K   = matern(|x~_a|^2 + |x~_b|^2 - 2 S) (FP32 + 2 MUFU per entry)
//   O_I += K V_J                            (packed FFMA2 from a transposed K tile)
// O is flushed with one atomic add per output element per CTA (several CTAs
// share a row tile so that the grid fills the GPU).
#include <algorithm>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr int BM = 128;        // rows per CTA tile
constexpr int BN = 64;         // columns per J tile
constexpr int KC = 32;         // feature chunk
constexpr int SXS = KC + 4;    // smem row stride of feature tiles (floats)
constexpr int SKS = BM + 4;    // smem row stride of the K^T tile
constexpr int NT = 256;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// k/s as a function of u^2 in prepared units (u = sqrt5 r log2 e).
__device__ __forceinline__ float matern_unit(float u2) {
  u2 = fmaxf(u2, 0.f);
  const float u = sqrt_approx(u2);
  const float p = fmaf(u2, kC2, fmaf(u, kC1, 1.f));
  return p * ex2_approx(-u);
}

template <int TC>
__global__ void __launch_bounds__(NT, 2)
kmv_plain_kernel(const float* __restrict__ xr, const float* __restrict__ nr,
                 int64_t nrows, const float* __restrict__ xc,
                 const float* __restrict__ nc, int64_t ncols, int d_pad,
                 const float* __restrict__ V, int64_t ldv, int t,
                 float* __restrict__ out, int64_t ldo, float s, int sym,
                 int tiles_per_split) {
  extern __shared__ __align__(16) float smem[];
  float* sXI = smem;                   // BM x SXS
  float* sXJ = sXI + BM * SXS;         // BN x SXS
  float* sKT = sXJ + BN * SXS;         // BN x SKS   (K^T: [col][row])
  float* sVT = sKT + BN * SKS;         // TC x (BN + 1)
  float* sNI = sVT + TC * (BN + 1);    // BM
  float* sNJ = sNI + BM;               // BN

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t n_col_tiles = (ncols + BN - 1) / BN;
  const int64_t jt0 = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t jt1 = min(n_col_tiles, jt0 + (int64_t)tiles_per_split);
  if (jt0 >= jt1) return;

  if (tid < BM) sNI[tid] = nr[row0 + tid];
  constexpr int QN = TC / 16;
  float acc_o[8][QN], acc_c[8][QN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      acc_o[i][q] = 0.f;
      acc_c[i][q] = 0.f;
    }

  for (int64_t jt = jt0; jt < jt1; ++jt) {
    const int64_t col0 = jt * BN;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < d_pad; k0 += KC) {
      __syncthreads();
      for (int i = tid; i < BM * (KC / 4); i += NT) {
        const int r = i / (KC / 4), q = i % (KC / 4);
        *reinterpret_cast<float4*>(sXI + r * SXS + q * 4) =
            *reinterpret_cast<const float4*>(xr + (row0 + r) * d_pad + k0 + q * 4);
      }
      for (int i = tid; i < BN * (KC / 4); i += NT) {
        const int r = i / (KC / 4), q = i % (KC / 4);
        *reinterpret_cast<float4*>(sXJ + r * SXS + q * 4) =
            *reinterpret_cast<const float4*>(xc + (col0 + r) * d_pad + k0 + q * 4);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < KC; kk += 4) {
        float4 b[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          b[j] = *reinterpret_cast<const float4*>(sXJ + (tx + 16 * j) * SXS + kk);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 a = *reinterpret_cast<const float4*>(sXI + (ty * 8 + i) * SXS + kk);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float v = acc[i][j];
            v = fmaf(a.x, b[j].x, v);
            v = fmaf(a.y, b[j].y, v);
            v = fmaf(a.z, b[j].z, v);
            v = fmaf(a.w, b[j].w, v);
            acc[i][j] = v;
          }
        }
      }
    }
    // column norms and the V_J^T tile
    if (tid < BN) sNJ[tid] = nc[col0 + tid];
    for (int i = tid; i < TC * BN; i += NT) {
      const int c = i / BN, b = i % BN;
      const int64_t col = col0 + b;
      sVT[c * (BN + 1) + b] = (c < t && col < ncols) ? V[(int64_t)c * ldv + col] : 0.f;
    }
    __syncthreads();
    const bool diag = sym && (row0 < col0 + BN) && (col0 < row0 + BM);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = tx + 16 * j;
      const float nb = sNJ[cc];
      float kv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = ty * 8 + i;
        kv[i] = matern_unit(fmaf(-2.f, acc[i][j], sNI[r] + nb));
        if (diag && row0 + r == col0 + cc) kv[i] = 1.f;
      }
      *reinterpret_cast<float4*>(sKT + cc * SKS + ty * 8) = make_float4(kv[0], kv[1], kv[2], kv[3]);
      *reinterpret_cast<float4*>(sKT + cc * SKS + ty * 8 + 4) = make_float4(kv[4], kv[5], kv[6], kv[7]);
    }
    __syncthreads();
    // the contraction with V_J, two rows per packed FP32x2 instruction
    float2 tile_o[4][QN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < QN; ++q) tile_o[i][q] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int b = 0; b < BN; ++b) {
      const float4 k0 = *reinterpret_cast<const float4*>(sKT + b * SKS + ty * 8);
      const float4 k1 = *reinterpret_cast<const float4*>(sKT + b * SKS + ty * 8 + 4);
      const float2 kr[4] = {make_float2(k0.x, k0.y), make_float2(k0.z, k0.w), make_float2(k1.x, k1.y),
                            make_float2(k1.z, k1.w)};
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        const float v = sVT[(tx + 16 * q) * (BN + 1) + b];
        const float2 v2 = make_float2(v, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) tile_o[i][q] = __ffma2_rn(kr[i], v2, tile_o[i][q]);
      }
    }
    // compensated (Kahan) running sum of the per-tile partial sums: over
    // ~1e5 significant columns a plain FP32 running sum drifts by ~1e-5
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        const float to = (i & 1) ? tile_o[i >> 1][q].y : tile_o[i >> 1][q].x;
        const float yv = to - acc_c[i][q];
        const float tv = acc_o[i][q] + yv;
        acc_c[i][q] = (tv - acc_o[i][q]) - yv;
        acc_o[i][q] = tv;
      }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t r = row0 + ty * 8 + i;
    if (r >= nrows) continue;
#pragma unroll
    for (int q = 0; q < QN; ++q) {
      const int c = tx + 16 * q;
      if (c < t) atomicAdd(out + (int64_t)c * ldo + r, s * (acc_o[i][q] - acc_c[i][q]));
    }
  }
}

__global__ void init_out_kernel(const float* __restrict__ V, int64_t ldv, int t,
                                int64_t n, float* __restrict__ out, int64_t ldo,
                                float sigma2) {
  const int64_t total = n * t;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / n, a = i % n;
    out[c * ldo + a] = V ? sigma2 * V[c * ldv + a] : 0.f;
  }
}

template <int TC>
int launch_plain(gp_ctx* ctx, const Prep& rows, const Prep& cols,
                 const float* V, int64_t ldv, int t, float* out, int64_t ldo,
                 float s, bool sym) {
  const size_t smem = sizeof(float) * (BM * SXS + BN * SXS + BN * SKS +
                                       TC * (BN + 1) + BM + BN);
  static std::atomic<uint64_t> attr{0};
  GP_TRY(smem_attr_once(ctx, kmv_plain_kernel<TC>, smem, attr));
  const int64_t row_tiles = ceil_div(rows.n, BM);
  const int64_t col_tiles = ceil_div(cols.n, BN);
  // enough CTAs for ~4 waves at 2 CTAs per SM, at least 4 J tiles per CTA
  const int64_t want = 8LL * ctx->num_sms;
  int64_t splits = std::max<int64_t>(1, ceil_div(want, row_tiles));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, col_tiles / 4));
  const int64_t per = ceil_div(col_tiles, splits);
  splits = ceil_div(col_tiles, per);
  dim3 grid((unsigned)row_tiles, (unsigned)splits);
  kmv_plain_kernel<TC><<<grid, NT, smem, ctx->stream>>>(
      rows.xt, rows.norm, rows.n, cols.xt, cols.norm, cols.n, rows.d_pad, V,
      ldv, t, out, ldo, s, sym ? 1 : 0, (int)per);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

}  // namespace

int kmv_init_out(gp_ctx* ctx, const float* V, int64_t ldv, int t, int64_t n,
                 float* out, int64_t ldo, float sigma2) {
  const int64_t total = n * t;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(total, 256), 16LL * ctx->num_sms);
  init_out_kernel<<<std::max(1u, grid), 256, 0, ctx->stream>>>(V, ldv, t, n, out, ldo, sigma2);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

int kmv_plain(gp_ctx* ctx, const Prep& rows, const Prep& cols, const float* V,
              int64_t ldv, int t, float* out, int64_t ldo, float s, bool sym) {
  for (int c0 = 0; c0 < t; c0 += 32) {
    const int tc = std::min(32, t - c0);
    const float* Vc = V + (int64_t)c0 * ldv;
    float* Oc = out + (int64_t)c0 * ldo;
    if (tc <= 16) {
      GP_TRY(launch_plain<16>(ctx, rows, cols, Vc, ldv, tc, Oc, ldo, s, sym));
    } else {
      GP_TRY(launch_plain<32>(ctx, rows, cols, Vc, ldv, tc, Oc, ldo, s, sym));
    }
  }
  return GP_OK;
}

int kmv(gp_ctx* ctx, const Prep& rows, const Prep& cols, const float* V,
        int64_t ldv, int t, float* out, int64_t ldo, double s, double sigma2,
        bool sym, int precision) {
  if (precision != GP_FP32_PLAIN && !kmv_tc_supported(rows, t, precision))
    return set_err(ctx, GP_EINVAL, "precision %d not supported for d=%d, t=%d",
                   precision, rows.d, t);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->prof) {
    if (ctx->ev_used == ctx->ev.size()) {
      cudaEvent_t a, b;
      GP_CUDA(ctx, cudaEventCreate(&a));
      GP_CUDA(ctx, cudaEventCreate(&b));
      ctx->ev.emplace_back(a, b);
    }
    e0 = ctx->ev[ctx->ev_used].first;
    e1 = ctx->ev[ctx->ev_used].second;
    ctx->ev_used++;
    ctx->prof_flops += 2.0 * (double)rows.n * (double)cols.n * (double)(rows.d + t);
    ctx->prof_elems += kmv_uses_sym(ctx, rows, cols, sym, precision) ? kmv_sym_entries(rows.n)
                                                                 : (double)rows.n * (double)cols.n;
  }
  GP_TRY(kmv_init_out(ctx, sym ? V : nullptr, ldv, t, rows.n, out, ldo, (float)sigma2));
  if (e0) GP_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
  if (precision != GP_FP32_PLAIN)
    GP_TRY(kmv_tc(ctx, rows, cols, V, ldv, t, out, ldo, (float)s, sym, precision));
  else
    GP_TRY(kmv_plain(ctx, rows, cols, V, ldv, t, out, ldo, (float)s, sym));
  if (e1) GP_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
  return GP_OK;
}

}  // namespace gp
