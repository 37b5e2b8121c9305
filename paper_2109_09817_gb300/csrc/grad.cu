// Backward tiles (A9): dL/dtheta for the lengthscales and outputscale.
//
// arXiv 2109.09817 Sec. 2.2 (hyperparameters maximise Eq. ll) and Sec. 3.2
// (mBCG estimates the derivatives).  With a = K-hat^{-1} y, probes z_c,
// u_c = K-hat^{-1} z_c and w_c = P^{-1} z_c,
//   dL/dtheta = sum_ab M_ab dK-hat_ab/dtheta,
//   M = 1/2 a a^T - 1/(2t) sum_c u_c w_c^T,
// and since dK-hat is symmetric M may be replaced by
//   M_sym = 1/2 (U W^T + W U^T),  U = [a, u_1..u_t], W = [a/2, -w_c/(2t)].
// For the Matern-5/2 ARD kernel (Sec. 4)
//   dk/dl_j = s f(r) (x_j - x'_j)^2 / l_j^3,  f = (5/3)(1 + sqrt5 r) e^{-sqrt5 r},
//   dk/ds   = k / s,
// and with F = f o M_sym (symmetric)
//   sum_ab F_ab (x~_aj - x~_bj)^2 = 2 [ sum_a x~_aj^2 (F 1)_a - sum_a x~_aj (F X~)_aj ].
// Per CTA: a 128-row tile I and a range of 64-column tiles J; K is
// recomputed per tile and never stored.  Accumulated (FP64 atomics):
//   G[j] += sum_{a in I} x~_aj^2 (F 1)_a - x~_aj (F X~)_aj   (prepared units)
//   G[d_pad] += sum_{a in I, b} k_ab/s M_sym,ab
#include <algorithm>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr int BM = 128, BN = 64, NT = 256;
constexpr int SKS = BM + 4;

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

template <int DP, int PW>   // DP = padded features, PW = 2 * T1 (padded to 32)
__global__ void __launch_bounds__(NT, 1)
grad_kernel(const float* __restrict__ xt, const float* __restrict__ nrm,
            int64_t n, int64_t ld, const float* __restrict__ U,
            const float* __restrict__ W, int T1, double* __restrict__ G,
            int tiles_per_split) {
  constexpr int SX = DP + 4;
  constexpr int SP = PW + 4;
  extern __shared__ __align__(16) float smem[];
  float* sXI = smem;               // BM x SX
  float* sXJ = sXI + BM * SX;      // BN x SX
  float* sPI = sXJ + BN * SX;      // BM x SP   ([U | W] rows of I)
  float* sPJ = sPI + BM * SP;      // BN x SP   ([W | U] rows of J)
  float* sCT = sPJ + BN * SP;      // BN x SKS  (F^T)
  float* sNI = sCT + BN * SKS;     // BM
  float* sNJ = sNI + BM;           // BN
  float* sRS = sNJ + BN;           // BM row sums
  double* sG = reinterpret_cast<double*>(sRS + BM);   // 16 x DP partials + 32

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t n_col_tiles = (n + BN - 1) / BN;
  const int64_t jt0 = (int64_t)blockIdx.y * tiles_per_split;
  const int64_t jt1 = min(n_col_tiles, jt0 + (int64_t)tiles_per_split);
  if (jt0 >= jt1) return;

  for (int i = tid; i < BM * (DP / 4); i += NT) {
    const int r = i / (DP / 4), q = i % (DP / 4);
    *reinterpret_cast<float4*>(sXI + r * SX + q * 4) =
        *reinterpret_cast<const float4*>(xt + (row0 + r) * DP + q * 4);
  }
  for (int i = tid; i < BM * PW; i += NT) {
    const int q = i / BM, r = i % BM;
    float v = 0.f;
    if (q < T1) v = U[(int64_t)q * ld + row0 + r];
    else if (q < 2 * T1) v = W[(int64_t)(q - T1) * ld + row0 + r];
    sPI[r * SP + q] = v;
  }
  if (tid < BM) {
    sNI[tid] = nrm[row0 + tid];
    sRS[tid] = 0.f;
  }
  constexpr int QD = DP / 16;
  float cx[8][QD];
  float rs[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    rs[i] = 0.f;
#pragma unroll
    for (int q = 0; q < QD; ++q) cx[i][q] = 0.f;
  }
  double gs = 0.0;

  for (int64_t jt = jt0; jt < jt1; ++jt) {
    const int64_t col0 = jt * BN;
    __syncthreads();
    for (int i = tid; i < BN * (DP / 4); i += NT) {
      const int r = i / (DP / 4), q = i % (DP / 4);
      *reinterpret_cast<float4*>(sXJ + r * SX + q * 4) =
          *reinterpret_cast<const float4*>(xt + (col0 + r) * DP + q * 4);
    }
    for (int i = tid; i < BN * PW; i += NT) {
      const int q = i / BN, r = i % BN;
      float v = 0.f;
      if (q < T1) v = W[(int64_t)q * ld + col0 + r];
      else if (q < 2 * T1) v = U[(int64_t)(q - T1) * ld + col0 + r];
      sPJ[r * SP + q] = v;
    }
    if (tid < BN) sNJ[tid] = nrm[col0 + tid];
    __syncthreads();
    float acc[8][4], mm[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j] = 0.f;
        mm[i][j] = 0.f;
      }
#pragma unroll 2
    for (int kk = 0; kk < DP; kk += 4) {
      float4 b[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = *reinterpret_cast<const float4*>(sXJ + (tx + 16 * j) * SX + kk);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 a = *reinterpret_cast<const float4*>(sXI + (ty * 8 + i) * SX + kk);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float v = acc[i][j];
          v = fmaf(a.x, b[j].x, v); v = fmaf(a.y, b[j].y, v);
          v = fmaf(a.z, b[j].z, v); v = fmaf(a.w, b[j].w, v);
          acc[i][j] = v;
        }
      }
    }
#pragma unroll 2
    for (int kk = 0; kk < PW; kk += 4) {
      float4 b[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = *reinterpret_cast<const float4*>(sPJ + (tx + 16 * j) * SP + kk);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 a = *reinterpret_cast<const float4*>(sPI + (ty * 8 + i) * SP + kk);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float v = mm[i][j];
          v = fmaf(a.x, b[j].x, v); v = fmaf(a.y, b[j].y, v);
          v = fmaf(a.z, b[j].z, v); v = fmaf(a.w, b[j].w, v);
          mm[i][j] = v;
        }
      }
    }
    const bool diag = (row0 < col0 + BN) && (col0 < row0 + BM);
    float gsf = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cc = tx + 16 * j;
      const bool colok = col0 + cc < n;
      float fv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = ty * 8 + i;
        const float u2 = fmaxf(fmaf(-2.f, acc[i][j], sNI[r] + sNJ[cc]), 0.f);
        const float u = sqrt_approx(u2);
        const float e = ex2_approx(-u);
        float ku = fmaf(u2, kC2, fmaf(u, kC1, 1.f)) * e;
        float f = (5.f / 3.f) * fmaf(u, kC1, 1.f) * e;
        if (diag && row0 + r == col0 + cc) {
          ku = 1.f;
          f = 5.f / 3.f;
        }
        const float msym = colok ? 0.5f * mm[i][j] : 0.f;
        gsf = fmaf(ku, msym, gsf);
        fv[i] = f * msym;
        rs[i] += fv[i];
      }
      *reinterpret_cast<float4*>(sCT + cc * SKS + ty * 8) = make_float4(fv[0], fv[1], fv[2], fv[3]);
      *reinterpret_cast<float4*>(sCT + cc * SKS + ty * 8 + 4) = make_float4(fv[4], fv[5], fv[6], fv[7]);
    }
    gs += (double)gsf;
    __syncthreads();
#pragma unroll 4
    for (int b = 0; b < BN; ++b) {
      const float4 k0 = *reinterpret_cast<const float4*>(sCT + b * SKS + ty * 8);
      const float4 k1 = *reinterpret_cast<const float4*>(sCT + b * SKS + ty * 8 + 4);
      const float kr[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
#pragma unroll
      for (int q = 0; q < QD; ++q) {
        const float v = sXJ[b * SX + tx + 16 * q];
#pragma unroll
        for (int i = 0; i < 8; ++i) cx[i][q] = fmaf(kr[i], v, cx[i][q]);
      }
    }
  }
  // ---- reduce: row sums across tx, then per-feature partials across rows
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 8; ++i) atomicAdd(&sRS[ty * 8 + i], rs[i]);
  __syncthreads();
  double gq[QD];
#pragma unroll
  for (int q = 0; q < QD; ++q) gq[q] = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = ty * 8 + i;
    if (row0 + r >= n) continue;
    const double rsum = (double)sRS[r];
#pragma unroll
    for (int q = 0; q < QD; ++q) {
      const double x = (double)sXI[r * SX + tx + 16 * q];
      gq[q] += x * x * rsum - x * (double)cx[i][q];
    }
  }
#pragma unroll
  for (int q = 0; q < QD; ++q) sG[ty * DP + tx + 16 * q] = gq[q];
  // gs: warp reduce then one atomic per warp
  for (int off = 16; off > 0; off >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, off);
  __syncthreads();
  for (int j = tid; j < DP; j += NT) {
    double s = 0.0;
    for (int y = 0; y < 16; ++y) s += sG[y * DP + j];
    atomicAdd(G + j, s);
  }
  if ((tid & 31) == 0) atomicAdd(G + DP, gs);
}

template <int DP, int PW>
int launch_grad(gp_ctx* ctx, const Prep& p, const float* U, const float* W,
                int T1, double* G) {
  constexpr int SX = DP + 4, SP = PW + 4;
  const size_t smem = sizeof(float) * (size_t)(BM * SX + BN * SX + BM * SP + BN * SP +
                                               BN * SKS + BM + BN + BM) +
                      sizeof(double) * (16 * DP + 32);
  static std::atomic<uint64_t> attr{0};
  GP_TRY(smem_attr_once(ctx, grad_kernel<DP, PW>, smem, attr));
  const int64_t row_tiles = ceil_div(p.n, BM), col_tiles = ceil_div(p.n, BN);
  int64_t splits = std::max<int64_t>(1, ceil_div(4LL * ctx->num_sms, row_tiles));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, col_tiles / 4));
  const int64_t per = ceil_div(col_tiles, splits);
  splits = ceil_div(col_tiles, per);
  grad_kernel<DP, PW><<<dim3((unsigned)row_tiles, (unsigned)splits), NT, smem, ctx->stream>>>(
      p.xt, p.norm, p.n, p.n_pad, U, W, T1, G, (int)per);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

template <int DP>
int launch_grad_pw(gp_ctx* ctx, const Prep& p, const float* U, const float* W,
                   int T1, double* G) {
  const int pw = 2 * T1;
  if (pw <= 32) return launch_grad<DP, 32>(ctx, p, U, W, T1, G);
  if (pw <= 64) return launch_grad<DP, 64>(ctx, p, U, W, T1, G);
  if (pw <= 96) return launch_grad<DP, 96>(ctx, p, U, W, T1, G);
  return launch_grad<DP, 128>(ctx, p, U, W, T1, G);
}

}  // namespace

int grad_tiles(gp_ctx* ctx, const Prep& p, const float* U, const float* W,
               int T1, double* G, double* gs, int precision) {
  (void)gs;   // G[d_pad] holds the outputscale sum
  // the split FP16 form keeps the TF32 split features for this kernel
  if ((precision == GP_FP32_SPLIT_TF32 || precision == GP_FP32_SPLIT_F16) && grad_tc_supported(p, T1))
    return grad_tc(ctx, p, U, W, T1, G);
  if (2 * T1 > 128) return set_err(ctx, GP_EINVAL, "gradient: at most 63 probes");
  switch (p.d_pad) {
    case 32: return launch_grad_pw<32>(ctx, p, U, W, T1, G);
    case 64: return launch_grad_pw<64>(ctx, p, U, W, T1, G);
    case 96: return launch_grad_pw<96>(ctx, p, U, W, T1, G);
    case 128: return launch_grad_pw<128>(ctx, p, U, W, T1, G);
    default: return set_err(ctx, GP_EINVAL, "gradient: d = %d > 128 not supported", p.d);
  }
}

}  // namespace gp
