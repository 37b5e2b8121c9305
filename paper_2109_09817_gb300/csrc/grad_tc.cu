// Backward tiles on tensor cores (split TF32): dL/dtheta for the lengthscales
// and the outputscale.
//
// arXiv 2109.09817 Sec. 2.2 (hyperparameters maximise Eq. ll) and Sec. 3.2
// (mBCG estimates the derivatives).  The quantities are those of the CUDA-core
// backward (grad.cu): with U = [a, u_1..u_t] and W = [a/2, -w_c/(2t)],
//   M_sym = 1/2 (U W^T + W U^T),   F = f o M_sym,
//   f = (5/3)(1 + sqrt5 r) e^{-sqrt5 r} = (5/3)(1 + ln2 u) 2^{-u} (prepared u),
//   G[j]  += sum_a x~_aj^2 (F 1)_a - x~_aj (F X~)_aj,
//   G[d]  += sum_ab k_ab/s M_sym,ab.
// Per CTA: a 128-row tile I and a range of 64-column tiles J.  Per J tile:
//   MMA1  S  = X~_I X~_J^T          (split: hi.[hi;lo]^T + lo.hi^T, SMEM x SMEM)
//   MMA_M M  = P_I Q_J^T            P = [U | W], Q = [W | U] (rows = points),
//                                   A from TMEM, split like MMA1
//   epi   F = f(u) o M/2, row sums of F, sum k o M/2; F written over S as
//         F_hi = tf32(F) and F_lo = F - F_hi
//   MMA3  CX += F X~_J              A = F from TMEM, B = X~^T (features x
//                                   points, K-major over the points of J),
//                                   split: F_hi.[X^T_hi; X^T_lo] + F_lo.X^T_hi
// CX (128 x d) accumulates over all J tiles of the CTA in TMEM; at the end it
// is drained and combined with the row sums.  S, M and F share one TMEM
// buffer, so a tile's MMAs wait for its epilogue; the MMA1/MMA_M of tile j+1
// queue right behind MMA3 of tile j.  Warp roles: 0 TMA producer, 1 MMA
// issuer, 2 TMEM allocator, 4..11 epilogue (two warps per TMEM lane quarter,
// one per 32-column half).  Every wait is bounded (GP_ETIMEOUT on timeout).
#include <algorithm>

#include "gp_internal.cuh"
#include "tc_ptx.cuh"

namespace gp {
namespace {
using namespace tc;

constexpr int GBM = 128;
constexpr int GBN = 64;
constexpr int GNT = 384;        // 4 control warps + 8 epilogue warps
constexpr int GEPI0 = 4;

template <int DP, int PW>
struct GLayout {
  static constexpr int KB = DP / 32;            // 128-byte K boxes of X~
  static constexpr int KP = PW / 32;            // 128-byte K boxes of P, Q
  // one slot of the X~_J / Q_J ring: the tile's next loads overlap its
  // epilogue and MMA3, which the single TMEM buffer serialises anyway
  static constexpr int XS = 1;
  static constexpr int TS = 2;                  // slots of the X~_J^T ring
  static constexpr int A_BOX = GBM * 128;
  static constexpr int J_BOX = GBN * 128;
  static constexpr int A_HI = 0;
  static constexpr int A_LO = KB * A_BOX;
  // ring A slot: per kb [X hi 64 rows][X lo 64 rows], then per kp [Q hi][Q lo]
  static constexpr int RA_X = 0;
  static constexpr int RA_Q = KB * 2 * J_BOX;
  static constexpr int RA_SLOT = RA_Q + KP * 2 * J_BOX;
  // ring B slot: per 32-point atom [X^T hi DP rows][X^T lo DP rows]
  static constexpr int T_ATOM = 2 * DP * 128;
  static constexpr int RB_SLOT = 2 * T_ATOM;
  static constexpr int RA0 = 2 * KB * A_BOX;
  static constexpr int RB0 = RA0 + XS * RA_SLOT;
  static constexpr int BAR = RB0 + TS * RB_SLOT;
  static constexpr int NBAR = 1 + 2 * XS + 2 * TS + 3;
  static constexpr int SRS = BAR + NBAR * 8 + 16;           // 128 row sums (double)
  static constexpr int SG = SRS + GBM * 8;                  // DP + 1 partials (double)
  static constexpr int TOTAL = SG + (DP + 8) * 8;
  static constexpr uint32_t TX_A = 2u * KB * A_BOX;
  static constexpr uint32_t TX_RA = (uint32_t)RA_SLOT;
  static constexpr uint32_t TX_RB = (uint32_t)RB_SLOT;
  // TMEM columns
  static constexpr uint32_t T_S = 0;            // S_hh / F_hi [0,64), S_x / F_lo [64,128)
  static constexpr uint32_t T_M = 128;          // M_hh [128,192), M_x [192,256)
  static constexpr uint32_t T_CX = 256;         // CX_hh [256, 256+DP), CX_x [.., +DP)
  static constexpr uint32_t T_P = T_CX + 2 * DP;  // P_I hi [T_P, +PW), lo [+PW, +2PW)
  static constexpr uint32_t T_COLS = 512;
  static_assert(T_P + 2 * PW <= T_COLS, "TMEM columns");
  // dynamic + 1024 alignment slack + 1024 static (the failure flag) <= 227 KB
  static_assert(TOTAL + 2048 <= 232448, "shared memory");
};

struct GParams {
  const float* nrm;       // row norms (padded), |hi + lo|^2
  const float* xt;        // prepared features (padded rows x DP), FP32
  const float* p_hi;      // P = [U | W] rows, hi / lo (padded rows x PW)
  const float* p_lo;
  int64_t n;
  int tiles_per_split;
  double* G;              // DP + 1 accumulators
  int* status;
};

// MMA_M k-steps: A = P_I from TMEM (hi / lo), B = Q_J slot [hi; lo] per kp.
template <class Ly, int KK, int NK>
__device__ __forceinline__ void mmam_steps(uint32_t dm, uint32_t p_hi, uint32_t p_lo, uint64_t dQ,
                                           uint32_t idw, uint32_t id) {
  if constexpr (KK < NK) {
    constexpr uint32_t BO = ((KK >> 2) * 2 * Ly::J_BOX + (KK & 3) * 32) >> 4;
    mma_ts_imm<KK * 8, BO>(dm, p_hi, dQ, idw, KK ? 1u : 0u);
    mma_ts_imm<KK * 8, BO>(dm + 64, p_lo, dQ, id, 1u);
    mmam_steps<Ly, KK + 1, NK>(dm, p_hi, p_lo, dQ, idw, id);
  }
}
// MMA3 k-steps over the 64 points of J: A = F from TMEM, B = X~^T slot.
template <class Ly, int DP, int KK, int NK>
__device__ __forceinline__ void mma3_steps(uint32_t dcx, uint32_t f_hi, uint32_t f_lo, uint64_t dT,
                                           uint32_t idw, uint32_t id, uint32_t acc0) {
  if constexpr (KK < NK) {
    constexpr uint32_t BO = ((KK >> 2) * Ly::T_ATOM + (KK & 3) * 32) >> 4;
    mma_ts_imm<KK * 8, BO>(dcx, f_hi, dT, idw, KK == 0 ? acc0 : 1u);
    mma_ts_imm<KK * 8, BO>(dcx + DP, f_lo, dT, id, 1u);
    mma3_steps<Ly, DP, KK + 1, NK>(dcx, f_hi, f_lo, dT, idw, id, acc0);
  }
}
// MMA1 k-steps (cross term), as in the fused K-hat V kernel.
template <class Ly, int KK, int NK>
__device__ __forceinline__ void gmma1_steps(uint32_t dhh, uint32_t dx, uint64_t dA_hi, uint64_t dA_lo,
                                            uint64_t dX, uint32_t idw, uint32_t id) {
  if constexpr (KK < NK) {
    constexpr uint32_t AO = ((KK >> 2) * Ly::A_BOX + (KK & 3) * 32) >> 4;
    constexpr uint32_t BO = ((KK >> 2) * 2 * Ly::J_BOX + (KK & 3) * 32) >> 4;
    mma_ss_imm<AO, BO>(dhh, dA_hi, dX, idw, KK ? 1u : 0u);
    mma_ss_imm<AO, BO>(dx, dA_lo, dX, id, 1u);
    gmma1_steps<Ly, KK + 1, NK>(dhh, dx, dA_hi, dA_lo, dX, idw, id);
  }
}

template <int DP, int PW>
__global__ void __launch_bounds__(GNT, 1)
grad_tc_kernel(const __grid_constant__ CUtensorMap map_r_hi, const __grid_constant__ CUtensorMap map_r_lo,
               const __grid_constant__ CUtensorMap map_c_hi, const __grid_constant__ CUtensorMap map_c_lo,
               const __grid_constant__ CUtensorMap map_q_hi, const __grid_constant__ CUtensorMap map_q_lo,
               const __grid_constant__ CUtensorMap map_t_hi, const __grid_constant__ CUtensorMap map_t_lo,
               const GParams p) {
  using Ly = GLayout<DP, PW>;
  constexpr int XS = Ly::XS, TS = Ly::TS;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Ly::BAR);
  uint64_t* bar_a = bars;
  uint64_t* bar_af = bars + 1;          // [XS] ring A slot loaded
  uint64_t* bar_ae = bar_af + XS;       // [XS] ... consumed by MMA1 / MMA_M
  uint64_t* bar_bf = bar_ae + XS;       // [TS] ring B slot loaded
  uint64_t* bar_be = bar_bf + TS;       // [TS] ... consumed by MMA3
  uint64_t* bar_s = bar_be + TS;        // S and M of the tile ready
  uint64_t* bar_f = bar_s + 1;          // F of the tile written (8 warps)
  uint64_t* bar_fin = bar_f + 1;        // all MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + Ly::NBAR);
  double* sRS = reinterpret_cast<double*>(smem + Ly::SRS);
  double* sG = reinterpret_cast<double*>(smem + Ly::SG);
  __shared__ int fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * GBM;
  const int64_t n_col_tiles = (p.n + GBN - 1) / GBN;
  const int64_t jt0 = (int64_t)blockIdx.y * p.tiles_per_split;
  const int64_t jt1 = min(n_col_tiles, jt0 + (int64_t)p.tiles_per_split);
  const int ntiles = (int)(jt1 - jt0);
  if (ntiles <= 0) return;

  if (threadIdx.x == 0) {
    fail = 0;
    mbar_init(bar_a, 1);
    for (int i = 0; i < XS; ++i) {
      mbar_init(bar_af + i, 1);
      mbar_init(bar_ae + i, 1);
    }
    for (int i = 0; i < TS; ++i) {
      mbar_init(bar_bf + i, 1);
      mbar_init(bar_be + i, 1);
    }
    mbar_init(bar_s, 1);
    mbar_init(bar_f, 8);
    mbar_init(bar_fin, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (threadIdx.x < GBM) sRS[threadIdx.x] = 0.0;
  if (threadIdx.x < DP + 8) sG[threadIdx.x] = 0.0;
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(Ly::T_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tmem_slot;

  // P_I (hi / lo) into TMEM: the epilogue warps of column half 0 write their
  // lane quarter's 32 rows
  if (warp >= GEPI0 && ((warp - GEPI0) >> 2) == 0) {
    const int q = warp & 3;
    const int64_t r = row0 + q * 32 + lane;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
#pragma unroll
    for (int c0 = 0; c0 < PW; c0 += 16) {
      uint32_t vh[16], vl[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        vh[c] = __float_as_uint(p.p_hi[r * PW + c0 + c]);
        vl[c] = __float_as_uint(p.p_lo[r * PW + c0 + c]);
      }
      tmem_st16(tbase + lane_off + Ly::T_P + c0, vh);
      tmem_st16(tbase + lane_off + Ly::T_P + PW + c0, vl);
    }
    tmem_wait_st();
  }
  fence_before();
  __syncthreads();
  fence_after();

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------- TMA producer --
    mbar_expect_tx(bar_a, Ly::TX_A);
    for (int kb = 0; kb < Ly::KB; ++kb) {
      tma_2d(smem + Ly::A_HI + kb * Ly::A_BOX, &map_r_hi, bar_a, kb * 32, (int)row0);
      tma_2d(smem + Ly::A_LO + kb * Ly::A_BOX, &map_r_lo, bar_a, kb * 32, (int)row0);
    }
    int armed_a = 0, armed_b = 0;
    for (int j = 0; j < ntiles; ++j) {
      const int col0 = (int)((jt0 + j) * GBN);
      const int xs = j % XS, ts = j % TS;
      if (j >= XS && !mbar_wait(bar_ae + xs, ((j / XS) - 1) & 1, &fail)) break;
      uint8_t* ra = smem + Ly::RA0 + xs * Ly::RA_SLOT;
      mbar_expect_tx(bar_af + xs, Ly::TX_RA);
      for (int kb = 0; kb < Ly::KB; ++kb) {
        tma_2d(ra + Ly::RA_X + (2 * kb) * Ly::J_BOX, &map_c_hi, bar_af + xs, kb * 32, col0);
        tma_2d(ra + Ly::RA_X + (2 * kb + 1) * Ly::J_BOX, &map_c_lo, bar_af + xs, kb * 32, col0);
      }
      for (int kp = 0; kp < Ly::KP; ++kp) {
        tma_2d(ra + Ly::RA_Q + (2 * kp) * Ly::J_BOX, &map_q_hi, bar_af + xs, kp * 32, col0);
        tma_2d(ra + Ly::RA_Q + (2 * kp + 1) * Ly::J_BOX, &map_q_lo, bar_af + xs, kp * 32, col0);
      }
      armed_a = j + 1;
      if (j >= TS && !mbar_wait(bar_be + ts, ((j / TS) - 1) & 1, &fail)) break;
      uint8_t* rb = smem + Ly::RB0 + ts * Ly::RB_SLOT;
      mbar_expect_tx(bar_bf + ts, Ly::TX_RB);
      for (int at = 0; at < 2; ++at) {
        tma_2d(rb + at * Ly::T_ATOM, &map_t_hi, bar_bf + ts, col0 + at * 32, 0);
        tma_2d(rb + at * Ly::T_ATOM + DP * 128, &map_t_lo, bar_bf + ts, col0 + at * 32, 0);
      }
      armed_b = j + 1;
    }
    mbar_wait_exit(bar_a, 0);
    for (int j = max(0, armed_a - XS); j < armed_a; ++j) mbar_wait_exit(bar_af + (j % XS), (j / XS) & 1);
    for (int j = max(0, armed_b - TS); j < armed_b; ++j) mbar_wait_exit(bar_bf + (j % TS), (j / TS) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------- MMA issuer --
    constexpr uint32_t ID1W = idesc_tf32(GBM, 2 * GBN), ID1 = idesc_tf32(GBM, GBN);
    constexpr uint32_t ID3W = idesc_tf32(GBM, 2 * DP), ID3 = idesc_tf32(GBM, DP);
    const uint64_t dA_hi = sdesc(su32(smem + Ly::A_HI)), dA_lo = sdesc(su32(smem + Ly::A_LO));
    const uint64_t dRA0 = sdesc(su32(smem + Ly::RA0)), dRB0 = sdesc(su32(smem + Ly::RB0));
    const uint32_t tS = tbase + Ly::T_S, tM = tbase + Ly::T_M, tCX = tbase + Ly::T_CX, tP = tbase + Ly::T_P;
    bool ok = mbar_wait(bar_a, 0, &fail);
    fence_after();
    for (int j = 0; ok && j < ntiles; ++j) {
      const int xs = j % XS, ts = j % TS;
      if (!(ok = mbar_wait(bar_af + xs, (j / XS) & 1, &fail))) break;
      fence_after();
      const uint64_t dX = dRA0 + (uint64_t)((xs * Ly::RA_SLOT + Ly::RA_X) >> 4);
      const uint64_t dQ = dRA0 + (uint64_t)((xs * Ly::RA_SLOT + Ly::RA_Q) >> 4);
      gmma1_steps<Ly, 0, DP / 8>(tS, tS + 64, dA_hi, dA_lo, dX, ID1W, ID1);
      mmam_steps<Ly, 0, PW / 8>(tM, tP, tP + PW, dQ, ID1W, ID1);
      mma_commit(bar_ae + xs);
      mma_commit(bar_s);
      if (!(ok = mbar_wait(bar_f, j & 1, &fail))) break;
      fence_after();
      if (!(ok = mbar_wait(bar_bf + ts, (j / TS) & 1, &fail))) break;
      fence_after();
      const uint64_t dT = dRB0 + (uint64_t)((ts * Ly::RB_SLOT) >> 4);
      mma3_steps<Ly, DP, 0, GBN / 8>(tCX, tS, tS + 64, dT, ID3W, ID3, j == 0 ? 0u : 1u);
      mma_commit(bar_be + ts);
    }
    mma_commit(bar_fin);
    mbar_wait_exit(bar_fin, 0);
  } else if (warp >= GEPI0) {
    // ----------------------------------------------------------- epilogue --
    const int e = warp - GEPI0;
    const int q = warp & 3;               // TMEM lane quarter
    const int h = e >> 2;                 // column half (32 columns)
    const int r = q * 32 + lane;
    const int64_t grow = row0 + r;
    const float na = p.nrm[grow];
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    double rs = 0.0, gs = 0.0;
    bool ok = true;
    for (int j = 0; j < ntiles; ++j) {
      const int64_t col0 = (jt0 + j) * GBN;
      if (!(ok = mbar_wait(bar_s, j & 1, &fail))) break;
      fence_after();
      const bool diag = row0 < col0 + GBN && col0 < row0 + GBM;
      float rsf = 0.f, gsf = 0.f;
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        const int cb = h * 32 + half * 16;
        const uint32_t sa = tbase + lane_off + Ly::T_S + cb;
        const uint32_t ma = tbase + lane_off + Ly::T_M + cb;
        uint32_t sh[16], sx[16], mh[16], mx[16];
        tmem_ld16(sa, sh);
        tmem_ld16(sa + 64, sx);
        tmem_ld16(ma, mh);
        tmem_ld16(ma + 64, mx);
        tmem_wait_ld();
        const float4* nb4 = reinterpret_cast<const float4*>(p.nrm + col0 + cb);
        const int64_t dc = grow - (col0 + cb);
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
          const float4 n4 = __ldg(nb4 + c4);
          const float nbv[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int c = c4 * 4 + i;
            const float sab = __uint_as_float(sh[c]) + __uint_as_float(sx[c]);
            const float u2 = fmaxf(fmaf(-2.f, sab, na + nbv[i]), 1e-30f);
            const float uu = u2 * rsqrt_approx(u2);
            const float ex = ex2_approx(-uu);
            float ku = fmaf(u2, kC2, fmaf(uu, kC1, 1.f)) * ex;
            float fv = (5.f / 3.f) * fmaf(uu, kC1, 1.f) * ex;
            if (diag && dc == c) {
              ku = 1.f;
              fv = 5.f / 3.f;
            }
            const float msym = 0.5f * (__uint_as_float(mh[c]) + __uint_as_float(mx[c]));
            const float F = fv * msym;
            rsf += F;
            gsf = fmaf(ku, msym, gsf);
            const float fh = tf32_rna(F);
            sh[c] = __float_as_uint(fh);
            sx[c] = __float_as_uint(F - fh);
          }
        }
        tmem_st16(sa, sh);
        tmem_st16(sa + 64, sx);
      }
      rs += (double)rsf;
      gs += (double)gsf;
      tmem_wait_st();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_f);
    }
    // ---- drain CX, combine with the row sums
    if (ok) ok = mbar_wait(bar_fin, 0, &fail);
    fence_after();
    atomicAdd(&sRS[r], rs);
    for (int off = 16; off > 0; off >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, off);
    if (lane == 0) atomicAdd(&sG[DP], gs);
    asm volatile("bar.sync 1, 256;" ::: "memory");   // the 8 epilogue warps
    if (ok) {
      const double rsum = sRS[r];
      constexpr int FH = DP / 2;          // features of this warp's half
#pragma unroll
      for (int f0 = 0; f0 < FH; f0 += 8) {
        uint32_t ch[8], cx[8];
        const uint32_t ca = tbase + lane_off + Ly::T_CX + h * FH + f0;
        tmem_ld8(ca, ch);
        tmem_ld8(ca + DP, cx);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int fj = h * FH + f0 + i;
          const double x = (grow < p.n) ? (double)p.xt[grow * DP + fj] : 0.0;
          double v = x * x * rsum - x * ((double)__uint_as_float(ch[i]) + (double)__uint_as_float(cx[i]));
          for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          if (lane == 0) atomicAdd(&sG[fj], v);
        }
      }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    if (ok && warp == GEPI0)
      for (int jf = lane; jf <= DP; jf += 32) atomicAdd(p.G + jf, sG[jf]);
  }
  // ------------------------------------------------------------- teardown --
  fence_before();
  __syncthreads();
  if (warp == 2) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(Ly::T_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && fail) atomicExch(p.status, GP_ETIMEOUT);
}

// P = [U | W], Q = [W | U] as (padded rows x PW) hi / lo; rows >= n and
// columns >= 2 T1 are zero.
__global__ void pq_kernel(const float* __restrict__ U, const float* __restrict__ W, int64_t ld, int T1,
                          int64_t n, int64_t npad, int PW, float* __restrict__ ph, float* __restrict__ pl,
                          float* __restrict__ qh, float* __restrict__ ql) {
  const int64_t total = npad * PW;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = i / PW;
    const int c = (int)(i % PW);
    float pv = 0.f, qv = 0.f;
    if (a < n && c < 2 * T1) {
      const float u = c < T1 ? U[(int64_t)c * ld + a] : W[(int64_t)(c - T1) * ld + a];
      const float w = c < T1 ? W[(int64_t)c * ld + a] : U[(int64_t)(c - T1) * ld + a];
      pv = u;
      qv = w;
    }
    const float p1 = tf32_rna(pv), q1 = tf32_rna(qv);
    ph[i] = p1;
    pl[i] = tf32_rna(pv - p1);
    qh[i] = q1;
    ql[i] = tf32_rna(qv - q1);
  }
}

// X~^T hi / lo (DP x padded rows) from the row-major hi / lo features.
__global__ void xt_transpose_kernel(const float* __restrict__ xh, const float* __restrict__ xl, int64_t npad,
                                    int DP, float* __restrict__ th, float* __restrict__ tl) {
  __shared__ float sh[32][33], sl[32][33];
  const int64_t a0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    sh[i][threadIdx.x] = xh[(a0 + i) * DP + j0 + threadIdx.x];
    sl[i][threadIdx.x] = xl[(a0 + i) * DP + j0 + threadIdx.x];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    th[(int64_t)(j0 + i) * npad + a0 + threadIdx.x] = sh[threadIdx.x][i];
    tl[(int64_t)(j0 + i) * npad + a0 + threadIdx.x] = sl[threadIdx.x][i];
  }
}

template <int DP, int PW>
int launch_grad_tc(gp_ctx* ctx, const Prep& pr, const float* U, const float* W, int T1, double* G) {
  using Ly = GLayout<DP, PW>;
  const int64_t npad = pr.n_pad;
  float* ph = ws<float>(ctx, WS_GT_P, (size_t)4 * npad * PW);
  float* th = ws<float>(ctx, WS_GT_T, (size_t)2 * npad * DP);
  if (!ph || !th) return set_err(ctx, GP_ENOMEM, "workspace (tensor-core gradient)");
  float* pl = ph + (size_t)npad * PW;
  float* qh = pl + (size_t)npad * PW;
  float* ql = qh + (size_t)npad * PW;
  float* tl = th + (size_t)npad * DP;
  const unsigned g = (unsigned)std::min<int64_t>(ceil_div(npad * PW, 256), 16LL * ctx->num_sms);
  pq_kernel<<<g, 256, 0, ctx->stream>>>(U, W, npad, T1, pr.n, npad, PW, ph, pl, qh, ql);
  GP_LAUNCHED(ctx);
  xt_transpose_kernel<<<dim3((unsigned)(npad / 32), DP / 32), dim3(32, 8), 0, ctx->stream>>>(
      pr.xt_hi, pr.xt_lo, npad, DP, th, tl);
  GP_LAUNCHED(ctx);
  CUtensorMap mrh, mrl, mch, mcl, mqh, mql, mth, mtl;
  GP_TRY(make_map(ctx, &mrh, pr.xt_hi, npad, DP, DP, GBM));
  GP_TRY(make_map(ctx, &mrl, pr.xt_lo, npad, DP, DP, GBM));
  GP_TRY(make_map(ctx, &mch, pr.xt_hi, npad, DP, DP, GBN));
  GP_TRY(make_map(ctx, &mcl, pr.xt_lo, npad, DP, DP, GBN));
  GP_TRY(make_map(ctx, &mqh, qh, npad, PW, PW, GBN));
  GP_TRY(make_map(ctx, &mql, ql, npad, PW, PW, GBN));
  GP_TRY(make_map(ctx, &mth, th, DP, npad, npad, DP));
  GP_TRY(make_map(ctx, &mtl, tl, DP, npad, npad, DP));
  int* status = device_status(ctx);
  if (!status) return set_err(ctx, GP_ENOMEM, "workspace (status)");
  const size_t smem = Ly::TOTAL + 1024;
  static std::atomic<uint64_t> attr{0};
  GP_TRY(smem_attr_once(ctx, grad_tc_kernel<DP, PW>, smem, attr));
  const int64_t row_tiles = ceil_div(pr.n, GBM), col_tiles = ceil_div(pr.n, GBN);
  int64_t splits = std::max<int64_t>(1, ceil_div(4LL * ctx->num_sms, row_tiles));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, col_tiles / 4));
  // L2-sized column bands, as in the forward product
  const int64_t tile_bytes = (int64_t)GBN * (2 * DP + 2 * PW + 2 * DP) * 4;
  splits = std::max<int64_t>(splits, ceil_div(col_tiles, std::max<int64_t>(64, (48LL << 20) / tile_bytes)));
  const int64_t per = ceil_div(col_tiles, splits);
  splits = ceil_div(col_tiles, per);
  GParams prm;
  prm.nrm = pr.norm;
  prm.xt = pr.xt;
  prm.p_hi = ph;
  prm.p_lo = pl;
  prm.n = pr.n;
  prm.tiles_per_split = (int)per;
  prm.G = G;
  prm.status = status;
  grad_tc_kernel<DP, PW><<<dim3((unsigned)row_tiles, (unsigned)splits), GNT, smem, ctx->stream>>>(
      mrh, mrl, mch, mcl, mqh, mql, mth, mtl, prm);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

}  // namespace

bool grad_tc_supported(const Prep& p, int T1) {
  return p.xt_hi && p.xt_lo && p.xt && (p.d_pad == 32 || p.d_pad == 64) && 2 * T1 <= 64;
}

int grad_tc(gp_ctx* ctx, const Prep& p, const float* U, const float* W, int T1, double* G) {
  if (!grad_tc_supported(p, T1)) return set_err(ctx, GP_EINVAL, "tensor-core gradient: unsupported shape");
  if (p.d_pad == 32)
    return 2 * T1 <= 32 ? launch_grad_tc<32, 32>(ctx, p, U, W, T1, G) : launch_grad_tc<32, 64>(ctx, p, U, W, T1, G);
  return 2 * T1 <= 32 ? launch_grad_tc<64, 32>(ctx, p, U, W, T1, G) : launch_grad_tc<64, 64>(ctx, p, U, W, T1, G);
}

}  // namespace gp
