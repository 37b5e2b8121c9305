// Symmetric split-FP16 K-hat V on sm_103a: each kernel tile of the upper
// block triangle is formed once and contracted twice.
//
// arXiv 2109.09817 Sec. 3.1-3.2 (blackbox products with K-hat, O(N) memory)
// and Sec. 4 (kernel tiles).  K(X, X) is symmetric, so the tile K_IJ of a
// 128-row tile I and a 64-column tile J serves both
//   O_I += K_IJ V_J        (the row tile's own output)
//   O_J += K_IJ^T V_I      (the column tile's output)
// and only tiles J at or right of the diagonal block are formed: a row tile
// I covers column tiles 2I, 2I + 1 (its diagonal block, which takes the
// first contraction only) and every tile 2I + 2, 2I + 3, ... (both).  The
// Matern epilogue, the binding cost of the full-grid kernel (kmv_tc.cu), is
// therefore paid for about half of the N^2 entries.
//
// Per CTA: one segment = a row tile I and a run of its column tiles inside
// one column band (bands keep the streamed X~_J / V_J and the transposed
// outputs O_J of the CTAs in flight inside L2).  Per column tile J:
//   MMA1  S = X~_I X~_J^T (three FP16 split products, M = 128, N = 64,
//         K = 16 per MMA); X~_I hi and lo sit in TMEM for the whole segment
//         (A operand from TMEM), X~_J arrives by TMA in a ring
//   epi   K = matern(n_a + n_b - 2 S) as 2^14 K split into FP16 hi + lo,
//         written to TMEM over S (A of the first contraction) and to a
//         128B-swizzled SMEM tile K[a][b] (A of the second, read MN-major)
//   MMA2  O_I += K_hi [V_hi; V_lo]_J + K_lo V_hi,J  (M = 128, A from TMEM)
//   MMAT  for a pair of consecutive column tiles J, J + 1 (128 columns b):
//         D = K_hi^T [V_hi; V_lo]_I + K_lo^T V_hi,I (M = 128, A = K^T of both
//         tiles read MN-major from their adjacent SMEM tiles; V_I loaded
//         once per segment)
//   epi   O_I drained into per-thread compensated sums every OGROUP tiles of
//         a group; each pair's D drained once and added into out with atomics
// Warp roles: 0 TMA producer, 1 MMA1 issuer, 2 TMEM allocator and MMAT
// issuer, 3 MMA2 issuer, 4..19 two epilogue groups of 8 warps (group g takes
// tiles j with j % 2 == g, and drains the pairs p with p % 2 == g).  MMA1
// runs per tile, so the two groups receive their S half a tile apart and
// their compute phases stay staggered on the shared schedulers; one N = 128
// cross term per pair would hand both groups their S together (measured
// 6.5 % slower).  Every mbarrier wait is bounded; a timeout records
// GP_ETIMEOUT in the status word and every role leaves its loop.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "gp_internal.cuh"
#include "tc_ptx.cuh"

namespace gp {
namespace {
using namespace tc;

constexpr int BM = 128;
constexpr int BN = 64;
constexpr int NTHREADS = 640;
constexpr int EPI_WARP0 = 4;
constexpr int GROUP_WARPS = 8;
constexpr int OGROUP = 4;       // a group's tiles accumulated in TMEM per O_I drain
constexpr int DPH = kHalfCols;  // FP16 features per row: one 128-byte box

template <int T>
struct SymLayout {
  // S/K buffers (TMEM and SMEM), an even number: the tiles of a pair sit in
  // adjacent buffers, so that one MN-major descriptor spans both.  Four
  // buffers (two pairs in flight) at both T; at T = 32 the TMEM budget then
  // leaves one O_I accumulator per group and one pair D, and shared memory
  // two X~_J slots.
  static constexpr int NSB = 4;
  static constexpr int XS = T <= 16 ? 3 : 2;     // X~_J ring slots
  static constexpr int VS = 4;                   // V_J ring slots
  static constexpr int OB = T <= 16 ? 2 : 1;     // O_I accumulators per epilogue group
  static constexpr int DP = T <= 16 ? 2 : 1;     // pair D accumulators (M = 128, 2T columns)
  static constexpr int XJ_BOX = BN * 128;        // 64 rows x 128 B
  static constexpr int V_BOX = T * 128;          // T vectors x 64 FP16 columns
  static constexpr int KT = BM * 128;            // one K part: 128 rows a x 64 columns b, FP16
  // shared memory (every tile 1024-byte aligned for the 128B swizzle)
  static constexpr int K0 = 0;                   // [NSB][hi, lo] K tiles
  static constexpr int VI_BOX = 2 * V_BOX;       // per 64 rows of I: [hi T rows][lo T rows]
  static constexpr int VI0 = K0 + NSB * 2 * KT;
  static constexpr int X_SLOT = 2 * XJ_BOX;      // [hi 64 rows][lo 64 rows]
  static constexpr int X0 = VI0 + 2 * VI_BOX;
  static constexpr int V_NRM = 2 * V_BOX;        // [hi T rows][lo T rows][64 column norms]
  static constexpr int V_SLOT = (V_NRM + 256 + 1023) / 1024 * 1024;
  static constexpr int V0 = X0 + XS * X_SLOT;
  static constexpr int BAR = V0 + VS * V_SLOT;
  static constexpr int NBAR = 2 * XS + 2 * VS + 1 + 3 * NSB + 4 * OB + 2 * DP + 1;
  static constexpr int TOTAL = BAR + NBAR * 8 + 16;
  static constexpr uint32_t TX_X = 2u * XJ_BOX;
  static constexpr uint32_t TX_V = 2u * V_BOX + 256u;
  static constexpr uint32_t TX_VI = 2u * VI_BOX;
  // TMEM columns
  static constexpr uint32_t T_XA = 0;                      // X~_I: hi [0, 32), lo [32, 64)
  static constexpr uint32_t T_S = 64;                      // S/K buffers, 64 columns each
  static constexpr uint32_t T_O = T_S + NSB * 64;          // O_I [group][buffer] x 2T
  static constexpr uint32_t T_D = T_O + 2 * OB * 2 * T;    // pair D [buffer] x 2T
  static constexpr uint32_t T_COLS = 512;
  static_assert(T_D + DP * 2 * T <= T_COLS, "TMEM columns");
  static_assert(NSB % 2 == 0, "pairs need adjacent buffers");
  static_assert(TOTAL + 2048 <= 232448, "shared memory");
};

struct SymParams {
  const __half* xh_hi;   // prepared FP16 split features, n_pad x 64 (rows = columns)
  const __half* xh_lo;
  const float* norm;     // |hi + lo|^2 2^-2e per row, n_pad
  const float* xs;       // device scalar 2^-e
  const float* vsc;      // per vector 2^-(e_c + 14)
  int64_t n;             // points
  int row_tiles, col_tiles, band;
  float* out;
  int64_t ldo;
  int t;                 // live vectors in this chunk
  float s;
  int* status;
};

// Segment of a CTA: bands of `band` column tiles in launch order; inside
// band b every row tile I with 2I below the band's end, in increasing I; the
// segment covers column tiles [max(2I, b band), band end).
__device__ __forceinline__ bool segment_of(const SymParams& p, int blk, int* I, int* jt0, int* jt1) {
  int rem = blk;
  for (int b = 0; b * p.band < p.col_tiles; ++b) {
    const int hi = min((b + 1) * p.band, p.col_tiles);
    const int cnt = min(p.row_tiles, (hi + 1) / 2);
    if (rem < cnt) {
      *I = rem;
      *jt0 = max(2 * rem, b * p.band);
      *jt1 = hi;
      return true;
    }
    rem -= cnt;
  }
  return false;
}

// SMEM descriptor of an MN-major operand in the 128B-swizzled layout: rows
// of 128 bytes are consecutive K indices, each holding 64 FP16 along M; 8
// such rows form a 1024-byte atom, atoms follow each other along K (SBO =
// 1024 bytes); the second 64 elements of M (the pair's second tile) sit
// `lbo` bytes on (the leading byte offset).
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr, uint32_t lbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// A operand MN-major (bit 15 of the instruction descriptor)
__host__ __device__ constexpr uint32_t idesc_f16_amn(int M, int N) { return idesc_f16(M, N) | (1u << 15); }

// MMA1: S = A_hi X_hi^T + A_hi X_lo^T + A_lo X_hi^T, A = X~_I from TMEM
// (FP16 pairs, k-step kk at column 8 kk; lo 32 columns on), B = the X~_J
// slot (hi rows, then lo rows XJ_BOX bytes on; 32 bytes per k-step).
template <class Ly, int KK>
__device__ __forceinline__ void mma1_sym_steps(uint32_t d, uint32_t xa, uint64_t dX, uint32_t id) {
  if constexpr (KK < DPH / 16) {
    constexpr uint32_t BO = (KK * 32) >> 4;
    constexpr uint32_t BL = BO + (Ly::XJ_BOX >> 4);
    mma_ts_bf16_imm<8 * KK, BO>(d, xa, dX, id, KK ? 1u : 0u);
    mma_ts_bf16_imm<8 * KK, BL>(d, xa, dX, id, 1u);
    mma_ts_bf16_imm<32 + 8 * KK, BO>(d, xa, dX, id, 1u);
    mma1_sym_steps<Ly, KK + 1>(d, xa, dX, id);
  }
}
// First contraction, as in kmv_tc.cu: O[0, 2T) += K_hi [V_hi; V_lo],
// O[0, T) += K_lo V_hi; K_hi of columns [32h + 16 half, +16) in TMEM columns
// [32h + 8 half, +8) of the S/K buffer, K_lo 16 columns further on.
template <class Ly, int KK>
__device__ __forceinline__ void mma2_sym_steps(uint32_t d, uint32_t khi, uint64_t dV, uint32_t id2w, uint32_t id2,
                                               uint32_t acc0) {
  if constexpr (KK < BN / 16) {
    constexpr uint32_t AO = (KK >> 1) * 32 + (KK & 1) * 8;
    constexpr uint32_t BO = (KK * 32) >> 4;
    mma_ts_bf16_imm<AO, BO>(d, khi, dV, id2w, KK == 0 ? acc0 : 1u);
    mma_ts_bf16_imm<AO + 16, BO>(d, khi, dV, id2, 1u);
    mma2_sym_steps<Ly, KK + 1>(d, khi, dV, id2w, id2, acc0);
  }
}
// Second contraction of a pair: D[0, 2T) = K_hi^T [V_hi; V_lo]_I, D[0, T)
// += K_lo^T V_hi,I, M = 128 (the 64 columns b of each tile), K = the 128 rows
// a in k-steps of 16: A = K^T read MN-major from the two SMEM tiles (16 rows
// a = 2048 bytes per k-step), B = the V_I slot (64 rows a per 128-byte box,
// 32 bytes per k-step).
template <class Ly, int KK>
__device__ __forceinline__ void mmat_sym_steps(uint32_t d, uint64_t dKh, uint64_t dKl, uint64_t dVI, uint32_t idw,
                                               uint32_t id) {
  if constexpr (KK < BM / 16) {
    constexpr uint32_t AO = (KK * 2048) >> 4;
    constexpr uint32_t BO = ((KK >> 2) * Ly::VI_BOX + (KK & 3) * 32) >> 4;
    mma_ss_f16_imm<AO, BO>(d, dKh, dVI, idw, KK ? 1u : 0u);
    mma_ss_f16_imm<AO, BO>(d, dKl, dVI, id, 1u);
    mmat_sym_steps<Ly, KK + 1>(d, dKh, dKl, dVI, idw, id);
  }
}

__device__ __forceinline__ void st_shared_v4(uint8_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(su32(p)), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}

template <int T>
__global__ void __launch_bounds__(NTHREADS, 1)
kmv_sym_kernel(const __grid_constant__ CUtensorMap map_c_hi, const __grid_constant__ CUtensorMap map_c_lo,
               const __grid_constant__ CUtensorMap map_v_hi, const __grid_constant__ CUtensorMap map_v_lo,
               const SymParams p) {
  using Ly = SymLayout<T>;
  constexpr int NSB = Ly::NSB, XS = Ly::XS, VS = Ly::VS, OB = Ly::OB, DP = Ly::DP;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Ly::BAR);
  uint64_t* bar_xf = bars;                 // [XS]  X~_J slot loaded
  uint64_t* bar_xe = bar_xf + XS;          // [XS]  ... consumed by MMA1
  uint64_t* bar_vf = bar_xe + XS;          // [VS]  V_J slot (and norms) loaded
  uint64_t* bar_ve = bar_vf + VS;          // [VS]  ... consumed by MMA2
  uint64_t* bar_vi = bar_ve + VS;          // V_I loaded
  uint64_t* bar_s = bar_vi + 1;            // [NSB] S in buffer b ready
  uint64_t* bar_k = bar_s + NSB;           // [NSB] K of buffer b written (TMEM and SMEM)
  uint64_t* bar_kf = bar_k + NSB;          // [NSB] ... read by both contractions (2 arrivals)
  uint64_t* bar_of = bar_kf + NSB;         // [2 OB] O_I of group g, buffer u ready
  uint64_t* bar_oe = bar_of + 2 * OB;      // [2 OB] ... drained
  uint64_t* bar_df = bar_oe + 2 * OB;      // [DP] pair D in buffer v ready
  uint64_t* bar_de = bar_df + DP;          // [DP] ... drained
  uint64_t* bar_fin = bar_de + DP;         // the three MMA issuers drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + Ly::NBAR);
  __shared__ int fail;
  __shared__ __align__(16) float out_scale[T];   // s 2^-(e_c + 14) per output vector

  int I, jt0, jt1;
  if (!segment_of(p, blockIdx.x, &I, &jt0, &jt1)) return;
  // a CTA of this launch (or an earlier one) already gave up on a wait: the
  // product is void, so the remaining CTAs leave at once
  if (*reinterpret_cast<volatile int*>(p.status) != 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)I * BM;
  const int ntiles = jt1 - jt0;
  const int jt_off = 2 * I + 2;            // tiles from here on are off the diagonal block

  if (threadIdx.x < T) out_scale[threadIdx.x] = threadIdx.x < p.t ? p.s * p.vsc[threadIdx.x] : 0.f;
  if (threadIdx.x == 0) {
    fail = 0;
    for (int i = 0; i < XS; ++i) {
      mbar_init(bar_xf + i, 1);
      mbar_init(bar_xe + i, 1);
    }
    for (int i = 0; i < VS; ++i) {
      mbar_init(bar_vf + i, 1);
      mbar_init(bar_ve + i, 1);
    }
    mbar_init(bar_vi, 1);
    for (int i = 0; i < NSB; ++i) {
      mbar_init(bar_s + i, 1);
      mbar_init(bar_k + i, GROUP_WARPS);
      mbar_init(bar_kf + i, 2);
    }
    for (int i = 0; i < 2 * OB; ++i) {
      mbar_init(bar_of + i, 1);
      mbar_init(bar_oe + i, GROUP_WARPS);
    }
    for (int i = 0; i < DP; ++i) {
      mbar_init(bar_df + i, 1);
      mbar_init(bar_de + i, GROUP_WARPS);
    }
    mbar_init(bar_fin, 3);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
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
  // X~_I hi and lo into TMEM for the whole segment (epilogue group 0: warp
  // quarter q holds rows 32q.., h = 0 the hi part, h = 1 the lo part)
  if (warp >= EPI_WARP0 && warp < EPI_WARP0 + GROUP_WARPS) {
    const int q = warp & 3, h = (warp - EPI_WARP0) >> 2;
    const uint4* src = reinterpret_cast<const uint4*>((h ? p.xh_lo : p.xh_hi) + (row0 + q * 32 + lane) * DPH);
    uint32_t r[32];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint4 v = src[i];
      r[4 * i] = v.x;
      r[4 * i + 1] = v.y;
      r[4 * i + 2] = v.z;
      r[4 * i + 3] = v.w;
    }
    tmem_st32(tbase + ((uint32_t)(q * 32) << 16) + Ly::T_XA + 32 * h, r);
    tmem_wait_st();
  }
  fence_before();
  __syncthreads();
  fence_after();

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------- TMA producer --
    // V_I: the row tile's vectors, B operand of the second contraction
    mbar_expect_tx(bar_vi, Ly::TX_VI);
    for (int kb = 0; kb < 2; ++kb) {
      tma_2d(smem + Ly::VI0 + kb * Ly::VI_BOX, &map_v_hi, bar_vi, (int)row0 + 64 * kb, 0);
      tma_2d(smem + Ly::VI0 + kb * Ly::VI_BOX + Ly::V_BOX, &map_v_lo, bar_vi, (int)row0 + 64 * kb, 0);
    }
    int armed = 0;
    for (int j = 0; j < ntiles; ++j) {
      const int col0 = (jt0 + j) * BN;
      const int xs = j % XS, vs = j % VS;
      if (j >= XS && !mbar_wait(bar_xe + xs, ((j / XS) - 1) & 1, &fail)) break;
      uint8_t* xb = smem + Ly::X0 + xs * Ly::X_SLOT;
      mbar_expect_tx(bar_xf + xs, Ly::TX_X);
      tma_2d(xb, &map_c_hi, bar_xf + xs, 0, col0);
      tma_2d(xb + Ly::XJ_BOX, &map_c_lo, bar_xf + xs, 0, col0);
      if (j >= VS && !mbar_wait(bar_ve + vs, ((j / VS) - 1) & 1, &fail)) {
        mbar_wait_exit(bar_xf + xs, (j / XS) & 1);
        break;
      }
      uint8_t* vb = smem + Ly::V0 + vs * Ly::V_SLOT;
      mbar_expect_tx(bar_vf + vs, Ly::TX_V);
      tma_2d(vb, &map_v_hi, bar_vf + vs, col0, 0);
      tma_2d(vb + Ly::V_BOX, &map_v_lo, bar_vf + vs, col0, 0);
      bulk_g2s(vb + Ly::V_NRM, p.norm + col0, 256, bar_vf + vs);
      armed = j + 1;
    }
    // never leave with bulk copies still landing in this CTA's memory
    mbar_wait_exit(bar_vi, 0);
    for (int j = max(0, armed - XS); j < armed; ++j) mbar_wait_exit(bar_xf + (j % XS), (j / XS) & 1);
    for (int j = max(0, armed - VS); j < armed; ++j) mbar_wait_exit(bar_vf + (j % VS), (j / VS) & 1);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------- MMA1 issuer --
    constexpr uint32_t ID1 = idesc_f16(BM, BN);
    const uint64_t dX0 = sdesc(su32(smem + Ly::X0));
    bool ok = true;
    for (int j = 0; ok && j < ntiles; ++j) {
      const int xs = j % XS, b = j % NSB;
      if (j >= NSB) {
        if (!(ok = mbar_wait(bar_kf + b, ((j / NSB) - 1) & 1, &fail))) break;
        fence_after();
      }
      if (!(ok = mbar_wait(bar_xf + xs, (j / XS) & 1, &fail))) break;
      fence_after();
      const uint64_t dX = dX0 + (uint64_t)(xs * (Ly::X_SLOT >> 4));
      mma1_sym_steps<Ly, 0>(tbase + Ly::T_S + b * 64, tbase + Ly::T_XA, dX, ID1);
      mma_commit(bar_xe + xs);
      mma_commit(bar_s + b);
    }
    mma_commit(bar_fin);
    mbar_wait_exit(bar_fin, 0);
  } else if (warp == 3 && lane == 0) {
    // ------------------------------------------------ first contraction --
    // Tile j: S/K buffer b = j % NSB, group g = j & 1, the group's i-th tile
    // with i = j >> 1; O_I accumulates OGROUP of the group's tiles in buffer
    // u = (i / OGROUP) % OB.
    constexpr uint32_t ID2 = idesc_f16(BM, T), ID2W = idesc_f16(BM, 2 * T);
    const uint64_t dV0 = sdesc(su32(smem + Ly::V0));
    bool ok = true;
    for (int j = 0; ok && j < ntiles; ++j) {
      const int b = j % NSB, vs = j % VS, g = j & 1, i = j >> 1;
      const int og = i / OGROUP, u = og % OB;
      const bool first = (i % OGROUP) == 0;
      const bool last = (i % OGROUP) == OGROUP - 1 || j + 2 >= ntiles;
      if (!(ok = mbar_wait(bar_k + b, (j / NSB) & 1, &fail))) break;
      fence_after();
      if (first && og >= OB) {
        if (!(ok = mbar_wait(bar_oe + g * OB + u, ((og - OB) / OB) & 1, &fail))) break;
        fence_after();
      }
      if (!(ok = mbar_wait(bar_vf + vs, (j / VS) & 1, &fail))) break;
      fence_after();
      const uint64_t dV = dV0 + (uint64_t)(vs * (Ly::V_SLOT >> 4));
      mma2_sym_steps<Ly, 0>(tbase + Ly::T_O + (g * OB + u) * 2 * T, tbase + Ly::T_S + b * 64, dV, ID2W, ID2,
                            first ? 0u : 1u);
      if (last) mma_commit(bar_of + g * OB + u);
      mma_commit(bar_ve + vs);
      mma_commit(bar_kf + b);
    }
    mma_commit(bar_fin);
    mbar_wait_exit(bar_fin, 0);
  } else if (warp == 2 && lane == 0) {
    // ----------------------------------------------- second contraction --
    // Pair p = tiles 2p, 2p + 1 (the second may not exist at the end of a
    // segment; its half of D is then not drained), in buffers b0 = 2p % NSB
    // and b0 + 1, D in buffer v = p % DP.  The diagonal block is always a
    // whole pair (the first of a row tile's first segment) and takes no
    // second contraction, but commits the same barriers, so that every
    // barrier's phase counts pairs and tiles.
    constexpr uint32_t IDT = idesc_f16_amn(BM, T), IDTW = idesc_f16_amn(BM, 2 * T);
    const uint64_t dVI = sdesc(su32(smem + Ly::VI0));
    const uint64_t dK0 = sdesc_mn(su32(smem + Ly::K0), 2 * Ly::KT);
    const int npairs = (ntiles + 1) / 2;
    bool ok = true, vi_ready = false;
    for (int pr = 0; ok && pr < npairs; ++pr) {
      const int j0 = 2 * pr, b0 = j0 % NSB, v = pr % DP;
      const bool two = j0 + 1 < ntiles;
      if (!(ok = mbar_wait(bar_k + b0, (j0 / NSB) & 1, &fail))) break;
      if (two && !(ok = mbar_wait(bar_k + b0 + 1, ((j0 + 1) / NSB) & 1, &fail))) break;
      fence_after();
      if (pr >= DP) {
        if (!(ok = mbar_wait(bar_de + v, ((pr - DP) / DP) & 1, &fail))) break;
        fence_after();
      }
      if (jt0 + j0 >= jt_off) {
        if (!vi_ready) {
          if (!(ok = mbar_wait(bar_vi, 0, &fail))) break;
          fence_after();
          vi_ready = true;
        }
        const uint64_t dKh = dK0 + (uint64_t)((b0 * 2 * Ly::KT) >> 4);
        mmat_sym_steps<Ly, 0>(tbase + Ly::T_D + v * 2 * T, dKh, dKh + (Ly::KT >> 4), dVI, IDTW, IDT);
      }
      mma_commit(bar_df + v);
      mma_commit(bar_kf + b0);
      if (two) mma_commit(bar_kf + b0 + 1);
    }
    mma_commit(bar_fin);
    mbar_wait_exit(bar_fin, 0);
  } else if (warp >= EPI_WARP0) {
    // ----------------------------------------------------------- epilogue --
    const int e = warp - EPI_WARP0;
    const int g = e / GROUP_WARPS;
    const int q = warp & 3;                  // TMEM lane quarter
    const int h = (e % GROUP_WARPS) >> 2;    // column half (32 columns)
    const int r = q * 32 + lane;             // row a within the tile
    const int64_t grow = row0 + r;
    const float na = p.norm[grow];
    const float xs = p.xs[0];
    const float m2 = -2.f * xs * xs;
    const float2 na2 = make_float2(na, na), m22 = make_float2(m2, m2);
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int my_tiles = (ntiles - g + 1) / 2;
    constexpr int TH = T / 2;                // outputs drained by this warp
    float acc[TH], cmp[TH];
#pragma unroll
    for (int c = 0; c < TH; ++c) {
      acc[c] = 0.f;
      cmp[c] = 0.f;
    }
    auto kahan = [&](int c, float v) {
      const float yv = v - cmp[c];
      const float tv = acc[c] + yv;
      cmp[c] = (tv - acc[c]) - yv;
      acc[c] = tv;
    };
    auto drain_o = [&](int og) -> bool {
      const int u = og % OB;
      if (!mbar_wait(bar_of + g * OB + u, (og / OB) & 1, &fail)) return false;
      fence_after();
      const uint32_t oa = tbase + lane_off + Ly::T_O + (g * OB + u) * 2 * T + h * TH;
#pragma unroll
      for (int c8 = 0; c8 < TH; c8 += 8) {
        uint32_t rr[8], rx[8];
        tmem_ld8(oa + c8, rr);
        tmem_ld8(oa + T + c8, rx);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 8; ++c) kahan(c8 + c, __uint_as_float(rr[c]) + __uint_as_float(rx[c]));
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_oe + g * OB + u);
      return true;
    };
    // The pair's D (M = 128): row r = 32 q + lane is column b = 64 (jt0 + 2p)
    // + r of K (rows 64.. belong to the pair's second tile); warp half h adds
    // outputs [h TH, +TH) of its rows into out
    const int npairs = (ntiles + 1) / 2;
    auto drain_d = [&](int pr) -> bool {
      const int v = pr % DP;
      if (!mbar_wait(bar_df + v, (pr / DP) & 1, &fail)) return false;
      fence_after();
      if (jt0 + 2 * pr >= jt_off) {
        const uint32_t da = tbase + lane_off + Ly::T_D + v * 2 * T + h * TH;
        const int64_t bcol = (int64_t)(jt0 + 2 * pr) * BN + r;
        const bool live = bcol < p.n && bcol < (int64_t)(jt0 + ntiles) * BN;
#pragma unroll
        for (int c8 = 0; c8 < TH; c8 += 8) {
          uint32_t rr[8], rx[8];
          tmem_ld8(da + c8, rr);
          tmem_ld8(da + T + c8, rx);
          tmem_wait_ld();
          if (live) {
            // the 8 output factors in two vector loads; a full chunk of
            // vectors (t = T) takes no per-column bound
            const float4 sc0 = reinterpret_cast<const float4*>(out_scale)[(h * TH + c8) >> 2];
            const float4 sc1 = reinterpret_cast<const float4*>(out_scale)[((h * TH + c8) >> 2) + 1];
            const float scv[8] = {sc0.x, sc0.y, sc0.z, sc0.w, sc1.x, sc1.y, sc1.z, sc1.w};
            float* o = p.out + (int64_t)(h * TH + c8) * p.ldo + bcol;
            if (p.t == T) {
#pragma unroll
              for (int c = 0; c < 8; ++c)
                atomicAdd(o + c * p.ldo, scv[c] * (__uint_as_float(rr[c]) + __uint_as_float(rx[c])));
            } else {
#pragma unroll
              for (int c = 0; c < 8; ++c)
                if (h * TH + c8 + c < p.t)
                  atomicAdd(o + c * p.ldo, scv[c] * (__uint_as_float(rr[c]) + __uint_as_float(rx[c])));
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_de + v);
      return true;
    };
    bool ok = true;
    for (int i = 0; i < my_tiles; ++i) {
      const int j = 2 * i + g;
      const int b = j % NSB, vs = j % VS;
      const int64_t col0 = (int64_t)(jt0 + j) * BN;
      if (!(ok = mbar_wait(bar_s + b, (j / NSB) & 1, &fail))) break;
      if (!(ok = mbar_wait(bar_vf + vs, (j / VS) & 1, &fail))) break;
      fence_after();
      const bool diag = row0 < col0 + BN && col0 < row0 + BM;
      const float4* snb = reinterpret_cast<const float4*>(smem + Ly::V0 + vs * Ly::V_SLOT + Ly::V_NRM) + h * 8;
      const uint32_t sa = tbase + lane_off + Ly::T_S + b * 64 + h * 32;
      uint8_t* krow = smem + Ly::K0 + b * 2 * Ly::KT + r * 128;
      uint32_t s32[32];
      tmem_ld32(sa, s32);
      tmem_wait_ld();
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        // two entries per packed FP32x2 instruction
        float2 kf[8];
#pragma unroll
        for (int c2 = 0; c2 < 8; ++c2) {
          const int cc = half * 16 + 2 * c2;
          const float4 n4 = snb[cc >> 2];
          const float2 nb = (cc & 2) ? make_float2(n4.z, n4.w) : make_float2(n4.x, n4.y);
          kf[c2] = matern2_scaled(make_float2(__uint_as_float(s32[cc]), __uint_as_float(s32[cc + 1])), nb,
                                  na2, m22);
        }
        if (diag) {
          const int64_t dc = grow - (col0 + h * 32 + half * 16);
          const uint32_t dmask = (dc >= 0 && dc < 16) ? (1u << (int)dc) : 0u;
#pragma unroll
          for (int c2 = 0; c2 < 8; ++c2) {
            kf[c2].x = ((dmask >> (2 * c2)) & 1u) ? (float)(1 << kKExp) : kf[c2].x;
            kf[c2].y = ((dmask >> (2 * c2 + 1)) & 1u) ? (float)(1 << kKExp) : kf[c2].y;
          }
        }
        uint32_t hi2[8], lo2[8];
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) split_h2(kf[k2], hi2[k2], lo2[k2]);
        tmem_st8(sa + half * 8, hi2);
        tmem_st8(sa + 16 + half * 8, lo2);
        // the same values into the SMEM tile: row a = r, 16-byte chunks
        // (columns / 8) placed at chunk ^ (a mod 8)
        const int ch = 4 * h + 2 * half, sw = r & 7;
        st_shared_v4(krow + ((ch ^ sw) << 4), hi2[0], hi2[1], hi2[2], hi2[3]);
        st_shared_v4(krow + (((ch + 1) ^ sw) << 4), hi2[4], hi2[5], hi2[6], hi2[7]);
        st_shared_v4(krow + Ly::KT + ((ch ^ sw) << 4), lo2[0], lo2[1], lo2[2], lo2[3]);
        st_shared_v4(krow + Ly::KT + (((ch + 1) ^ sw) << 4), lo2[4], lo2[5], lo2[6], lo2[7]);
      }
      // the SMEM tile is read by the tensor core (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tmem_wait_st();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_k + b);
      if ((i % OGROUP) == 0 && i > 0 && !(ok = drain_o(i / OGROUP - 1))) break;
      // pair i - 1 (tiles 2i - 2, 2i - 1) is complete once both groups have
      // passed it; the group of its parity drains it
      if (i > 0 && ((i - 1) & 1) == g && !(ok = drain_d(i - 1))) break;
    }
    if (ok && my_tiles > 0) ok = drain_o((my_tiles - 1) / OGROUP);
    for (int pr = max(0, my_tiles - 1); ok && pr < npairs; ++pr)
      if ((pr & 1) == g) ok = drain_d(pr);
    if (ok && my_tiles > 0 && grow < p.n) {
#pragma unroll
      for (int c = 0; c < TH; ++c) {
        const int col = h * TH + c;
        if (col < p.t) atomicAdd(p.out + (int64_t)col * p.ldo + grow, out_scale[col] * (acc[c] - cmp[c]));
      }
    }
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

struct SymGrid {
  int row_tiles, col_tiles, band;
  int64_t segments, tiles;
};

SymGrid sym_grid(int64_t n, int T, int num_sms) {
  SymGrid g;
  g.row_tiles = (int)ceil_div(n, BM);
  g.col_tiles = (int)ceil_div(n, BN);
  // tiles formed: sum over I of (col_tiles - 2I); col_tiles >= 2 row_tiles - 1
  g.tiles = (int64_t)g.row_tiles * g.col_tiles - (int64_t)g.row_tiles * (g.row_tiles - 1);
  // bands of column tiles whose X~_J and V_J (and the O_J they receive) stay
  // in L2 while the CTAs in flight stream them; narrower bands when the
  // problem is small, so that the segments still fill the GPU several times
  const int64_t tile_bytes = (int64_t)BN * (DPH + T) * 2 * 2 + 256 + (int64_t)BN * T * 4;
  const int64_t band_l2 = std::max<int64_t>(64, (48LL << 20) / tile_bytes);
  const int64_t band_fill = g.tiles / (4LL * num_sms);
  // even, so that every segment starts on an even column tile and the pairs
  // of the second contraction never straddle the diagonal block
  g.band = (int)(std::max<int64_t>(2, std::min(band_l2, band_fill)) & ~int64_t(1));
  g.segments = 0;
  for (int64_t b = 0; b * g.band < g.col_tiles; ++b) {
    const int64_t hi = std::min<int64_t>((b + 1) * g.band, g.col_tiles);
    g.segments += std::min<int64_t>(g.row_tiles, (hi + 1) / 2);
  }
  return g;
}

template <int T>
int launch_sym(gp_ctx* ctx, const Prep& p, const __half* vhi, const __half* vlo, const float* vsc, int64_t vld,
               int t, float* out, int64_t ldo, float s, int* status) {
  using Ly = SymLayout<T>;
  CUtensorMap mch, mcl, mvh, mvl;
  GP_TRY(make_map(ctx, &mch, p.xh_hi, p.n_pad, DPH, DPH, BN, 64, true, true));
  GP_TRY(make_map(ctx, &mcl, p.xh_lo, p.n_pad, DPH, DPH, BN, 64, true, true));
  GP_TRY(make_map(ctx, &mvh, vhi, T, p.n_pad, vld, T, 64, true, true));
  GP_TRY(make_map(ctx, &mvl, vlo, T, p.n_pad, vld, T, 64, true, true));
  const size_t smem = Ly::TOTAL + 1024;
  static std::atomic<uint64_t> attr{0};
  GP_TRY(smem_attr_once(ctx, kmv_sym_kernel<T>, smem, attr));
  const SymGrid grid = sym_grid(p.n, T, ctx->num_sms);
  SymParams prm;
  prm.xh_hi = p.xh_hi;
  prm.xh_lo = p.xh_lo;
  prm.norm = p.norm_h;
  prm.xs = p.xh_scale;
  prm.vsc = vsc;
  prm.n = p.n;
  prm.row_tiles = grid.row_tiles;
  prm.col_tiles = grid.col_tiles;
  prm.band = grid.band;
  prm.out = out;
  prm.ldo = ldo;
  prm.t = t;
  prm.s = s;
  prm.status = status;
  kmv_sym_kernel<T><<<(unsigned)grid.segments, NTHREADS, smem, ctx->stream>>>(mch, mcl, mvh, mvl, prm);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

}  // namespace

double kmv_sym_entries(int64_t n) {
  return (double)sym_grid(n, 16, 152).tiles * BM * BN;
}

int kmv_sym_f16(gp_ctx* ctx, const Prep& p, const __half* vhi, const __half* vlo, const float* vsc, int64_t vld,
                int t, int T, float* out, int64_t ldo, float s, int* status) {
  if (!p.xh_hi || !p.xh_lo || !p.norm_h || p.d_pad > DPH)
    return set_err(ctx, GP_EINVAL, "symmetric K-hat V: FP16 features not prepared");
  return T == 16 ? launch_sym<16>(ctx, p, vhi, vlo, vsc, vld, t, out, ldo, s, status)
                 : launch_sym<32>(ctx, p, vhi, vlo, vsc, vld, t, out, ldo, s, status);
}

}  // namespace gp
