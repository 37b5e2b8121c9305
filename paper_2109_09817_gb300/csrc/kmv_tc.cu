// Tensor-core K-hat V on sm_103a (tcgen05 + TMEM + TMA): split TF32, single
// TF32, and split FP16 (kind::f16, power-of-two scaled operands).
//
// arXiv 2109.09817 Sec. 3.1-3.2 (blackbox products with K-hat, O(N)
// memory) and Sec. 4 (kernel tiles).  Per CTA: a 128-row tile I and a range
// of 64-column tiles J.  Per J tile:
//   MMA1  S = X~_I X~_J^T          operands in 128B-swizzled SMEM (TMA),
//                                  accumulator in TMEM; split forms:
//                                  S = hi.hi^T + hi.lo^T + lo.hi^T
//         TF32: hi.[hi; lo]^T as one N = 128 MMA plus lo.hi^T, two 64-column
//         accumulators; FP16: three N = 64 MMAs into one accumulator (16
//         features per MMA)
//   epi   K = matern(n_a + n_b - 2S) on the FP32/MUFU pipes (8 warps), written
//         back to TMEM over S as hi + lo parts (TF32 hi and BF16 lo, or FP16
//         hi and lo of 2^14 K)
//   MMA2  O_J = K_hi [V_hi V_lo] + K_lo V_hi, A from TMEM.  TF32 form: the
//         first term kind::tf32, the second kind::f16 with BF16 operands
//         (K_lo is 2^-11 of K, so BF16 keeps the term to 2^-20 of K V and
//         covers 16 columns per MMA instead of 8).  FP16 form: both kind::f16
//   epi   O_J drained from TMEM and added into per-thread registers with a
//         compensated (Kahan) sum; flushed once per CTA with atomics.
// The tensor pipe loses roughly 500 cycles whenever it drains, so MMA1 runs
// NSB tiles ahead of MMA2: S/K lives in NSB TMEM buffers, and MMA1 and MMA2
// are issued by two threads so that a wait in one does not starve the pipe.
// X~_J tiles and V_J tiles travel in separate TMA rings, so an X~_J slot is
// recycled as soon as its MMA1 has run.  Warp roles: 0 TMA producer, 1 MMA1
// issuer, 2 TMEM allocator, 3 MMA2 issuer, 4..19 epilogue in two groups of 8
// (group g takes tiles j with j % 2 == g).
// Every mbarrier wait is bounded: on a timeout the kernel records
// GP_ETIMEOUT in a status word and all roles leave their loops.
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
constexpr int NTHREADS = 640;     // 4 control warps + 2 x 8 epilogue warps
constexpr int EPI_WARP0 = 4;
constexpr int GROUP_WARPS = 8;    // one epilogue group: 2 warps per TMEM lane quarter
constexpr int OGROUP = 2;         // a group's J tiles accumulated in TMEM per O drain

// ------------------------------------------------------------- layout ------
// F16: operands are FP16 (2 bytes), so a 128-byte K box holds 64 elements
// and one MMA k-step (32 bytes) covers 16 of them instead of 8.
template <int DP, int T, bool F16 = false>
struct TcLayout {
  static constexpr int ES = F16 ? 2 : 4;               // operand element bytes
  static constexpr int BOXE = 128 / ES;                // elements per K box
  static constexpr int KSTEP = 32 / ES;                // K elements per MMA
  static constexpr int KB = DP / BOXE;                 // 128-byte K boxes of X~
  // FP16: the three split products accumulate into one 64-column S buffer;
  // TF32: hi.hi and the two cross products in two 64-column halves
  static constexpr uint32_t SBW = F16 ? 64 : 128;      // TMEM columns per S/K buffer
  static constexpr int NSB = F16 ? 4 : (T <= 16 ? 3 : 2);  // S/K buffers in TMEM
  static constexpr int XS = F16 ? 6 : (DP <= 32 ? 4 : 3);  // X~_J ring slots
  static constexpr int VS = T <= 16 ? NSB + 2 : NSB + 1;  // V_J ring slots (>= NSB)
  static constexpr int A_BOX = BM * 128;               // bytes per K box, A
  static constexpr int XJ_BOX = BN * 128;              // bytes per K box, X~_J
  static constexpr int V_BOX = T * 128;                // bytes per K box of V_J
  static constexpr int A_HI = 0;
  static constexpr int A_LO = A_HI + KB * A_BOX;
  // X~_J slot: per 128-byte K box kb: [hi rows 0..63][lo rows 0..63], so that
  // hi and lo stack into one N = 128 B operand
  static constexpr int X_SLOT = KB * 2 * XJ_BOX;
  static constexpr int X0 = A_LO + KB * A_BOX;
  // V_J slot, TF32: per 32-column box vb: [hi T rows][lo T rows]; then V_hi
  // in BF16 (T rows of 64 columns = one 128-byte atom row each).  FP16: one
  // 64-column box [hi T rows][lo T rows].  Then the 64 column norms.
  static constexpr int V_BF = 2 * 2 * V_BOX;
  static constexpr int V_NRM = F16 ? 2 * V_BOX : V_BF + T * 128;
  static constexpr int V_SLOT = (V_NRM + 256 + 1023) / 1024 * 1024;
  static constexpr int V0 = X0 + XS * X_SLOT;
  static constexpr int BAR = V0 + VS * V_SLOT;
  static constexpr int NBAR = 1 + 2 * XS + 2 * VS + 3 * NSB + 8 + 1;
  static constexpr int TOTAL = BAR + NBAR * 8 + 16;
  static constexpr uint32_t TX_A = 2u * KB * A_BOX;
  static constexpr uint32_t TX_X = 2u * KB * XJ_BOX;
  static constexpr uint32_t TX_V = F16 ? 2u * V_BOX + 256u : 4u * V_BOX + T * 128u + 256u;  // split forms
  static constexpr uint32_t TX_V1 = 2u * V_BOX + 256u;             // single TF32
  // TMEM columns
  // per S buffer b: [b*128, +64) the hi.hi product, then K_hi;
  //                 [b*128+64, +64) the hi.lo + lo.hi products, then K_lo
  // (FP16 K_hi and K_lo, and BF16 K_lo, two per 32-bit column)
  static constexpr uint32_t T_S = 0;
  static constexpr uint32_t T_X = 64;
  static constexpr uint32_t T_O = NSB * SBW;  // 2 epilogue groups x 2 x 2T: O (hh | hi.lo part)
  static constexpr uint32_t T_COLS = 512;
  static_assert(T_O + 8 * T <= T_COLS, "TMEM columns");
  static_assert(KB >= 1 && DP % BOXE == 0, "feature width");
  // dynamic + 1024 alignment slack + 1024 static (the failure flag) <= 227 KB
  static_assert(TOTAL + 2048 <= 232448, "shared memory");
};

struct TcParams {
  const float* nr;      // row norms (padded)
  const float* nc;      // column norms (padded)
  int64_t nrows, ncols;
  float* out;
  int64_t ldo;
  int t;                // live vectors in this chunk
  float s;
  int sym;
  int tiles_per_split;
  int* status;
  // FP16 form only (device scalars): row and column feature scales 2^-e,
  // and per output vector the factor 2^-(e_c + 14) that undoes the scaling
  // of V_c and of K
  const float* xs_r;
  const float* xs_c;
  const float* vsc;
};

// MMA1 k-steps KK..NK-1 of the TF32 forms (8 features = 32 B per step
// inside 128 B atoms).
template <class Ly, bool SPLIT, int KK, int NK>
__device__ __forceinline__ void mma1_steps(uint32_t dhh, uint32_t dx, uint64_t dA_hi, uint64_t dA_lo, uint64_t dX,
                                           uint32_t id1w, uint32_t id1) {
  if constexpr (KK < NK) {
    constexpr uint32_t AO = ((KK >> 2) * Ly::A_BOX + (KK & 3) * 32) >> 4;
    constexpr uint32_t BO = ((KK >> 2) * 2 * Ly::XJ_BOX + (KK & 3) * 32) >> 4;
    if constexpr (SPLIT) {
      mma_ss_imm<AO, BO>(dhh, dA_hi, dX, id1w, KK ? 1u : 0u);
      mma_ss_imm<AO, BO>(dx, dA_lo, dX, id1, 1u);
    } else {
      mma_ss_imm<AO, BO>(dhh, dA_hi, dX, id1, KK ? 1u : 0u);
    }
    mma1_steps<Ly, SPLIT, KK + 1, NK>(dhh, dx, dA_hi, dA_lo, dX, id1w, id1);
  }
}
// MMA2 k-steps over the 64 columns of the K tile (A = K from TMEM).
template <class Ly, bool SPLIT, int KK, int NK>
__device__ __forceinline__ void mma2_steps(uint32_t d, uint32_t khi, uint32_t klo, uint64_t dV, uint32_t id2w,
                                           uint32_t id2, uint32_t acc0) {
  if constexpr (KK < NK) {
    constexpr uint32_t BO = ((KK >> 2) * 2 * Ly::V_BOX + (KK & 3) * 32) >> 4;
    const uint32_t acc = KK == 0 ? acc0 : 1u;
    if constexpr (SPLIT) {
      mma_ts_imm<KK * 8, BO>(d, khi, dV, id2w, acc);
    } else {
      mma_ts_imm<KK * 8, BO>(d, khi, dV, id2, acc);
    }
    mma2_steps<Ly, SPLIT, KK + 1, NK>(d, khi, klo, dV, id2w, id2, acc0);
  }
}
// K_lo V_hi in BF16, 16 columns per k-step.  The epilogue packs K_lo of
// columns [32h, 32h + 32) into TMEM columns [32h, 32h + 16) of the S_x
// region, two BF16 per 32-bit column, so k-step kk reads 8 columns at
// (kk >> 1) * 32 + (kk & 1) * 8; B = V_hi (BF16), 32 bytes per k-step.
template <class Ly, int KK, int NK>
__device__ __forceinline__ void mma2_lo_steps(uint32_t d, uint32_t klo, uint64_t dVb, uint32_t id) {
  if constexpr (KK < NK) {
    mma_ts_bf16_imm<(KK >> 1) * 32 + (KK & 1) * 8, ((KK * 32) >> 4)>(d, klo, dVb, id, 1u);
    mma2_lo_steps<Ly, KK + 1, NK>(d, klo, dVb, id);
  }
}

// FP16 cross term with the three split products in one accumulator:
// S += A_hi X_hi^T + A_hi X_lo^T + A_lo X_hi^T, three N = 64 MMAs per k-step.
template <class Ly, int KK, int NK>
__device__ __forceinline__ void mma1_one_steps(uint32_t d, uint64_t dA_hi, uint64_t dA_lo, uint64_t dX,
                                               uint32_t id1) {
  if constexpr (KK < NK) {
    constexpr uint32_t AO = ((KK >> 2) * Ly::A_BOX + (KK & 3) * 32) >> 4;
    constexpr uint32_t BO = ((KK >> 2) * 2 * Ly::XJ_BOX + (KK & 3) * 32) >> 4;
    constexpr uint32_t BL = BO + (Ly::XJ_BOX >> 4);
    mma_ss_f16_imm<AO, BO>(d, dA_hi, dX, id1, KK ? 1u : 0u);
    mma_ss_f16_imm<AO, BL>(d, dA_hi, dX, id1, 1u);
    mma_ss_f16_imm<AO, BO>(d, dA_lo, dX, id1, 1u);
    mma1_one_steps<Ly, KK + 1, NK>(d, dA_hi, dA_lo, dX, id1);
  }
}

// FP16 contraction, 16 columns per k-step: O[0, 2T) += K_hi [V_hi; V_lo]
// (N = 2T), then O[0, T) += K_lo V_hi (N = T).  K_hi and K_lo of columns
// [32h + 16 half, +16) sit, two FP16 per 32-bit column, in TMEM columns
// [32h + 8 half, +8) of their regions, so k-step kk reads 8 columns at
// (kk >> 1) * 32 + (kk & 1) * 8; B advances 32 bytes per k-step inside the
// 128-byte rows of the V slot.
template <class Ly, int KK, int NK>
__device__ __forceinline__ void mma2_f16_steps(uint32_t d, uint32_t khi, uint32_t klo, uint64_t dV,
                                               uint32_t id2w, uint32_t id2, uint32_t acc0) {
  if constexpr (KK < NK) {
    constexpr uint32_t AO = (KK >> 1) * 32 + (KK & 1) * 8;
    constexpr uint32_t BO = (KK * 32) >> 4;
    mma_ts_bf16_imm<AO, BO>(d, khi, dV, id2w, KK == 0 ? acc0 : 1u);
    mma_ts_bf16_imm<AO, BO>(d, klo, dV, id2, 1u);
    mma2_f16_steps<Ly, KK + 1, NK>(d, khi, klo, dV, id2w, id2, acc0);
  }
}

// OP: 0 = single TF32, 1 = split TF32 (hi/lo products), 2 = split FP16.
template <int DP, int T, int OP>
__global__ void __launch_bounds__(NTHREADS, 1)
kmv_tc_kernel(const __grid_constant__ CUtensorMap map_r_hi, const __grid_constant__ CUtensorMap map_r_lo,
              const __grid_constant__ CUtensorMap map_c_hi, const __grid_constant__ CUtensorMap map_c_lo,
              const __grid_constant__ CUtensorMap map_v_hi, const __grid_constant__ CUtensorMap map_v_lo,
              const __grid_constant__ CUtensorMap map_v_bf, const TcParams p) {
  constexpr bool SPLIT = OP != 0, F16 = OP == 2;
  using Ly = TcLayout<DP, T, F16>;
  constexpr int NSB = Ly::NSB, XS = Ly::XS, VS = Ly::VS;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Ly::BAR);
  uint64_t* bar_a = bars;
  uint64_t* bar_xf = bars + 1;              // [XS]   X~_J slot loaded
  uint64_t* bar_xe = bar_xf + XS;           // [XS]   ... consumed by MMA1
  uint64_t* bar_vf = bar_xe + XS;           // [VS]   V_J slot (and norms) loaded
  uint64_t* bar_ve = bar_vf + VS;           // [VS]   ... consumed by MMA2
  uint64_t* bar_s = bar_ve + VS;            // [NSB]  S in buffer b ready
  uint64_t* bar_k = bar_s + NSB;            // [NSB]  K in buffer b written
  uint64_t* bar_kf = bar_k + NSB;           // [NSB]  K in buffer b read by MMA2
  uint64_t* bar_of = bar_kf + NSB;          // [2][2] O of group g, buffer u ready
  uint64_t* bar_oe = bar_of + 4;            // [2][2] ... drained
  uint64_t* bar_fin = bar_oe + 4;           // both MMA issuers drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + Ly::NBAR);
  __shared__ int fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t n_col_tiles = (p.ncols + BN - 1) / BN;
  const int64_t jt0 = (int64_t)blockIdx.y * p.tiles_per_split;
  const int64_t jt1 = min(n_col_tiles, jt0 + (int64_t)p.tiles_per_split);
  const int ntiles = (int)(jt1 - jt0);
  if (ntiles <= 0) return;

  if (threadIdx.x == 0) {
    fail = 0;
    mbar_init(bar_a, 1);
    for (int i = 0; i < XS; ++i) {
      mbar_init(bar_xf + i, 1);
      mbar_init(bar_xe + i, 1);
    }
    for (int i = 0; i < VS; ++i) {
      mbar_init(bar_vf + i, 1);
      mbar_init(bar_ve + i, 1);
    }
    for (int i = 0; i < NSB; ++i) {
      mbar_init(bar_s + i, 1);
      mbar_init(bar_k + i, GROUP_WARPS);
      mbar_init(bar_kf + i, 1);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(bar_of + i, 1);
      mbar_init(bar_oe + i, GROUP_WARPS);
    }
    mbar_init(bar_fin, 2);
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

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------------- TMA producer --
    mbar_expect_tx(bar_a, SPLIT ? Ly::TX_A : Ly::TX_A / 2);
    for (int kb = 0; kb < Ly::KB; ++kb) {
      tma_2d(smem + Ly::A_HI + kb * Ly::A_BOX, &map_r_hi, bar_a, kb * Ly::BOXE, (int)row0);
      if (SPLIT) tma_2d(smem + Ly::A_LO + kb * Ly::A_BOX, &map_r_lo, bar_a, kb * Ly::BOXE, (int)row0);
    }
    int armed = 0;   // tiles whose loads (both rings) have been issued
    for (int j = 0; j < ntiles; ++j) {
      const int col0 = (int)((jt0 + j) * BN);
      const int xs = j % XS, vs = j % VS;
      if (j >= XS && !mbar_wait(bar_xe + xs, ((j / XS) - 1) & 1, &fail)) break;
      uint8_t* xb = smem + Ly::X0 + xs * Ly::X_SLOT;
      mbar_expect_tx(bar_xf + xs, SPLIT ? Ly::TX_X : Ly::TX_X / 2);
      for (int kb = 0; kb < Ly::KB; ++kb) {
        tma_2d(xb + (2 * kb) * Ly::XJ_BOX, &map_c_hi, bar_xf + xs, kb * Ly::BOXE, col0);
        if (SPLIT) tma_2d(xb + (2 * kb + 1) * Ly::XJ_BOX, &map_c_lo, bar_xf + xs, kb * Ly::BOXE, col0);
      }
      if (j >= VS && !mbar_wait(bar_ve + vs, ((j / VS) - 1) & 1, &fail)) {
        // the X~_J loads of this tile are in flight: let them land first
        mbar_wait_exit(bar_xf + xs, (j / XS) & 1);
        break;
      }
      uint8_t* vb = smem + Ly::V0 + vs * Ly::V_SLOT;
      mbar_expect_tx(bar_vf + vs, SPLIT ? Ly::TX_V : Ly::TX_V1);
      if constexpr (F16) {
        tma_2d(vb, &map_v_hi, bar_vf + vs, col0, 0);
        tma_2d(vb + Ly::V_BOX, &map_v_lo, bar_vf + vs, col0, 0);
      } else {
        for (int b = 0; b < 2; ++b) {
          tma_2d(vb + (2 * b) * Ly::V_BOX, &map_v_hi, bar_vf + vs, col0 + b * 32, 0);
          if (SPLIT) tma_2d(vb + (2 * b + 1) * Ly::V_BOX, &map_v_lo, bar_vf + vs, col0 + b * 32, 0);
        }
        if (SPLIT) tma_2d(vb + Ly::V_BF, &map_v_bf, bar_vf + vs, col0, 0);
      }
      bulk_g2s(vb + Ly::V_NRM, p.nc + col0, 256, bar_vf + vs);
      armed = j + 1;
    }
    // never leave with bulk copies still landing in this CTA's memory
    mbar_wait_exit(bar_a, 0);
    for (int j = max(0, armed - XS); j < armed; ++j) mbar_wait_exit(bar_xf + (j % XS), (j / XS) & 1);
    for (int j = max(0, armed - VS); j < armed; ++j) mbar_wait_exit(bar_vf + (j % VS), (j / VS) & 1);
  } else if ((warp == 1 || warp == 3) && lane == 0) {
    // --------------------------------------------------------- MMA issuers --
    // Two issuing threads: warp 1 issues MMA1 (cross terms), warp 3 issues
    // MMA2 (contractions).  Each waits on its own barriers, so one keeps the
    // tensor pipe fed while the other waits.  Tile j: S/K buffer b = j % NSB,
    // epilogue group g = j & 1, the group's i-th tile with i = j >> 1; the
    // group's O accumulates OGROUP of its tiles in buffer u = (i / OGROUP) & 1.
    // MMA1(j) reuses buffer b only after MMA2(j - NSB) has completed.
    constexpr uint32_t ID1 = F16 ? idesc_f16(BM, BN) : idesc_tf32(BM, BN);            // N = 64
    constexpr uint32_t ID1W = F16 ? idesc_f16(BM, 2 * BN) : idesc_tf32(BM, 2 * BN);   // N = 128: [hi; lo]
    constexpr uint32_t ID2 = F16 ? idesc_f16(BM, T) : idesc_tf32(BM, T);
    constexpr uint32_t ID2W = F16 ? idesc_f16(BM, 2 * T) : idesc_tf32(BM, 2 * T);
    constexpr uint32_t ID2B = idesc_bf16(BM, T);
    // SMEM descriptors are built once; an operand at byte offset o from a
    // 1024-aligned base has descriptor desc(base) + (o >> 4), so every MMA
    // below issues with constant offsets (a single issuing thread would
    // otherwise spend tens of cycles per MMA on descriptor arithmetic)
    const uint64_t dA_hi = sdesc(su32(smem + Ly::A_HI)), dA_lo = sdesc(su32(smem + Ly::A_LO));
    const uint64_t dX0 = sdesc(su32(smem + Ly::X0)), dV0 = sdesc(su32(smem + Ly::V0));
    bool ok = mbar_wait(bar_a, 0, &fail);
    fence_after();
    // Columns [b*128, +64) get A_hi B_hi^T and [b*128+64, +64) get
    // A_hi B_lo^T + A_lo B_hi^T: one N = 128 MMA writes both halves
    // (B = [hi; lo] rows), a second N = 64 MMA adds A_lo B_hi^T.  Every
    // tcgen05.mma costs a roughly fixed time at small N, so products are
    // stacked along N rather than issued separately.
    auto mma1 = [&](int j) -> bool {
      const int xs = j % XS, b = j % NSB;
      if (!mbar_wait(bar_xf + xs, (j / XS) & 1, &fail)) return false;
      fence_after();
      const uint64_t dX = dX0 + (uint64_t)(xs * (Ly::X_SLOT >> 4));
      const uint32_t dhh = tbase + Ly::T_S + b * Ly::SBW;
      const uint32_t dx = dhh + Ly::T_X;
      if constexpr (F16)
        mma1_one_steps<Ly, 0, DP / Ly::KSTEP>(dhh, dA_hi, dA_lo, dX, ID1);
      else
        mma1_steps<Ly, SPLIT, 0, DP / Ly::KSTEP>(dhh, dx, dA_hi, dA_lo, dX, ID1W, ID1);
      mma_commit(bar_xe + xs);
      mma_commit(bar_s + b);
      return true;
    };
    // O[0, T) += K_hi V_hi + K_lo V_hi and O[T, 2T) += K_hi V_lo: the first
    // MMA stacks [V_hi; V_lo] along N (A from TMEM)
    auto mma2 = [&](int j, uint32_t ocol, bool first) -> bool {
      const int vs = j % VS, b = j % NSB;
      if (!mbar_wait(bar_vf + vs, (j / VS) & 1, &fail)) return false;
      fence_after();
      const uint64_t dV = dV0 + (uint64_t)(vs * (Ly::V_SLOT >> 4));
      const uint32_t d = tbase + ocol;
      const uint32_t khi = tbase + Ly::T_S + b * Ly::SBW, klo = khi + (F16 ? 16u : Ly::T_X);
      if constexpr (F16) {
        mma2_f16_steps<Ly, 0, BN / 16>(d, khi, klo, dV, ID2W, ID2, first ? 0u : 1u);
      } else {
        mma2_steps<Ly, SPLIT, 0, BN / 8>(d, khi, klo, dV, ID2W, ID2, first ? 0u : 1u);
        if constexpr (SPLIT) mma2_lo_steps<Ly, 0, BN / 16>(d, klo, dV + (Ly::V_BF >> 4), ID2B);
      }
      return true;
    };
    if (warp == 1) {
      for (int j = 0; ok && j < ntiles; ++j) {
        const int b = j % NSB;
        if (j >= NSB) {
          if (!(ok = mbar_wait(bar_kf + b, ((j / NSB) - 1) & 1, &fail))) break;
          fence_after();
        }
        ok = mma1(j);
      }
    } else {
      for (int j = 0; ok && j < ntiles; ++j) {
        const int b = j % NSB, g = j & 1, i = j >> 1;
        const int og = i / OGROUP, u = og & 1;
        const bool first = (i % OGROUP) == 0;
        const bool last = (i % OGROUP) == OGROUP - 1 || j + 2 >= ntiles;
        if (!(ok = mbar_wait(bar_k + b, (j / NSB) & 1, &fail))) break;
        fence_after();
        if (first && og >= 2) {
          if (!(ok = mbar_wait(bar_oe + 2 * g + u, ((og - 2) >> 1) & 1, &fail))) break;
          fence_after();
        }
        if (!(ok = mma2(j, Ly::T_O + (2 * g + u) * 2 * T, first))) break;
        if (last) mma_commit(bar_of + 2 * g + u);
        mma_commit(bar_ve + (j % VS));
        mma_commit(bar_kf + b);
      }
    }
    // every MMA issued by either thread has completed before TMEM is released
    mma_commit(bar_fin);
    mbar_wait_exit(bar_fin, 0);
  } else if (warp >= EPI_WARP0) {
    // ----------------------------------------------------------- epilogue --
    const int e = warp - EPI_WARP0;
    const int g = e / GROUP_WARPS;       // epilogue group: tiles j with j & 1 == g
    const int q = warp & 3;              // TMEM lane quarter of this warp
    const int h = (e % GROUP_WARPS) >> 2;  // column half (32 columns)
    const int r = q * 32 + lane;         // row within the tile
    const int64_t grow = row0 + r;
    const float na = p.nr[grow];
    // u^2 = n_a + n_b + m2 S: the FP16 cross term carries the feature scales
    const float m2 = F16 ? -2.f * p.xs_r[0] * p.xs_c[0] : -2.f;
    const float2 na2 = make_float2(na, na), m22 = make_float2(m2, m2);
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int my_tiles = (ntiles - g + 1) / 2;   // tiles j = g, g + 2, ...
    constexpr int TH = T / 2;            // O columns drained by this warp
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
    auto drain = [&](int og) -> bool {
      const int u = og & 1;
      if (!mbar_wait(bar_of + 2 * g + u, (og >> 1) & 1, &fail)) return false;
      fence_after();
      const uint32_t oa = tbase + lane_off + Ly::T_O + (2 * g + u) * 2 * T + h * TH;
      // two 8-column pieces: O[0, T) (K_hi V_hi + K_lo V_hi) and O[T, 2T) (K_hi V_lo)
#pragma unroll
      for (int c8 = 0; c8 < TH; c8 += 8) {
        uint32_t rr[8], rx[8];
        tmem_ld8(oa + c8, rr);
        if (SPLIT) tmem_ld8(oa + T + c8, rx);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 8; ++c)
          kahan(c8 + c, __uint_as_float(rr[c]) + (SPLIT ? __uint_as_float(rx[c]) : 0.f));
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_oe + 2 * g + u);
      return true;
    };
    bool ok = true;
    for (int i = 0; i < my_tiles; ++i) {
      const int j = 2 * i + g;
      const int b = j % NSB, vs = j % VS;
      const int64_t col0 = (jt0 + j) * BN;
      if (!(ok = mbar_wait(bar_s + b, (j / NSB) & 1, &fail))) break;
      // the slot's norms: the wait makes the async-proxy writes visible here
      if (!(ok = mbar_wait(bar_vf + vs, (j / VS) & 1, &fail))) break;
      fence_after();
      const bool diag = p.sym && row0 < col0 + BN && col0 < row0 + BM;
      if constexpr (F16) {
        // All 32 of this warp's S columns at once.  u^2 = n_a + n_b + m2 S and
        // u = sqrt(|u^2|) in one MUFU op (the modulus absorbs a u^2 rounded
        // below zero).  K is held as 2^14 K (the scale rides in the
        // polynomial's coefficients) and split into FP16
        // hi = fp16(K) and lo = fp16(K - hi), K - hi being exact in FP32, so
        // hi + lo = K to 2^-22.  They are packed two per 32-bit column (even
        // column in the low half): K_hi of columns [32h + 16 half, +16) to
        // [32h + 8 half, +8), K_lo 16 columns further on, both inside the
        // columns already loaded.
        const float4* snb = reinterpret_cast<const float4*>(smem + Ly::V0 + vs * Ly::V_SLOT + Ly::V_NRM) + h * 8;
        const uint32_t sa = tbase + lane_off + Ly::T_S + b * Ly::SBW + h * 32;
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
          for (int i = 0; i < 8; ++i) split_h2(kf[i], hi2[i], lo2[i]);
          tmem_st8(sa + half * 8, hi2);
          tmem_st8(sa + 16 + half * 8, lo2);
        }
      }
      if constexpr (!F16) {
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        const int cb = h * 32 + half * 16;   // first of these 16 columns
        const float4* snb = reinterpret_cast<const float4*>(smem + Ly::V0 + vs * Ly::V_SLOT + Ly::V_NRM) + cb / 4;
        const uint32_t sa = tbase + lane_off + Ly::T_S + b * Ly::SBW + cb;
        uint32_t sh[16], sx[16];
        tmem_ld16(sa, sh);
        if (SPLIT) tmem_ld16(sa + Ly::T_X, sx);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const float4 n4 = snb[c >> 2];      // broadcast load, 4 norms per LDS.128
          const float nbc = (c & 3) == 0 ? n4.x : (c & 3) == 1 ? n4.y : (c & 3) == 2 ? n4.z : n4.w;
          float sab = __uint_as_float(sh[c]);
          if (SPLIT) sab += __uint_as_float(sx[c]);
          // u = u2 / sqrt(u2) with one MUFU op; one clamp serves both the
          // rounding below zero and the rsqrt (u = 1e-15 for u2 <= 0 gives
          // k = 1 to FP32 precision)
          const float u2 = fmaxf(fmaf(m2, sab, na + nbc), 1e-30f);
          const float uu = u2 * rsqrt_approx(u2);
          const float kv = fmaf(u2, kC2, fmaf(uu, kC1, 1.f)) * ex2_approx(-uu);
          // K = hi + lo exactly: hi = K rounded to TF32, lo the remainder;
          // |lo| <= 2^-11 |K|, so lo rounded to BF16 costs <= 2^-20 |K|
          const float hi = tf32_rna(kv);
          sh[c] = __float_as_uint(hi);
          sx[c] = __float_as_uint(kv - hi);
        }
        if (diag) {
          // diagonal tile: the entry a = b is exactly k(0) = 1
          const int64_t dc = grow - (col0 + cb);
          const uint32_t dmask = (dc >= 0 && dc < 16) ? (1u << (int)dc) : 0u;
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const bool on = (dmask >> c) & 1u;
            sh[c] = on ? __float_as_uint(1.0f) : sh[c];
            sx[c] = on ? 0u : sx[c];
          }
        }
        tmem_st16(sa, sh);
        if (SPLIT) {
          // K_lo as BF16 pairs (even column in the low half) into this warp's
          // own S_x columns, already read above: [32h + 8 half, +8)
          uint32_t lo2[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const __nv_bfloat162 v =
                __floats2bfloat162_rn(__uint_as_float(sx[2 * i]), __uint_as_float(sx[2 * i + 1]));
            lo2[i] = *reinterpret_cast<const uint32_t*>(&v);
          }
          tmem_st8(tbase + lane_off + Ly::T_S + b * Ly::SBW + Ly::T_X + h * 32 + half * 8, lo2);
        }
      }
      }
      tmem_wait_st();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_k + b);
      // drain this group's previous O buffer once its last MMA2 was issued
      if ((i % OGROUP) == 0 && i > 0 && !(ok = drain(i / OGROUP - 1))) break;
    }
    if (ok && my_tiles > 0) ok = drain((my_tiles - 1) / OGROUP);
    if (ok && my_tiles > 0 && grow < p.nrows) {
#pragma unroll
      for (int c = 0; c < TH; ++c) {
        const int col = h * TH + c;
        if (col < p.t)
          atomicAdd(p.out + (int64_t)col * p.ldo + grow, p.s * (acc[c] - cmp[c]) * (F16 ? p.vsc[col] : 1.f));
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

// V (t vectors, ld ldv, n valid) -> hi/lo TF32 parts, T_pad vectors of
// length n_pad (zero padding).
__global__ void split_v_kernel(const float* __restrict__ V, int64_t ldv, int t, int64_t n,
                               int tpad, int64_t npad, float* __restrict__ vhi,
                               float* __restrict__ vlo, __nv_bfloat16* __restrict__ vbf) {
  const int64_t total = (int64_t)tpad * npad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / npad, a = i % npad;
    const float v = (c < t && a < n) ? V[c * ldv + a] : 0.f;
    const float h = tf32_rna(v);
    vhi[i] = h;
    vlo[i] = tf32_rna(v - h);
    if (vbf) vbf[i] = __float2bfloat16_rn(h);
  }
}

// Per-vector max |v| for the FP16 split: grid (blocks, t), the bits of a
// non-negative float (integer order = float order).
__global__ void vmax_kernel(const float* __restrict__ V, int64_t ldv, int64_t n, unsigned* __restrict__ vmax) {
  const int c = blockIdx.y;
  float m = 0.f;
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(V[c * ldv + a]));
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(vmax + c, __float_as_uint(m));
}

// V -> FP16 hi/lo of 2^e_c V_c, e_c putting max |V_c| into [2^14, 2^15);
// vsc[c] = 2^-(e_c + 14) undoes that scale and the 2^14 of K.
__global__ void split_vh_kernel(const float* __restrict__ V, int64_t ldv, int t, int64_t n, int tpad,
                                int64_t npad, const unsigned* __restrict__ vmax, __half* __restrict__ vhi,
                                __half* __restrict__ vlo, float* __restrict__ vsc) {
  const int64_t total = (int64_t)tpad * npad;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / npad, a = i % npad;
    const float m = c < t ? __uint_as_float(vmax[c]) : 0.f;
    int e = 0;
    if (m > 0.f) {
      int ex;
      frexpf(m, &ex);
      e = kHalfTop - ex;
    }
    const float v = (c < t && a < n) ? ldexpf(V[c * ldv + a], e) : 0.f;
    const __half h = __float2half_rn(v);
    vhi[i] = h;
    vlo[i] = __float2half_rn(v - __half2float(h));
    if (a == 0) vsc[c] = ldexpf(1.f, -(e + kKExp));
  }
}

// ------------------------------------------------------------- host side ----
template <int DP, int T, int OP>
int launch_tc(gp_ctx* ctx, const Prep& rows, const Prep& cols, const void* vhi, const void* vlo,
              const __nv_bfloat16* vbf, const float* vsc, int64_t vld, int t, float* out, int64_t ldo, float s,
              bool sym, int* status) {
  constexpr bool SPLIT = OP != 0, F16 = OP == 2;
  using Ly = TcLayout<DP, T, F16>;
  CUtensorMap mrh, mrl, mch, mcl, mvh, mvl, mvb;
  if constexpr (F16) {
    // 16-bit elements: 64 features (128 bytes) per box row
    GP_TRY(make_map(ctx, &mrh, rows.xh_hi, rows.n_pad, DP, DP, BM, 64, true, true));
    GP_TRY(make_map(ctx, &mrl, rows.xh_lo, rows.n_pad, DP, DP, BM, 64, true, true));
    GP_TRY(make_map(ctx, &mch, cols.xh_hi, cols.n_pad, DP, DP, BN, 64, true, true));
    GP_TRY(make_map(ctx, &mcl, cols.xh_lo, cols.n_pad, DP, DP, BN, 64, true, true));
    GP_TRY(make_map(ctx, &mvh, vhi, T, cols.n_pad, vld, T, 64, true, true));
    GP_TRY(make_map(ctx, &mvl, vlo, T, cols.n_pad, vld, T, 64, true, true));
    mvb = mvh;
  } else {
    const float* rlo = SPLIT ? rows.xt_lo : rows.xt_hi;
    const float* clo = SPLIT ? cols.xt_lo : cols.xt_hi;
    GP_TRY(make_map(ctx, &mrh, rows.xt_hi, rows.n_pad, DP, DP, BM));
    GP_TRY(make_map(ctx, &mrl, rlo, rows.n_pad, DP, DP, BM));
    GP_TRY(make_map(ctx, &mch, cols.xt_hi, cols.n_pad, DP, DP, BN));
    GP_TRY(make_map(ctx, &mcl, clo, cols.n_pad, DP, DP, BN));
    GP_TRY(make_map(ctx, &mvh, vhi, T, cols.n_pad, vld, T));
    GP_TRY(make_map(ctx, &mvl, SPLIT ? vlo : vhi, T, cols.n_pad, vld, T));
    // V_hi in BF16: boxes of 64 columns (128 bytes) x T rows
    if (SPLIT) {
      GP_TRY(make_map(ctx, &mvb, vbf, T, cols.n_pad, vld, T, 64, true, true));
    } else {
      mvb = mvh;
    }
  }
  const size_t smem = Ly::TOTAL + 1024;
  static std::atomic<uint64_t> attr{0};
  GP_TRY(smem_attr_once(ctx, kmv_tc_kernel<DP, T, OP>, smem, attr));
  const int64_t row_tiles = ceil_div(rows.n, BM);
  const int64_t col_tiles = ceil_div(cols.n, BN);
  int64_t splits = std::max<int64_t>(1, ceil_div(4LL * ctx->num_sms, row_tiles));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, col_tiles / 4));
  // Column bands that fit in L2: blockIdx.x (row tiles) varies fastest in
  // launch order, so every row tile finishes band y before band y + 1 starts
  // and each band of X~_J / V_J is read from DRAM about once, instead of once
  // per wave of CTAs that have drifted apart.
  const int64_t tile_bytes =
      F16 ? (int64_t)BN * (DP + T) * 2 * 2 + 256
          : (int64_t)BN * (DP + T) * 4 * (SPLIT ? 2 : 1) + (SPLIT ? (int64_t)BN * T * 2 : 0) + 256;
  const int64_t band_tiles = std::max<int64_t>(64, (48LL << 20) / tile_bytes);
  splits = std::max<int64_t>(splits, ceil_div(col_tiles, band_tiles));
  const int64_t per = ceil_div(col_tiles, splits);
  splits = ceil_div(col_tiles, per);
  TcParams prm;
  prm.nr = F16 ? rows.norm_h : rows.norm;
  prm.nc = F16 ? cols.norm_h : cols.norm;
  prm.nrows = rows.n;
  prm.ncols = cols.n;
  prm.out = out;
  prm.ldo = ldo;
  prm.t = t;
  prm.s = s;
  prm.sym = sym ? 1 : 0;
  prm.tiles_per_split = (int)per;
  prm.status = status;
  prm.xs_r = rows.xh_scale;
  prm.xs_c = cols.xh_scale;
  prm.vsc = vsc;
  kmv_tc_kernel<DP, T, OP><<<dim3((unsigned)row_tiles, (unsigned)splits), NTHREADS, smem, ctx->stream>>>(
      mrh, mrl, mch, mcl, mvh, mvl, mvb, prm);
  GP_LAUNCHED(ctx);
  return GP_OK;
}

}  // namespace

bool kmv_uses_sym(const gp_ctx* ctx, const Prep& rows, const Prep& cols, bool sym, int precision) {
  return ctx->sym_kmv && sym && precision == GP_FP32_SPLIT_F16 && rows.xh_hi != nullptr && rows.xh_hi == cols.xh_hi &&
         rows.n == cols.n;
}

bool kmv_tc_supported(const Prep& rows, int t, int precision) {
  (void)t;
  if (precision == GP_FP32_SPLIT_F16) return rows.xh_hi != nullptr && rows.d_pad <= kHalfCols;
  if (precision != GP_FP32_SPLIT_TF32 && precision != GP_TF32) return false;
  return rows.d_pad == 32 || rows.d_pad == 64;
}

int* device_status(gp_ctx* ctx) {
  int* st = static_cast<int*>(ws_get(ctx, WS_STATUS, 64));
  if (st && !ctx->status_init) {
    if (cudaMemsetAsync(st, 0, 64, ctx->stream) != cudaSuccess) return nullptr;
    ctx->status_init = true;
  }
  return st;
}

int check_status(gp_ctx* ctx) {
  if (!ctx->status_init) return GP_OK;
  int* st = static_cast<int*>(ws_get(ctx, WS_STATUS, 64));
  if (!ctx->status_host && cudaMallocHost(&ctx->status_host, 64) != cudaSuccess) {
    cudaGetLastError();
    ctx->status_host = nullptr;
  }
  int* h = ctx->status_host;
  if (!st || !h) return set_err(ctx, GP_ENOMEM, "status readback");
  GP_CUDA(ctx, cudaMemcpyAsync(h, st, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GP_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int code = h[0];
  if (code != 0) {
    GP_CUDA(ctx, cudaMemsetAsync(st, 0, 64, ctx->stream));
    return set_err(ctx, code, "a tensor-core K-hat V wait timed out (status %d)", code);
  }
  return GP_OK;
}

int kmv_tc(gp_ctx* ctx, const Prep& rows, const Prep& cols, const float* V, int64_t ldv, int t,
           float* out, int64_t ldo, float s, bool sym, int precision) {
  const bool f16 = precision == GP_FP32_SPLIT_F16;
  const bool split = precision == GP_FP32_SPLIT_TF32;
  if (f16 ? (!rows.xh_hi || !cols.xh_hi) : (!rows.xt_hi || !cols.xt_hi))
    return set_err(ctx, GP_EINVAL, "tensor-core features not prepared");
  int* status = device_status(ctx);
  if (!status) return set_err(ctx, GP_ENOMEM, "workspace (status)");
  const int64_t npad = cols.n_pad;
  for (int c0 = 0; c0 < t; c0 += 32) {
    const int tc = std::min(32, t - c0);
    const int T = tc <= 16 ? 16 : 32;
    const int64_t total = (int64_t)T * npad;
    const unsigned g = (unsigned)std::min<int64_t>(ceil_div(total, 256), 16LL * ctx->num_sms);
    const float* Vc = V + (int64_t)c0 * ldv;
    float* oc = out + (int64_t)c0 * ldo;
    int rc;
    if (f16) {
      __half* vhi = ws<__half>(ctx, WS_VHI, (size_t)T * npad);
      __half* vlo = ws<__half>(ctx, WS_VLO, (size_t)T * npad);
      unsigned* vmax = ws<unsigned>(ctx, WS_VMAX, 64);   // [0, 32) max bits, [32, 64) vsc
      if (!vhi || !vlo || !vmax) return set_err(ctx, GP_ENOMEM, "workspace (V split)");
      float* vsc = reinterpret_cast<float*>(vmax + 32);
      GP_CUDA(ctx, cudaMemsetAsync(vmax, 0, sizeof(unsigned) * 32, ctx->stream));
      const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(cols.n, 1024), 2LL * ctx->num_sms));
      vmax_kernel<<<dim3(gb, (unsigned)tc), 256, 0, ctx->stream>>>(Vc, ldv, cols.n, vmax);
      GP_LAUNCHED(ctx);
      split_vh_kernel<<<g, 256, 0, ctx->stream>>>(Vc, ldv, tc, cols.n, T, npad, vmax, vhi, vlo, vsc);
      GP_LAUNCHED(ctx);
      if (kmv_uses_sym(ctx, rows, cols, sym, precision))
        rc = kmv_sym_f16(ctx, rows, vhi, vlo, vsc, npad, tc, T, oc, ldo, s, status);
      else
        rc = T == 16 ? launch_tc<kHalfCols, 16, 2>(ctx, rows, cols, vhi, vlo, nullptr, vsc, npad, tc, oc, ldo, s,
                                                   sym, status)
                     : launch_tc<kHalfCols, 32, 2>(ctx, rows, cols, vhi, vlo, nullptr, vsc, npad, tc, oc, ldo, s,
                                                   sym, status);
      if (rc != GP_OK) return rc;
      continue;
    }
    float* vhi = ws<float>(ctx, WS_VHI, (size_t)T * npad);
    float* vlo = ws<float>(ctx, WS_VLO, (size_t)T * npad);
    __nv_bfloat16* vbf = split ? ws<__nv_bfloat16>(ctx, WS_VBHI, (size_t)T * npad) : nullptr;
    if (!vhi || !vlo || (split && !vbf)) return set_err(ctx, GP_ENOMEM, "workspace (V split)");
    split_v_kernel<<<g, 256, 0, ctx->stream>>>(Vc, ldv, tc, cols.n, T, npad, vhi, vlo, vbf);
    GP_LAUNCHED(ctx);
    if (split) {
      if (rows.d_pad == 32)
        rc = T == 16 ? launch_tc<32, 16, 1>(ctx, rows, cols, vhi, vlo, vbf, nullptr, npad, tc, oc, ldo, s, sym, status)
                     : launch_tc<32, 32, 1>(ctx, rows, cols, vhi, vlo, vbf, nullptr, npad, tc, oc, ldo, s, sym, status);
      else
        rc = T == 16 ? launch_tc<64, 16, 1>(ctx, rows, cols, vhi, vlo, vbf, nullptr, npad, tc, oc, ldo, s, sym, status)
                     : launch_tc<64, 32, 1>(ctx, rows, cols, vhi, vlo, vbf, nullptr, npad, tc, oc, ldo, s, sym, status);
    } else {
      if (rows.d_pad == 32)
        rc = T == 16 ? launch_tc<32, 16, 0>(ctx, rows, cols, vhi, vlo, vbf, nullptr, npad, tc, oc, ldo, s, sym, status)
                     : launch_tc<32, 32, 0>(ctx, rows, cols, vhi, vlo, vbf, nullptr, npad, tc, oc, ldo, s, sym, status);
      else
        rc = T == 16 ? launch_tc<64, 16, 0>(ctx, rows, cols, vhi, vlo, vbf, nullptr, npad, tc, oc, ldo, s, sym, status)
                     : launch_tc<64, 32, 0>(ctx, rows, cols, vhi, vlo, vbf, nullptr, npad, tc, oc, ldo, s, sym, status);
    }
    if (rc != GP_OK) return rc;
  }
  return GP_OK;
}

}  // namespace gp
