// PTX helpers shared by the tcgen05 kernels (fused K-hat V and the backward
// tiles): mbarriers with bounded waits, TMA loads, shared-memory matrix
// descriptors, tcgen05.mma / ld / st wrappers, and the host-side tensor-map
// encoder.  Every wait is bounded by kWaitCycles; a timeout sets the CTA's
// failure flag instead of trapping.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "gp_internal.cuh"

namespace gp {
namespace tc {

constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait with a suspend-time hint: the thread sleeps until the phase
// completes or about `ns` nanoseconds pass, instead of spinning on issue
// slots that the other warps of the SM need.
__device__ __forceinline__ bool mbar_test_sleep(uint64_t* b, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Bounded wait: false on timeout or when another role already failed.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* fail) {
  if (mbar_test(b, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t i = 1;; ++i) {
    if (mbar_test_sleep(b, parity, 20000u)) return true;
    if ((i & 15) == 0) {
      if (*reinterpret_cast<volatile int*>(fail)) return false;
      if (clock64() - t0 > kWaitCycles) {
        atomicExch(fail, 1);
        return false;
      }
    }
  }
}
// Bounded wait used on the way out (ignores the failure flag).
__device__ __forceinline__ bool mbar_wait_exit(uint64_t* b, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(b, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          su32(dst)),
      "l"(map), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// SMEM matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor: kind::f16 with BF16 A and B, D = F32, K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor: kind::f16 with FP16 A and B, D = F32, K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor: kind::tf32, D = F32, A and B K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// tcgen05.mma kind::tf32 (A from SMEM: _ss, from TMEM: _ts) with compile-time
// byte/16 offsets added to the SMEM descriptors (and to the TMEM A address)
// inside the asm, so that the offsets stay immediates instead of registers
// held across the tile loop.
template <uint32_t AO, uint32_t BO>
__device__ __forceinline__ void mma_ss_imm(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b64 da, db;\n add.s64 da, %1, %5;\n add.s64 db, %2, %6;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], da, db, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc), "n"(AO), "n"(BO)
      : "memory");
}
// kind::f16 (FP16 or BF16 operands, as the instruction descriptor says), A
// and B from SMEM.
template <uint32_t AO, uint32_t BO>
__device__ __forceinline__ void mma_ss_f16_imm(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b64 da, db;\n add.s64 da, %1, %5;\n add.s64 db, %2, %6;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc), "n"(AO), "n"(BO)
      : "memory");
}
template <uint32_t AO, uint32_t BO>
__device__ __forceinline__ void mma_ts_imm(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b32 ta;\n .reg .b64 db;\n add.u32 ta, %1, %5;\n add.s64 db, %2, %6;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [ta], db, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc), "n"(AO), "n"(BO)
      : "memory");
}
template <uint32_t AO, uint32_t BO>
__device__ __forceinline__ void mma_ts_bf16_imm(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                                uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b32 ta;\n .reg .b64 db;\n add.u32 ta, %1, %5;\n add.s64 db, %2, %6;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [ta], db, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc), "n"(AO), "n"(BO)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
[[maybe_unused]] __device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
}
[[maybe_unused]] __device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// 2^-x on the MUFU pipe (the negation is an operand modifier of the op)
__device__ __forceinline__ float ex2_neg_approx(float x) {
  float y;
  asm("{\n .reg .f32 t;\n neg.f32 t, %1;\n ex2.approx.ftz.f32 %0, t;\n}\n" : "=f"(y) : "f"(x));
  return y;
}
// sqrt(|x|) on the MUFU pipe: the modulus absorbs a u^2 rounded below zero
// and sqrt(0) = 0, so the caller needs no clamp.  The modulus is the plain
// (non-flushing) abs, which rides on the MUFU operand as a modifier; the
// square root's own ftz flushes a subnormal |x| to 0.
__device__ __forceinline__ float sqrt_abs_approx(float x) {
  float y;
  asm("{\n .reg .f32 t;\n abs.f32 t, %1;\n sqrt.approx.ftz.f32 %0, t;\n}\n" : "=f"(y) : "f"(x));
  return y;
}
// 2^14 k/s of two kernel entries of one row (columns b, b + 1) from the
// cross term s = x~_a . x~_b in FP16-scaled units: u^2 = m2 s + (n_a + n_b),
// u = sqrt(|u^2|), (2^14 + 2^14 ln2 u + 2^14 (ln2)^2 u^2 / 3) 2^-u.  The
// FP32 steps run as packed FP32x2 instructions (two entries per
// instruction, each lane rounded to nearest as the scalar ops are); the
// square roots and exponentials stay on the MUFU pipe.
__device__ __forceinline__ float2 matern2_scaled(float2 s, float2 nb, float2 na2, float2 m22) {
  const float2 u2 = __ffma2_rn(m22, s, __fadd2_rn(na2, nb));
  const float2 uu = make_float2(sqrt_abs_approx(u2.x), sqrt_abs_approx(u2.y));
  float2 p = __ffma2_rn(uu, make_float2(kC1s, kC1s), make_float2(kP0s, kP0s));
  p = __ffma2_rn(u2, make_float2(kC2s, kC2s), p);
  return __fmul2_rn(p, make_float2(ex2_neg_approx(uu.x), ex2_neg_approx(uu.y)));
}
// FP16 hi and lo parts of two values, packed two per 32-bit word (first
// value in the low half): hi = fp16(v), lo = fp16(v - hi), v - hi exact in
// FP32, so hi + lo = v to 2^-22.  v - hi is one mixed-precision FMA per
// value (FP16 hi times FP16 -1 plus the FP32 v, rounded once), so hi is
// never widened back to FP32 by a separate conversion.
__device__ __forceinline__ void split_h2(float2 v, uint32_t& hi, uint32_t& lo) {
  const __half2 hv = __floats2half2_rn(v.x, v.y);
  hi = *reinterpret_cast<const uint32_t*>(&hv);
  float r0, r1;
  asm("{\n .reg .b16 a, b, m;\n mov.b32 {a, b}, %2;\n mov.b16 m, 0xBC00;\n"
      " fma.rn.f32.f16 %0, a, m, %3;\n fma.rn.f32.f16 %1, b, m, %4;\n}\n"
      : "=f"(r0), "=f"(r1)
      : "r"(hi), "f"(v.x), "f"(v.y));
  const __half2 lv = __floats2half2_rn(r0, r1);
  lo = *reinterpret_cast<const uint32_t*>(&lv);
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}


// ------------------------------------------------------------- host side ----
inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D FP32 tensor [rows][cols] (cols contiguous), box = 32 cols x box_rows,
// 128-byte swizzle.
inline int make_map(gp_ctx* ctx, CUtensorMap* m, const void* base, int64_t rows, int64_t cols,
             int64_t ld, int box_rows, int box_cols = 32, bool swizzle = true, bool bf16 = false) {
  auto fn = encode_fn();
  if (!fn) return set_err(ctx, GP_ECUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const size_t es_bytes = bf16 ? 2 : 4;
  cuuint64_t gstr[1] = {(cuuint64_t)ld * es_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1u, 1u};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  const_cast<void*>(base), gdim, gstr, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_err(ctx, GP_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return GP_OK;
}


}  // namespace tc
}  // namespace gp
