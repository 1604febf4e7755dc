// tcgen05 / TMA / mbarrier helpers shared by the plane kernels (inline PTX
// for sm_103a): shared-memory matrix descriptors in the no-swizzle
// core-matrix layout, the BF16 x BF16 -> FP32 tcgen05.mma with its commit,
// tensor-memory loads, bounded mbarrier waits, bulk copies.
#pragma once
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"

namespace tts {
namespace tc {

constexpr int kS1 = 144;                 // bytes between core matrices along i_1 (k of B)
constexpr int kS4 = 16 * kS1;            // 2304: bytes between core matrices along i_d (n of B)
static_assert(kS4 == kTcGroupBytes, "block image layout");
constexpr int kTileB = 16 * kS4;         // one 128 x 128 BF16 tile
constexpr int kStageB = 2 * kTileB;      // hi + lo
constexpr long long kWaitCycles = 4000000000LL;  // bounded waits (~2 s)
constexpr int kMaxChainL = 256;                   // accumulating MMAs per accumulator between flushes
constexpr int kMaxChainS = 32;                    // the same with TT_FLAG_SHORT_CHAINS

struct SkTc {
  int64_t rows, off, wdiv, hstride;
  int64_t tab;  // byte offset of the staged blocks in the workspace, -1: generated per plane
  int sid;
  int kr;       // global sketch index when the test matrix is Khatri-Rao, -1: dense
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of
// 16), completing `bytes` of transaction count on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// L2 prefetch of `bytes` (a multiple of 16) from a 16-byte aligned global address.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; on give-up raises the abort flag and the timeout status bit.
static __device__ bool mbar_wait_for(uint32_t a, uint32_t parity, volatile int* abort_flag, int* status,
                              long long limit) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort_flag) return false;
      if (clock64() - t0 > limit) {
        *abort_flag = 1;
        atomicOr(status, ST_TIMEOUT);
        return false;
      }
    }
  }
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int* status) {
  return mbar_wait_for(a, parity, abort_flag, status, kWaitCycles);
}
// Wait by every lane of a warp; the result is the same on all lanes (false if
// any lane gave up), so control flow after it stays converged.
__device__ __forceinline__ bool warp_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, int* status) {
  const bool ok = mbar_wait_for(a, parity, abort_flag, status, kWaitCycles);
  return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor, no swizzle: start, leading (K-direction)
// and stride (M/N-direction) byte offsets of the core matrices, version 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor, kind::f16: BF16 x BF16 (or, f16, FP16 x FP16) ->
// F32, M = 128.  A and B always have the same type.
__host__ __device__ constexpr uint32_t make_idesc(int n, bool a_mn_major, bool f16 = false) {
  return (1u << 4) | (f16 ? 0u : (1u << 7) | (1u << 10)) | ((a_mn_major ? 1u : 0u) << 15) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma16_ss(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// Same, with the descriptors given as 32-bit halves (a k-step only moves the
// start-address field, which lives in the low half).
__device__ __forceinline__ void mma16_ss_lo(uint32_t dtmem, uint32_t alo, uint32_t ahi, uint32_t blo,
                                               uint32_t bhi, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t.reg .b64 ad, bd;\n\t"
      "mov.b64 ad, {%1, %2};\n\tmov.b64 bd, {%3, %4};\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], ad, bd, %5, p;\n\t}"
      ::"r"(dtmem), "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc));
}
// One lane of a converged warp (the lowest active lane) is elected; the MMA
// warp runs its control flow on all lanes and issues through the elected lane,
// so descriptors and loop state stay warp-uniform.
__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "elect.sync _|P, 0xffffffff;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(pred));
  return pred != 0;
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
template <int ELL>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float v[ELL]) {
  static_assert(ELL == 8 || ELL == 16, "sketch width of the plane kernel");
  if constexpr (ELL == 16) tmem_ld16(taddr, v);
  else tmem_ld8(taddr, v);
}
// Two FP32 values rounded to nearest-even and packed, `lo` in the low half
// (cvt packs its first source into the upper half).
__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ uint32_t f16x2_bits(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// The 16-bit MMA operand type of a kernel instance: BF16, or FP16 when F16.
template <bool F16>
__device__ __forceinline__ uint32_t op16x2_bits(float lo, float hi) {
  if constexpr (F16) return f16x2_bits(lo, hi);
  else return bf16x2_bits(lo, hi);
}
template <bool F16>
__device__ __forceinline__ uint16_t op16_bits(float v) {
  if constexpr (F16) return __half_as_ushort(__float2half_rn(v));
  else return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
// X = hi + lo in the 16-bit operand type, two entries at a time: hi is the
// nearest value of the type, lo the nearest to the exact FP32 remainder.
template <bool F16>
__device__ __forceinline__ void split_hi_lo(float x0, float x1, uint32_t& hb, uint32_t& lb) {
  if constexpr (F16) {
    hb = f16x2_bits(x0, x1);
    const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&hb));
    lb = f16x2_bits(__fsub_rn(x0, hf.x), __fsub_rn(x1, hf.y));
  } else {
    hb = bf16x2_bits(x0, x1);
    const float h0 = __uint_as_float(hb << 16), h1 = __uint_as_float(hb & 0xFFFF0000u);
    lb = bf16x2_bits(__fsub_rn(x0, h0), __fsub_rn(x1, h1));
  }
}
template <bool F16>
__device__ __forceinline__ float round_op16(float v) {
  if constexpr (F16) return __half2float(__float2half_rn(v));
  else return __bfloat162float(__float2bfloat16_rn(v));
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void st_shared_b32(uint32_t a, uint32_t x) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(x) : "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

}  // namespace tc
}  // namespace tts
