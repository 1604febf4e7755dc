// Device side of the library's Gaussian stream.
//
// The paper draws the test matrices of Algorithm 2 (and of the one-pass
// variant, eq. (3.3)) with i.i.d. standard Gaussian entries; this library
// regenerates them on the fly from a counter-based generator instead of
// storing them.  Definition (independent of, and identical in meaning to, the
// host-side definition used by the tests):
//   Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of
//     (hi0, lo0) = c0 * 0xD2511F53, (hi1, lo1) = c2 * 0xCD9E8D57,
//     c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
//   key bumped by (0x9E3779B9, 0xBB67AE85) after each round.
//   key = (seed lo, seed hi); entry (row, j) of stream s uses the counter
//   (row lo, row hi, j / 4, s) and Box-Muller on the four output words:
//   rho = sqrt(-2 ln u(x0)), theta = 2 pi u(x1) -> (rho cos, rho sin) for
//   j % 4 = 0, 1 and likewise (x2, x3) for j % 4 = 2, 3.
//   FP64 uniforms: u = (x + 1/2) 2^-32.
//   FP32 (mixed precision): the same u evaluated in FP32 as
//   fma(float(x), 2^-32, 2^-33) (relative error <= 2^-24), rho from logf and
//   sqrt, and the angle taken centred, theta - pi = 2 pi u - pi in (-pi, pi],
//   through the fast sine/cosine (cos theta = -cos(theta - pi), likewise
//   sin); the normal differs from the FP64 one by about 1e-7 relative and at
//   most a few 1e-6 absolute.
#pragma once
#include <cstdint>

#include <cuda_fp16.h>

namespace tts {

__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u;  // one 32x32 -> 64-bit multiply each
    const uint64_t p1 = (uint64_t)c2 * 0xCD9E8D57u;
    c0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    c1 = (uint32_t)p1;
    c2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c3 = (uint32_t)p0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// Four consecutive FP64 normals z[4q..4q+3] of row `row` of stream `sid`.
__device__ __forceinline__ void normals4_f64(uint64_t seed, uint32_t sid, uint64_t row, uint32_t q,
                                             double z[4]) {
  uint32_t c0 = (uint32_t)row, c1 = (uint32_t)(row >> 32), c2 = q, c3 = sid;
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u0 = ((double)c0 + 0.5) * 0x1p-32;
  const double u1 = ((double)c1 + 0.5) * 0x1p-32;
  const double u2 = ((double)c2 + 0.5) * 0x1p-32;
  const double u3 = ((double)c3 + 0.5) * 0x1p-32;
  const double ra = sqrt(-2.0 * log(u0));
  const double rb = sqrt(-2.0 * log(u2));
  double sa, ca, sb, cb;
  sincospi(2.0 * u1, &sa, &ca);
  sincospi(2.0 * u3, &sb, &cb);
  z[0] = ra * ca;
  z[1] = ra * sa;
  z[2] = rb * cb;
  z[3] = rb * sb;
}

// Four consecutive FP32 normals of the mixed-precision sketches.  Every
// operation below is an explicitly rounded intrinsic (or logf), so the
// compiler has no contraction or reassociation freedom: every inlined copy,
// in every kernel that regenerates these entries (the sketch, the staged
// test-matrix tables, the middle-core matrix B, the backward), computes the
// same bits.
__device__ __forceinline__ float4 normals4_f32(uint64_t seed, uint32_t sid, uint64_t row, uint32_t q) {
  uint32_t c0 = (uint32_t)row, c1 = (uint32_t)(row >> 32), c2 = q, c3 = sid;
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  // u = (x + 1/2) 2^-32 in FP32: x is rounded to 24 bits (relative error
  // 2^-24 at any magnitude), then scaled exactly and offset by 2^-33.
  const float u0 = __fmaf_rn(__uint2float_rn(c0), 0x1p-32f, 0x1p-33f);
  const float u1 = __fmaf_rn(__uint2float_rn(c1), 0x1p-32f, 0x1p-33f);
  const float u2 = __fmaf_rn(__uint2float_rn(c2), 0x1p-32f, 0x1p-33f);
  const float u3 = __fmaf_rn(__uint2float_rn(c3), 0x1p-32f, 0x1p-33f);
  const float ra = __fsqrt_rn(__fmul_rn(-2.0f, logf(u0)));
  const float rb = __fsqrt_rn(__fmul_rn(-2.0f, logf(u2)));
  // centred angles 2 pi u - pi in (-pi, pi]: cos(2 pi u) = -cos(.), sin likewise
  const float ta = __fmaf_rn(u1, 6.28318530717958647692f, -3.14159265358979323846f);
  const float tb = __fmaf_rn(u3, 6.28318530717958647692f, -3.14159265358979323846f);
  float sa, ca, sb, cb;
  __sincosf(ta, &sa, &ca);
  __sincosf(tb, &sb, &cb);
  return make_float4(-__fmul_rn(ra, ca), -__fmul_rn(ra, sa), -__fmul_rn(rb, cb), -__fmul_rn(rb, sb));
}

// Round an FP32 value to the MMA input type, nearest-even, returned as FP32.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  const uint32_t lsb = (u >> 13) & 1u;
  u = (u + 0xFFFu + lsb) & ~0x1FFFu;
  return __uint_as_float(u);
}
__device__ __forceinline__ float round_bf16(float x) {
  uint32_t u = __float_as_uint(x);
  const uint32_t lsb = (u >> 16) & 1u;
  u = (u + 0x7FFFu + lsb) & ~0xFFFFu;
  return __uint_as_float(u);
}
__device__ __forceinline__ float round_f16(float x) { return __half2float(__float2half_rn(x)); }
__device__ __forceinline__ float round_prec(float x, int prec) {
  return prec == TT_PREC_TF32 ? round_tf32(x) : prec == TT_PREC_FP16 ? round_f16(x) : round_bf16(x);
}

}  // namespace tts
