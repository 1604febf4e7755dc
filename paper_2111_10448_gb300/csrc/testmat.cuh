// Test-matrix entries as every kernel of the library regenerates them: the
// dense Gaussian stream of philox.cuh, or (TT_FLAG_KR) the Khatri-Rao product
// of per-mode Gaussian factors (Sec. 3.2, eq. (sketch_orig)) whose factors
// were staged in the workspace at the start of the call (krdrm.cu).
//
// A Khatri-Rao row index is the column-major multi-index over the sketch's
// factor modes (first mode fastest); its entry j is the product of the factor
// entries F_t(i_t, j), taken in increasing mode order for a column sketch and
// in decreasing order for a row sketch (DevSketch::kr_dec).  The products use
// explicitly rounded multiplies, so every kernel computes the same bits.
#pragma once
#include <cstdint>

#include "internal.cuh"
#include "philox.cuh"

namespace tts {

// The device sketch table of a workspace (uploaded with the plan tables).
__device__ __forceinline__ const DevSketch* ws_sketches(const void* wsb) {
  const char* b = reinterpret_cast<const char*>(wsb);
  const DevTables& T = *reinterpret_cast<const DevTables*>(b + 256);
  return reinterpret_cast<const DevSketch*>(b + T.off_sketches);
}

// Digit of mode t of a Khatri-Rao row: increasing order peels the fastest
// mode off by a remainder, decreasing order the slowest by a quotient (32-bit
// arithmetic when the row fits, which it does for every shape up to 2^32 rows).
__device__ __forceinline__ int64_t kr_digit_inc(uint64_t& row, int64_t n, bool last) {
  if (last) return (int64_t)row;
  if (row < 0x100000000ull && n < 0x100000000ll) {
    const uint32_t r = (uint32_t)row, nn = (uint32_t)n;
    const uint32_t q = r / nn;
    row = q;
    return (int64_t)(r - q * nn);
  }
  const uint64_t q = row / (uint64_t)n;
  const int64_t i = (int64_t)(row - q * (uint64_t)n);
  row = q;
  return i;
}
__device__ __forceinline__ int64_t kr_digit_dec(uint64_t& row, int64_t stride, bool last) {
  if (last) return (int64_t)row;
  uint64_t i;
  if (row < 0x100000000ull && stride < 0x100000000ll) i = (uint32_t)row / (uint32_t)stride;
  else i = row / (uint64_t)stride;
  row -= i * (uint64_t)stride;
  return (int64_t)i;
}

// Columns 4q..4q+3 of Khatri-Rao row `row` (FP32 factors, FP32 product).
__device__ __forceinline__ float4 kr_quad_f32(const void* wsb, const DevSketch& s, uint64_t row, uint32_t q) {
  const float* tab = reinterpret_cast<const float*>(reinterpret_cast<const char*>(wsb) + s.kr_tab);
  float4 v = make_float4(1.f, 1.f, 1.f, 1.f);
  for (int u = 0; u < s.kr_nm; ++u) {
    const int t = s.kr_dec ? s.kr_nm - 1 - u : u;
    const bool last = u + 1 == s.kr_nm;
    const int64_t i = s.kr_dec ? kr_digit_dec(row, s.kr_stride[t], last) : kr_digit_inc(row, s.kr_n[t], last);
    const float4 f = *reinterpret_cast<const float4*>(tab + s.kr_off[t] + i * s.kr_lp + 4 * q);
    if (u == 0) {
      v = f;
    } else {
      v.x = __fmul_rn(v.x, f.x);
      v.y = __fmul_rn(v.y, f.y);
      v.z = __fmul_rn(v.z, f.z);
      v.w = __fmul_rn(v.w, f.w);
    }
  }
  return v;
}

// Same in FP64 (FP64 factors and product).
__device__ __forceinline__ void kr_quad_f64(const void* wsb, const DevSketch& s, uint64_t row, uint32_t q,
                                            double z[4]) {
  const double* tab = reinterpret_cast<const double*>(reinterpret_cast<const char*>(wsb) + s.kr_tab);
  for (int u = 0; u < s.kr_nm; ++u) {
    const int t = s.kr_dec ? s.kr_nm - 1 - u : u;
    const bool last = u + 1 == s.kr_nm;
    const int64_t i = s.kr_dec ? kr_digit_dec(row, s.kr_stride[t], last) : kr_digit_inc(row, s.kr_n[t], last);
    const double2* f = reinterpret_cast<const double2*>(tab + s.kr_off[t] + i * s.kr_lp + 4 * q);
    const double2 a = f[0], b = f[1];
    if (u == 0) {
      z[0] = a.x; z[1] = a.y; z[2] = b.x; z[3] = b.y;
    } else {
      z[0] = __dmul_rn(z[0], a.x);
      z[1] = __dmul_rn(z[1], a.y);
      z[2] = __dmul_rn(z[2], b.x);
      z[3] = __dmul_rn(z[3], b.y);
    }
  }
}

// Mode-by-mode row sketch of X_{d-1} (DevSketch::kr_mbm): the mode-1 factor
// quad of i_1 (FP32, unrounded; an MMA operand after rounding) ...
__device__ __forceinline__ float4 kr_f1_quad(const void* wsb, const DevSketch& s, int64_t i1, uint32_t q) {
  const float* tab = reinterpret_cast<const float*>(reinterpret_cast<const char*>(wsb) + s.kr_tab);
  return *reinterpret_cast<const float4*>(tab + s.kr_off[0] + i1 * s.kr_lp + 4 * q);
}
// ... and the column scale of block `rest` (the row index divided by n_1): the
// product of the rows of modes k..2 (decreasing order), FP32, rounded to the
// MMA type `prec`.
__device__ __forceinline__ float4 kr_scale_quad(const void* wsb, const DevSketch& s, uint64_t rest, uint32_t q,
                                                int prec) {
  const float* tab = reinterpret_cast<const float*>(reinterpret_cast<const char*>(wsb) + s.kr_tab);
  uint64_t row = rest * (uint64_t)s.kr_n[0];
  float4 v = make_float4(1.f, 1.f, 1.f, 1.f);
  for (int t = s.kr_nm - 1; t >= 1; --t) {
    const int64_t i = kr_digit_dec(row, s.kr_stride[t], false);
    const float4 f = *reinterpret_cast<const float4*>(tab + s.kr_off[t] + i * s.kr_lp + 4 * q);
    if (t == s.kr_nm - 1) {
      v = f;
    } else {
      v.x = __fmul_rn(v.x, f.x);
      v.y = __fmul_rn(v.y, f.y);
      v.z = __fmul_rn(v.z, f.z);
      v.w = __fmul_rn(v.w, f.w);
    }
  }
  return make_float4(round_prec(v.x, prec), round_prec(v.y, prec), round_prec(v.z, prec), round_prec(v.w, prec));
}

// The quad a kernel uses: kr = the sketch's device record when its test
// matrix is Khatri-Rao, nullptr for the dense stream.
__device__ __forceinline__ float4 tm_quad_f32(const void* wsb, const DevSketch* kr, uint64_t seed, uint32_t sid,
                                              uint64_t row, uint32_t q) {
  if (kr) return kr_quad_f32(wsb, *kr, row, q);
  return normals4_f32(seed, sid, row, q);
}
__device__ __forceinline__ void tm_quad_f64(const void* wsb, const DevSketch* kr, uint64_t seed, uint32_t sid,
                                            uint64_t row, uint32_t q, double z[4]) {
  if (kr) kr_quad_f64(wsb, *kr, row, q, z);
  else normals4_f64(seed, sid, row, q, z);
}
// Final test-matrix entries of a TF32 / BF16 path as FP32 values (for the
// kernels that use them in FP32 / FP64 arithmetic: the middle-core matrix B
// and the backward): entries rounded to the MMA type, except a mode-by-mode
// Khatri-Rao sketch, whose entry is the exact FP32 product of its two rounded
// parts.
__device__ __forceinline__ float4 tm_quad_mixed(const void* wsb, const DevSketch* kr, uint64_t seed, uint32_t sid,
                                                uint64_t row, uint32_t q, int prec) {
  if (kr && kr->kr_mbm) {
    const uint64_t rest = row / (uint64_t)kr->kr_n[0];
    const float4 f = kr_f1_quad(wsb, *kr, (int64_t)(row - rest * (uint64_t)kr->kr_n[0]), q);
    const float4 c = kr_scale_quad(wsb, *kr, rest, q, prec);
    return make_float4(__fmul_rn(round_prec(f.x, prec), c.x), __fmul_rn(round_prec(f.y, prec), c.y),
                       __fmul_rn(round_prec(f.z, prec), c.z), __fmul_rn(round_prec(f.w, prec), c.w));
  }
  const float4 z = tm_quad_f32(wsb, kr, seed, sid, row, q);
  return make_float4(round_prec(z.x, prec), round_prec(z.y, prec), round_prec(z.z, prec), round_prec(z.w, prec));
}

// Device record of sketch gsk of the workspace, or nullptr (gsk < 0: dense).
__device__ __forceinline__ const DevSketch* kr_of(const void* wsb, int gsk) {
  return gsk >= 0 ? ws_sketches(wsb) + gsk : nullptr;
}

}  // namespace tts
