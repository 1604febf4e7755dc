// Mixed-precision (TF32 / BF16 / FP16 tensor-core) sketch path and everything that
// must regenerate its test matrices bit-identically (the middle-core matrix
// B = P^T Omega_{d*} of the one-pass solve, and the test-matrix export).
// All of them use the FP32 generator of philox.cuh.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "philox.cuh"
#include "testmat.cuh"
#include "tc_common.cuh"

namespace tts {

namespace {

__global__ void test_matrix_mixed_kernel(uint64_t seed, int sid, int64_t row0, int64_t nrows, int ncols,
                                         int prec, double* out) {
  const int nq = (ncols + 3) / 4;
  const int64_t total = nrows * nq;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % nrows;
    const int q = (int)(e / nrows);
    const float4 z4 = normals4_f32(seed, (uint32_t)sid, (uint64_t)(row0 + r), (uint32_t)q);
    const float z[4] = {z4.x, z4.y, z4.z, z4.w};
    for (int t = 0; t < 4; ++t)
      if (4 * q + t < ncols) out[r + nrows * (4 * q + t)] = (double)round_prec(z[t], prec);
  }
}

constexpr int64_t kTableOffB = 256;

// B = P_{d*}^T Omega^_{d*}, Omega^ = the rounded FP32 entries the sketch used.
// item < 0: batched launch, item = blockIdx.y
__global__ void __launch_bounds__(256) mid_b_kernel_mixed(char* wsb, int item_arg, const int* ranks) {
  const int item = item_arg >= 0 ? item_arg : (int)blockIdx.y;
  constexpr int CH = 32;
  __shared__ double Ps[CH * TT_MAXL];
  __shared__ double Gs[CH * (TT_MAXL + 1)];
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
  const DevItem& it = reinterpret_cast<const DevItem*>(wsb + T.off_items)[item];
  const DevSketch* sks = reinterpret_cast<const DevSketch*>(wsb + T.off_sketches);
  const DevSketch& sp = sks[it.basis_of_k[it.mbk]];
  // the middle test matrix is the one the least-squares sketch used
  const DevSketch* kr_mid = sks[it.mid_sk].kr_nm ? &sks[it.mid_sk] : nullptr;
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + it.mbk];
  const int l = it.lmid;
  const int64_t M = sp.rows;
  const double* Pm = ws + sp.lev_z[0];
  // with r l <= blockDim pairs each thread keeps its pair's sum across the
  // block's row chunks and adds it to B once
  const bool keep = r * l <= (int)blockDim.x;
  double kept = 0.0;
  for (int64_t v0 = (int64_t)blockIdx.x * CH; v0 < M; v0 += (int64_t)gridDim.x * CH) {
    const int nv = (int)imin64(CH, M - v0);
    __syncthreads();
    for (int o = threadIdx.x; o < CH * r; o += blockDim.x) {
      const int v = o % CH, c = o / CH;
      Ps[v + CH * c] = v < nv ? Pm[v0 + v + M * c] : 0.0;
    }
    const int nq = (l + 3) / 4;
    for (int o = threadIdx.x; o < nv * nq; o += blockDim.x) {
      const int v = o % nv, q = o / nv;
      const float4 z4 =
          tm_quad_mixed(wsb, kr_mid, it.seed, (uint32_t)it.mstream, (uint64_t)(v0 + v), (uint32_t)q, it.prec);
      const float z[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < l) Gs[v + CH * (4 * q + t)] = (double)z[t];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < r * l; o += blockDim.x) {
      const int c = o % r, j = o / r;
      double acc = 0.0;
      for (int v = 0; v < nv; ++v) acc = fma(Ps[v + CH * c], Gs[v + CH * j], acc);
      if (keep) kept += acc;
      else atomicAdd(ws + it.off_B + c + (int64_t)it.rpad[it.mbk] * j, acc);
    }
  }
  if (keep && (int)threadIdx.x < r * l) {
    const int c = (int)threadIdx.x % r, j = (int)threadIdx.x / r;
    atomicAdd(ws + it.off_B + c + (int64_t)it.rpad[it.mbk] * j, kept);
  }
}

}  // namespace

const DevSketch* plan_sketches_host(const Plan* p);

cudaError_t launch_test_matrix_mixed(uint64_t seed, int sid, int64_t row0, int64_t nrows, int ncols,
                                     int prec, double* out, cudaStream_t st) {
  const int64_t n = nrows * ((ncols + 3) / 4);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16LL * device_sm_count()));
  count_launch();
  test_matrix_mixed_kernel<<<grid, 256, 0, st>>>(seed, sid, row0, nrows, ncols, prec, out);
  return cudaGetLastError();
}

cudaError_t launch_mid_b_mixed_batched(const Plan& P, void* ws, const int* ranks, cudaStream_t st) {
  int64_t Mmax = 1;
  for (int i = 0; i < plan_num_items(&P); ++i) {
    const DevItem& it = plan_items_host(&P)[i];
    Mmax = std::max(Mmax, plan_sketches_host(&P)[it.basis_of_k[it.mbk]].rows);
  }
  const unsigned gx = (unsigned)std::min<int64_t>((Mmax + 31) / 32, 64);
  count_launch();
  mid_b_kernel_mixed<<<dim3(gx, (unsigned)plan_num_items(&P)), 256, 0, st>>>((char*)ws, -1, ranks);
  return cudaGetLastError();
}

cudaError_t launch_mid_b_mixed(const Plan& P, int item, void* ws, const int* ranks, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  const int64_t M = plan_sketches_host(&P)[it.basis_of_k[it.mbk]].rows;
  const int grid = (int)std::min<int64_t>((M + 31) / 32, 2LL * device_sm_count());
  count_launch();
  mid_b_kernel_mixed<<<grid, 256, 0, st>>>((char*)ws, item, ranks);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Generic mixed-precision fused sketch (any shape): the plane/tile structure of
// the FP64 kernel, with the tile products on the tensor cores.  For one tile
// (a-block x b-block of plane w) and one sketch the product is taken
// transposed, D^T = G^T X', so that the thin side (l, padded to 16) is the MMA
// M dimension and the tile's rows or columns are N:
//   column sketch: D^T[j, a] = sum_b G[b, j] X[a, b]   (G = Omega_k rows)
//   row sketch:    D^T[j, b] = sum_a G[a, j] X[a, b]   (G = Psi_k rows)
// X is split as X = X_hi + X_lo in the MMA type (two MMAs per k-step); G is
// rounded once.  FP32 accumulation per tile, flushed to the FP64 sketches.
namespace {

constexpr int gTA = 64;
constexpr int gTB = 32;
constexpr int gThreads = 256;

struct SkArgM {
  int64_t rows, off, wdiv, hstride;
  int64_t tab;  // byte offset (from the workspace base) of the staged test-matrix rows, -1: none
  int type, width, sid;
  int kr;       // global sketch index when the test matrix is Khatri-Rao, -1: dense
};

struct MixArgs {
  const float* X;
  double* ws;
  int64_t n1, cnt, first, W, Nd1;
  uint64_t seed;
  int nsk, prec;
  float xscale;  // FP16: 2^s, X is split as X 2^s (1 otherwise)
  SkArgM sk[kMaxSk];
};

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_f16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One (m-tile, n-tile) of D^T = G^T X' for the current tile and sketch, TF32
// (m16n8k8) fragments read element by element from the FP32 tiles.
// Gs: rows x LDG (row = contraction index k, col = j).  X'[k][o] = X(o, k)
// (column sketch, X[o + LDX k]) or X(k, o) (row sketch, X[k + LDX o]).
template <bool COL>
__device__ __forceinline__ void tile_mma_tf32(const float* Gs, int LDG, const float* Xh, const float* Xl, int LDX,
                                              int kreal, int kext, int m0, int n0, float acc[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  auto Aj = [&](int j, int k) -> float { return (k < kreal) ? Gs[k * LDG + j] : 0.0f; };
  auto Bx = [&](const float* Xs, int k, int o) -> float {
    if (k >= kreal) return 0.0f;
    return COL ? Xs[o + LDX * k] : Xs[k + LDX * o];
  };
  for (int k0 = 0; k0 < kext; k0 += 8) {
    uint32_t a[4];
    a[0] = __float_as_uint(Aj(m0 + g, k0 + t));
    a[1] = __float_as_uint(Aj(m0 + g + 8, k0 + t));
    a[2] = __float_as_uint(Aj(m0 + g, k0 + t + 4));
    a[3] = __float_as_uint(Aj(m0 + g + 8, k0 + t + 4));
    const int o = n0 + g;
    mma_tf32(acc, a, __float_as_uint(Bx(Xh, k0 + t, o)), __float_as_uint(Bx(Xh, k0 + t + 4, o)));
    mma_tf32(acc, a, __float_as_uint(Bx(Xl, k0 + t, o)), __float_as_uint(Bx(Xl, k0 + t + 4, o)));
  }
}

__device__ __forceinline__ uint32_t g_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void g_ldsm_x4_trans(const void* p, uint32_t r[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(g_smem_u32(p)));
}
__device__ __forceinline__ void g_ldsm_x2(const void* p, uint32_t r[2]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(g_smem_u32(p)));
}
__device__ __forceinline__ void g_ldsm_x2_trans(const void* p, uint32_t r[2]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(g_smem_u32(p)));
}

// 16-bit operand tiles, BF16 or FP16 (in the same dynamic shared memory as
// the FP32 ones):
// X hi / lo as [b][a] (a contiguous) and the test-matrix rows as [k][j] (j
// contiguous), rows of 72 elements (144 bytes: the eight row addresses of an
// ldmatrix fall on distinct banks).  The MMA fragments come from ldmatrix:
// A = G^T from [k][j] transposed, B from [b][a] transposed (column sketches,
// k = b) or as stored (row sketches, k = a).
constexpr int gLDX = gTA + 8;
constexpr int gLDG = TT_MAXL + 8;

// One tile (gTA rows of i_1 x gTB columns of i_d of plane w) into every sketch.
// F16: the 16-bit operands are FP16 (X scaled by 2^s first), else BF16.
template <bool F16>
__device__ void mma_tile(const MixArgs& a, int64_t item, float* fsm) {
  constexpr int LDX = gTA + 1;
  float* Xh = fsm;                  // LDX x gTB  (X[a + LDX b])        (TF32)
  float* Xl = Xh + LDX * gTB;
  float* Gs = Xl + LDX * gTB;       // rows (<= gTA) x LDG              (TF32)
  uint16_t* XhB = reinterpret_cast<uint16_t*>(fsm);   // gTB x gLDX (16-bit)
  uint16_t* XlB = XhB + gLDX * gTB;
  uint16_t* GsB = XlB + gLDX * gTB;                   // gTA x gLDG (16-bit)
  const bool bf = a.prec == TT_PREC_BF16 || F16;      // 16-bit operands (m16n8k16)
  // rounding to the MMA type: FP16 in the F16 instance, else TF32 or BF16
  const bool tf = a.prec == TT_PREC_TF32;
  auto rnd = [tf](float x) -> float {
    if constexpr (F16) return round_f16(x);
    else return tf ? round_tf32(x) : round_bf16(x);
  };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nA = (a.n1 + gTA - 1) / gTA;
  const int64_t nB = (a.cnt + gTB - 1) / gTB;
  {
    const int64_t w = item / (nA * nB);
    const int64_t rem = item - w * nA * nB;
    const int64_t bb = rem / nA, ab = rem - bb * nA;
    const int64_t a0 = ab * gTA, b0 = bb * gTB;
    const int ta = (int)imin64(gTA, a.n1 - a0);
    const int tb = (int)imin64(gTB, a.cnt - b0);
    __syncthreads();
    for (int o = tid; o < gTA * gTB; o += gThreads) {
      const int ia = o % gTA, ib = o / gTA;
      float v = 0.0f;
      if (ia < ta && ib < tb) v = __ldg(a.X + (a0 + ia) + a.n1 * w + a.Nd1 * (b0 + ib));
      if constexpr (F16) v = __fmul_rn(v, a.xscale);
      const float hi = rnd(v);
      const float lo = rnd(__fsub_rn(v, hi));
      if (bf) {  // exact: hi, lo are values of the 16-bit type
        XhB[ib * gLDX + ia] = tc::op16_bits<F16>(hi);
        XlB[ib * gLDX + ia] = tc::op16_bits<F16>(lo);
      } else {
        Xh[ia + LDX * ib] = hi;
        Xl[ia + LDX * ib] = lo;
      }
    }
    for (int s = 0; s < a.nsk; ++s) {
      const SkArgM sk = a.sk[s];
      const int l = sk.width;
      const int lpad = (l + 15) & ~15;
      const int LDG = lpad + 4;
      const int64_t wlo = w % sk.wdiv, whi = w / sk.wdiv;
      const bool col = sk.type == SK_COL;
      const int nr = col ? tb : ta;          // contraction extent of this product
      const int nout = col ? ta : tb;        // output extent (N)
      const int nq = lpad / 4;
      const int kext = bf ? ((nr + 15) & ~15) : ((nr + 7) & ~7);
      __syncthreads();
      if (sk.tab >= 0) {
        // staged rows: (key, row) at element (key nrows + row) lpad, where the
        // column side keys by w / wdiv over the slab's i_d and the row side by
        // w % wdiv over i_1
        const int64_t trow = col ? whi * a.cnt + b0 : wlo * a.n1 + a0;
        const int esz = bf ? 2 : 4;
        const int cpr = lpad * esz / 16;  // 16-byte chunks a row
        const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(a.ws) + sk.tab +
                                                          trow * lpad * esz);
        for (int o = tid; o < nr * cpr; o += gThreads) {
          const int r = o / cpr, c = o - r * cpr;
          const uint4 v = __ldg(src + (int64_t)r * cpr + c);
          if (bf) reinterpret_cast<uint4*>(GsB + r * gLDG)[c] = v;
          else reinterpret_cast<uint4*>(Gs + r * LDG)[c] = v;
        }
      } else {  // regenerate the rows
        for (int o = tid; o < nr * nq; o += gThreads) {
          const int r = o % nr, q = o / nr;
          const uint64_t grow = col ? (uint64_t)(whi + sk.hstride * (a.first + b0 + r))
                                    : (uint64_t)((a0 + r) + a.n1 * wlo);
          const DevSketch* krs = kr_of(a.ws, sk.kr);
          // a mode-by-mode sketch takes its mode-1 factor here (scaled at the flush)
          const float4 z4 = (krs && krs->kr_mbm) ? kr_f1_quad(a.ws, *krs, a0 + r, (uint32_t)q)
                                                 : tm_quad_f32(a.ws, krs, a.seed, (uint32_t)sk.sid, grow, (uint32_t)q);
          const float z[4] = {z4.x, z4.y, z4.z, z4.w};
          if (bf) {
            float zz[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) zz[u] = (4 * q + u < l) ? rnd(z[u]) : 0.0f;
            uint32_t* gp = reinterpret_cast<uint32_t*>(GsB + r * gLDG + 4 * q);
            gp[0] = tc::op16x2_bits<F16>(zz[0], zz[1]);
            gp[1] = tc::op16x2_bits<F16>(zz[2], zz[3]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) Gs[r * LDG + 4 * q + u] = (4 * q + u < l) ? rnd(z[u]) : 0.0f;
          }
        }
      }
      if (bf)  // contraction padding rows [nr, kext) (another sketch may have left rows there)
        for (int o = tid; o < (kext - nr) * (lpad / 2); o += gThreads) {
          const int r = nr + o / (lpad / 2), c2 = o % (lpad / 2);
          reinterpret_cast<uint32_t*>(GsB + r * gLDG)[c2] = 0u;
        }
      __syncthreads();
      const int mt = lpad / 16, nt = (nout + 7) / 8;
      double* out = a.ws + sk.off;
      for (int job = warp; job < mt * nt; job += gThreads / 32) {
        const int m0 = (job % mt) * 16, n0 = (job / mt) * 8;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (bf) {
          for (int k0 = 0; k0 < kext; k0 += 16) {
            uint32_t af[4], bh[2], bl[2];
            g_ldsm_x4_trans(GsB + (k0 + (lane & 7) + 8 * (lane >> 4)) * gLDG + m0 + 8 * ((lane >> 3) & 1), af);
            if (col) {  // B[k][o] = X(o, k), k = b: the [b][a] tile read transposed
              const int off = (k0 + (lane & 7) + 8 * ((lane >> 3) & 1)) * gLDX + n0;
              g_ldsm_x2_trans(XhB + off, bh);
              g_ldsm_x2_trans(XlB + off, bl);
            } else {    // B[k][o] = X(k, o), k = a: the [b][a] tile read as stored
              const int off = (n0 + (lane & 7)) * gLDX + k0 + 8 * ((lane >> 3) & 1);
              g_ldsm_x2(XhB + off, bh);
              g_ldsm_x2(XlB + off, bl);
            }
            if constexpr (F16) {
              mma_f16(acc, af, bh[0], bh[1]);
              mma_f16(acc, af, bl[0], bl[1]);
            } else {
              mma_bf16(acc, af, bh[0], bh[1]);
              mma_bf16(acc, af, bl[0], bl[1]);
            }
          }
        } else {
          if (col) tile_mma_tf32<true>(Gs, LDG, Xh, Xl, LDX, nr, kext, m0, n0, acc);
          else tile_mma_tf32<false>(Gs, LDG, Xh, Xl, LDX, nr, kext, m0, n0, acc);
        }
        const int g = lane >> 2, t = lane & 3;
        // mode-by-mode Khatri-Rao sketch: scale column j by the rounded product
        // of the other modes' rows of this plane
        float sc[2] = {1.0f, 1.0f};
        const DevSketch* krs = kr_of(a.ws, sk.kr);
        if (krs && krs->kr_mbm) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = min(m0 + g + 8 * h, lpad - 1);
            const float4 c = kr_scale_quad(a.ws, *krs, (uint64_t)wlo, (uint32_t)(j >> 2), a.prec);
            sc[h] = (j & 3) == 0 ? c.x : (j & 3) == 1 ? c.y : (j & 3) == 2 ? c.z : c.w;
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = m0 + g + ((e >> 1) << 3);
          const int oo = n0 + 2 * t + (e & 1);
          if (j < l && oo < nout) {
            const int64_t row = col ? (a0 + oo + a.n1 * wlo) : (whi + sk.hstride * (a.first + b0 + oo));
            atomicAdd(out + row + sk.rows * j, (double)(acc[e] * sc[e >> 1]));
          }
        }
      }
    }
  }
}


template <bool F16>
__global__ void __launch_bounds__(gThreads, 4) sketch_mma_kernel(const MixArgs a) {
  extern __shared__ float fsm[];
  const int64_t total = a.W * ((a.n1 + gTA - 1) / gTA) * ((a.cnt + gTB - 1) / gTB);
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) mma_tile<F16>(a, item, fsm);
}

// Batched form (same scheduling as the FP64 batched kernel): persistent CTAs
// take `chunk` consecutive tiles of the cost-ordered tile sequence at a time.
template <bool F16>
__global__ void __launch_bounds__(gThreads) sketch_mma_batched_kernel(const BatchLaunch b) {
  extern __shared__ float fsm[];
  __shared__ MixArgs sa;
  __shared__ int64_t s_base;
  __shared__ int s_pos;
  const DevTables& T = *reinterpret_cast<const DevTables*>(b.wsb + kTableOffB);
  const DevItem* items = reinterpret_cast<const DevItem*>(b.wsb + T.off_items);
  const DevSketch* sks = reinterpret_cast<const DevSketch*>(b.wsb + T.off_sketches);
  const int* order = reinterpret_cast<const int*>(b.wsb + T.off_border);
  const int64_t* prefix = reinterpret_cast<const int64_t*>(b.wsb + T.off_bprefix);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(b.wsb + T.off_bcounter);
  const int64_t total = prefix[T.nitems];
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) {
      s_base = (int64_t)atomicAdd(counter, (unsigned long long)b.chunk);
      int lo = 0, hi = T.nitems - 1;
      if (s_base < total) {
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (prefix[mid] <= s_base) lo = mid;
          else hi = mid - 1;
        }
      }
      s_pos = lo;
    }
    __syncthreads();
    const int64_t base = s_base;
    int pos = s_pos;
    if (base >= total) break;
    const int64_t end = imin64(base + b.chunk, total);
    for (int64_t t = base; t < end; ++t) {
      while (prefix[pos + 1] <= t) ++pos;
      const int it_idx = order[pos];
      if (it_idx != cur) {
        __syncthreads();
        if (threadIdx.x == 0) {
          const DevItem& it = items[it_idx];
          sa.X = reinterpret_cast<const float*>(b.X[it_idx]);
          sa.ws = reinterpret_cast<double*>(b.wsb);
          sa.n1 = it.n[0];
          sa.cnt = it.n[it.d - 1];
          sa.first = 0;
          sa.W = it.W;
          sa.Nd1 = it.N[it.d - 1];
          sa.seed = it.seed;
          sa.nsk = it.nsk;
          sa.prec = it.prec;
          sa.xscale = it.prec == TT_PREC_FP16 ? it.xscale : 1.0f;
          for (int s = 0; s < it.nsk; ++s) {
            const DevSketch& d = sks[it.sk0 + s];
            sa.sk[s] = SkArgM{d.rows, d.off, d.wdiv, d.hstride, -1, d.type, d.width, d.stream_id, -1};
          }
        }
        __syncthreads();
        cur = it_idx;
      }
      mma_tile<F16>(sa, t - prefix[pos], fsm);
    }
    __syncthreads();
  }
}

}  // namespace

// ----------------------------------------------------------------------------
// tcgen05 plane kernel: the fused multi-sketch for large planes (n_1 and the
// slab's last-mode extent both 128 or 256, d = 3 or 4), BF16 with X split into
// hi + lo, FP32 accumulators in tensor memory, FP64 flush.
//
// Per plane w the column sketches form ONE product D_L = X(:, w, :) [B_1 | B_2]
// (M = i_1, K = i_d, N = l * #column sketches) and the row sketches ONE product
// D_R = X(:, w, :)^T [C_1 | C_2] (M = i_d, K = i_1), where the B / C blocks are
// the test-matrix rows the plane needs (regenerated here).  The plane is
// processed in 128 x 128 quarters.  A quarter is stored once in shared memory,
// as BF16 hi and lo tiles in the no-swizzle core-matrix layout (8 x 8 blocks,
// i_1 contiguous inside a 16-byte row, i_d the row index); that single layout
// is the MN-major A operand of D_L and the K-major A operand of D_R, so every
// X element is written to shared memory once and read by the tensor core
// twice per part.  Core matrices are 144 bytes apart along i_1 (16 bytes of
// padding), which makes the producers' 16-byte stores conflict-free.
//
// Accumulator slots: w = kL + WL kR with WL = N_{d*}/n_1.  All column-sketch
// output rows depend on w only through kL, all row-sketch rows only through
// kR.  A tile is a block of T2 kL values x T3 kR values; tiles are numbered
// kL-block-major and every CTA takes one contiguous run of them, so its tiles
// share the kL block except at most once.  The D_L slots (one per kL) stay in
// tensor memory for the whole run of a kL block and are flushed when the block
// changes; the D_R slots (one per kR) are double-buffered and flushed after
// every tile while the next tile is being computed.  Flushes add FP32 tensor-
// memory values into the FP64 sketches with atomics.
//
// Warp roles (640 threads, one CTA per SM): warps 0-3 epilogue (TMEM lanes
// 0-127), warp 4 TMEM allocation + MMA issue (one thread), warps 5-12
// producers (X -> BF16 hi/lo), warps 13-19 test-matrix generation.  Stages
// are handed over with mbarriers; every wait is bounded (about 2 s), after
// which the CTA raises the timeout status bit, stops, drains its MMAs and
// frees its tensor memory.
namespace tc {

constexpr int kStages = 2;
constexpr int kBBlkB = 4 * kS4;          // one test-matrix block, N <= 32
constexpr int kBBlks = 4;                // L[h4=0,1], R[h1=0,1] per plane
constexpr int kBBufs = 2;
constexpr int kWarps = 20;  // 5 per scheduler: 96 registers per thread
constexpr int kThreads = kWarps * 32;
constexpr int kEpiWarps = 4, kMmaWarp = 4, kProdWarp0 = 5, kProdWarps = 8, kRngWarp0 = 13, kRngWarps = 7;
constexpr int kOffB = kStages * kStageB;
constexpr int kOffBar = kOffB + kBBufs * kBBlks * kBBlkB;
constexpr int kSmemBytes = kOffBar + 256 + 1024;  // barriers + alignment slack


struct TcArgs {
  const float* X;
  double* ws;
  int* status;
  int64_t n1, first, W, WL, WR, Nd1, tilesL, tilesR;
  uint64_t seed;
  int H1, H4, T2, T3, ell, nL, nR, NL, NR, tmem_cols;
  int64_t runL;  // tiles of one kL block accumulated in the L slots before a flush
  int genL[4], genR[4], ngenL, ngenR;  // sketches whose blocks the RNG warps generate
  uint32_t tab_tx;                     // bytes of staged blocks copied per plane
  float xscale;                        // FP16 operands: 2^s, X is split as X 2^s (1 with BF16)
  int f16;                             // FP16 operands (else BF16), for the table kernel
  SkTc col[4], row[4];
};

// Self-test of the give-up path: one thread waits, with the kernels' own
// bounded wait, on an mbarrier that nothing will ever arrive at.
__global__ void wait_timeout_kernel(long long limit, int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_for(smem_u32(&bar), 0, &abort_flag, status, limit);
}
// Iteration helper shared by all roles: plane (a, b) of tile t is valid when
// both keys are in range.
struct TileInfo {
  int64_t kL0, kR0;
  int nA, nB;
};
__device__ __forceinline__ TileInfo tile_info(const TcArgs& g, int64_t t) {
  TileInfo ti;
  const int64_t tl = t / g.tilesR, tr = t % g.tilesR;  // kL-block-major
  ti.kL0 = tl * g.T2;
  ti.kR0 = tr * g.T3;
  ti.nA = (int)imin64(g.T2, g.WL - ti.kL0);
  ti.nB = (int)imin64(g.T3, g.WR - ti.kR0);
  return ti;
}

// The L slots of one kL block are flushed after at most runL tiles.  The error
// of the tensor core's FP32 accumulation in tensor memory grows about linearly
// with the number of MMAs accumulated into one slot (measured on the 256^4
// Hilbert-type tensor: 8192 accumulating MMAs per slot gave 4.7e-5 relative
// reconstruction error, 64 gave 2.3e-6), so a chain is kept to a few hundred
// MMAs and the sum continues in FP64.
__device__ __forceinline__ int64_t l_group(const TcArgs& g, int64_t t) {
  const int64_t tl = t / g.tilesR, tr = t % g.tilesR;
  return tl * ((g.tilesR + g.runL - 1) / g.runL) + tr / g.runL;
}

// The test-matrix row of a plane w = kL + WL kR depends on w / wdiv (column
// sketches) or w % wdiv (row sketches), with wdiv one of 1, WL, W for d <= 4;
// these keys avoid a 64-bit division per generated row.
__device__ __forceinline__ int64_t col_key(const TcArgs& g, const SkTc& sk, int64_t w, int64_t kR) {
  if (sk.wdiv == 1) return w;
  if (sk.wdiv == g.WL) return kR;
  if (sk.wdiv == g.W) return 0;
  return w / sk.wdiv;
}
__device__ __forceinline__ int64_t row_key(const TcArgs& g, const SkTc& sk, int64_t w, int64_t kL) {
  if (sk.wdiv == 1) return 0;
  if (sk.wdiv == g.WL) return kL;
  if (sk.wdiv == g.W) return w;
  return w % sk.wdiv;
}

template <int ELL, bool F16>
__global__ void __launch_bounds__(kThreads, 1) sketch_tc_kernel(const TcArgs g) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kOffBar);
  // barrier indices
  const int FULL_A = 0, EMPTY_A = 2, FULL_B = 4, EMPTY_B = 6, TML_FULL = 8, TML_EMPTY = 9, DRAIN = 10,
            TMR_FULL = 11, TMR_EMPTY = 13, TAB_FULL = 15;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kOffBar + 192);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffBar + 200);
  // sketch descriptors in shared memory: every role indexes them by a runtime
  // sketch number
  __shared__ SkTc s_col[4], s_row[4];
  __shared__ int s_gen[8];  // generated sketches: column side 0..3, row side 4..7
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };

  if (threadIdx.x < 4) {
    s_col[threadIdx.x] = g.col[threadIdx.x];
    s_row[threadIdx.x] = g.row[threadIdx.x];
    s_gen[threadIdx.x] = g.genL[threadIdx.x];
    s_gen[4 + threadIdx.x] = g.genR[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(bar(FULL_A + s), kProdWarps);
      mbar_init(bar(EMPTY_A + s), 1);
      mbar_init(bar(FULL_B + s), kRngWarps);
      mbar_init(bar(TAB_FULL + s), 1);  // staged-block copies of a plane
      mbar_init(bar(EMPTY_B + s), 1);
    }
    mbar_init(bar(TML_FULL), 1);
    mbar_init(bar(TML_EMPTY), kEpiWarps);
    mbar_init(bar(DRAIN), 1);
    for (int s2 = 0; s2 < 2; ++s2) {
      mbar_init(bar(TMR_FULL + s2), 1);
      mbar_init(bar(TMR_EMPTY + s2), kEpiWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)g.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t ntiles_all = g.tilesL * g.tilesR;
  // this CTA's contiguous run of tiles [t_beg, ntiles)
  const int64_t t_beg = ntiles_all * blockIdx.x / gridDim.x;
  const int64_t ntiles = ntiles_all * (blockIdx.x + 1) / gridDim.x;
  const uint32_t sA = smem_u32(sm);
  const uint32_t sB = smem_u32(sm + kOffB);
  constexpr int ell = ELL;

  if (warp >= kProdWarp0 && warp < kProdWarp0 + kProdWarps) {
    // ------------------------------------------------------------ producers
    const int pt = threadIdx.x - kProdWarp0 * 32;   // 0..255
    const int cb1 = pt & 15, rsub = pt >> 4;         // i_1 core block, row group
    // The loads of the next quarter are issued before waiting for its stage,
    // so their latency overlaps the tensor-core work on the stage.
    const int nq = g.H1 * g.H4;
    // Cursor over (quarter, plane, tile) in the order every role uses; it runs
    // two quarters ahead of the quarter held in registers.
    int64_t t = t_beg;
    int a = 0, b = 0, q = 0;
    TileInfo ti = tile_info(g, t);
    auto advance = [&]() {
      if (++q == nq) {
        q = 0;
        if (++a == ti.nA) {
          a = 0;
          if (++b == ti.nB) {
            b = 0;
            t += 1;
            if (t < ntiles) ti = tile_info(g, t);
          }
        }
      }
    };
    // this thread's first element of the quarter at the cursor
    auto cursor_src = [&]() -> const float* {
      if (t >= ntiles) return nullptr;
      const int64_t w = (ti.kL0 + a) + g.WL * (ti.kR0 + b);
      const int h1 = q % g.H1, h4 = q / g.H1;
      return g.X + (h1 * 128 + cb1 * 8) + g.n1 * w + g.Nd1 * (int64_t)(h4 * 128 + rsub);
    };
    // L2 prefetch of a quarter: the four threads that share a 128-byte line
    // (cb1 & 3 = 0..3) take two of its eight rows each.
    auto prefetch = [&](const float* src) {
      const int c = cb1 & 3;
      const float* line = src - c * 8;
      prefetch_l2(line + g.Nd1 * (int64_t)(16 * (2 * c)));
      prefetch_l2(line + g.Nd1 * (int64_t)(16 * (2 * c + 1)));
    };
    float4 v[16];
    const float xs = g.xscale;
    auto sx = [&](float f) -> float {
      if constexpr (F16) return __fmul_rn(f, xs);
      else return f;
    };
    auto issue = [&](const float* src) {
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float4* p4 = reinterpret_cast<const float4*>(src + g.Nd1 * (int64_t)(16 * m));
        v[2 * m] = __ldcs(p4);
        v[2 * m + 1] = __ldcs(p4 + 1);
      }
    };
    // The loads of the next quarter are issued before waiting for its stage,
    // so their latency overlaps the tensor-core work on the stage; the one
    // after it is prefetched into L2, which puts more of X in flight than the
    // registers can hold.
    const float* src0 = cursor_src();
    bool have = src0 != nullptr;
    if (have) issue(src0);
    advance();
    const float* src1 = cursor_src();
    if (src1) prefetch(src1);
    advance();
    uint32_t qi = 0;
    while (have && !*abort_flag) {
      const int st = qi & 1;
      if (!mbar_wait(bar(EMPTY_A + st), ((qi >> 1) & 1) ^ 1, abort_flag, g.status)) break;
      const uint32_t tileA = sA + st * kStageB;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int i4 = rsub + 16 * m;
        const float x[8] = {sx(v[2 * m].x),     sx(v[2 * m].y),     sx(v[2 * m].z),     sx(v[2 * m].w),
                            sx(v[2 * m + 1].x), sx(v[2 * m + 1].y), sx(v[2 * m + 1].z), sx(v[2 * m + 1].w)};
        uint32_t hb[4], lb[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_hi_lo<F16>(x[2 * e], x[2 * e + 1], hb[e], lb[e]);
        const uint32_t off = cb1 * kS1 + (i4 >> 3) * kS4 + (i4 & 7) * 16;
        st_shared_v4(tileA + off, hb[0], hb[1], hb[2], hb[3]);
        st_shared_v4(tileA + kTileB + off, lb[0], lb[1], lb[2], lb[3]);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(FULL_A + st));
      ++qi;
      have = src1 != nullptr;
      if (have) issue(src1);
      src1 = cursor_src();
      if (src1) prefetch(src1);
      advance();
    }
  } else if (warp >= kRngWarp0 && warp < kRngWarp0 + kRngWarps) {
    // ------------------------------------------------- test-matrix blocks
    const int rt = threadIdx.x - kRngWarp0 * 32;  // 0..223
    constexpr int qps = ell / 4;                  // column quads per sketch
    // Work of one plane: 2-row units (two rows x four columns, two Philox
    // calls) of the generated 128-row blocks, column-side blocks first; each
    // thread takes a contiguous range of units, so no thread does more than
    // one unit above the average.
    constexpr int upb = 64 * qps;                 // units per block
    const int nbL = g.H4 * g.ngenL, nbR = g.H1 * g.ngenR;
    const int nunits = (nbL + nbR) * upb;
    const int u_beg = nunits * rt / (kRngWarps * 32), u_end = nunits * (rt + 1) / (kRngWarps * 32);
    // position of the first unit (the same on every plane)
    const int bi_beg = u_beg / upb, rp_beg = (u_beg % upb) / qps, nq_beg = u_beg % qps;
    // Per-plane state of the block a unit lies in: unit (rp, nq) covers rows
    // row0 + rstep * {2 rp, 2 rp + 1} of stream sid, columns n0 .. n0 + 3.
    struct Blk {
      int64_t row0, rstep;
      uint32_t dst0, sid;
      int n0;
      const DevSketch* kr;  // Khatri-Rao record, nullptr: dense stream
    };
    auto block_state = [&](int bi, int64_t w, int64_t kLp, int64_t kRp, int buf) {
      Blk bs;
      const bool colside = bi < nbL;
      const int bj = colside ? bi : bi - nbL;
      const int H = colside ? g.H4 : g.H1;
      const int blk = bj % H, gi = bj / H;
      const int sn = s_gen[(colside ? 0 : 4) + gi];
      const SkTc& sk = colside ? s_col[sn] : s_row[sn];
      // column side: row = key + hstride * i_d; row side: row = i_1 + n1 * key
      bs.row0 = colside ? col_key(g, sk, w, kRp) + sk.hstride * (g.first + blk * 128)
                        : blk * 128 + g.n1 * row_key(g, sk, w, kLp);
      bs.rstep = colside ? sk.hstride : 1;
      bs.sid = (uint32_t)sk.sid;
      bs.kr = kr_of(g.ws, sk.kr);
      bs.n0 = sn * ell;
      bs.dst0 = sB + (buf * kBBlks + (colside ? blk : 2 + blk)) * kBBlkB;
      return bs;
    };
    uint32_t pi = 0;
    int64_t tab_last[2] = {-1, -1};  // last plane whose staged copies used each buffer
    for (int64_t t = t_beg; t < ntiles && !*abort_flag; ++t) {
      const TileInfo ti = tile_info(g, t);
      for (int b = 0; b < ti.nB && !*abort_flag; ++b)
        for (int a = 0; a < ti.nA && !*abort_flag; ++a, ++pi) {
          const int64_t kLp = ti.kL0 + a, kRp = ti.kR0 + b;
          const int64_t w = kLp + g.WL * kRp;
          const int buf = pi & 1;
          if (!mbar_wait(bar(EMPTY_B + buf), ((pi >> 1) & 1) ^ 1, abort_flag, g.status)) break;
          // blocks: 0..H4-1 = column side (k = i_d), 2..2+H1-1 = row side (k = i_1)
          if (rt == 0 && g.tab_tx) {
            // blocks shared by many planes come from the staged tables
            mbar_arrive_expect_tx(bar(TAB_FULL + buf), g.tab_tx);
            tab_last[buf] = pi;
            const char* wsb = reinterpret_cast<const char*>(g.ws);
            constexpr uint32_t bytes = (uint32_t)(ell / 8) * kS4;
            for (int s = 0; s < g.nL; ++s) {
              const SkTc& sk = s_col[s];
              if (sk.tab < 0) continue;
              for (int h4 = 0; h4 < g.H4; ++h4)
                bulk_g2s(sB + (buf * kBBlks + h4) * kBBlkB + (s * ell / 8) * kS4,
                         wsb + sk.tab + (col_key(g, sk, w, kRp) * g.H4 + h4) * (int64_t)bytes, bytes,
                         bar(TAB_FULL + buf));
            }
            for (int s = 0; s < g.nR; ++s) {
              const SkTc& sk = s_row[s];
              if (sk.tab < 0) continue;
              for (int h1 = 0; h1 < g.H1; ++h1)
                bulk_g2s(sB + (buf * kBBlks + 2 + h1) * kBBlkB + (s * ell / 8) * kS4,
                         wsb + sk.tab + (row_key(g, sk, w, kLp) * g.H1 + h1) * (int64_t)bytes, bytes,
                         bar(TAB_FULL + buf));
            }
          }
          // this thread's units in order: two Philox chains per unit
          if (u_beg < u_end) {
            int bi = bi_beg, rp = rp_beg, nq = nq_beg;
            Blk bs = block_state(bi, w, kLp, kRp, buf);
            for (int u = u_beg; u < u_end; ++u) {
              const int k = 2 * rp;  // row of the block (i_d or i_1 offset)
              const int64_t row = bs.row0 + bs.rstep * k;
              const float4 ra = tm_quad_f32(g.ws, bs.kr, g.seed, bs.sid, (uint64_t)row, (uint32_t)nq);
              const float4 rb = tm_quad_f32(g.ws, bs.kr, g.seed, bs.sid, (uint64_t)(row + bs.rstep), (uint32_t)nq);
              const int n0 = bs.n0 + 4 * nq;  // a multiple of 4: one core matrix holds n0 .. n0 + 3
              const uint32_t dst = bs.dst0 + (k >> 3) * kS1 + (n0 >> 3) * kS4 + (n0 & 7) * 16 + (k & 7) * 2;
              st_shared_b32(dst, op16x2_bits<F16>(ra.x, rb.x));
              st_shared_b32(dst + 16, op16x2_bits<F16>(ra.y, rb.y));
              st_shared_b32(dst + 32, op16x2_bits<F16>(ra.z, rb.z));
              st_shared_b32(dst + 48, op16x2_bits<F16>(ra.w, rb.w));
              if (++nq == qps) {
                nq = 0;
                if (++rp == 64) {
                  rp = 0;
                  ++bi;
                  if (u + 1 < u_end) bs = block_state(bi, w, kLp, kRp, buf);
                }
              }
            }
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(FULL_B + buf));
        }
    }
    // Copies still in flight when the CTA gave up must land before it exits.
    if (rt == 0)
      for (int b2 = 0; b2 < 2; ++b2)
        if (tab_last[b2] >= 0) {
          const long long t0 = clock64();
          while (!mbar_try(bar(TAB_FULL + b2), (uint32_t)((tab_last[b2] >> 1) & 1)) &&
                 clock64() - t0 < kWaitCycles) {
          }
        }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    // Every lane runs the schedule and waits; the elected lane issues the
    // MMAs and commits (the same lane each time: the warp is converged).
    const uint32_t idL = make_idesc(g.NL, true, F16), idR = make_idesc(g.NR, false, F16);
    const uint32_t colR0 = (uint32_t)(g.T2 * g.H1 * g.NL);
    const uint32_t colRB = (uint32_t)(g.T3 * g.H4 * g.NR);  // one R buffer
    uint32_t qi = 0, pi = 0, lf = 0, ti = 0;
    int64_t cur_tl = -1;
    uint32_t initL = 0;
    bool ok = true;
    for (int64_t t = t_beg; t < ntiles && ok; ++t, ++ti) {
      const TileInfo tinf = tile_info(g, t);
      const int64_t tl = l_group(g, t);
      if (tl != cur_tl) {
        // a new L group: the previous group's L slots go to the epilogue
        if (cur_tl >= 0) {
          if (elect_one()) mma_commit(bar(TML_FULL));
          __syncwarp();
          ++lf;
        }
        ok = warp_wait(bar(TML_EMPTY), (lf & 1) ^ 1, abort_flag, g.status);
        if (!ok) break;
        tc_fence_after();
        initL = 0;
        cur_tl = tl;
      }
      const uint32_t rb = ti & 1;
      ok = warp_wait(bar(TMR_EMPTY + rb), ((ti >> 1) & 1) ^ 1, abort_flag, g.status);
      if (!ok) break;
      tc_fence_after();
      uint32_t initR = 0;
      for (int b = 0; b < tinf.nB && ok; ++b)
        for (int a = 0; a < tinf.nA && ok; ++a, ++pi) {
          const int buf = pi & 1;
          ok = warp_wait(bar(FULL_B + buf), (pi >> 1) & 1, abort_flag, g.status);
          if (ok && g.tab_tx) ok = warp_wait(bar(TAB_FULL + buf), (pi >> 1) & 1, abort_flag, g.status);
          if (!ok) break;
          tc_fence_after();
          for (int q = 0; q < g.H1 * g.H4; ++q, ++qi) {
            const int h1 = q % g.H1, h4 = q / g.H1;
            const int st = qi & 1;
            ok = warp_wait(bar(FULL_A + st), (qi >> 1) & 1, abort_flag, g.status);
            if (!ok) break;
            tc_fence_after();
            const uint32_t tileA = sA + st * kStageB;
            const uint32_t bL = sB + (buf * kBBlks + h4) * kBBlkB;
            const uint32_t bR = sB + (buf * kBBlks + 2 + h1) * kBBlkB;
            const int slotL = a * g.H1 + h1, slotR = b * g.H4 + h4;
            const uint32_t dL = tmem + (uint32_t)(slotL * g.NL);
            const uint32_t dR = tmem + colR0 + rb * colRB + (uint32_t)(slotR * g.NR);
            // descriptors of k-step 0; a k-step advances the start address
            // field (16-byte units) by a constant
            const uint64_t aL0 = make_desc(tileA, kS4, kS1), aR0 = make_desc(tileA, kS1, kS4);
            const uint64_t bL0 = make_desc(bL, kS1, kS4), bR0 = make_desc(bR, kS1, kS4);
            const uint32_t accL0 = (initL >> slotL) & 1u, accR0 = (initR >> slotR) & 1u;
            if (elect_one()) {
#pragma unroll
              for (int ks = 0; ks < 8; ++ks) {
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                  const uint64_t po = (uint64_t)((part * kTileB) >> 4);
                  mma16_ss(dL, aL0 + po + (uint64_t)((ks * 2 * kS4) >> 4), bL0 + (uint64_t)((ks * 2 * kS1) >> 4),
                              idL, accL0 | (uint32_t)(ks | part));
                  mma16_ss(dR, aR0 + po + (uint64_t)((ks * 2 * kS1) >> 4), bR0 + (uint64_t)((ks * 2 * kS1) >> 4),
                              idR, accR0 | (uint32_t)(ks | part));
                }
              }
              mma_commit(bar(EMPTY_A + st));
            }
            __syncwarp();
            initL |= 1u << slotL;
            initR |= 1u << slotR;
          }
          if (ok) {
            if (elect_one()) mma_commit(bar(EMPTY_B + buf));
            __syncwarp();
          }
        }
      if (ok) {
        if (elect_one()) mma_commit(bar(TMR_FULL + rb));
        __syncwarp();
      }
    }
    if (ok && cur_tl >= 0) {
      if (elect_one()) mma_commit(bar(TML_FULL));
      __syncwarp();
    }
    // drain the issued MMAs before the tensor memory is freed
    if (elect_one()) mma_commit(bar(DRAIN));
    __syncwarp();
    const long long t0 = clock64();
    while (!mbar_try(bar(DRAIN), 0) && clock64() - t0 < kWaitCycles) {
    }
    __syncwarp();
  } else if (warp < kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int lrow = warp * 32 + lane;  // TMEM lane = row within a 128 half
    const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
    const uint32_t colR0 = (uint32_t)(g.T2 * g.H1 * g.NL);
    const uint32_t colRB = (uint32_t)(g.T3 * g.H4 * g.NR);
    // L slots of kL block [kL0, kL0 + nA) -> column sketches.  A sketch whose
    // rows do not depend on the plane (wdiv = 1) is pre-summed in FP32 over
    // the few slots of one flush; the others go to their rows directly.
    auto flush_L = [&](int64_t kL0, int nA, uint32_t lf) -> bool {
      if (!mbar_wait(bar(TML_FULL), lf & 1, abort_flag, g.status)) return false;
      tc_fence_after();
      for (int h1 = 0; h1 < g.H1; ++h1) {
        const int64_t i1 = h1 * 128 + lrow;
        for (int s = 0; s < g.nL; ++s) {
          const SkTc& sk = s_col[s];
          const bool presum = sk.wdiv == 1;
          double* dst = g.ws + sk.off;
          float acc[ell];
#pragma unroll
          for (int j = 0; j < ell; ++j) acc[j] = 0.0f;
          for (int a = 0; a < nA; ++a) {
            float v[ell];
            tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)((a * g.H1 + h1) * g.NL + s * ell), v);
            if (presum) {
#pragma unroll
              for (int j = 0; j < ell; ++j) acc[j] += v[j];
            } else {
              const int64_t row = i1 + g.n1 * ((kL0 + a) % sk.wdiv);
#pragma unroll
              for (int j = 0; j < ell; ++j) atomicAdd(dst + row + sk.rows * j, (double)v[j]);
            }
          }
          if (presum) {
#pragma unroll
            for (int j = 0; j < ell; ++j) atomicAdd(dst + i1 + sk.rows * j, (double)acc[j]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(TML_EMPTY));
      return true;
    };
    uint32_t lf = 0, ti = 0;
    int64_t cur_tl = -1, cur_kL0 = 0;
    int cur_nA = 0;
    bool ok = true;
    for (int64_t t = t_beg; t < ntiles && ok && !*abort_flag; ++t, ++ti) {
      const TileInfo tinf = tile_info(g, t);
      const int64_t tl = l_group(g, t);
      if (tl != cur_tl) {
        if (cur_tl >= 0) {
          ok = flush_L(cur_kL0, cur_nA, lf);
          ++lf;
          if (!ok) break;
        }
        cur_tl = tl;
        cur_kL0 = tinf.kL0;
        cur_nA = tinf.nA;
      }
      // R slots of this tile (buffer ti & 1) -> row sketches; a sketch whose
      // rows do not depend on the plane (wdiv = W) is pre-summed over the tile
      const uint32_t rb = ti & 1;
      if (!mbar_wait(bar(TMR_FULL + rb), (ti >> 1) & 1, abort_flag, g.status)) break;
      tc_fence_after();
      for (int h4 = 0; h4 < g.H4; ++h4) {
        const int64_t bg = g.first + h4 * 128 + lrow;
        for (int s = 0; s < g.nR; ++s) {
          const SkTc& sk = s_row[s];
          const bool presum = sk.wdiv == g.W;
          double* dst = g.ws + sk.off;
          float acc[ell];
#pragma unroll
          for (int j = 0; j < ell; ++j) acc[j] = 0.0f;
          for (int b = 0; b < tinf.nB; ++b) {
            float v[ell];
            tmem_ld_cols<ell>(tmem + lane_addr + colR0 + rb * colRB + (uint32_t)((b * g.H4 + h4) * g.NR + s * ell), v);
            if (presum) {
#pragma unroll
              for (int j = 0; j < ell; ++j) acc[j] += v[j];
            } else {
              const int64_t whi = (tinf.kR0 + b) / (sk.wdiv / g.WL);
              const int64_t row = whi + sk.hstride * bg;
#pragma unroll
              for (int j = 0; j < ell; ++j) atomicAdd(dst + row + sk.rows * j, (double)v[j]);
            }
          }
          if (presum) {
#pragma unroll
            for (int j = 0; j < ell; ++j) atomicAdd(dst + bg * sk.hstride + sk.rows * j, (double)acc[j]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(TMR_EMPTY + rb));
    }
    if (ok && cur_tl >= 0 && !*abort_flag) flush_L(cur_kL0, cur_nA, lf);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)g.tmem_cols));
  }
}

// Staged test-matrix blocks of sketch (side, s): block (v, h), h < H, holds the
// 128 rows v + hstride (first + 128 h + k) (column side) or 128 h + k + n1 v
// (row side), k = 0..127, as the K-major core-matrix image the MMA reads (BF16
// or FP16: the same layout and rounding the RNG warps produce).
__global__ void tc_table_kernel(const TcArgs g, int colside, int s, int64_t nv, int H) {
  const SkTc sk = colside ? g.col[s] : g.row[s];
  const int qps = g.ell / 4;
  const int64_t blkB = (int64_t)(g.ell / 8) * kS4;
  const int64_t total = nv * H * 16 * qps * 8;
  char* tab = reinterpret_cast<char*>(g.ws) + sk.tab;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r8 = (int)(e & 7);
    int64_t rest = e >> 3;
    const int q = (int)(rest % qps);
    rest /= qps;
    const int kg = (int)(rest & 15);
    rest >>= 4;
    const int h = (int)(rest % H);
    const int64_t v = rest / H;
    const int64_t k = 128 * h + 8 * kg + r8;
    const uint64_t row = colside ? (uint64_t)(v + sk.hstride * (g.first + k)) : (uint64_t)(k + g.n1 * v);
    const float4 z = tm_quad_f32(g.ws, kr_of(g.ws, sk.kr), g.seed, (uint32_t)sk.sid, row, (uint32_t)q);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    char* blk = tab + (v * H + h) * blkB;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * q + u;
      *reinterpret_cast<uint16_t*>(blk + kg * kS1 + (j >> 3) * kS4 + (j & 7) * 16 + r8 * 2) =
          g.f16 ? op16_bits<true>(zz[u]) : op16_bits<false>(zz[u]);
    }
  }
}

// Shape rules of the plane kernel; fills the launch arguments when it applies.
bool plan_tc(const Plan& P, int item, int64_t count, TcArgs* out) {
  const DevItem& it = plan_items_host(&P)[item];
  if ((it.prec != TT_PREC_BF16 && it.prec != TT_PREC_FP16) || it.x_f64) return false;
  // Khatri-Rao plans go to the slab kernel (the mode-by-mode last row sketch
  // needs a per-plane scale that this kernel's accumulators cannot take)
  if (plan_sketches_host(&P)[it.sk0].kr_nm) return false;
  if (it.d != 3 && it.d != 4) return false;
  if (it.n[0] != 128 && it.n[0] != 256) return false;
  if (count != 128 && count != 256) return false;
  const DevSketch* sks = plan_sketches_host(&P);
  TcArgs g;
  memset(&g, 0, sizeof(g));
  const int ell = sks[it.sk0].width;
  int nL = 0, nR = 0;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& d = sks[it.sk0 + s];
    if (d.width != ell) return false;
    SkTc t{d.rows, d.off, d.wdiv, d.hstride, -1, d.stream_id, d.kr_nm ? it.sk0 + s : -1};
    if (d.type == SK_COL) {
      if (nL >= 4) return false;
      g.col[nL++] = t;
    } else {
      if (nR >= 4) return false;
      g.row[nR++] = t;
    }
  }
  if (ell != 8 && ell != 16) return false;  // the kernel is compiled for these widths
  const int NL = nL * ell, NR = nR * ell;
  if (NL < 16 || NR < 16 || NL > 32 || NR > 32 || NL % 16 || NR % 16) return false;
  g.n1 = it.n[0];
  g.W = it.W;
  g.WL = it.N[it.ds] / it.n[0];
  g.WR = g.W / g.WL;
  g.Nd1 = it.N[it.d - 1];
  g.H1 = (int)(it.n[0] / 128);
  g.H4 = (int)(count / 128);
  // tile: T2 x T3 planes, all slots resident in 512 TMEM columns
  // tile: T2 kL x T3 kR planes; TMEM holds the L slots and two R buffers
  int T2 = (int)std::min<int64_t>(g.WL, 4), T3 = (int)std::min<int64_t>(g.WR, 2);
  auto cols = [&](int a, int b) { return a * g.H1 * NL + 2 * b * g.H4 * NR; };
  while (cols(T2, T3) > 512 && (T2 > 1 || T3 > 1)) {
    if (T2 >= 2 * T3 && T2 > 1) --T2;
    else if (T3 > 1) --T3;
    else --T2;
  }
  while (T2 < g.WL && T2 < 16 && cols(T2 + 1, T3) <= 512) ++T2;
  while (T3 < g.WR && T3 < 16 && cols(T2, T3 + 1) <= 512) ++T3;
  if (cols(T2, T3) > 512) return false;
  g.T2 = T2;
  g.T3 = T3;
  int tc = 32;
  while (tc < cols(T2, T3)) tc <<= 1;
  g.tmem_cols = tc;
  g.tilesL = (g.WL + T2 - 1) / T2;
  g.tilesR = (g.WR + T3 - 1) / T3;
  // accumulating MMAs per L slot and tile: T3 planes x H4 quarters x 8 k-steps x (hi, lo)
  g.runL = std::max<int64_t>(1, (it.short_chains ? kMaxChainS : kMaxChainL) / (T3 * g.H4 * 16));
  g.ell = ell;
  g.nL = nL;
  g.nR = nR;
  // Test-matrix blocks whose rows do not depend on the plane (column sketches
  // with wdiv > 1: rows depend on w / wdiv only; row sketches with wdiv < W:
  // on w % wdiv only) are generated once per launch into the staging area and
  // copied per plane; the others are generated per plane.
  {
    const int64_t hd = (std::min<int64_t>(it.n[it.d - 1], 256) + 127) / 128;
    const int64_t blk = (int64_t)((ell + 7) / 8) * kS4;
    int64_t cur = it.off_tctab * 8;
    const bool staged = it.tctab_doubles > 0 && ell % 8 == 0;
    g.tab_tx = 0;
    for (int s = 0; s < nL; ++s) {
      if (staged && g.col[s].wdiv > 1) {
        g.col[s].tab = cur;
        cur += (g.W / g.col[s].wdiv) * hd * blk;
        g.tab_tx += (uint32_t)(g.H4 * blk);
      } else {
        g.genL[g.ngenL++] = s;
      }
    }
    for (int s = 0; s < nR; ++s) {
      if (staged && g.row[s].wdiv < g.W) {
        g.row[s].tab = cur;
        cur += g.row[s].wdiv * g.H1 * blk;
        g.tab_tx += (uint32_t)(g.H1 * blk);
      } else {
        g.genR[g.ngenR++] = s;
      }
    }
    if (cur > (it.off_tctab + it.tctab_doubles) * 8 && g.tab_tx) return false;
  }
  g.NL = NL;
  g.NR = NR;
  g.seed = it.seed;
  g.f16 = it.prec == TT_PREC_FP16 ? 1 : 0;
  g.xscale = g.f16 ? it.xscale : 1.0f;
  *out = g;
  return true;
}

}  // namespace tc

// ----------------------------------------------------------------------------
// Backward kernels that regenerate test matrices (same generator and rounding
// as the forward sketch of the item's precision).
namespace {

template <typename Real>
__device__ __forceinline__ void test_row(const void* wsb, const DevSketch* kr, int prec, uint64_t seed, int sid,
                                         uint64_t row, int l, Real* out) {
  for (int q = 0; q < (l + 3) / 4; ++q) {
    double z[4];
    if (prec == TT_PREC_FP64) {
      tm_quad_f64(wsb, kr, seed, (uint32_t)sid, row, (uint32_t)q, z);
    } else {
      const float4 f = tm_quad_mixed(wsb, kr, seed, (uint32_t)sid, row, (uint32_t)q, prec);
      z[0] = f.x;
      z[1] = f.y;
      z[2] = f.z;
      z[3] = f.w;
    }
    for (int t = 0; t < 4; ++t)
      if (4 * q + t < l) out[4 * q + t] = (Real)z[t];
  }
}

// Pbar_{d*}(v, c) += sum_j Omega_{d*}(v, j) Bbar(c, j)
__global__ void pbar_ls_kernel(char* wsb, int item, const int* ranks) {
  __shared__ double Bb[TT_MAXL * TT_MAXL];
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + 256);
  const DevItem& it = reinterpret_cast<const DevItem*>(wsb + T.off_items)[item];
  const DevSketch* sks = reinterpret_cast<const DevSketch*>(wsb + T.off_sketches);
  const DevSketch& sp = sks[it.basis_of_k[it.ds]];
  const DevSketch* kr_mid = sks[it.mid_sk].kr_nm ? &sks[it.mid_sk] : nullptr;
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + it.ds];
  const int rp = it.rpad[it.ds];
  const int l = it.lmid;
  for (int o = threadIdx.x; o < rp * l; o += blockDim.x) Bb[o] = ws[it.off_bbar + o];
  __syncthreads();
  double* Pb = ws + it.off_qbar[it.ds];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < sp.rows; v += (int64_t)gridDim.x * blockDim.x) {
    double om[TT_MAXL];
    test_row(wsb, kr_mid, it.prec, it.seed, it.ds, (uint64_t)v, l, om);
    for (int c = 0; c < r; ++c) {
      double acc = 0.0;
      for (int j = 0; j < l; ++j) acc += om[j] * Bb[c + rp * j];
      Pb[v + sp.rows * c] += acc;
    }
  }
}

// dX(a, w, b) = sum_col sum_j Sbar_k[a + n1 wlo, j] Omega_k[whi + hs b, j]
//             + sum_row sum_j Psi_k[a + n1 wlo, j] Rbar_k[whi + hs b, j]
// (one tile of 64 x 32 entries of one plane per iteration; written once).
// Real = double for the FP64 path; float for the TF32 / BF16 paths, whose
// test-matrix entries are exact in FP32 and whose forward sketch accumulates
// in FP32 (the adjoints S-bar / R-bar are rounded to FP32 on load).
template <typename Real>
__global__ void __launch_bounds__(256) sketch_adjoint_kernel(char* wsb, int item, void* dX) {
  constexpr int TA = 64, TB = 32, LD = TT_MAXL + 1;
  __shared__ Real Lf[TA * LD];
  __shared__ Real Rf[TB * LD];
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + 256);
  const DevItem& it = reinterpret_cast<const DevItem*>(wsb + T.off_items)[item];
  const DevSketch* S = reinterpret_cast<const DevSketch*>(wsb + T.off_sketches);
  const double* ws = reinterpret_cast<const double*>(wsb);
  const int64_t n1 = it.n[0], nd = it.n[it.d - 1], W = it.W, Nd1 = it.N[it.d - 1];
  const int64_t nA = (n1 + TA - 1) / TA, nB = (nd + TB - 1) / TB;
  const int64_t total = W * nA * nB;
  const int tid = threadIdx.x;
  const int ia = tid % TA, ib0 = tid / TA;  // rows ia, columns ib0 + 4 m
  for (int64_t job = blockIdx.x; job < total; job += gridDim.x) {
    const int64_t w = job / (nA * nB);
    const int64_t rem = job - w * nA * nB;
    const int64_t bb = rem / nA, ab = rem - bb * nA;
    const int64_t a0 = ab * TA, b0 = bb * TB;
    const int ta = (int)imin64(TA, n1 - a0), tb = (int)imin64(TB, nd - b0);
    Real acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int s = 0; s < it.nsk; ++s) {
      const DevSketch& sk = S[it.sk0 + s];
      const DevSketch* kr = sk.kr_nm ? &sk : nullptr;
      const int l = sk.width;
      const int64_t wlo = w % sk.wdiv, whi = w / sk.wdiv;
      const double* bar = ws + it.off_sbar[s];
      __syncthreads();
      if (sk.type == SK_COL) {
        for (int o = tid; o < ta * l; o += blockDim.x) {
          const int a = o % ta, j = o / ta;
          Lf[a * LD + j] = (Real)bar[(a0 + a + n1 * wlo) + sk.rows * j];
        }
        for (int b = tid; b < tb; b += blockDim.x)
          test_row(wsb, kr, it.prec, it.seed, sk.stream_id, (uint64_t)(whi + sk.hstride * (b0 + b)), l, Rf + b * LD);
      } else {
        for (int a = tid; a < ta; a += blockDim.x)
          test_row(wsb, kr, it.prec, it.seed, sk.stream_id, (uint64_t)((a0 + a) + n1 * wlo), l, Lf + a * LD);
        for (int o = tid; o < tb * l; o += blockDim.x) {
          const int b = o % tb, j = o / tb;
          Rf[b * LD + j] = (Real)bar[(whi + sk.hstride * (b0 + b)) + sk.rows * j];
        }
      }
      __syncthreads();
      if (ia < ta) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int b = ib0 + 4 * m;
          if (b < tb) {
            Real v = 0;
            for (int j = 0; j < l; ++j) v += Lf[ia * LD + j] * Rf[b * LD + j];
            acc[m] += v;
          }
        }
      }
    }
    if (ia < ta) {
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int b = ib0 + 4 * m;
        if (b < tb) {
          const int64_t idx = (a0 + ia) + n1 * w + Nd1 * (b0 + b);
          if (it.x_f64) ((double*)dX)[idx] = (double)acc[m];
          else ((float*)dX)[idx] = (float)acc[m];
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_pbar_ls(const Plan& P, int item, void* ws, const int* ranks, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  const int64_t M = plan_sketches_host(&P)[it.basis_of_k[it.ds]].rows;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((M + 127) / 128, 8LL * device_sm_count()));
  count_launch();
  pbar_ls_kernel<<<grid, 128, 0, st>>>((char*)ws, item, ranks);
  return cudaGetLastError();
}

cudaError_t launch_sketch_adjoint(const Plan& P, int item, void* dX, void* ws, cudaStream_t st) {
  // planes of at most 32 x 32 with dense TF32 / BF16 test matrices: the
  // tensor-core form (one warp a plane, rank-l products on mma.sync)
  if (adjoint_sp_eligible(P, item)) return launch_adjoint_sp(P, item, dX, ws, st);
  const DevItem& it = plan_items_host(&P)[item];
  const int64_t nA = (it.n[0] + 63) / 64, nB = (it.n[it.d - 1] + 31) / 32;
  const int64_t total = it.W * nA * nB;
  const int grid = (int)std::min<int64_t>(total, 8LL * device_sm_count());
  count_launch();
  if (it.prec == TT_PREC_FP64) sketch_adjoint_kernel<double><<<grid, 256, 0, st>>>((char*)ws, item, dX);
  else sketch_adjoint_kernel<float><<<grid, 256, 0, st>>>((char*)ws, item, dX);
  return cudaGetLastError();
}

bool mixed_tc_supported(const Plan& P, int item, int64_t) {
  const DevItem& it = plan_items_host(&P)[item];
  return it.prec == TT_PREC_TF32 || it.prec == TT_PREC_BF16 || it.prec == TT_PREC_FP16;
}

cudaError_t launch_sketch_mma(const Plan& P, int item, const void* X, int64_t first, int64_t count,
                              void* ws, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  const DevSketch* sks = plan_sketches_host(&P);
  MixArgs a;
  a.X = (const float*)X;
  a.ws = (double*)ws;
  a.n1 = it.n[0];
  a.cnt = count;
  a.first = first;
  a.W = it.W;
  a.Nd1 = it.N[it.d - 1];
  a.seed = it.seed;
  a.nsk = it.nsk;
  a.prec = it.prec;
  a.xscale = it.prec == TT_PREC_FP16 ? it.xscale : 1.0f;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& d = sks[it.sk0 + s];
    a.sk[s] = SkArgM{d.rows, d.off, d.wdiv, d.hstride, -1, d.type, d.width, d.stream_id, d.kr_nm ? it.sk0 + s : -1};
    if (d.gen_tab >= 0 && it.gentab_doubles > 0) {
      // stage the sketch's rows for this call: the slab's i_d (column side) or i_1 (row side)
      const int lpad = (d.width + 15) / 16 * 16;
      const bool col = d.type == SK_COL;
      a.sk[s].tab = it.off_gentab * 8 + d.gen_tab;
      cudaError_t e = launch_rows_table(d, it.sk0 + s, (const char*)ws, it.seed, first, a.n1,
                                        col ? (int)count : (int)a.n1, lpad,
                                        col ? it.W / d.wdiv : d.wdiv, (char*)ws + a.sk[s].tab,
                                        it.prec, st);
      if (e != cudaSuccess) return e;
    }
  }
  const size_t smem = sizeof(float) * (2 * (gTA + 1) * gTB + (size_t)gTA * (TT_MAXL + 4));
  static bool attr_set = false;
  if (!attr_set) {
    for (auto f : {sketch_mma_kernel<false>, sketch_mma_kernel<true>}) {
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    attr_set = true;
  }
  const int64_t nA = (a.n1 + gTA - 1) / gTA, nB = (count + gTB - 1) / gTB;
  const int64_t total = a.W * nA * nB;
  const int64_t grid = std::min<int64_t>(total, (int64_t)device_sm_count() * 8);
  count_launch();
  if (it.prec == TT_PREC_FP16) sketch_mma_kernel<true><<<(unsigned)grid, gThreads, smem, st>>>(a);
  else sketch_mma_kernel<false><<<(unsigned)grid, gThreads, smem, st>>>(a);
  return cudaGetLastError();
}

int64_t batched_tiles_mma(int64_t W, int64_t n1, int64_t cnt, int) {
  return W * ((n1 + gTA - 1) / gTA) * ((cnt + gTB - 1) / gTB);
}

cudaError_t launch_sketch_mma_batched(const BatchLaunch& b, const BatchCfg& cfg, bool f16, cudaStream_t st) {
  const size_t smem = sizeof(float) * (2 * (gTA + 1) * gTB + (size_t)gTA * (TT_MAXL + 4));
  static bool attr_set = false;
  if (!attr_set) {
    for (auto f : {sketch_mma_batched_kernel<false>, sketch_mma_batched_kernel<true>}) {
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    attr_set = true;
  }
  count_launch();
  if (f16) sketch_mma_batched_kernel<true><<<cfg.ctas_per_sm * device_sm_count(), gThreads, smem, st>>>(b);
  else sketch_mma_batched_kernel<false><<<cfg.ctas_per_sm * device_sm_count(), gThreads, smem, st>>>(b);
  return cudaGetLastError();
}

// The plane kernel needs one CTA of 640 threads with 217 KB of shared memory
// per SM; checked once against the compiled function and the device.
static bool tc_kernel_launchable() {
  static int ok = -1;
  if (ok < 0) {
    cudaFuncAttributes fa, fb;
    int dev = 0, smem_optin = 0;
    ok = cudaFuncGetAttributes(&fa, tc::sketch_tc_kernel<16, false>) == cudaSuccess &&
         cudaFuncGetAttributes(&fb, tc::sketch_tc_kernel<8, false>) == cudaSuccess &&
         cudaGetDevice(&dev) == cudaSuccess &&
         fb.maxThreadsPerBlock >= tc::kThreads &&
         cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
         fa.maxThreadsPerBlock >= tc::kThreads && smem_optin >= tc::kSmemBytes;
  }
  return ok == 1;
}

cudaError_t launch_sketch_tc(const Plan& P, int item, const void* X, int64_t first, int64_t count, void* ws,
                             cudaStream_t st) {
  tc::TcArgs g;
  if (!tc::plan_tc(P, item, count, &g)) return cudaErrorNotSupported;
  g.X = (const float*)X;
  g.ws = (double*)ws;
  g.status = reinterpret_cast<int*>((char*)ws + kStatusOff);
  g.first = first;
  using KernelFn = void (*)(tc::TcArgs);
  const KernelFn kernels[2][2] = {{tc::sketch_tc_kernel<8, false>, tc::sketch_tc_kernel<16, false>},
                                  {tc::sketch_tc_kernel<8, true>, tc::sketch_tc_kernel<16, true>}};
  static bool attr_set = false;
  if (!attr_set) {
    for (int f = 0; f < 2; ++f)
      for (int i = 0; i < 2; ++i) {
        const cudaError_t e =
            cudaFuncSetAttribute(kernels[f][i], cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
        if (e != cudaSuccess) return e;
      }
    attr_set = true;
  }
  if (!tc_kernel_launchable()) return launch_sketch_mma(P, item, X, first, count, ws, st);
  // the staging area is rewritten here in this kernel's layout: a later slab-
  // kernel launch of the same decomposition must stage its own blocks again
  plan_stream_tables(const_cast<Plan&>(P)) = false;
  for (int side = 0; side < 2; ++side)
    for (int s = 0; s < (side ? g.nR : g.nL); ++s) {
      const tc::SkTc& sk = side ? g.row[s] : g.col[s];
      if (sk.tab < 0) continue;
      const int64_t nv = side ? sk.wdiv : g.W / sk.wdiv;
      const int H = side ? g.H1 : g.H4;
      const int64_t total = nv * H * 16 * (g.ell / 4) * 8;
      const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8 * device_sm_count());
      count_launch();
      tc::tc_table_kernel<<<blocks, 256, 0, st>>>(g, side ? 0 : 1, s, nv, H);
    }
  const int64_t ntiles = g.tilesL * g.tilesR;
  const int grid = (int)std::min<int64_t>(ntiles, device_sm_count());
  count_launch();
  kernels[g.f16][g.ell == 16 ? 1 : 0]<<<grid, tc::kThreads, tc::kSmemBytes, st>>>(g);
  return cudaGetLastError();
}

}  // namespace tts

extern "C" tt_status tt_selftest_wait_timeout(int64_t limit_cycles, int* status_dev, tt_stream_t stream) {
  if (!status_dev || limit_cycles < 1 || limit_cycles > (int64_t)tts::tc::kWaitCycles) return TT_ERR_INVALID_ARG;
  tts::count_launch();
  tts::tc::wait_timeout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((long long)limit_cycles, status_dev);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

namespace tts {

// Which mixed kernel a launch uses: the tcgen05 plane kernel when its shape
// rules hold.
bool use_tc_kernel(const Plan& P, int item, int64_t count) {
  // the plane kernel is built for the two-sided split (at most two sketches
  // per side); one-sided plans go to the other kernels
  if (plan_items_host(&P)[item].sided1) return false;
  tc::TcArgs g;
  return tc::plan_tc(P, item, count, &g);
}

cudaError_t launch_sketch_mixed(const Plan& P, int item, const void* X, int64_t first, int64_t count,
                                void* ws, cudaStream_t st) {
  if (use_tc_kernel(P, item, count)) return launch_sketch_tc(P, item, X, first, count, ws, st);
  if (use_slab_kernel(P, item, count)) {
    const cudaError_t e = launch_sketch_slab(P, item, X, first, count, ws, st);
    if (e != cudaErrorNotSupported) return e;
  }
  if (use_sp_kernel(P, item, count)) return launch_sketch_sp(P, item, X, first, count, ws, st);
  return launch_sketch_mma(P, item, X, first, count, ws, st);
}

}  // namespace tts
