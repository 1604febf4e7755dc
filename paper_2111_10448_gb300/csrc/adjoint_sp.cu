// Tensor-core sketch adjoint of the backward (the last step of the adjoint of
// the one-pass map, the differentiation form): for planes of at most 32 x 32
// entries (n_1, n_d <= 32), TF32 / BF16 plans with dense Gaussian test
// matrices.
//
// X enters the one-pass map only through the sketches (Sec. 3.2), so
//   dX(a, w, b) = sum_{column sketches} sum_j Sbar_k[a + n_1 wlo, j] Omega_k[whi + hs b, j]
//               + sum_{row sketches}    sum_j Psi_k[a + n_1 wlo, j] Rbar_k[whi + hs b, j],
// i.e. per plane w a sum of rank-l products L_s R_s^T with L_s the n_1 x l
// rows on the i_1 side (Sbar or Psi) and R_s the n_d x l rows on the i_d side
// (Omega or Rbar).  One warp takes one plane and accumulates all of them with
// mma.sync (FP32 accumulation): the test-matrix entries are exact in the MMA
// type (they are rounded to it by definition), and each sketch adjoint, which
// is FP64, is rounded to FP32 and split into three terms of the MMA type by a
// pass before the kernel (three products; the terms hold the FP32 value, so
// the error is that of FP32 rounding and accumulation, 2^-24 relative to the
// sum of the magnitudes: the gradient of the map can cancel across sketches,
// which a two-term BF16 split, 2^-17, did not survive).
//
// Test-matrix rows: the rows that many planes share come from the small-plane
// kernel's staging tables, restaged here for the whole last mode; the rows of
// Omega_1 and Psi_{d-1} (and of any sketch without a table) are unique to the
// plane and are generated into the warp's shared-memory buffer.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "philox.cuh"

namespace tts {

const DevSketch* plan_sketches_host(const Plan* p);
cudaError_t launch_rows_table(const DevSketch& d, int gsk, const char* wsb, uint64_t seed, int64_t first, int64_t n1,
                              int nr, int lpad, int64_t nkeys, char* tab, int prec, cudaStream_t st);

namespace adj {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kLDG = 40;  // element row stride of the per-warp generated rows (32 rows)
constexpr int64_t kTableOffB = 256;

struct AdjSk {
  int64_t rows, wdiv, hstride;
  int64_t adj;   // byte offset of the split adjoint (kAdjParts row blocks), row-major rows x lpad
  int64_t tab;   // byte offset of the staged test-matrix rows (-1: generated per plane)
  int col, sid, ell, pad_;
};

struct AdjArgs {
  char* wsb;
  float* dX;
  uint64_t seed;
  int64_t n1, nd, W, Nd1, WL;
  int nsk;
  AdjSk sk[kMaxSk];
};

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
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

// Split the FP64 sketch adjoints into kAdjParts terms of the MMA type
// (t_0 = rn(v), t_1 = rn(v - t_0), t_2 = rn(v - t_0 - t_1), each difference
// exact in FP32): row-major rows x lpad per term, zero past the sketch's
// width.
template <bool TF>
__global__ void split_kernel(char* wsb, int item, int lpad) {
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
  const DevItem& it = reinterpret_cast<const DevItem*>(wsb + T.off_items)[item];
  const DevSketch* S = reinterpret_cast<const DevSketch*>(wsb + T.off_sketches);
  const double* ws = reinterpret_cast<const double*>(wsb);
  using E = typename std::conditional<TF, float, __nv_bfloat16>::type;
  int64_t base = it.off_adjtab * 8;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& sk = S[it.sk0 + s];
    const double* bar = ws + it.off_sbar[s];
    E* t = reinterpret_cast<E*>(wsb + base);
    const int64_t total = sk.rows * lpad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t r = e / lpad;
      const int j = (int)(e - r * lpad);
      float v = j < sk.width ? (float)bar[r + sk.rows * j] : 0.0f;
#pragma unroll
      for (int part = 0; part < kAdjParts; ++part) {
        if constexpr (TF) {
          const float h = round_tf32(v);
          t[part * total + e] = h;
          v = __fsub_rn(v, h);
        } else {
          const __nv_bfloat16 h = __float2bfloat16_rn(v);
          t[part * total + e] = h;
          v = __fsub_rn(v, __bfloat162float(h));
        }
      }
    }
    base += total * (int64_t)sizeof(E) * kAdjParts;
  }
}

// One warp, one plane: D (n_1 x n_d, two m-tiles x four n-tiles of 16 x 8)
// = sum over sketches of L R^T.  Fragments are 32-bit loads of two adjacent
// elements of a row-major rows x lpad source (the split adjoint, a staged
// table or the warp's generated rows).
template <int LPAD, bool TF>
__global__ void __launch_bounds__(kThreads, 2) adjoint_kernel(const AdjArgs ga) {
  using E = typename std::conditional<TF, float, __nv_bfloat16>::type;
  constexpr int KS = TF ? 8 : 16;  // k per MMA
  __shared__ AdjArgs g;
  __shared__ __align__(16) E gen[kWarps][32 * kLDG];
  if (threadIdx.x == 0) g = ga;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const int n1 = (int)g.n1, nd = (int)g.nd;
  E* mine = gen[warp];
  for (int64_t w = (int64_t)blockIdx.x * kWarps + warp; w < g.W; w += (int64_t)gridDim.x * kWarps) {
    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
    for (int si = 0; si < g.nsk; ++si) {
      const AdjSk& s = g.sk[si];
      const int64_t wlo = w % s.wdiv, whi = w / s.wdiv;
      // the test-matrix side: rows of the i_d side (column sketch: Omega rows
      // whi + hs b) or of the i_1 side (row sketch: Psi rows a + n1 wlo)
      const int nr = s.col ? nd : n1;
      const E* test;
      int ldt;
      if (s.tab >= 0) {
        const int64_t key = s.col ? whi : wlo;
        test = reinterpret_cast<const E*>(g.wsb + s.tab) + key * nr * LPAD;
        ldt = LPAD;
      } else {
        __syncwarp();
        const int nq = LPAD / 4;
        for (int c = lane; c < nr * nq; c += 32) {
          const int r = c / nq, q = c - r * nq;
          const uint64_t row = s.col ? (uint64_t)(whi + s.hstride * r) : (uint64_t)(r + g.n1 * wlo);
          float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
          if (4 * q < s.ell) z = normals4_f32(g.seed, (uint32_t)s.sid, row, (uint32_t)q);
          const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float v = 4 * q + u < s.ell ? zz[u] : 0.0f;
            if constexpr (TF) mine[r * kLDG + 4 * q + u] = round_tf32(v);
            else mine[r * kLDG + 4 * q + u] = __float2bfloat16_rn(v);
          }
        }
        __syncwarp();
        test = mine;
        ldt = kLDG;
      }
      // the adjoint side: Sbar rows a + n1 wlo (column sketch) or Rbar rows
      // whi + hs b (row sketch), one row block per term of the split
      const E* adj = reinterpret_cast<const E*>(g.wsb + s.adj);
      const int64_t pstride = s.rows * LPAD;
      const int64_t arow0 = s.col ? g.n1 * wlo : whi;
      const int64_t astep = s.col ? 1 : s.hstride;
      // L rows (i_1 side, m = a) and R rows (i_d side, n = b)
      auto lrow = [&](int part, int a) -> const E* {
        if (!s.col) return test + (int64_t)a * ldt;
        return adj + part * pstride + (arow0 + a) * LPAD;
      };
      auto rrow = [&](int part, int b) -> const E* {
        if (s.col) return test + (int64_t)b * ldt;
        return adj + part * pstride + (arow0 + astep * b) * LPAD;
      };
      // fragments: A (m = a) from L rows, B (n = b) from R rows; the test side
      // is loaded once per k-step, the adjoint side once per term
      for (int k0 = 0; k0 < LPAD; k0 += KS) {
        uint32_t af[2][4], bf[4][2];
        auto fill_a = [&](int part) {
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            const int a0 = mt * 16 + gq, a1 = a0 + 8;
            if constexpr (TF) {
              const float* r0 = reinterpret_cast<const float*>(lrow(part, a0 < n1 ? a0 : 0));
              const float* r1 = reinterpret_cast<const float*>(lrow(part, a1 < n1 ? a1 : 0));
              af[mt][0] = a0 < n1 ? __float_as_uint(r0[k0 + tq]) : 0u;
              af[mt][1] = a1 < n1 ? __float_as_uint(r1[k0 + tq]) : 0u;
              af[mt][2] = a0 < n1 ? __float_as_uint(r0[k0 + tq + 4]) : 0u;
              af[mt][3] = a1 < n1 ? __float_as_uint(r1[k0 + tq + 4]) : 0u;
            } else {
              const uint32_t* r0 = reinterpret_cast<const uint32_t*>(lrow(part, a0 < n1 ? a0 : 0) + k0);
              const uint32_t* r1 = reinterpret_cast<const uint32_t*>(lrow(part, a1 < n1 ? a1 : 0) + k0);
              af[mt][0] = a0 < n1 ? r0[tq] : 0u;
              af[mt][1] = a1 < n1 ? r1[tq] : 0u;
              af[mt][2] = a0 < n1 ? r0[tq + 4] : 0u;
              af[mt][3] = a1 < n1 ? r1[tq + 4] : 0u;
            }
          }
        };
        auto fill_b = [&](int part) {
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const int b = nt * 8 + gq;
            if constexpr (TF) {
              const float* rb = reinterpret_cast<const float*>(rrow(part, b < nd ? b : 0));
              bf[nt][0] = b < nd ? __float_as_uint(rb[k0 + tq]) : 0u;
              bf[nt][1] = b < nd ? __float_as_uint(rb[k0 + tq + 4]) : 0u;
            } else {
              const uint32_t* rb = reinterpret_cast<const uint32_t*>(rrow(part, b < nd ? b : 0) + k0);
              bf[nt][0] = b < nd ? rb[tq] : 0u;
              bf[nt][1] = b < nd ? rb[tq + 4] : 0u;
            }
          }
        };
        // the test side: R rows (column sketch) or L rows (row sketch), part 0
        if (s.col) fill_b(0);
        else fill_a(0);
#pragma unroll
        for (int part = 0; part < kAdjParts; ++part) {
          if (s.col) fill_a(part);
          else fill_b(part);
#pragma unroll
          for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              if constexpr (TF) mma_tf32(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
              else mma_bf16(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
            }
        }
      }
    }
    // dX(a, w, b): lanes of a quad hold b = 2 tq, 2 tq + 1 of rows a = gq, gq + 8
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int a = mt * 16 + gq + 8 * (e >> 1), b = nt * 8 + 2 * tq + (e & 1);
          if (a < n1 && b < nd) g.dX[a + g.n1 * w + g.Nd1 * b] = acc[mt][nt][e];
        }
  }
}

}  // namespace adj

bool adjoint_sp_eligible(const Plan& P, int item) {
  const DevItem& it = plan_items_host(&P)[item];
  if (it.adjtab_doubles <= 0 || it.x_f64) return false;
  if (it.prec != TT_PREC_BF16 && it.prec != TT_PREC_TF32) return false;
  if (it.n[0] > 32 || it.n[it.d - 1] > 32) return false;
  const DevSketch* sks = plan_sketches_host(&P);
  for (int s = 0; s < it.nsk; ++s)
    if (sks[it.sk0 + s].width > 32 || sks[it.sk0 + s].kr_nm) return false;
  return true;
}

cudaError_t launch_adjoint_sp(const Plan& P, int item, void* dX, void* ws, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  const DevSketch* sks = plan_sketches_host(&P);
  const bool tf = it.prec == TT_PREC_TF32;
  int lmax = 0;
  for (int s = 0; s < it.nsk; ++s) lmax = std::max(lmax, sks[it.sk0 + s].width);
  const int lpad = lmax <= 16 ? 16 : 32;
  const int64_t esz = tf ? 4 : 2;
  adj::AdjArgs g;
  memset(&g, 0, sizeof(g));
  g.wsb = (char*)ws;
  g.dX = (float*)dX;
  g.seed = it.seed;
  g.n1 = it.n[0];
  g.nd = it.n[it.d - 1];
  g.W = it.W;
  g.Nd1 = it.N[it.d - 1];
  g.nsk = it.nsk;
  int64_t base = it.off_adjtab * 8;
  cudaError_t e;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& d = sks[it.sk0 + s];
    adj::AdjSk& k = g.sk[s];
    k.rows = d.rows;
    k.wdiv = d.wdiv;
    k.hstride = d.hstride;
    k.adj = base;
    base += d.rows * lpad * esz * kAdjParts;
    k.col = d.type == SK_COL ? 1 : 0;
    k.sid = d.stream_id;
    k.ell = d.width;
    k.tab = -1;
    if (d.sp_tab >= 0) {
      // restage the shared rows for the whole last mode (the forward may
      // have streamed slabs, whose tables held the last slab's rows)
      k.tab = it.off_sptab * 8 + d.sp_tab;
      const int nr = k.col ? (int)g.nd : (int)g.n1;
      const int64_t nkeys = k.col ? it.W / d.wdiv : d.wdiv;
      e = launch_rows_table(d, it.sk0 + s, (const char*)ws, it.seed, 0, g.n1, nr, lpad, nkeys, (char*)ws + k.tab,
                            it.prec, st);
      if (e != cudaSuccess) return e;
    }
  }
  {
    int64_t rows = 0;
    for (int s = 0; s < it.nsk; ++s) rows += sks[it.sk0 + s].rows;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((rows * lpad + 255) / 256, 8LL * device_sm_count()));
    count_launch();
    if (tf) adj::split_kernel<true><<<blocks, 256, 0, st>>>((char*)ws, item, lpad);
    else adj::split_kernel<false><<<blocks, 256, 0, st>>>((char*)ws, item, lpad);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((it.W + adj::kWarps - 1) / adj::kWarps,
                                                                4LL * device_sm_count()));
  count_launch();
  if (tf) {
    if (lpad == 16) adj::adjoint_kernel<16, true><<<(unsigned)grid, adj::kThreads, 0, st>>>(g);
    else adj::adjoint_kernel<32, true><<<(unsigned)grid, adj::kThreads, 0, st>>>(g);
  } else {
    if (lpad == 16) adj::adjoint_kernel<16, false><<<(unsigned)grid, adj::kThreads, 0, st>>>(g);
    else adj::adjoint_kernel<32, false><<<(unsigned)grid, adj::kThreads, 0, st>>>(g);
  }
  return cudaGetLastError();
}

}  // namespace tts
