// Mixed-precision (TF32 / BF16 tensor-core) sketch path and everything that
// must regenerate its test matrices bit-identically (the middle-core matrix
// B = P^T Omega_{d*} of the one-pass solve, and the test-matrix export).
// All of them live in this translation unit and call the one out-of-line FP32
// generator below.
#include <algorithm>

#include "internal.cuh"
#include "philox.cuh"

namespace tts {

__device__ __noinline__ void normals4_f32(uint64_t seed, uint32_t sid, uint64_t row, uint32_t q,
                                          float z[4]) {
  uint32_t c0 = (uint32_t)row, c1 = (uint32_t)(row >> 32), c2 = q, c3 = sid;
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u0 = __fmul_rn((float)((c0 >> 9) * 2u + 1u), 0x1p-24f);
  const float u1 = __fmul_rn((float)((c1 >> 9) * 2u + 1u), 0x1p-24f);
  const float u2 = __fmul_rn((float)((c2 >> 9) * 2u + 1u), 0x1p-24f);
  const float u3 = __fmul_rn((float)((c3 >> 9) * 2u + 1u), 0x1p-24f);
  const float ra = __fsqrt_rn(__fmul_rn(-2.0f, logf(u0)));
  const float rb = __fsqrt_rn(__fmul_rn(-2.0f, logf(u2)));
  float sa, ca, sb, cb;
  sincospif(__fmul_rn(2.0f, u1), &sa, &ca);
  sincospif(__fmul_rn(2.0f, u3), &sb, &cb);
  z[0] = __fmul_rn(ra, ca);
  z[1] = __fmul_rn(ra, sa);
  z[2] = __fmul_rn(rb, cb);
  z[3] = __fmul_rn(rb, sb);
}

namespace {

__global__ void test_matrix_mixed_kernel(uint64_t seed, int sid, int64_t row0, int64_t nrows, int ncols,
                                         int prec, double* out) {
  const int nq = (ncols + 3) / 4;
  const int64_t total = nrows * nq;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % nrows;
    const int q = (int)(e / nrows);
    float z[4];
    normals4_f32(seed, (uint32_t)sid, (uint64_t)(row0 + r), (uint32_t)q, z);
    for (int t = 0; t < 4; ++t)
      if (4 * q + t < ncols) out[r + nrows * (4 * q + t)] = (double)round_prec(z[t], prec);
  }
}

constexpr int64_t kTableOffB = 256;

// B = P_{d*}^T Omega^_{d*}, Omega^ = the rounded FP32 entries the sketch used.
__global__ void __launch_bounds__(256) mid_b_kernel_mixed(char* wsb, int item, const int* ranks) {
  constexpr int CH = 32;
  __shared__ double Ps[CH * TT_MAXL];
  __shared__ double Gs[CH * (TT_MAXL + 1)];
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
  const DevItem& it = reinterpret_cast<const DevItem*>(wsb + T.off_items)[item];
  const DevSketch sp = reinterpret_cast<const DevSketch*>(wsb + T.off_sketches)[it.basis_of_k[it.ds]];
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + it.ds];
  const int l = it.lmid;
  const int64_t M = sp.rows;
  const double* Pm = ws + sp.lev_z[0];
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
      float z[4];
      normals4_f32(it.seed, (uint32_t)it.ds, (uint64_t)(v0 + v), (uint32_t)q, z);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < l) Gs[v + CH * (4 * q + t)] = (double)round_prec(z[t], it.prec);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < r * l; o += blockDim.x) {
      const int c = o % r, j = o / r;
      double acc = 0.0;
      for (int v = 0; v < nv; ++v) acc += Ps[v + CH * c] * Gs[v + CH * j];
      atomicAdd(ws + it.off_B + c + (int64_t)it.rpad[it.ds] * j, acc);
    }
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

cudaError_t launch_mid_b_mixed(const Plan& P, int item, void* ws, const int* ranks, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  const int64_t M = plan_sketches_host(&P)[it.basis_of_k[it.ds]].rows;
  const int grid = (int)std::min<int64_t>((M + 31) / 32, 4LL * device_sm_count());
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
  int type, width, sid, pad_;
};

struct MixArgs {
  const float* X;
  double* ws;
  int64_t n1, cnt, first, W, Nd1;
  uint64_t seed;
  int nsk, prec;
  SkArgM sk[kMaxSk];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
  // two bf16-exact floats -> bf16x2 (first argument in the low half)
  return (__float_as_uint(lo_k) >> 16) | (__float_as_uint(hi_k) & 0xFFFF0000u);
}

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

// One (m-tile, n-tile) of D^T = G^T X' for the current tile and sketch.
// Gs: rows x LDG (row = contraction index k, col = j).  Xh/Xl: LDX layout with
// X'[k][o] = col sketch: X[o + LDX k] ... see callers (getx).
template <bool COL>
__device__ __forceinline__ void tile_mma(int prec, const float* Gs, int LDG, const float* Xh, const float* Xl,
                                         int LDX, int kreal, int kext, int m0, int n0, float acc[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // element accessors: A[j][k] = G[k][j];  B[k][o] = X(o, k) (COL) or X(k, o) (ROW)
  auto Aj = [&](int j, int k) -> float { return (k < kreal) ? Gs[k * LDG + j] : 0.0f; };
  auto Bx = [&](const float* Xs, int k, int o) -> float {
    if (k >= kreal) return 0.0f;
    return COL ? Xs[o + LDX * k] : Xs[k + LDX * o];
  };
  if (prec == TT_PREC_BF16) {
    for (int k0 = 0; k0 < kext; k0 += 16) {
      uint32_t a[4];
      a[0] = pack_bf16(Aj(m0 + g, k0 + 2 * t), Aj(m0 + g, k0 + 2 * t + 1));
      a[1] = pack_bf16(Aj(m0 + g + 8, k0 + 2 * t), Aj(m0 + g + 8, k0 + 2 * t + 1));
      a[2] = pack_bf16(Aj(m0 + g, k0 + 2 * t + 8), Aj(m0 + g, k0 + 2 * t + 9));
      a[3] = pack_bf16(Aj(m0 + g + 8, k0 + 2 * t + 8), Aj(m0 + g + 8, k0 + 2 * t + 9));
      const int o = n0 + g;
      const uint32_t bh0 = pack_bf16(Bx(Xh, k0 + 2 * t, o), Bx(Xh, k0 + 2 * t + 1, o));
      const uint32_t bh1 = pack_bf16(Bx(Xh, k0 + 2 * t + 8, o), Bx(Xh, k0 + 2 * t + 9, o));
      const uint32_t bl0 = pack_bf16(Bx(Xl, k0 + 2 * t, o), Bx(Xl, k0 + 2 * t + 1, o));
      const uint32_t bl1 = pack_bf16(Bx(Xl, k0 + 2 * t + 8, o), Bx(Xl, k0 + 2 * t + 9, o));
      mma_bf16(acc, a, bh0, bh1);
      mma_bf16(acc, a, bl0, bl1);
    }
  } else {
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
}

__global__ void __launch_bounds__(gThreads) sketch_mma_kernel(const MixArgs a) {
  extern __shared__ float fsm[];
  constexpr int LDX = gTA + 1;
  float* Xh = fsm;                  // LDX x gTB  (X[a + LDX b])
  float* Xl = Xh + LDX * gTB;
  float* Gs = Xl + LDX * gTB;       // rows (<= gTA) x LDG
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nA = (a.n1 + gTA - 1) / gTA;
  const int64_t nB = (a.cnt + gTB - 1) / gTB;
  const int64_t total = a.W * nA * nB;
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
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
      const float hi = round_prec(v, a.prec);
      const float lo = round_prec(__fsub_rn(v, hi), a.prec);
      Xh[ia + LDX * ib] = hi;
      Xl[ia + LDX * ib] = lo;
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
      __syncthreads();
      for (int o = tid; o < nr * nq; o += gThreads) {
        const int r = o % nr, q = o / nr;
        const uint64_t grow = col ? (uint64_t)(whi + sk.hstride * (a.first + b0 + r))
                                  : (uint64_t)((a0 + r) + a.n1 * wlo);
        float z[4];
        normals4_f32(a.seed, (uint32_t)sk.sid, grow, (uint32_t)q, z);
#pragma unroll
        for (int u = 0; u < 4; ++u) Gs[r * LDG + 4 * q + u] = (4 * q + u < l) ? round_prec(z[u], a.prec) : 0.0f;
      }
      __syncthreads();
      const int mt = lpad / 16, nt = (nout + 7) / 8;
      double* out = a.ws + sk.off;
      const int kext = (a.prec == TT_PREC_BF16) ? ((nr + 15) & ~15) : ((nr + 7) & ~7);
      for (int job = warp; job < mt * nt; job += gThreads / 32) {
        const int m0 = (job % mt) * 16, n0 = (job / mt) * 8;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if (col) tile_mma<true>(a.prec, Gs, LDG, Xh, Xl, LDX, nr, kext, m0, n0, acc);
        else tile_mma<false>(a.prec, Gs, LDG, Xh, Xl, LDX, nr, kext, m0, n0, acc);
        const int g = lane >> 2, t = lane & 3;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = m0 + g + ((e >> 1) << 3);
          const int oo = n0 + 2 * t + (e & 1);
          if (j < l && oo < nout) {
            const int64_t row = col ? (a0 + oo + a.n1 * wlo) : (whi + sk.hstride * (a.first + b0 + oo));
            atomicAdd(out + row + sk.rows * j, (double)acc[e]);
          }
        }
      }
    }
  }
}

}  // namespace

bool mixed_tc_supported(const Plan& P, int item, int64_t) {
  const DevItem& it = plan_items_host(&P)[item];
  return it.prec == TT_PREC_TF32 || it.prec == TT_PREC_BF16;
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
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& d = sks[it.sk0 + s];
    a.sk[s] = SkArgM{d.rows, d.off, d.wdiv, d.hstride, d.type, d.width, d.stream_id, 0};
  }
  const size_t smem = sizeof(float) * (2 * (gTA + 1) * gTB + (size_t)gTA * (TT_MAXL + 4));
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(sketch_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t nA = (a.n1 + gTA - 1) / gTA, nB = (count + gTB - 1) / gTB;
  const int64_t total = a.W * nA * nB;
  const int64_t grid = std::min<int64_t>(total, (int64_t)device_sm_count() * 8);
  count_launch();
  sketch_mma_kernel<<<(unsigned)grid, gThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sketch_mixed(const Plan& P, int item, const void* X, int64_t first, int64_t count,
                                void* ws, cudaStream_t st) {
  return launch_sketch_mma(P, item, X, first, count, ws, st);
}

}  // namespace tts
