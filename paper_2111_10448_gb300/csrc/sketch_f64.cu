// FP64 fused multi-sketch (the correctness path of the sketch step, Sec. 3.2
// and Algorithm 5: one read of each tile of X feeds every sketch).
//
// X is seen as planes X(:, w, :) (n_1 x n_d, see internal.cuh).  A work item is
// one tile (a-block x b-block) of one plane; it is staged in shared memory
// once, then every sketch adds its contribution:
//   column sketch: S_k[a + n_1 wlo, j] += sum_b X(a, w, b) Omega_k[whi + hs b, j]
//   row sketch:    R_k[whi + hs b, j]  += sum_a X(a, w, b) Psi_k[a + n_1 wlo, j]
// with the test-matrix tile regenerated from Philox into shared memory.  The
// per-tile partial sums are added to the FP64 sketches with atomics.  On
// GB300 FP64 arithmetic is the bound of this kernel (not HBM).
#include <algorithm>

#include "internal.cuh"
#include "philox.cuh"

namespace tts {
const DevSketch* plan_sketches_host(const Plan* p);
namespace {

constexpr int kTA = 64;   // rows (i_1) per tile
constexpr int kTB = 32;   // columns (i_d) per tile
constexpr int kThreads = 256;

struct SkArg {
  int64_t rows, off, wdiv, hstride;
  int type, width, sid, pad_;
};

struct F64Args {
  const void* X;
  double* ws;
  int64_t n1, cnt, first, W, Nd1;
  uint64_t seed;
  int x_f64, nsk;
  SkArg sk[kMaxSk];
};

__device__ __forceinline__ double load_x(const void* X, int x_f64, int64_t i) {
  return x_f64 ? __ldg((const double*)X + i) : (double)__ldg((const float*)X + i);
}

__global__ void __launch_bounds__(kThreads) sketch_f64_kernel(const F64Args a) {
  extern __shared__ double smem[];
  constexpr int LDX = kTA + 1;
  double* Xs = smem;                         // LDX x kTB
  double* Gs = smem + LDX * kTB;             // max(kTA, kTB) rows x LDG
  const int tid = threadIdx.x;
  const int64_t nA = (a.n1 + kTA - 1) / kTA;
  const int64_t nB = (a.cnt + kTB - 1) / kTB;
  const int64_t total = a.W * nA * nB;
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int64_t w = item / (nA * nB);
    const int64_t rem = item - w * nA * nB;
    const int64_t bb = rem / nA, ab = rem - bb * nA;
    const int64_t a0 = ab * kTA, b0 = bb * kTB;
    const int ta = (int)imin64(kTA, a.n1 - a0);
    const int tb = (int)imin64(kTB, a.cnt - b0);
    __syncthreads();
    for (int o = tid; o < kTA * kTB; o += kThreads) {
      const int ia = o % kTA, ib = o / kTA;
      double v = 0.0;
      if (ia < ta && ib < tb) v = load_x(a.X, a.x_f64, (a0 + ia) + a.n1 * w + a.Nd1 * (b0 + ib));
      Xs[ia + LDX * ib] = v;
    }
    for (int s = 0; s < a.nsk; ++s) {
      const SkArg sk = a.sk[s];
      const int l = sk.width;
      const int LDG = l + 1;
      const int64_t wlo = w % sk.wdiv, whi = w / sk.wdiv;
      const int nr = sk.type == SK_COL ? tb : ta;
      const int nq = (l + 3) / 4;
      __syncthreads();
      for (int o = tid; o < nr * nq; o += kThreads) {
        const int r = o % nr, q = o / nr;
        const uint64_t grow = sk.type == SK_COL
                                  ? (uint64_t)(whi + sk.hstride * (a.first + b0 + r))
                                  : (uint64_t)((a0 + r) + a.n1 * wlo);
        double z[4];
        normals4_f64(a.seed, (uint32_t)sk.sid, grow, (uint32_t)q, z);
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (4 * q + t < l) Gs[r * LDG + 4 * q + t] = z[t];
      }
      __syncthreads();
      double* out = a.ws + sk.off;
      if (sk.type == SK_COL) {
        for (int o = tid; o < kTA * l; o += kThreads) {
          const int ia = o % kTA, j = o / kTA;
          if (ia >= ta) continue;
          double acc = 0.0;
          for (int ib = 0; ib < tb; ++ib) acc = fma(Xs[ia + LDX * ib], Gs[ib * LDG + j], acc);
          atomicAdd(out + (a0 + ia + a.n1 * wlo) + sk.rows * j, acc);
        }
      } else {
        for (int o = tid; o < kTB * l; o += kThreads) {
          const int ib = o % kTB, j = o / kTB;
          if (ib >= tb) continue;
          double acc = 0.0;
          for (int ia = 0; ia < ta; ++ia) acc = fma(Xs[ia + LDX * ib], Gs[ia * LDG + j], acc);
          atomicAdd(out + (whi + sk.hstride * (a.first + b0 + ib)) + sk.rows * j, acc);
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_sketch_f64(const Plan& P, int item, const void* X, int64_t first, int64_t count,
                              void* ws, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  F64Args a;
  a.X = X;
  a.ws = (double*)ws;
  a.n1 = it.n[0];
  a.cnt = count;
  a.first = first;
  a.W = it.W;
  a.Nd1 = it.N[it.d - 1];
  a.seed = it.seed;
  a.x_f64 = it.x_f64;
  a.nsk = it.nsk;
  const DevSketch* sks = plan_sketches_host(&P);
  int lmax = 1;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& d = sks[it.sk0 + s];
    a.sk[s] = SkArg{d.rows, d.off, d.wdiv, d.hstride, d.type, d.width, d.stream_id, 0};
    lmax = d.width > lmax ? d.width : lmax;
  }
  const size_t smem = sizeof(double) * ((kTA + 1) * kTB + (size_t)kTA * (lmax + 1));
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(sketch_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         96 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t nA = (a.n1 + kTA - 1) / kTA, nB = (count + kTB - 1) / kTB;
  const int64_t total = a.W * nA * nB;
  const int64_t grid = std::min<int64_t>(total, (int64_t)device_sm_count() * 8);
  count_launch();
  sketch_f64_kernel<<<(unsigned)grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace tts
