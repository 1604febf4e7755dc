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
#include "testmat.cuh"

namespace tts {
const DevSketch* plan_sketches_host(const Plan* p);
namespace {

constexpr int64_t kTableOffB = 256;
constexpr int kTA = 64;   // rows (i_1) per tile of the single-tensor launch
constexpr int kTB = 32;   // columns (i_d) per tile
constexpr int kThreads = 256;

struct SkArg {
  int64_t rows, off, wdiv, hstride;
  int type, width, sid;
  int kr;  // global sketch index when the test matrix is Khatri-Rao, -1: dense
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

template <int TA, int TB>
__host__ __device__ constexpr int64_t f64_tiles(int64_t W, int64_t n1, int64_t cnt) {
  return W * ((n1 + TA - 1) / TA) * ((cnt + TB - 1) / TB);
}

// One tile (TA rows of i_1 x TB columns of i_d of plane w) into every sketch.
template <int TA, int TB>
__device__ void f64_tile(const F64Args& a, int64_t item, double* smem) {
  constexpr int LDX = TA + 1;
  double* Xs = smem;                         // LDX x TB
  double* Gs = smem + LDX * TB;              // max(TA, TB) rows x LDG
  const int tid = threadIdx.x;
  const int64_t nA = (a.n1 + TA - 1) / TA;
  const int64_t nB = (a.cnt + TB - 1) / TB;
  const int64_t w = item / (nA * nB);
  const int64_t rem = item - w * nA * nB;
  const int64_t bb = rem / nA, ab = rem - bb * nA;
  const int64_t a0 = ab * TA, b0 = bb * TB;
  const int ta = (int)imin64(TA, a.n1 - a0);
  const int tb = (int)imin64(TB, a.cnt - b0);
  __syncthreads();
  for (int o = tid; o < TA * TB; o += kThreads) {
    const int ia = o % TA, ib = o / TA;
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
      tm_quad_f64(a.ws, kr_of(a.ws, sk.kr), a.seed, (uint32_t)sk.sid, grow, (uint32_t)q, z);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < l) Gs[r * LDG + 4 * q + t] = z[t];
    }
    __syncthreads();
    double* out = a.ws + sk.off;
    if (sk.type == SK_COL) {
      for (int o = tid; o < TA * l; o += kThreads) {
        const int ia = o % TA, j = o / TA;
        if (ia >= ta) continue;
        double acc = 0.0;
        for (int ib = 0; ib < tb; ++ib) acc = fma(Xs[ia + LDX * ib], Gs[ib * LDG + j], acc);
        atomicAdd(out + (a0 + ia + a.n1 * wlo) + sk.rows * j, acc);
      }
    } else {
      for (int o = tid; o < TB * l; o += kThreads) {
        const int ib = o % TB, j = o / TB;
        if (ib >= tb) continue;
        double acc = 0.0;
        for (int ia = 0; ia < ta; ++ia) acc = fma(Xs[ia + LDX * ib], Gs[ia * LDG + j], acc);
        atomicAdd(out + (whi + sk.hstride * (a.first + b0 + ib)) + sk.rows * j, acc);
      }
    }
  }
}

template <int TA, int TB>
__host__ __device__ constexpr size_t f64_smem(int lmax) {
  return sizeof(double) * ((size_t)(TA + 1) * TB + (size_t)(TA > TB ? TA : TB) * (lmax + 1));
}

__global__ void __launch_bounds__(kThreads) sketch_f64_kernel(const F64Args a) {
  extern __shared__ double smem[];
  const int64_t total = f64_tiles<kTA, kTB>(a.W, a.n1, a.cnt);
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) f64_tile<kTA, kTB>(a, item, smem);
}

// Batched form: one persistent launch over the tiles of every tensor of the
// plan.  The tensors are visited in the plan's cost order (largest first) and
// their tiles numbered consecutively (prefix[] = first tile of each); a CTA
// takes `chunk` consecutive tiles at a time from a global counter.
template <int TA, int TB>
__global__ void __launch_bounds__(kThreads) sketch_f64_batched_kernel(const BatchLaunch b) {
  extern __shared__ double smem[];
  __shared__ F64Args sa;
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
      // position of the tensor holding tile s_base (last prefix <= s_base)
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
          sa.X = b.X[it_idx];
          sa.ws = reinterpret_cast<double*>(b.wsb);
          sa.n1 = it.n[0];
          sa.cnt = it.n[it.d - 1];
          sa.first = 0;
          sa.W = it.W;
          sa.Nd1 = it.N[it.d - 1];
          sa.seed = it.seed;
          sa.x_f64 = it.x_f64;
          sa.nsk = it.nsk;
          for (int s = 0; s < it.nsk; ++s) {
            const DevSketch& d = sks[it.sk0 + s];
            sa.sk[s] = SkArg{d.rows, d.off, d.wdiv, d.hstride, d.type, d.width, d.stream_id, -1};
          }
        }
        __syncthreads();
        cur = it_idx;
      }
      f64_tile<TA, TB>(sa, t - prefix[pos], smem);
    }
    __syncthreads();
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
    a.sk[s] = SkArg{d.rows, d.off, d.wdiv, d.hstride, d.type, d.width, d.stream_id, d.kr_nm ? it.sk0 + s : -1};
    lmax = d.width > lmax ? d.width : lmax;
  }
  const size_t smem = f64_smem<kTA, kTB>(lmax);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(sketch_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         96 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t total = f64_tiles<kTA, kTB>(a.W, a.n1, count);
  const int64_t grid = std::min<int64_t>(total, (int64_t)device_sm_count() * 8);
  count_launch();
  sketch_f64_kernel<<<(unsigned)grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

int64_t batched_tiles_f64(int64_t W, int64_t n1, int64_t cnt, int ta) {
  return ta == 32 ? f64_tiles<32, kTB>(W, n1, cnt) : f64_tiles<64, kTB>(W, n1, cnt);
}

cudaError_t launch_sketch_f64_batched(const BatchLaunch& b, const BatchCfg& cfg, int lmax, cudaStream_t st) {
  const size_t smem = cfg.ta == 32 ? f64_smem<32, kTB>(lmax) : f64_smem<64, kTB>(lmax);
  auto kern = cfg.ta == 32 ? sketch_f64_batched_kernel<32, kTB> : sketch_f64_batched_kernel<64, kTB>;
  static bool attr_set[2] = {false, false};
  if (!attr_set[cfg.ta == 32]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    if (e != cudaSuccess) return e;
    attr_set[cfg.ta == 32] = true;
  }
  count_launch();
  kern<<<cfg.ctas_per_sm * device_sm_count(), kThreads, smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace tts
