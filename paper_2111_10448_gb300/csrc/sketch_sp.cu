// Small-plane fused multi-sketch (BF16, FP16 or TF32 tensor cores, X split
// into hi + lo; the description below uses BF16)
// for tensors whose first and last modes are small (n_1, n_d <= 32), e.g. the
// d = 6, n = 24 random-TT workload and the many small tensors of a batch.
//
// Every plane X(:, w, :) (n_1 x n_d, w = kL + WL kR with WL = N_{d*}/n_1)
// contributes a plain product to every sketch of the one-pass sketch
// (Sec. 3.2): column sketch k, S_k[a + n_1 (w mod N_k/n_1), j] +=
// sum_b X(a, w, b) Omega_k[w div (N_k/n_1) + hs b, j], and row sketch k,
// R_k[w div (N_k/n_1) + hs b, j] += sum_a X(a, w, b) Psi_k[a + n_1 (w mod
// N_k/n_1), j].  Column-sketch rows depend on w only through kL and row-sketch
// rows only through kR (N_k/n_1 divides WL for k <= d*, and WL divides it
// for k >= d*).
//
// Why a separate kernel: with n = 24 and l = 26 a plane holds 576 entries but
// each sketch needs 24 test-matrix rows of 26 normals.  Only the outermost
// sketches (Omega_1: rows w + W b; Psi_{d-1}: rows a + n_1 w) have rows no
// other plane uses; every other test matrix row is shared by many planes, so
// those rows are generated once per call into a BF16 table (L2-resident for
// the workloads here) and copied per plane.  That leaves about 2 l / n normals
// per entry, the least any dense Gaussian sketch of these unfoldings needs.
//
// Organisation: one CTA of 16 warps per SM takes a contiguous run of blocks of
// T2 x T3 = 16 planes (kL-major; 4 x 4, or 8 x 2 / 16 x 1 when there are only
// two / one kR values), one plane per warp; a warp converts its plane
// to BF16 hi / lo in shared memory ([b][a], a contiguous), then for each
// sketch builds the test-matrix block [k][j] and runs mma.sync m16n8k16 with
// ldmatrix fragments (A = block^T, B = the plane or its transpose), adding
// the FP32 results into shared accumulators with shared-memory atomics.
// Accumulator slots: a column sketch has one slot per kL of the block (one if
// its rows do not depend on w), a row sketch one per kR (one if its rows do not
// depend on w).  Row slots are added into the FP64 sketches after every
// block; column slots (and plane-independent row slots) when the kL block
// changes or after kColFlushBlocks blocks, which bounds the FP32 chains.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "philox.cuh"
#include "testmat.cuh"

namespace tts {

const DevItem* plan_items_host(const Plan* p);
const DevSketch* plan_sketches_host(const Plan* p);
int plan_num_items(const Plan* p);

namespace sp {

constexpr int kBlockPlanes = 16;  // planes per block: T2 values of kL x T3 values of kR
constexpr int kLD = 40;           // element row stride of the 32-row tiles
constexpr int kTileElems = 32 * kLD;
constexpr int kColFlushBlocks = 16;
// Operand formats of a kernel instance (template argument FMT).
constexpr int kFmtBF16 = 0, kFmtTF32 = 1, kFmtFP16 = 2;
__host__ __device__ constexpr int fmt_of(int prec) {
  return prec == TT_PREC_TF32 ? kFmtTF32 : prec == TT_PREC_FP16 ? kFmtFP16 : kFmtBF16;
}
// Per precision: BF16 / FP16 tiles (80-byte rows) leave room for 16 warps, one
// plane each per block; TF32 tiles hold FP32 words (160-byte rows), 8 warps,
// two planes each per block.
template <int FMT>
struct Prec {
  static constexpr bool TF = FMT == kFmtTF32;
  static constexpr int kWarps = TF ? 8 : 16;
  static constexpr int kThreads = kWarps * 32;
  static constexpr int kEsz = TF ? 4 : 2;
  static constexpr int kWarpBytes = 3 * kTileElems * kEsz;  // plane hi, plane lo, test-matrix block
};
constexpr int kMaxSmem = 227 * 1024 - 2048;
constexpr int64_t kTableOffB = 256;  // dynamic shared memory; the static part is below 2 KB

struct SpSk {
  int64_t rows, off, wdiv, hstride, tab;  // tab: byte offset of the staged rows, -1: generated per plane
  int col, sid, nslot, slot0, lflush;     // lflush: flushed on the column-side schedule
  int dep;                                // output rows depend on the plane (through kL or kR)
  int ell;                                // this sketch's width (<= the padded width of the launch)
  int kr;                                 // global sketch index of a Khatri-Rao test matrix, -1: dense
};

struct SpArgs {
  const float* X;
  char* wsb;
  uint64_t seed;
  int64_t n1, cnt, first, W, WL, WR, Nd1, tilesL, tilesR, tab0;
  int nsk, ell, nq, nslots, ldo;  // ell: the largest sketch width (sets the padding), nq its column quads
  int T2, T3;  // block shape
  float xscale;  // FP16: 2^s, X is split as X 2^s (1 otherwise)
  SpSk sk[kMaxSk];
};

// Block shape of an item: 16 planes, as many kR values as there are, at
// most t3max (1, 2, 4 or 8; the batched autotuner chooses it, single calls
// use 4).
__host__ __device__ inline void sp_block_shape(int64_t WL, int64_t WR, int t3max, int* T2, int* T3) {
  const int t3 = WR >= t3max ? t3max : (int)WR;
  int t2 = kBlockPlanes / t3;
  if (t2 > WL) t2 = (int)WL;
  *T2 = t2;
  *T3 = t3;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t a, uint32_t r[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t a, uint32_t r[2]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t a, uint32_t r[2]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma_f16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma_tf32(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t f16x2(float lo, float hi) {
  __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t op16x2(bool f16, float lo, float hi) {
  return f16 ? f16x2(lo, hi) : bf16x2(lo, hi);
}

// Staged test-matrix rows of one sketch: entry (key, r, j), r < nr, j < lpad,
// at element (key nr + r) lpad + j of `tab`: the normal of row key + hstride
// (first + r) (column side) or r + n1 key (row side) rounded to the operand
// type of precision `prec`: BF16 or FP16 (2-byte elements) or TF32 (4-byte
// FP32 words), zero for j >= l.  Threads tid0, tid0 + nthr, ... of the caller
// take the entries.
__device__ void sp_table_fill(const char* wsb, const SpSk& s, uint64_t seed, int64_t first, int64_t n1, int nr,
                              int ell, int lpad, int64_t nkeys, char* tab, int64_t tid0, int64_t nthr, int prec) {
  const bool tf = prec == TT_PREC_TF32, f16 = prec == TT_PREC_FP16;
  const DevSketch* kr = kr_of(wsb, s.kr);
  const int qpr = lpad / 4;
  const int64_t total = nkeys * nr * qpr;
  for (int64_t e = tid0; e < total; e += nthr) {
    const int q = (int)(e % qpr);
    const int64_t rest = e / qpr;
    const int r = (int)(rest % nr);
    const int64_t key = rest / nr;
    const uint64_t row = s.col ? (uint64_t)(key + s.hstride * (first + r)) : (uint64_t)(r + n1 * key);
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (4 * q < ell) z = tm_quad_f32(wsb, kr, seed, (uint32_t)s.sid, row, (uint32_t)q);
    const int64_t el = (key * nr + r) * lpad + 4 * q;
    if (tf) {
      *reinterpret_cast<float4*>(tab + el * 4) =
          make_float4(4 * q < ell ? round_tf32(z.x) : 0.f, 4 * q + 1 < ell ? round_tf32(z.y) : 0.f,
                      4 * q + 2 < ell ? round_tf32(z.z) : 0.f, 4 * q + 3 < ell ? round_tf32(z.w) : 0.f);
    } else {
      const uint32_t lo = op16x2(f16, 4 * q < ell ? z.x : 0.f, 4 * q + 1 < ell ? z.y : 0.f);
      const uint32_t hi = op16x2(f16, 4 * q + 2 < ell ? z.z : 0.f, 4 * q + 3 < ell ? z.w : 0.f);
      *reinterpret_cast<uint2*>(tab + el * 2) = make_uint2(lo, hi);
    }
  }
}

__global__ void sp_table_kernel(const char* wsb, SpSk s, uint64_t seed, int64_t first, int64_t n1, int nr, int ell,
                                int lpad, int64_t nkeys, char* tab, int prec) {
  sp_table_fill(wsb, s, seed, first, n1, nr, ell, lpad, nkeys, tab,
                (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, prec);
}

// Launch arguments of one item (the whole last mode when count = n_d), shared
// by the host launch and the batched kernel.
__host__ __device__ inline void sp_fill(const DevItem& it, const DevSketch* sks, int64_t count, SpArgs& g,
                                        int t3max = 4) {
  g.n1 = it.n[0];
  g.cnt = count;
  g.W = it.W;
  g.WL = it.N[it.ds] / it.n[0];
  g.WR = g.W / g.WL;
  g.Nd1 = it.N[it.d - 1];
  sp_block_shape(g.WL, g.WR, t3max, &g.T2, &g.T3);
  g.tilesL = (g.WL + g.T2 - 1) / g.T2;
  g.tilesR = (g.WR + g.T3 - 1) / g.T3;
  g.tab0 = it.off_sptab * 8;
  g.seed = it.seed;
  g.xscale = it.prec == TT_PREC_FP16 ? it.xscale : 1.0f;
  g.nsk = it.nsk;
  g.ell = 0;
  for (int s = 0; s < it.nsk; ++s) g.ell = sks[it.sk0 + s].width > g.ell ? sks[it.sk0 + s].width : g.ell;
  g.nq = (g.ell + 3) / 4;
  const int64_t mx = g.n1 > count ? g.n1 : count;
  g.ldo = (int)((mx + 7) / 8 * 8);
  int slots = 0;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& d = sks[it.sk0 + s];
    SpSk k;
    k.rows = d.rows;
    k.off = d.off;
    k.wdiv = d.wdiv;
    k.hstride = d.hstride;
    k.tab = d.sp_tab;
    k.col = d.type == SK_COL ? 1 : 0;
    k.sid = d.stream_id;
    k.ell = d.width;
    k.kr = d.kr_nm ? it.sk0 + s : -1;
    const bool per_plane_rows = k.col ? d.wdiv > 1 : d.wdiv < it.W;
    k.dep = per_plane_rows ? 1 : 0;
    k.nslot = per_plane_rows ? (k.col ? g.T2 : g.T3) : 1;
    k.slot0 = slots;
    // row slots of plane-dependent rows go out after every block (kR changes);
    // everything else is kept while the kL block stays
    k.lflush = (k.col || !k.dep) ? 1 : 0;
    slots += k.nslot;
    g.sk[s] = k;
  }
  g.nslots = slots;
}

// Adds the slots of one flush class into the FP64 sketches and clears them:
// warps take the (slot, j) rows, lanes the outputs o.
template <int LPAD, int FMT>
__device__ void sp_flush(const SpArgs& g, const SpSk* s_sk, float* acc, bool long_class, int64_t bL, int64_t bR) {
  constexpr int kWarps = Prec<FMT>::kWarps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n1 = (int)g.n1, cnt = (int)g.cnt;
  const int slot_elems = LPAD * g.ldo;
  double* ws = reinterpret_cast<double*>(g.wsb);
  {
    for (int si = 0; si < g.nsk; ++si) {
      const SpSk& s = s_sk[si];
      if ((s.lflush != 0) != long_class) continue;
      const int nout = s.col ? n1 : cnt;
      const int nrow = s.nslot * s.ell;
      for (int rr = warp; rr < nrow; rr += kWarps) {
        const int sl = rr / s.ell, j = rr - sl * s.ell;
        float* p = acc + (size_t)(s.slot0 + sl) * slot_elems + j * g.ldo;
        // kL < WL and kR < WR: 32-bit arithmetic (plan_sp requires W < 2^31)
        int64_t base;
        if (s.col) {
          const uint32_t kL = (uint32_t)(bL * g.T2 + sl);
          base = g.n1 * (int64_t)(s.dep ? kL % (uint32_t)s.wdiv : 0u);
        } else {
          const uint32_t kR = (uint32_t)(bR * g.T3 + sl);
          base = (int64_t)(s.dep ? kR / (uint32_t)(s.wdiv / g.WL) : 0u) + s.hstride * g.first;
        }
        for (int o = lane; o < nout; o += 32) {
          const float v = p[o];
          if (v == 0.0f) continue;
          p[o] = 0.0f;
          const int64_t row = s.col ? base + o : base + s.hstride * o;
          atomicAdd(ws + s.off + row + s.rows * j, (double)v);
        }
      }
    }
  }
}

// The planes of block (bL, bR), one per warp; no block-wide barrier inside.
// KR: the launch has Khatri-Rao test matrices (the dense instance leaves
// their code out, which keeps it within its registers).
template <int LPAD, int FMT, bool KR>
__device__ void sp_block(const SpArgs& g, const SpSk* s_sk, unsigned char* smraw, float* acc, int64_t bL, int64_t bR) {
  constexpr bool TF = FMT == kFmtTF32, F16 = FMT == kFmtFP16;
  using E = typename std::conditional<TF, float, uint16_t>::type;
  constexpr int kWarps = Prec<FMT>::kWarps, kEsz = Prec<FMT>::kEsz;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  E* Xh = reinterpret_cast<E*>(smraw + warp * Prec<FMT>::kWarpBytes);
  E* Xl = Xh + kTileElems;
  E* Gs = Xl + kTileElems;
  const int slot_elems = LPAD * g.ldo;
  const int n1 = (int)g.n1, cnt = (int)g.cnt;
  const int64_t kL0 = bL * g.T2, kR0 = bR * g.T3;
  const int nA = (int)imin64(g.T2, g.WL - kL0), nB = (int)imin64(g.T3, g.WR - kR0);
    for (int p = warp; p < nA * nB; p += kWarps) {
      const int sa = p % nA, sb = p / nA;
      const int64_t w = (kL0 + sa) + g.WL * (kR0 + sb);
      // ---- the plane, split into hi + lo in the MMA type, [b][a]
      {
        const float* xp = g.X + g.n1 * w + lane;
        float v[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) v[b] = (b < cnt && lane < n1) ? __ldcs(xp + g.Nd1 * b) : 0.0f;
        if (lane < n1) {
#pragma unroll
          for (int b = 0; b < 32; ++b) {
            if (b < cnt) {
              if constexpr (TF) {
                const float h = round_tf32(v[b]);
                Xh[b * kLD + lane] = h;
                Xl[b * kLD + lane] = round_tf32(__fsub_rn(v[b], h));
              } else if constexpr (F16) {
                const float xv = __fmul_rn(v[b], g.xscale);
                const __half h = __float2half_rn(xv);
                Xh[b * kLD + lane] = __half_as_ushort(h);
                Xl[b * kLD + lane] = __half_as_ushort(__float2half_rn(__fsub_rn(xv, __half2float(h))));
              } else {
                const __nv_bfloat16 h = __float2bfloat16_rn(v[b]);
                Xh[b * kLD + lane] = __bfloat16_as_ushort(h);
                Xl[b * kLD + lane] = __bfloat16_as_ushort(__float2bfloat16_rn(__fsub_rn(v[b], __bfloat162float(h))));
              }
            }
          }
        }
      }
      __syncwarp();
      const uint32_t kLp = (uint32_t)(kL0 + sa), kRp = (uint32_t)(kR0 + sb);
      for (int sj = 0; sj < g.nsk; ++sj) {
        // warps start at different sketches, so that at any moment they add
        // into different accumulator slots (less shared-atomic contention)
        const int si = (sj + warp) % g.nsk;
        const SpSk& s = s_sk[si];
        const int sell = s.ell;  // in a register: the tile stores below may alias s_sk
        const int nr = s.col ? cnt : n1;     // contraction extent
        const int nout = s.col ? n1 : cnt;   // output extent
        const int kext = TF ? (nr + 7) & ~7 : (nr + 15) & ~15;
        // key of the plane's test-matrix rows: w div wdiv (column side) or
        // w mod wdiv (row side); wdiv divides WL (column) or WL divides wdiv
        // (row), so both follow from kL and kR in 32-bit arithmetic
        const uint32_t wd = (uint32_t)s.wdiv, wl = (uint32_t)g.WL;
        const int64_t key = s.col ? (int64_t)(kLp / wd) + (int64_t)(wl / wd) * kRp
                                  : (int64_t)kLp + (int64_t)wl * (kRp % (wd / wl));
        // ---- test-matrix block Gs[k][j]
        if (s.tab >= 0) {
          constexpr int cpr = LPAD * kEsz / 16;  // 16-byte chunks per row
          const uint4* src = reinterpret_cast<const uint4*>(g.wsb + g.tab0 + s.tab + key * nr * LPAD * kEsz);
          for (int c = lane; c < nr * cpr; c += 32) {
            const int r = c / cpr, q = c - r * cpr;
            *reinterpret_cast<uint4*>(Gs + r * kLD + (16 / kEsz) * q) = __ldg(src + c);
          }
        } else {
          // jobs c = (row r, column quad q), two per lane at a time (independent
          // Philox chains); r = c div nq by a multiply-shift that is exact for
          // c < 2^10, nq <= 8
          const int njobs = nr * g.nq;
          const uint32_t inv = (65536u + (uint32_t)g.nq - 1u) / (uint32_t)g.nq;
          for (int c0 = lane; c0 < njobs; c0 += 64) {
            float4 z[2];
            int rr[2], qq[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int c = min(c0 + 32 * h, njobs - 1);
              rr[h] = (int)(((uint32_t)c * inv) >> 16);
              qq[h] = c - rr[h] * g.nq;
              const uint64_t row = s.col ? (uint64_t)(key + s.hstride * (g.first + rr[h]))
                                         : (uint64_t)(rr[h] + g.n1 * key);
              const DevSketch* krs = KR ? kr_of(g.wsb, s.kr) : nullptr;
              // a mode-by-mode sketch takes its mode-1 factor here (scaled below)
              z[h] = (krs && krs->kr_mbm) ? kr_f1_quad(g.wsb, *krs, rr[h], (uint32_t)qq[h])
                                          : tm_quad_f32(g.wsb, krs, g.seed, (uint32_t)s.sid, row, (uint32_t)qq[h]);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (c0 + 32 * h < njobs) {
                const int q = qq[h];
                if constexpr (TF) {
                  *reinterpret_cast<float4*>(Gs + rr[h] * kLD + 4 * q) = make_float4(
                      4 * q < sell ? round_tf32(z[h].x) : 0.f, 4 * q + 1 < sell ? round_tf32(z[h].y) : 0.f,
                      4 * q + 2 < sell ? round_tf32(z[h].z) : 0.f, 4 * q + 3 < sell ? round_tf32(z[h].w) : 0.f);
                } else {
                  const uint32_t lo = op16x2(F16, 4 * q < sell ? z[h].x : 0.f, 4 * q + 1 < sell ? z[h].y : 0.f);
                  const uint32_t hi = op16x2(F16, 4 * q + 2 < sell ? z[h].z : 0.f, 4 * q + 3 < sell ? z[h].w : 0.f);
                  *reinterpret_cast<uint2*>(Gs + rr[h] * kLD + 4 * q) = make_uint2(lo, hi);
                }
              }
            }
          }
        }
        // contraction padding rows [nr, kext) (another sketch may have left rows there)
        constexpr int zpr = LPAD * kEsz / 16;  // 16-byte chunks per row
        for (int c = lane; c < (kext - nr) * zpr; c += 32) {
          const int r = nr + c / zpr, q = c % zpr;
          *reinterpret_cast<uint4*>(Gs + r * kLD + (16 / kEsz) * q) = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncwarp();
        // ---- D[j][o] = sum_k Gs[k][j] Xs'[k][o], hi and lo parts
        const int ntn = (nout + 7) >> 3;
        const int sl = s.dep ? (s.col ? sa : sb) : 0;
        float* slot = acc + (size_t)(s.slot0 + sl) * slot_elems;
        const int gq = lane >> 2, tq = lane & 3;
        constexpr int MT = LPAD / 16;
        // every fragment of a k-step is loaded first, then the MMAs run over
        // independent accumulators (m-tile x n-tile; the hi and lo parts of X
        // go into the same one, as in the tcgen05 kernels), so consecutive
        // MMAs do not wait on each other
        float ch[MT][4][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) ch[mt][nt][e] = 0.0f;
        if constexpr (TF) {
          // m16n8k8 TF32 fragments straight from the FP32 tiles (row stride 40
          // words: the A loads and the column-product B loads are conflict-free)
          for (int k0 = 0; k0 < kext; k0 += 8) {
            uint32_t a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
              const float* gp = reinterpret_cast<const float*>(Gs) + (k0 + tq) * kLD + mt * 16 + gq;
              a[mt][0] = __float_as_uint(gp[0]);
              a[mt][1] = __float_as_uint(gp[8]);
              a[mt][2] = __float_as_uint(gp[4 * kLD]);
              a[mt][3] = __float_as_uint(gp[4 * kLD + 8]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              if (nt < ntn) {
                uint32_t bh0, bh1, bl0, bl1;
                const float* xh = reinterpret_cast<const float*>(Xh);
                const float* xl = reinterpret_cast<const float*>(Xl);
                if (s.col) {  // B[k][o] = X(o, k) = tile[k][o]
                  const int off = (k0 + tq) * kLD + nt * 8 + gq;
                  bh0 = __float_as_uint(xh[off]);
                  bh1 = __float_as_uint(xh[off + 4 * kLD]);
                  bl0 = __float_as_uint(xl[off]);
                  bl1 = __float_as_uint(xl[off + 4 * kLD]);
                } else {      // B[k][o] = X(k, o) = tile[o][k]
                  const int off = (nt * 8 + gq) * kLD + k0 + tq;
                  bh0 = __float_as_uint(xh[off]);
                  bh1 = __float_as_uint(xh[off + 4]);
                  bl0 = __float_as_uint(xl[off]);
                  bl1 = __float_as_uint(xl[off + 4]);
                }
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                  mma_tf32(ch[mt][nt], a[mt], bh0, bh1);
                  mma_tf32(ch[mt][nt], a[mt], bl0, bl1);
                }
              }
            }
          }
        } else {
#pragma unroll
        for (int k0 = 0; k0 < 32; k0 += 16) {
          if (k0 < kext) {
            uint32_t a[MT][4], bh[4][2], bl[4][2];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
              ldsm_x4_trans(smem_u32(Gs + (k0 + (lane & 7) + 8 * (lane >> 4)) * kLD + mt * 16 + 8 * ((lane >> 3) & 1)),
                            a[mt]);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              if (nt < ntn) {
                if (s.col) {  // B[k][o] = X(o, k): the [b][a] tile read transposed
                  const int off = (k0 + (lane & 7) + 8 * ((lane >> 3) & 1)) * kLD + nt * 8;
                  ldsm_x2_trans(smem_u32(Xh + off), bh[nt]);
                  ldsm_x2_trans(smem_u32(Xl + off), bl[nt]);
                } else {      // B[k][o] = X(k, o): the [b][a] tile read as is
                  const int off = (nt * 8 + (lane & 7)) * kLD + k0 + 8 * ((lane >> 3) & 1);
                  ldsm_x2(smem_u32(Xh + off), bh[nt]);
                  ldsm_x2(smem_u32(Xl + off), bl[nt]);
                }
              }
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
              for (int nt = 0; nt < 4; ++nt)
                if (nt < ntn) {
                  if constexpr (F16) mma_f16(ch[mt][nt], a[mt], bh[nt]);
                  else mma_bf16(ch[mt][nt], a[mt], bh[nt]);
                }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
              for (int nt = 0; nt < 4; ++nt)
                if (nt < ntn) {
                  if constexpr (F16) mma_f16(ch[mt][nt], a[mt], bl[nt]);
                  else mma_bf16(ch[mt][nt], a[mt], bl[nt]);
                }
          }
        }
        }
        // mode-by-mode Khatri-Rao sketch: column j scaled by the rounded product
        // of the other modes' rows of this plane (rows of the lane: gq, gq + 8
        // of each m-tile)
        float sc[MT][2];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) sc[mt][0] = sc[mt][1] = 1.0f;
        if constexpr (KR) {
          const DevSketch* krs = kr_of(g.wsb, s.kr);
          if (krs && krs->kr_mbm) {
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int j = mt * 16 + gq + 8 * h;
                const float4 c = kr_scale_quad(g.wsb, *krs, (uint64_t)key, (uint32_t)(j >> 2),
                                              TF ? TT_PREC_TF32 : F16 ? TT_PREC_FP16 : TT_PREC_BF16);
                sc[mt][h] = (j & 3) == 0 ? c.x : (j & 3) == 1 ? c.y : (j & 3) == 2 ? c.z : c.w;
              }
          }
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            if (nt < ntn) {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int j = mt * 16 + gq + 8 * (e >> 1), o = nt * 8 + 2 * tq + (e & 1);
                if (j < sell && o < nout) atomicAdd(slot + j * g.ldo + o, ch[mt][nt][e] * sc[mt][e >> 1]);
              }
            }
          }
        __syncwarp();  // every lane is done with Gs before the next sketch overwrites it
      }
    }
}

// Zeroes the per-warp tiles (their padding rows and columns stay zero) and
// the accumulator slots.
template <int FMT>
__device__ void sp_zero(unsigned char* smraw, float* acc, int acc_elems) {
  for (int i = threadIdx.x; i < Prec<FMT>::kWarps * Prec<FMT>::kWarpBytes / 16; i += Prec<FMT>::kThreads)
    reinterpret_cast<uint4*>(smraw)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = threadIdx.x; i < acc_elems; i += Prec<FMT>::kThreads) acc[i] = 0.0f;
}

template <int LPAD, int FMT, bool KR>
__global__ void __launch_bounds__(Prec<FMT>::kThreads, 1) sketch_sp_kernel(const SpArgs ga) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ SpArgs g;
  if (threadIdx.x == 0) g = ga;
  __syncthreads();
  float* acc = reinterpret_cast<float*>(smraw + Prec<FMT>::kWarps * Prec<FMT>::kWarpBytes);
  sp_zero<FMT>(smraw, acc, g.nslots * LPAD * g.ldo);
  __syncthreads();
  const int64_t nblocks = g.tilesL * g.tilesR;
  const int64_t b_beg = nblocks * blockIdx.x / gridDim.x, b_end = nblocks * (blockIdx.x + 1) / gridDim.x;
  int64_t cur_bL = -1;
  int age = 0;
  for (int64_t t = b_beg; t < b_end; ++t) {
    const int64_t bL = t / g.tilesR, bR = t - bL * g.tilesR;
    if (bL != cur_bL || age == kColFlushBlocks) {
      if (cur_bL >= 0) {
        sp_flush<LPAD, FMT>(g, g.sk, acc, true, cur_bL, 0);
        __syncthreads();
      }
      cur_bL = bL;
      age = 0;
    }
    ++age;
    sp_block<LPAD, FMT, KR>(g, g.sk, smraw, acc, bL, bR);
    __syncthreads();
    sp_flush<LPAD, FMT>(g, g.sk, acc, false, cur_bL, bR);
    __syncthreads();
  }
  if (cur_bL >= 0) sp_flush<LPAD, FMT>(g, g.sk, acc, true, cur_bL, 0);
}

// Batched form: persistent CTAs take `chunk` consecutive units (item, block)
// of the largest-first unit sequence at a time; row slots are flushed after
// every unit, the others when the item or the kL block changes.
template <int LPAD, int FMT>
__global__ void __launch_bounds__(Prec<FMT>::kThreads, 1) sketch_sp_batched_kernel(const BatchLaunch b) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ SpArgs g;
  __shared__ int64_t s_base;
  __shared__ int s_pos;
  const DevTables& T = *reinterpret_cast<const DevTables*>(b.wsb + kTableOffB);
  const DevItem* items = reinterpret_cast<const DevItem*>(b.wsb + T.off_items);
  const DevSketch* sks = reinterpret_cast<const DevSketch*>(b.wsb + T.off_sketches);
  const int* order = reinterpret_cast<const int*>(b.wsb + T.off_border);
  const int64_t* prefix = reinterpret_cast<const int64_t*>(b.wsb + T.off_bprefix);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(b.wsb + T.off_bcounter);
  const int64_t total = prefix[T.nitems];
  float* acc = reinterpret_cast<float*>(smraw + Prec<FMT>::kWarps * Prec<FMT>::kWarpBytes);
  sp_zero<FMT>(smraw, acc, 0);
  int cur = -1;
  int64_t cur_bL = -1;
  int age = 0;
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
    for (int64_t u = base; u < end; ++u) {
      while (prefix[pos + 1] <= u) ++pos;
      const int it_idx = order[pos];
      const int64_t lu = u - prefix[pos];
      // long-class slots (column sketches, plane-independent rows) are kept
      // while the item and the kL block stay the same, for at most
      // kColFlushBlocks units
      if (cur >= 0 && (it_idx != cur || lu / g.tilesR != cur_bL || age == kColFlushBlocks)) {
        sp_flush<LPAD, FMT>(g, g.sk, acc, true, cur_bL, 0);
        __syncthreads();
        age = 0;
        cur_bL = -1;
      }
      if (it_idx != cur) {
        __syncthreads();
        if (threadIdx.x == 0) {
          const DevItem& it = items[it_idx];
          sp_fill(it, sks, it.n[it.d - 1], g, b.t3max);
          g.X = reinterpret_cast<const float*>(b.X[it_idx]);
          g.wsb = b.wsb;
          g.first = 0;
        }
        __syncthreads();
        // slots of this item start at zero (every unit is flushed completely)
        for (int i = threadIdx.x; i < g.nslots * LPAD * g.ldo; i += Prec<FMT>::kThreads) acc[i] = 0.0f;
        __syncthreads();
        cur = it_idx;
      }
      const int64_t bL = lu / g.tilesR, bR = lu - bL * g.tilesR;
      cur_bL = bL;
      ++age;
      sp_block<LPAD, FMT, false>(g, g.sk, smraw, acc, bL, bR);  // batched plans refuse Khatri-Rao
      __syncthreads();
      sp_flush<LPAD, FMT>(g, g.sk, acc, false, bL, bR);
      __syncthreads();
    }
  }
  if (cur >= 0 && cur_bL >= 0) sp_flush<LPAD, FMT>(g, g.sk, acc, true, cur_bL, 0);
}

// Batched tables: blockIdx.y = item; its staged sketches one after another.
__global__ void sp_table_batched_kernel(char* wsb) {
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
  const DevItem& it = reinterpret_cast<const DevItem*>(wsb + T.off_items)[blockIdx.y];
  const DevSketch* sks = reinterpret_cast<const DevSketch*>(wsb + T.off_sketches);
  int lmax = 0;
  for (int si = 0; si < it.nsk; ++si) lmax = sks[it.sk0 + si].width > lmax ? sks[it.sk0 + si].width : lmax;
  const int lpad = lmax <= 16 ? 16 : 32;
  for (int si = 0; si < it.nsk; ++si) {
    const DevSketch& d = sks[it.sk0 + si];
    if (d.sp_tab < 0) continue;
    SpSk k;
    k.hstride = d.hstride;
    k.col = d.type == SK_COL ? 1 : 0;
    k.sid = d.stream_id;
    k.kr = -1;  // batched plans draw dense test matrices
    const int nr = k.col ? (int)it.n[it.d - 1] : (int)it.n[0];
    const int64_t nkeys = k.col ? it.W / d.wdiv : d.wdiv;
    sp_table_fill(wsb, k, it.seed, 0, it.n[0], nr, d.width, lpad, nkeys, wsb + it.off_sptab * 8 + d.sp_tab,
                  (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, it.prec);
  }
}

// Unit prefix of the batched form (largest items first); resets the work
// counter and the status word.
__global__ void __launch_bounds__(1024) sp_batch_prep_kernel(char* wsb, int t3max) {
  __shared__ int64_t cnt[kMaxBatchItems];
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
  const DevItem* items = reinterpret_cast<const DevItem*>(wsb + T.off_items);
  const int* order = reinterpret_cast<const int*>(wsb + T.off_border);
  int64_t* prefix = reinterpret_cast<int64_t*>(wsb + T.off_bprefix);
  for (int i = threadIdx.x; i < T.nitems; i += blockDim.x) {
    const DevItem& it = items[order[i]];
    const int64_t WL = it.N[it.ds] / it.n[0], WR = it.W / WL;
    int T2, T3;
    sp_block_shape(WL, WR, t3max, &T2, &T3);
    cnt[i] = ((WL + T2 - 1) / T2) * ((WR + T3 - 1) / T3);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t a = 0;
    for (int i = 0; i < T.nitems; ++i) {
      prefix[i] = a;
      a += cnt[i];
    }
    prefix[T.nitems] = a;
    *reinterpret_cast<unsigned long long*>(wsb + T.off_bcounter) = 0ull;
    *reinterpret_cast<int*>(wsb + kStatusOff) = 0;
  }
}

bool plan_sp(const Plan& P, int item, int64_t count, SpArgs* out, size_t* smem, int t3max = 4) {
  const DevItem& it = plan_items_host(&P)[item];
  if ((it.prec != TT_PREC_BF16 && it.prec != TT_PREC_TF32 && it.prec != TT_PREC_FP16) || it.x_f64 ||
      it.sptab_doubles == 0)
    return false;
  if (count < 1 || count > 32 || it.n[0] > 32 || it.W >= (1LL << 31)) return false;
  const DevSketch* sks = plan_sketches_host(&P);
  SpArgs g;
  memset(&g, 0, sizeof(g));
  sp_fill(it, sks, count, g, t3max);
  if (g.ell > 32) return false;
  const int lpad = g.ell <= 16 ? 16 : 32;
  const size_t tiles = it.prec == TT_PREC_TF32 ? (size_t)Prec<kFmtTF32>::kWarps * Prec<kFmtTF32>::kWarpBytes
                                               : (size_t)Prec<kFmtBF16>::kWarps * Prec<kFmtBF16>::kWarpBytes;
  const size_t need = tiles + sizeof(float) * (size_t)g.nslots * lpad * g.ldo;
  if (need > (size_t)kMaxSmem) return false;
  *out = g;
  *smem = need;
  return true;
}

}  // namespace sp

cudaError_t launch_rows_table(const DevSketch& d, int gsk, const char* wsb, uint64_t seed, int64_t first, int64_t n1,
                              int nr, int lpad, int64_t nkeys, char* tab, int prec, cudaStream_t st) {
  sp::SpSk k;
  memset(&k, 0, sizeof(k));
  k.hstride = d.hstride;
  k.col = d.type == SK_COL ? 1 : 0;
  k.sid = d.stream_id;
  k.kr = d.kr_nm ? gsk : -1;
  const int64_t total = nkeys * nr * (lpad / 4);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * device_sm_count()));
  count_launch();
  sp::sp_table_kernel<<<blocks, 256, 0, st>>>(wsb, k, seed, first, n1, nr, d.width, lpad, nkeys, tab, prec);
  return cudaGetLastError();
}

bool use_sp_kernel(const Plan& P, int item, int64_t count) {
  sp::SpArgs g;
  size_t smem;
  return sp::plan_sp(P, item, count, &g, &smem);
}

cudaError_t launch_sketch_sp(const Plan& P, int item, const void* X, int64_t first, int64_t count, void* ws,
                             cudaStream_t st) {
  sp::SpArgs g;
  size_t smem = 0;
  if (!sp::plan_sp(P, item, count, &g, &smem)) return cudaErrorNotSupported;
  g.X = (const float*)X;
  g.wsb = (char*)ws;
  g.first = first;
  const int lpad = g.ell <= 16 ? 16 : 32;
  const DevItem& it = plan_items_host(&P)[item];
  const int fmt = sp::fmt_of(it.prec);
  using KernelFn = void (*)(const sp::SpArgs);
#define TT_SP_K(F)                                                                      \
  {{sp::sketch_sp_kernel<16, F, false>, sp::sketch_sp_kernel<16, F, true>},             \
   {sp::sketch_sp_kernel<32, F, false>, sp::sketch_sp_kernel<32, F, true>}}
  const KernelFn kernels[3][2][2] = {TT_SP_K(sp::kFmtBF16), TT_SP_K(sp::kFmtTF32), TT_SP_K(sp::kFmtFP16)};
#undef TT_SP_K
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 3; ++f)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kernels[f][i][j], cudaFuncAttributeMaxDynamicSharedMemorySize, sp::kMaxSmem);
    if (e != cudaSuccess) {
      cudaGetLastError();  // leave no pending error for the caller's next runtime call
      return e;
    }
    attr_set = true;
  }
  for (int s = 0; s < g.nsk; ++s) {
    const sp::SpSk& k = g.sk[s];
    if (k.tab < 0) continue;
    const int nr = k.col ? (int)count : (int)g.n1;
    const int64_t nkeys = k.col ? it.W / k.wdiv : k.wdiv;
    const int64_t total = nkeys * nr * (lpad / 4);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 16LL * device_sm_count());
    count_launch();
    sp::sp_table_kernel<<<blocks, 256, 0, st>>>(g.wsb, k, g.seed, first, g.n1, nr, k.ell, lpad, nkeys,
                                                g.wsb + g.tab0 + k.tab, it.prec);
  }
  const int64_t nblocks = g.tilesL * g.tilesR;
  const int grid = (int)std::min<int64_t>(nblocks, device_sm_count());
  count_launch();
  bool kr = false;
  for (int s = 0; s < g.nsk; ++s) kr = kr || g.sk[s].kr >= 0;
  const KernelFn k = kernels[fmt][lpad == 16 ? 0 : 1][kr ? 1 : 0];
  k<<<grid, fmt == sp::kFmtTF32 ? sp::Prec<sp::kFmtTF32>::kThreads : sp::Prec<sp::kFmtBF16>::kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

// Batched form: every item must fit the small-plane kernel with the same
// padded width (the tables and tiles of a launch share it).
bool sp_batched_eligible(const Plan& P, size_t* smem_out, int* lpad_out, int t3max) {
  const int n = plan_num_items(&P);
  size_t smem = 0;
  int lpad = 0;
  for (int i = 0; i < n; ++i) {
    const DevItem& it = plan_items_host(&P)[i];
    if (it.prec != plan_items_host(&P)[0].prec) return false;
    sp::SpArgs g;
    size_t need = 0;
    if (!sp::plan_sp(P, i, it.n[it.d - 1], &g, &need, t3max)) return false;
    const int lp = g.ell <= 16 ? 16 : 32;
    if (lpad && lp != lpad) return false;
    lpad = lp;
    smem = std::max(smem, need);
  }
  if (smem_out) *smem_out = smem;
  if (lpad_out) *lpad_out = lpad;
  return n > 0 && n <= kMaxBatchItems;
}

cudaError_t launch_sketch_sp_batched(const Plan& P, const void* const* X, const BatchCfg& cfg, void* ws,
                                     cudaStream_t st) {
  // ta of the launch shape is the largest number of kR values per block here
  const int t3max = (cfg.ta == 1 || cfg.ta == 2 || cfg.ta == 4 || cfg.ta == 8) ? cfg.ta : 4;
  size_t smem = 0;
  int lpad = 0;
  if (!sp_batched_eligible(P, &smem, &lpad, t3max)) return cudaErrorNotSupported;
  const int nitems = plan_num_items(&P);
  static BatchLaunch b;  // 16 KB: kept off the host stack
  b.wsb = (char*)ws;
  b.chunk = std::max(1, cfg.chunk);
  b.t3max = t3max;
  for (int i = 0; i < nitems; ++i) b.X[i] = X[i];
  using KernelFn = void (*)(const BatchLaunch);
  const KernelFn kernels[3][2] = {
      {sp::sketch_sp_batched_kernel<16, sp::kFmtBF16>, sp::sketch_sp_batched_kernel<32, sp::kFmtBF16>},
      {sp::sketch_sp_batched_kernel<16, sp::kFmtTF32>, sp::sketch_sp_batched_kernel<32, sp::kFmtTF32>},
      {sp::sketch_sp_batched_kernel<16, sp::kFmtFP16>, sp::sketch_sp_batched_kernel<32, sp::kFmtFP16>}};
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < 3; ++f)
      for (int i = 0; i < 2; ++i)
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(kernels[f][i], cudaFuncAttributeMaxDynamicSharedMemorySize, sp::kMaxSmem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    attr_set = true;
  }
  const int fmt = sp::fmt_of(plan_items_host(&P)[0].prec);
  count_launch();
  sp::sp_batch_prep_kernel<<<1, 1024, 0, st>>>((char*)ws, t3max);
  count_launch();
  sp::sp_table_batched_kernel<<<dim3(16, (unsigned)nitems), 256, 0, st>>>((char*)ws);
  count_launch();
  const int nsm = device_sm_count();
  const int threads = fmt == sp::kFmtTF32 ? sp::Prec<sp::kFmtTF32>::kThreads : sp::Prec<sp::kFmtBF16>::kThreads;
  kernels[fmt][lpad == 16 ? 0 : 1]<<<nsm, threads, smem, st>>>(b);
  return cudaGetLastError();
}

}  // namespace tts
