// Slab form of the tcgen05 plane kernel: the fused multi-sketch of one slab of
// c = 16, 32 or 64 slices of the last mode of a 4-way tensor -- the unit of
// the paper's single stream over sub-tensors (Sec. 4.2, Algorithm 5; a 1 GiB
// slab of the 256^4 FP32 tensor is 16 slices).  BF16 or FP16 (X scaled by
// 2^s first) with X split into hi + lo, FP32 accumulators in tensor memory,
// FP64 flush, as the plane kernel.
//
// The plane kernel contracts a plane X(:, w, :) (n_1 x slab) over its 128-row
// quarters of i_4; a slab of 16 slices has no such quarter.  Here G = 128 / c
// planes that share i_2 (= kL) and have consecutive i_3 (kR) form one
// super-plane, an n_1 x 128 matrix whose column k = i_4' + c g (i_4' < c the
// slice within the slab, g < G the plane).  With w_g = kL + n_2 (G kRg + g):
//  * S_1 (rows i_1, test-matrix rows w_g + n_2 n_3 i_4) and S_2 (rows
//    i_1 + n_1 kL, rows kR_g + n_3 i_4): D_L = X_sp [B_1 | B_2], M = i_1,
//    K = k -- both sketches' output rows are the same for every k, so the
//    super-plane is an ordinary product;
//  * R_2 (rows kR_g + n_3 i_4, test-matrix rows i_1 + n_1 kL): D_R = X_sp^T C_2,
//    M = k, K = i_1 -- the test-matrix rows are the same for every k;
//  * R_3 (rows i_4, test-matrix rows i_1 + n_1 w_g): the test-matrix rows
//    depend on g, which runs along M, so the product is taken against all G
//    blocks side by side, D_Y = X_sp^T [C_3(g=0) | ... | C_3(g=G-1)]
//    (N = G l), and only its diagonal blocks (row group g, column block g) are
//    kept.  The tensor pipe does G times the R_3 work it needs; it has the
//    room (the kernel is bound by HBM).
// Test-matrix blocks: the L block (S_1, S_2; 128 composite rows) comes from
// the test-matrix warps for every super-plane; the R_2 block from a staged
// table (one per kL, generated at the first launch of a decomposition).  R_3
// with dense Gaussian test matrices: its rows belong to one plane each and
// regenerating them costs l / c normals per entry of X (1 at c = l = 16), so
// the G planes' blocks are generated once per decomposition into a table of
// block images and bulk-copied per quarter by one warp (when the plan has
// room for the table; else regenerated per quarter).  R_3 with Khatri-Rao
// test matrices (TT_FLAG_KR) is taken mode by mode: X_sp^T round(F_1) against
// one fixed block (the mode-1 factor), the plane's rounded mode-3 x mode-2
// row product applied by the epilogue as a column scale per super-plane.
//
// Accumulators: one L slot per (kL of the tile, i_1 half), kept for runL
// tiles (Khatri-Rao: each slot drained by the epilogue right after its last
// super-plane of the run, overlapping the rest of the tile); the R_2 slots (one per kR group of the tile) and the D_Y block of a
// tile are double-buffered with the epilogue; every accumulator sees at most
// 256 MMAs before a flush.  Khatri-Rao: the tensor cores' FP32 accumulation
// adds ~2e-8 relative error per accumulating MMA (measured), so D_Y and R_2
// get short chains: a buffer per super-plane (16 MMAs a half of i_1),
// double-buffered, which the epilogue sums in FP32 (D_Y scaled, and R_2 in
// shared memory, over a kR group's super-planes).  Flushes:
// FP64 atomics into S_1, R_2 and R_3; FP32 atomics into a staging copy of S_2
// (about four CTA partials per entry a launch), added into S_2 by
// s2_fold_kernel after the launch.
//
// Warp roles: 4 epilogue warps (the TMEM lane quarters), 1 MMA issuer, 8
// producers (X loads, hi / lo split into the 16-bit operand stages), and 7
// (dense) or 3 (Khatri-Rao) test-matrix warps.  Every mbarrier wait is
// bounded; a wait that gives up raises the CTA's abort flag and the timeout
// status bit, waits for its own copies and MMAs, frees TMEM and returns.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "philox.cuh"
#include "tc_common.cuh"
#include "testmat.cuh"

namespace tts {

const DevSketch* plan_sketches_host(const Plan* p);

namespace tc {
namespace slab {

constexpr int kEpiWarps = 4, kMmaWarp = 4, kProdWarp0 = 5, kProdWarps = 8, kRngWarp0 = 13;
// Test-matrix warps: seven draw the dense Gaussian blocks (Philox); three
// form the Khatri-Rao L blocks from factor rows.  The Khatri-Rao kernel has
// 16 warps and so 128 registers a thread (registers go to warps four at a
// time), which its roles need without spilling.
template <bool KRY>
struct Roles {
  static constexpr int rng = KRY ? 3 : 7;
  static constexpr int threads = (kRngWarp0 + rng) * 32;
};
constexpr int kLBlkB = 4 * kS4;   // L block: 128 rows x N <= 32
constexpr int kRBlkB = 2 * kS4;   // R_2 block: 128 rows x N <= 16
constexpr int kYBlkB = 16 * kS4;  // R_3 blocks side by side: 128 rows x N <= 128
constexpr int kOffL = 2 * kStageB;
constexpr int kOffR = kOffL + 2 * kLBlkB;
constexpr int kOffY = kOffR + 4 * kRBlkB;
constexpr int kOffBar = kOffY + kYBlkB;
// Khatri-Rao: the fixed mode-1 block takes the first two R_2-sized blocks of
// the R_3 area; the slab's mode-4 rows of S_1 and S_2 (FP32, c x l each)
// follow it
constexpr int kOffF4 = kOffY + 2 * kRBlkB;
// and the L flush's FP32 sums of S_1 over a run's kL values ([half][column][lane])
constexpr int kOffS1 = kOffF4 + 2 * 64 * 16 * 4;
static_assert(kOffS1 - kOffY + 2 * 16 * 128 * 4 <= kYBlkB, "Khatri-Rao blocks in the R_3 area");
// Khatri-Rao: the lanes' FP32 sums of R_2 over a kR group's super-planes
// ([column][lane]), after the barrier words
constexpr int kOffR2 = kOffBar + 256;
constexpr int kSmemBytes = kOffR2 + 16 * 128 * 4 + 1024;
constexpr int kTmemY = 0;         // D_Y buffers at columns 0 and 128, then the L slots, then R_2

struct SlabArgs {
  const float* X;
  double* ws;
  int* status;
  int64_t n1, first, W, WL, WR, Nd1;
  int64_t WRg;             // kR groups: WR / G
  int64_t tilesL, tilesR;  // tiles of T2 kL values x T3 kR groups
  uint64_t seed;
  int H1, T2, T3, ell, c, lc, G;
  int colL, colR;          // tensor-memory columns of the L slots and of the R_2 buffers
  int kry;                 // Khatri-Rao test matrices: R_3 mode by mode (fixed mode-1 block)
  int64_t runL;            // tiles of one kL block accumulated in the L slots before a flush
  uint32_t tab_tx;         // bytes of the staged R_2 blocks copied per super-plane
  float* s2stage;          // FP32 staging of S_2 (row-major: l floats a row), added into S_2 after the launch
  int64_t ytab;            // dense: byte offset of the staged R_3 blocks (-1: regenerated per quarter)
  float xscale;            // FP16 operands: 2^s, X is split as X 2^s (1 with BF16)
  int f16;                 // FP16 operands (else BF16), for the table kernels
  SkTc col[2], row[2];     // S_1, S_2 | R_2, R_3
};

struct TileInfo {
  int64_t kL0, kRg0;
  int nA, nB;
};
// dst[0 .. ELL) += v with four-wide FP32 reductions (dst 16-byte aligned).
template <int ELL>
__device__ __forceinline__ void red_add_row(float* dst, const float v[ELL]) {
#pragma unroll
  for (int q = 0; q < ELL / 4; ++q)
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4 * q), "f"(v[4 * q]),
                 "f"(v[4 * q + 1]), "f"(v[4 * q + 2]), "f"(v[4 * q + 3])
                 : "memory");
}
__device__ __forceinline__ TileInfo tile_info(const SlabArgs& g, int64_t t) {
  TileInfo ti;
  const int64_t tl = t / g.tilesR, tr = t % g.tilesR;  // kL-block-major
  ti.kL0 = tl * g.T2;
  ti.kRg0 = tr * g.T3;
  ti.nA = (int)imin64(g.T2, g.WL - ti.kL0);
  ti.nB = (int)imin64(g.T3, g.WRg - ti.kRg0);
  return ti;
}
__device__ __forceinline__ int64_t l_group(const SlabArgs& g, int64_t t) {
  const int64_t tl = t / g.tilesR, tr = t % g.tilesR;
  return tl * ((g.tilesR + g.runL - 1) / g.runL) + tr / g.runL;
}
// The super-plane after (a, b) of tile t in the order every role walks them
// (tile, then kR group b, then kL a): its kL and first kR; false past the
// CTA's last tile.
__device__ __forceinline__ bool next_super_plane(const SlabArgs& g, int64_t ntiles, int64_t t, int a, int b,
                                                 const TileInfo& ti, int64_t& kL, int64_t& kR0) {
  if (++a == ti.nA) {
    a = 0;
    if (++b == ti.nB) {
      b = 0;
      if (++t >= ntiles) return false;
      const TileInfo tn = tile_info(g, t);
      kL = tn.kL0;
      kR0 = tn.kRg0 * g.G;
      return true;
    }
  }
  kL = ti.kL0 + a;
  kR0 = (ti.kRg0 + b) * g.G;
  return true;
}

template <int ELL, int C, bool KRY, bool F16>
__global__ void __launch_bounds__(Roles<KRY>::threads, 1) sketch_slab_kernel(const SlabArgs g) {
  constexpr int kRngWarps = Roles<KRY>::rng;
  constexpr int kThreads = Roles<KRY>::threads;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kOffBar);
  // barrier indices
  // (TML_EMPTY + a: the L slots of the tile's a-th kL value are free, a < 8)
  const int FULL_A = 0, EMPTY_A = 2, FULL_L = 4, EMPTY_L = 6, TAB_FULL = 8, FULL_Y = 10, EMPTY_Y = 11,
            TML_FULL = 12, TMR_FULL = 14, TMR_EMPTY = 16, DRAIN = 18, TMY_FULL = 19, TMY_EMPTY = 21,
            TML_EMPTY = 23;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kOffBar + 248);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffBar + 252);
  __shared__ SkTc s_col[2], s_row[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };
  constexpr int ell = ELL;
  constexpr int NL = 2 * ELL;

  if (threadIdx.x < 2) {
    s_col[threadIdx.x] = g.col[threadIdx.x];
    s_row[threadIdx.x] = g.row[threadIdx.x];
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(bar(FULL_A + s), kProdWarps);
      mbar_init(bar(EMPTY_A + s), 1);
      mbar_init(bar(FULL_L + s), kRngWarps);
      mbar_init(bar(EMPTY_L + s), 1);
      mbar_init(bar(TAB_FULL + s), 1);
      mbar_init(bar(TMR_FULL + s), 1);
      mbar_init(bar(TMR_EMPTY + s), kEpiWarps);
    }
    mbar_init(bar(FULL_Y), g.ytab >= 0 ? 1 : kRngWarps);
    mbar_init(bar(EMPTY_Y), 1);
    for (int s2 = 0; s2 < 2; ++s2) {
      mbar_init(bar(TMY_FULL + s2), 1);
      mbar_init(bar(TMY_EMPTY + s2), kEpiWarps);
    }
    mbar_init(bar(TML_FULL), 1);
    for (int a = 0; a < 8; ++a) mbar_init(bar(TML_EMPTY + a), kEpiWarps);
    mbar_init(bar(DRAIN), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // Khatri-Rao test matrices: R_3 is taken mode by mode (eq. (sketch_orig)),
  // X_sp^T round(F_1) -- one fixed B block for the whole launch, here in the
  // R_3 block area -- with the rounded product of the plane's mode-2 and
  // mode-3 rows applied by the epilogue to each super-plane's partial sums.
  const DevSketch* kr3 = kr_of(g.ws, g.row[1].kr);
  if constexpr (KRY) {
    const float* f1 = reinterpret_cast<const float*>(reinterpret_cast<const char*>(g.ws) + kr3->kr_tab) +
                      kr3->kr_off[0];
    for (int e = threadIdx.x; e < g.H1 * 128 * ell; e += kThreads) {
      const int j = e % ell, i1 = e / ell, h1 = i1 >> 7, k = i1 & 127;
      *reinterpret_cast<uint16_t*>(sm + kOffY + h1 * kRBlkB + (k >> 3) * kS1 + (j >> 3) * kS4 + (j & 7) * 16 +
                                   (k & 7) * 2) = op16_bits<F16>(f1[(int64_t)i1 * kr3->kr_lp + j]);
    }
    // the mode-4 rows of the slab's slices for S_1 (its mode-4 factor is its
    // third) and S_2 (its second)
    const DevSketch* k0 = kr_of(g.ws, g.col[0].kr);
    const DevSketch* k1 = kr_of(g.ws, g.col[1].kr);
    if (k0 && k1) {
      float* f4s = reinterpret_cast<float*>(sm + kOffF4);
      for (int e = threadIdx.x; e < 2 * C * ell; e += kThreads) {
        const int sk = e / (C * ell), r = (e / ell) % C, j = e % ell;
        const DevSketch* kb = sk ? k1 : k0;
        const float* tb = reinterpret_cast<const float*>(reinterpret_cast<const char*>(g.ws) + kb->kr_tab);
        f4s[e] = tb[kb->kr_off[sk ? 1 : 2] + (g.first + r) * kb->kr_lp + j];
      }
    }
    float* s1z = reinterpret_cast<float*>(sm + kOffS1);
    for (int e = threadIdx.x; e < g.H1 * ell * 128; e += kThreads) s1z[e] = 0.0f;
    fence_async_smem();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t ntiles_all = g.tilesL * g.tilesR;
  const int64_t t_beg = ntiles_all * blockIdx.x / gridDim.x;
  const int64_t ntiles = ntiles_all * (blockIdx.x + 1) / gridDim.x;
  const uint32_t sA = smem_u32(sm);
  const uint32_t sL = smem_u32(sm + kOffL);
  const uint32_t sR = smem_u32(sm + kOffR);
  const uint32_t sY = smem_u32(sm + kOffY);
  constexpr int cmask = C - 1;
  constexpr int lc = C == 16 ? 4 : C == 32 ? 5 : 6;
  const int64_t gstride = g.n1 * g.WL;  // elements between the planes of a super-plane (kR + 1)

  if (warp >= kProdWarp0 && warp < kProdWarp0 + kProdWarps) {
    // ------------------------------------------------------------ producers
    const int pt = threadIdx.x - kProdWarp0 * 32;
    const int cb1 = pt & 15, rsub = pt >> 4;
    // composite row k = rsub + 16 m of a quarter: slice k & (c-1) of plane k >> lc
    auto rowoff = [&](int m) -> int64_t {
      const int k = rsub + 16 * m;
      return (int64_t)(k & cmask) * g.Nd1 + (int64_t)(k >> lc) * gstride;
    };
    int64_t t = t_beg;
    int a = 0, b = 0, q = 0;
    TileInfo ti = tile_info(g, t);
    auto advance = [&]() {
      if (++q == g.H1) {
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
    auto cursor_src = [&]() -> const float* {
      if (t >= ntiles) return nullptr;
      const int64_t w0 = (ti.kL0 + a) + g.WL * ((ti.kRg0 + b) * g.G);
      return g.X + (q * 128 + cb1 * 8) + g.n1 * w0;
    };
    auto prefetch = [&](const float* src) {
      const int cc = cb1 & 3;
      const float* line = src - cc * 8;
      prefetch_l2(line + rowoff(2 * cc));
      prefetch_l2(line + rowoff(2 * cc + 1));
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
        const float4* p4 = reinterpret_cast<const float4*>(src + rowoff(m));
        v[2 * m] = __ldcs(p4);
        v[2 * m + 1] = __ldcs(p4 + 1);
      }
    };
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
        const int k = rsub + 16 * m;
        const float x[8] = {sx(v[2 * m].x),     sx(v[2 * m].y),     sx(v[2 * m].z),     sx(v[2 * m].w),
                            sx(v[2 * m + 1].x), sx(v[2 * m + 1].y), sx(v[2 * m + 1].z), sx(v[2 * m + 1].w)};
        uint32_t hb[4], lb[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_hi_lo<F16>(x[2 * e], x[2 * e + 1], hb[e], lb[e]);
        const uint32_t off = cb1 * kS1 + (k >> 3) * kS4 + (k & 7) * 16;
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
    const int rt = threadIdx.x - kRngWarp0 * 32;  // 0 .. 32 kRngWarps - 1
    constexpr int qps = ell / 4;
    constexpr int upb = 64 * qps;  // 2-row units of one 128-row block
    // L block: S_1 then S_2, rows k = composite; contiguous unit ranges.  With
    // staged R_3 blocks the first warp only issues the bulk copies (its lane
    // 0 would otherwise hold the next quarter's copy behind its share of the
    // L block), and the other warps generate.
    const bool copier_warp = g.ytab >= 0 && rt < 32;
    const int gt = g.ytab >= 0 ? rt - 32 : rt, gn = (g.ytab >= 0 ? kRngWarps - 1 : kRngWarps) * 32;
    const int lu_beg = copier_warp ? 0 : 2 * upb * gt / gn, lu_end = copier_warp ? 0 : 2 * upb * (gt + 1) / gn;
    // R_3 blocks of a quarter: G blocks of 128 rows of i_1
    const int yn = g.G * upb;
    const int yu_beg = yn * rt / (kRngWarps * 32), yu_end = yn * (rt + 1) / (kRngWarps * 32);
    const DevSketch* krL0 = kr_of(g.ws, s_col[0].kr);
    const DevSketch* krL1 = kr_of(g.ws, s_col[1].kr);
    // Khatri-Rao L blocks by task: task u = (rp, nq) (u = qps rp + nq) is rows
    // k = 2 rp, 2 rp + 1 and column quad nq of both S_1 and S_2; thread rt
    // takes u = rt + 96 i, all with the same quad.  The mode-4 rows (slices
    // first + k mod c, + 1) come from shared memory, staged at the start; the
    // mode-2 / mode-3 rows of the next super-plane are loaded while this one
    // is stored.
    constexpr int kNT = Roles<true>::rng * 32;
    constexpr int kTasks = KRY ? (64 * qps + kNT - 1) / kNT : 1;
    static_assert(!KRY || kNT % qps == 0, "Khatri-Rao L tasks keep their quad");
    const bool kr_tasks = KRY && krL0 != nullptr && krL1 != nullptr;
    const int kq = rt % qps;
    int task_k[kTasks];
    bool task_on[kTasks];
    float4 f3r[2][kTasks], f2r = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4* f4s = reinterpret_cast<const float4*>(sm + kOffF4);  // [sketch][slice][l / 4]
    const float *kt0 = nullptr, *kt1 = nullptr;
    int64_t o2_0 = 0, o3_0 = 0, o3_1 = 0, lp0 = 0, lp1 = 0;
    auto kr_load_sp = [&](int64_t kL, int64_t kR0) {
      f2r = *reinterpret_cast<const float4*>(kt0 + o2_0 + kL * lp0 + 4 * kq);
#pragma unroll
      for (int i = 0; i < kTasks; ++i)
        if (task_on[i]) {
          const int64_t gg = task_k[i] >> lc;
          f3r[0][i] = *reinterpret_cast<const float4*>(kt0 + o3_0 + (kR0 + gg) * lp0 + 4 * kq);
          f3r[1][i] = *reinterpret_cast<const float4*>(kt1 + o3_1 + (kR0 + gg) * lp1 + 4 * kq);
        }
    };
    if (kr_tasks) {
      kt0 = reinterpret_cast<const float*>(reinterpret_cast<const char*>(g.ws) + krL0->kr_tab);
      kt1 = reinterpret_cast<const float*>(reinterpret_cast<const char*>(g.ws) + krL1->kr_tab);
      lp0 = krL0->kr_lp;
      lp1 = krL1->kr_lp;
      // S_1 over modes 2, 3, 4; S_2 over modes 3, 4
      o2_0 = krL0->kr_off[0];
      o3_0 = krL0->kr_off[1];
      o3_1 = krL1->kr_off[0];
#pragma unroll
      for (int i = 0; i < kTasks; ++i) {
        const int u = rt + kNT * i;
        task_on[i] = u < 64 * qps;
        task_k[i] = task_on[i] ? 2 * (u / qps) : 0;
      }
      if (t_beg < ntiles) {
        const TileInfo t0 = tile_info(g, t_beg);
        kr_load_sp(t0.kL0, t0.kRg0 * g.G);
      }
    }
    uint32_t pi = 0, qy = 0;
    int64_t tab_last[2] = {-1, -1}, y_last = -1;
    bool ok = true;
    for (int64_t t = t_beg; t < ntiles && ok && !*abort_flag; ++t) {
      const TileInfo ti = tile_info(g, t);
      for (int b = 0; b < ti.nB && ok; ++b)
        for (int a = 0; a < ti.nA && ok; ++a, ++pi) {
          const int64_t kL = ti.kL0 + a, kR0 = (ti.kRg0 + b) * g.G;
          const int64_t w0 = kL + g.WL * kR0;
          const int buf = pi & 1;
          if (!mbar_wait(bar(EMPTY_L + buf), ((pi >> 1) & 1) ^ 1, abort_flag, g.status)) {
            ok = false;
            break;
          }
          if (rt == 0 && g.tab_tx) {
            // the R_2 blocks of this kL from the staged table
            mbar_arrive_expect_tx(bar(TAB_FULL + buf), g.tab_tx);
            tab_last[buf] = pi;
            constexpr uint32_t bytes = (uint32_t)(ell / 8) * kS4;
            const char* wsb = reinterpret_cast<const char*>(g.ws);
            for (int h1 = 0; h1 < g.H1; ++h1)
              bulk_g2s(sR + (buf * 2 + h1) * kRBlkB, wsb + s_row[0].tab + (kL * g.H1 + h1) * (int64_t)bytes, bytes,
                       bar(TAB_FULL + buf));
          }
          // L block: S_1 rows w_g + W (first + i4'), S_2 rows kR_g + n3 (first + i4'),
          // k = i4' + c g
          auto store_pair = [&](int bi, int k, const float4& ra, const float4& rb) {
            const int n0 = bi * ell + 4 * kq;
            const uint32_t dst = sL + buf * kLBlkB + (k >> 3) * kS1 + (n0 >> 3) * kS4 + (n0 & 7) * 16 + (k & 7) * 2;
            st_shared_b32(dst, op16x2_bits<F16>(ra.x, rb.x));
            st_shared_b32(dst + 16, op16x2_bits<F16>(ra.y, rb.y));
            st_shared_b32(dst + 32, op16x2_bits<F16>(ra.z, rb.z));
            st_shared_b32(dst + 48, op16x2_bits<F16>(ra.w, rb.w));
          };
          auto mul4 = [](const float4& x, const float4& y) {
            return make_float4(__fmul_rn(x.x, y.x), __fmul_rn(x.y, y.y), __fmul_rn(x.z, y.z), __fmul_rn(x.w, y.w));
          };
          if (kr_tasks) {
            // increasing mode order: S_1 (F_2(kL) F_3(kR_g)) F_4(i4), S_2 F_3(kR_g) F_4(i4)
#pragma unroll
            for (int i = 0; i < kTasks; ++i)
              if (task_on[i]) {
                const int kk = task_k[i] & cmask;
                const float4 a0 = f4s[(0 * C + kk) * qps + kq], a1 = f4s[(0 * C + kk + 1) * qps + kq];
                const float4 b0 = f4s[(1 * C + kk) * qps + kq], b1 = f4s[(1 * C + kk + 1) * qps + kq];
                const float4 c1 = mul4(f2r, f3r[0][i]);
                store_pair(0, task_k[i], mul4(c1, a0), mul4(c1, a1));
                store_pair(1, task_k[i], mul4(f3r[1][i], b0), mul4(f3r[1][i], b1));
              }
            int64_t kLn, kR0n;
            if (next_super_plane(g, ntiles, t, a, b, ti, kLn, kR0n)) kr_load_sp(kLn, kR0n);
          }
          for (int u = lu_beg; u < (kr_tasks ? lu_beg : lu_end); ++u) {
            const int bi = u / upb, rp = (u % upb) / qps, nq = u % qps;
            const SkTc& sk = s_col[bi];
            const int k = 2 * rp;
            const int64_t gg = k >> lc, kk = k & cmask;
            float4 ra, rb;
            if (krL0) {
              // Khatri-Rao, increasing mode order: S_1 (F_2(kL) F_3(kR_g)) F_4(i4),
              // S_2 F_3(kR_g) F_4(i4)
              const DevSketch* kb = bi == 0 ? krL0 : krL1;
              const float* tb = reinterpret_cast<const float*>(reinterpret_cast<const char*>(g.ws) + kb->kr_tab);
              const int lp = kb->kr_lp, t4 = bi == 0 ? 2 : 1;
              float4 cw = *reinterpret_cast<const float4*>(tb + kb->kr_off[t4 - 1] + (kR0 + gg) * lp + 4 * nq);
              if (bi == 0) {
                const float4 f2 = *reinterpret_cast<const float4*>(tb + kb->kr_off[0] + kL * lp + 4 * nq);
                cw = make_float4(__fmul_rn(f2.x, cw.x), __fmul_rn(f2.y, cw.y), __fmul_rn(f2.z, cw.z),
                                 __fmul_rn(f2.w, cw.w));
              }
              const float* f4 = tb + kb->kr_off[t4] + (g.first + kk) * lp + 4 * nq;
              const float4 fa = *reinterpret_cast<const float4*>(f4);
              const float4 fb = *reinterpret_cast<const float4*>(f4 + lp);
              ra = make_float4(__fmul_rn(cw.x, fa.x), __fmul_rn(cw.y, fa.y), __fmul_rn(cw.z, fa.z),
                               __fmul_rn(cw.w, fa.w));
              rb = make_float4(__fmul_rn(cw.x, fb.x), __fmul_rn(cw.y, fb.y), __fmul_rn(cw.z, fb.z),
                               __fmul_rn(cw.w, fb.w));
            } else {
              const int64_t key = bi == 0 ? w0 + g.WL * gg : kR0 + gg;  // w / wdiv for wdiv = 1, n2
              const int64_t row = key + sk.hstride * (g.first + kk);
              ra = normals4_f32(g.seed, (uint32_t)sk.sid, (uint64_t)row, (uint32_t)nq);
              rb = normals4_f32(g.seed, (uint32_t)sk.sid, (uint64_t)(row + sk.hstride), (uint32_t)nq);
            }
            const int n0 = bi * ell + 4 * nq;
            const uint32_t dst = sL + buf * kLBlkB + (k >> 3) * kS1 + (n0 >> 3) * kS4 + (n0 & 7) * 16 + (k & 7) * 2;
            st_shared_b32(dst, op16x2_bits<F16>(ra.x, rb.x));
            st_shared_b32(dst + 16, op16x2_bits<F16>(ra.y, rb.y));
            st_shared_b32(dst + 32, op16x2_bits<F16>(ra.z, rb.z));
            st_shared_b32(dst + 48, op16x2_bits<F16>(ra.w, rb.w));
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(FULL_L + buf));
          // Khatri-Rao: R_3 needs no regenerated blocks (fixed mode-1 block)
          if constexpr (KRY) continue;
          // R_3 blocks, one quarter (half of i_1) at a time
          if (g.ytab >= 0) {
            // staged: one bulk copy of the super-plane's G blocks per quarter,
            // and an L2 prefetch of the next super-plane's
            constexpr uint32_t blkB = (uint32_t)(ell / 8) * kS4;
            const uint32_t bytes = (uint32_t)g.G * blkB;
            const char* ytab = reinterpret_cast<const char*>(g.ws) + g.ytab;
            auto ysrc = [&](int h1, int64_t kL, int64_t kR) {
              return ytab + ((h1 * g.WL + kL) * g.WR + kR) * (int64_t)blkB;
            };
            for (int h1 = 0; h1 < g.H1; ++h1, ++qy) {
              if (rt != 0) continue;
              if (!mbar_wait(bar(EMPTY_Y), (qy & 1) ^ 1, abort_flag, g.status)) {
                ok = false;
                break;
              }
              mbar_arrive_expect_tx(bar(FULL_Y), bytes);
              bulk_g2s(sY, ysrc(h1, kL, kR0), bytes, bar(FULL_Y));
              y_last = (int64_t)qy;
              int64_t kLn, kR0n;
              if (h1 == 0 && next_super_plane(g, ntiles, t, a, b, ti, kLn, kR0n))
                for (int h2 = 0; h2 < g.H1; ++h2) bulk_prefetch_l2(ysrc(h2, kLn, kR0n), bytes);
            }
            continue;
          }
          for (int h1 = 0; h1 < g.H1; ++h1, ++qy) {
            if (!mbar_wait(bar(EMPTY_Y), (qy & 1) ^ 1, abort_flag, g.status)) {
              ok = false;
              break;
            }
            // two units at a time: four independent Philox chains in flight
            const SkTc& sk = s_row[1];
            for (int u0 = yu_beg; u0 < yu_end; u0 += 2) {
              float4 z[2][2];
              int kk2[2], nn2[2];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int u = min(u0 + h, yu_end - 1);
                const int gp = u / upb, rp = (u % upb) / qps, nq = u % qps;
                kk2[h] = 2 * rp;
                nn2[h] = gp * ell + 4 * nq;
                const int64_t row = h1 * 128 + kk2[h] + g.n1 * (w0 + g.WL * gp);
                z[h][0] = normals4_f32(g.seed, (uint32_t)sk.sid, (uint64_t)row, (uint32_t)nq);
                z[h][1] = normals4_f32(g.seed, (uint32_t)sk.sid, (uint64_t)(row + 1), (uint32_t)nq);
              }
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                if (u0 + h >= yu_end) break;
                const int k = kk2[h], n0 = nn2[h];
                const float4 ra = z[h][0], rb = z[h][1];
                const uint32_t dst = sY + (k >> 3) * kS1 + (n0 >> 3) * kS4 + (n0 & 7) * 16 + (k & 7) * 2;
                st_shared_b32(dst, op16x2_bits<F16>(ra.x, rb.x));
                st_shared_b32(dst + 16, op16x2_bits<F16>(ra.y, rb.y));
                st_shared_b32(dst + 32, op16x2_bits<F16>(ra.z, rb.z));
                st_shared_b32(dst + 48, op16x2_bits<F16>(ra.w, rb.w));
              }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(FULL_Y));
          }
        }
    }
    // copies still in flight when the CTA gave up must land before it exits
    if (rt == 0 && y_last >= 0) {
      const long long t0 = clock64();
      while (!mbar_try(bar(FULL_Y), (uint32_t)(y_last & 1)) && clock64() - t0 < kWaitCycles) {
      }
    }
    if (rt == 0)
      for (int b2 = 0; b2 < 2; ++b2)
        if (tab_last[b2] >= 0) {
          const long long t0 = clock64();
          while (!mbar_try(bar(TAB_FULL + b2), (uint32_t)((tab_last[b2] >> 1) & 1)) && clock64() - t0 < kWaitCycles) {
          }
        }
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issue
    // Khatri-Rao: R_2 into a buffer per super-plane (16 MMAs a half of i_1)
    // that the epilogue sums in FP32: each accumulating MMA adds ~2e-8
    // relative error in FP32 (measured), which a chain over the tile's kL
    // values would bring to the rank rule's threshold.
    const uint32_t idL = make_idesc(NL, true, F16), idR = make_idesc(ell, false, F16),
                   idY = make_idesc(KRY ? ell : g.G * ell, false, F16);
    const uint32_t colYB = (uint32_t)(KRY ? ell : g.G * ell);
    uint32_t qi = 0, pi = 0, lf = 0, ti_n = 0;
    int64_t cur_tl = -1;
    uint32_t initL = 0, pendL = 0;
    bool ok = true;
    for (int64_t t = t_beg; t < ntiles && ok; ++t, ++ti_n) {
      const TileInfo tinf = tile_info(g, t);
      const int64_t tl = l_group(g, t);
      if (tl != cur_tl) {
        if (cur_tl >= 0) {
          // Khatri-Rao: the epilogue drains each slot after its last
          // super-plane of the run (no whole-run commit)
          if (!KRY && elect_one()) mma_commit(bar(TML_FULL));
          __syncwarp();
          ++lf;
        }
        // the epilogue frees the previous run's slots kL by kL: each is
        // awaited just before its first MMA of this run
        pendL = 0xFFu;
        initL = 0;
        cur_tl = tl;
      }
      const uint32_t rb = ti_n & 1;
      if (!KRY) {
        ok = warp_wait(bar(TMR_EMPTY + rb), ((ti_n >> 1) & 1) ^ 1, abort_flag, g.status);
        if (!ok) break;
        tc_fence_after();
      }
      uint32_t initR = 0;
      bool initY = false;
      const uint32_t dY = tmem + (uint32_t)kTmemY + rb * colYB;
      for (int b = 0; b < tinf.nB && ok; ++b)
        for (int a = 0; a < tinf.nA && ok; ++a, ++pi) {
          const int buf = pi & 1;
          if ((pendL >> a) & 1u) {
            ok = warp_wait(bar(TML_EMPTY + a), (lf & 1) ^ 1, abort_flag, g.status);
            if (!ok) break;
            tc_fence_after();
            pendL &= ~(1u << a);
          }
          ok = warp_wait(bar(FULL_L + buf), (pi >> 1) & 1, abort_flag, g.status);
          if (ok && g.tab_tx) ok = warp_wait(bar(TAB_FULL + buf), (pi >> 1) & 1, abort_flag, g.status);
          // Khatri-Rao: one D_Y accumulator per super-plane, double-buffered
          // with the epilogue (which scales it by the plane's factor rows)
          const uint32_t yb = pi & 1;
          if (KRY && ok) ok = warp_wait(bar(TMY_EMPTY + yb), ((pi >> 1) & 1) ^ 1, abort_flag, g.status);
          if (!ok) break;
          tc_fence_after();
          for (int h1 = 0; h1 < g.H1; ++h1, ++qi) {
            const int st = qi & 1;
            ok = warp_wait(bar(FULL_A + st), (qi >> 1) & 1, abort_flag, g.status);
            if (!KRY && ok) ok = warp_wait(bar(FULL_Y), qi & 1, abort_flag, g.status);
            if (!ok) break;
            tc_fence_after();
            const uint32_t tileA = sA + st * kStageB;
            const uint32_t bL = sL + buf * kLBlkB;
            const uint32_t bR = sR + (buf * 2 + h1) * kRBlkB;
            const int slotL = a * g.H1 + h1;
            const uint32_t dL = tmem + (uint32_t)g.colL + (uint32_t)(slotL * NL);
            const uint32_t dR = KRY ? tmem + (uint32_t)g.colR + yb * (uint32_t)ell
                                    : tmem + (uint32_t)g.colR + rb * (uint32_t)(g.T3 * ell) + (uint32_t)(b * ell);
            const uint64_t aL0 = make_desc(tileA, kS4, kS1), aR0 = make_desc(tileA, kS1, kS4);
            // Khatri-Rao: the fixed mode-1 block of this half of i_1, into the
            // super-plane's D_Y; dense: the G planes' R_3 blocks into the tile's
            const uint64_t bL0 = make_desc(bL, kS1, kS4), bR0 = make_desc(bR, kS1, kS4),
                           bY0 = make_desc(KRY ? sY + (uint32_t)(h1 * kRBlkB) : sY, kS1, kS4);
            const uint32_t dYq = KRY ? tmem + (uint32_t)kTmemY + yb * colYB : dY;
            const uint32_t accL0 = (initL >> slotL) & 1u,
                           accR0 = KRY ? (h1 > 0 ? 1u : 0u) : (initR >> b) & 1u,
                           accY0 = KRY ? (h1 > 0 ? 1u : 0u) : (initY ? 1u : 0u);
            if (elect_one()) {
              // the R_3 products first, so that the RNG warps can refill their
              // single buffer while the rest of the quarter runs
#pragma unroll
              for (int ks = 0; ks < 8; ++ks)
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                  const uint64_t po = (uint64_t)((part * kTileB) >> 4);
                  mma16_ss(dYq, aR0 + po + (uint64_t)((ks * 2 * kS1) >> 4), bY0 + (uint64_t)((ks * 2 * kS1) >> 4),
                              idY, accY0 | (uint32_t)(ks | part));
                }
              if (!KRY) mma_commit(bar(EMPTY_Y));
#pragma unroll
              for (int ks = 0; ks < 8; ++ks)
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                  const uint64_t po = (uint64_t)((part * kTileB) >> 4);
                  mma16_ss(dL, aL0 + po + (uint64_t)((ks * 2 * kS4) >> 4), bL0 + (uint64_t)((ks * 2 * kS1) >> 4), idL,
                              accL0 | (uint32_t)(ks | part));
                  mma16_ss(dR, aR0 + po + (uint64_t)((ks * 2 * kS1) >> 4), bR0 + (uint64_t)((ks * 2 * kS1) >> 4), idR,
                              accR0 | (uint32_t)(ks | part));
                }
              mma_commit(bar(EMPTY_A + st));
            }
            __syncwarp();
            initL |= 1u << slotL;
            initR |= 1u << b;
            initY = true;
          }
          if (ok) {
            if (elect_one()) {
              mma_commit(bar(EMPTY_L + buf));
              if (KRY) mma_commit(bar(TMY_FULL + yb));
            }
            __syncwarp();
          }
        }
      if (ok && !KRY) {
        if (elect_one()) mma_commit(bar(TMR_FULL + rb));
        __syncwarp();
      }
    }
    if (!KRY && ok && cur_tl >= 0) {
      if (elect_one()) mma_commit(bar(TML_FULL));
      __syncwarp();
    }
    if (elect_one()) mma_commit(bar(DRAIN));
    __syncwarp();
    const long long t0 = clock64();
    while (!mbar_try(bar(DRAIN), 0) && clock64() - t0 < kWaitCycles) {
    }
    __syncwarp();
  } else if (warp < kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int lrow = warp * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
    const uint32_t colYB = (uint32_t)(KRY ? ell : g.G * ell);
    // L slots of kL block [kL0, kL0 + nA): S_1 (rows i_1, pre-summed over the
    // kL values) and S_2 (rows i_1 + n_1 kL).
    // Khatri-Rao: slot a is drained right after the run's last super-plane
    // of kL0 + a (its MMAs are complete once that super-plane's D_Y is), so
    // the drain overlaps the rest of the tile and the MMA warp, which waits
    // for a slot only before its first MMA of the next run, never stalls on
    // it; S_1 is summed in shared memory over every run of the CTA and added
    // to the sketch once at its end (its rows are the same for every run).
    auto drain_slot = [&](int64_t kL, int a) {
      float* s1p = reinterpret_cast<float*>(sm + kOffS1);
      for (int h1 = 0; h1 < g.H1; ++h1) {
        float v[ell];
        tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)g.colL + (uint32_t)((a * g.H1 + h1) * NL), v);
#pragma unroll
        for (int j = 0; j < ell; ++j) s1p[(h1 * ell + j) * 128 + lrow] += v[j];
        tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)g.colL + (uint32_t)((a * g.H1 + h1) * NL + ell), v);
        // S_2: four-wide FP32 reductions into the row-major staging copy
        // (FP64 atomics here cost the launch ~25 us of drain)
        red_add_row<ell>(g.s2stage + (h1 * 128 + lrow + g.n1 * kL) * ell, v);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(TML_EMPTY + a));
    };
    // Dense: half by half (the R_3 area holds no room for S_1's sums), after
    // the run's last tile, the slots handed back at the end.
    auto flush_L = [&](int64_t kL0, int nA, uint32_t lf) -> bool {
      if (!mbar_wait(bar(TML_FULL), lf & 1, abort_flag, g.status)) return false;
      tc_fence_after();
      const SkTc& sk1 = s_col[0];
      double* dst1 = g.ws + sk1.off;
      {
        for (int h1 = 0; h1 < g.H1; ++h1) {
          const int64_t i1 = h1 * 128 + lrow;
          float acc[ell];
#pragma unroll
          for (int j = 0; j < ell; ++j) acc[j] = 0.0f;
          for (int a = 0; a < nA; ++a) {
            float v[ell];
            tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)g.colL + (uint32_t)((a * g.H1 + h1) * NL), v);
#pragma unroll
            for (int j = 0; j < ell; ++j) acc[j] += v[j];
            tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)g.colL + (uint32_t)((a * g.H1 + h1) * NL + ell), v);
            float* st2 = g.s2stage + (i1 + g.n1 * (kL0 + a)) * ell;
#pragma unroll
            for (int j = 0; j < ell; ++j) atomicAdd(st2 + j, v[j]);
          }
#pragma unroll
          for (int j = 0; j < ell; ++j) atomicAdd(dst1 + i1 + sk1.rows * j, (double)acc[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
          for (int a = 0; a < nA; ++a) mbar_arrive(bar(TML_EMPTY + a));
      }
      return true;
    };
    uint32_t lf = 0, ti_n = 0;
    int64_t cur_tl = -1, cur_kL0 = 0;
    int cur_nA = 0;
    bool ok = true;
    // composite row of this lane: slice kk of plane gl of the super-plane
    const int gl = lrow >> lc, kk = lrow & cmask;
    constexpr int kYTiles = 16;   // dense: tiles per R_3 flush
    constexpr int kYSuper = 16;   // Khatri-Rao: super-planes per R_3 flush
    int ytiles = 0;
    uint32_t spn = 0;             // super-planes handed over by the MMA warp so far
    float yacc[ell];
#pragma unroll
    for (int j = 0; j < ell; ++j) yacc[j] = 0.0f;
    float* racc = reinterpret_cast<float*>(sm + kOffR2);   // Khatri-Rao: [column][lane]
    if constexpr (KRY)
      for (int j = 0; j < ell; ++j) racc[j * 128 + lrow] = 0.0f;
    // Khatri-Rao: the plane's mode-3 and mode-2 factor rows, loaded one
    // super-plane ahead of their use
    float4 ef3[ell / 4], ef2[ell / 4];
    const float* ektab = KRY ? reinterpret_cast<const float*>(reinterpret_cast<const char*>(g.ws) + kr3->kr_tab) : nullptr;
    const int64_t eo2 = KRY ? kr3->kr_off[1] : 0, eo3 = KRY ? kr3->kr_off[2] : 0, elp = KRY ? kr3->kr_lp : 0;
    auto e_load = [&](int64_t kL, int64_t kR0) {
      const float4* f3 = reinterpret_cast<const float4*>(ektab + eo3 + (kR0 + gl) * elp);
      const float4* f2 = reinterpret_cast<const float4*>(ektab + eo2 + kL * elp);
#pragma unroll
      for (int q = 0; q < ell / 4; ++q) {
        ef3[q] = f3[q];
        ef2[q] = f2[q];
      }
    };
    if (KRY && t_beg < ntiles) {
      const TileInfo t0 = tile_info(g, t_beg);
      e_load(t0.kL0, t0.kRg0 * g.G);
    }
    // R_3 rows first + kk: at c = 16 lanes l and l + 16 hold the same slice of
    // two planes and are summed first
    auto flush_Y = [&]() {
      const SkTc& sk = s_row[1];
      double* dst = g.ws + sk.off;
      float y[ell];
#pragma unroll
      for (int j = 0; j < ell; ++j) {
        y[j] = yacc[j];
        if constexpr (C == 16) y[j] += __shfl_down_sync(0xffffffffu, y[j], 16);
        yacc[j] = 0.0f;
      }
      if (C != 16 || lane < 16) {
        const int64_t row = sk.hstride * (g.first + kk);
#pragma unroll
        for (int j = 0; j < ell; ++j) atomicAdd(dst + row + sk.rows * j, (double)y[j]);
      }
    };
    for (int64_t t = t_beg; t < ntiles && ok && !*abort_flag; ++t, ++ti_n) {
      const TileInfo tinf = tile_info(g, t);
      const int64_t tl = l_group(g, t);
      if (tl != cur_tl) {
        if (cur_tl >= 0) {
          if (!KRY) ok = flush_L(cur_kL0, cur_nA, lf);
          ++lf;
          if (!ok) break;
        }
        cur_tl = tl;
        cur_kL0 = tinf.kL0;
        cur_nA = tinf.nA;
      }
      if constexpr (KRY) {
        // Khatri-Rao R_3, super-plane by super-plane in the MMA's order: the
        // lane's row of D_Y (plane gl, slice kk) times the rounded product of
        // the plane's mode-3 and mode-2 rows, summed into the lane's R_3 row
        bool yok = true;
        // the run's last tile: each kL slot is drained after its last super-plane
        const bool run_end = t + 1 >= ntiles || l_group(g, t + 1) != tl;
        for (int b = 0; b < tinf.nB && yok; ++b) {
          for (int a = 0; a < tinf.nA; ++a, ++spn) {
            const uint32_t yb = spn & 1;
            if (!mbar_wait(bar(TMY_FULL + yb), (spn >> 1) & 1, abort_flag, g.status)) {
              yok = false;
              break;
            }
            tc_fence_after();
            {
              float y[ell];
              tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)kTmemY + yb * colYB, y);
              // the plane's rows of the mode-3 and mode-2 factors (i_3 = kR_g,
              // i_2 = kL, loaded during the previous super-plane); product in
              // the row sketch's decreasing mode order, rounded to the operand
              // type (the column scale)
#pragma unroll
              for (int q = 0; q < ell / 4; ++q) {
                yacc[4 * q] = fmaf(y[4 * q], round_op16<F16>(__fmul_rn(ef3[q].x, ef2[q].x)), yacc[4 * q]);
                yacc[4 * q + 1] = fmaf(y[4 * q + 1], round_op16<F16>(__fmul_rn(ef3[q].y, ef2[q].y)), yacc[4 * q + 1]);
                yacc[4 * q + 2] = fmaf(y[4 * q + 2], round_op16<F16>(__fmul_rn(ef3[q].z, ef2[q].z)), yacc[4 * q + 2]);
                yacc[4 * q + 3] = fmaf(y[4 * q + 3], round_op16<F16>(__fmul_rn(ef3[q].w, ef2[q].w)), yacc[4 * q + 3]);
              }
            }
            {  // the next super-plane's factor rows go out
              int64_t kLn, kR0n;
              if (next_super_plane(g, ntiles, t, a, b, tinf, kLn, kR0n)) e_load(kLn, kR0n);
            }
            {
              // the super-plane's R_2 partial (rows of the lane's slice), summed
              // over the kL values of this kR group
              float r[ell];
              tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)g.colR + yb * (uint32_t)ell, r);
#pragma unroll
              for (int j = 0; j < ell; ++j) racc[j * 128 + lrow] += r[j];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(TMY_EMPTY + yb));
            if (run_end && b == tinf.nB - 1) drain_slot(tinf.kL0 + a, a);
            if (++ytiles == kYSuper) {
              flush_Y();
              ytiles = 0;
            }
          }
          if (!yok) break;
          // R_2 rows kR_g + n_3 (first + kk) of this kR group
          const SkTc& sk = s_row[0];
          double* dst = g.ws + sk.off;
          const int64_t row = ((tinf.kRg0 + b) * g.G + gl) + sk.hstride * (g.first + kk);
#pragma unroll
          for (int j = 0; j < ell; ++j) {
            atomicAdd(dst + row + sk.rows * j, (double)racc[j * 128 + lrow]);
            racc[j * 128 + lrow] = 0.0f;
          }
        }
        if (!yok) break;
        continue;
      }
      const uint32_t rb = ti_n & 1;
      if (!mbar_wait(bar(TMR_FULL + rb), (ti_n >> 1) & 1, abort_flag, g.status)) break;
      tc_fence_after();
      // R_2: rows kR_g + n_3 (first + kk), one slot per kR group of the tile
      {
        const SkTc& sk = s_row[0];
        double* dst = g.ws + sk.off;
        for (int b = 0; b < tinf.nB; ++b) {
          float v[ell];
          tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)g.colR + rb * (uint32_t)(g.T3 * ell) + (uint32_t)(b * ell), v);
          const int64_t row = ((tinf.kRg0 + b) * g.G + gl) + sk.hstride * (g.first + kk);
#pragma unroll
          for (int j = 0; j < ell; ++j) atomicAdd(dst + row + sk.rows * j, (double)v[j]);
        }
      }
      // R_3 (dense): the diagonal block of D_Y (row group gl, column block gl).
      // Every tile adds to the same c rows (first + kk), so the lane keeps its
      // row's sum over the tiles of its run and adds it to the sketch once per
      // kYTiles tiles (an FP32 chain of at most that many tile sums): the
      // rows are few, and per-tile atomics would all meet at them.
      if constexpr (!KRY) {
        const int g_lo = (warp * 32) >> lc;  // first plane of this warp's lanes
        float y[ell];
        tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)kTmemY + rb * colYB + (uint32_t)(g_lo * ell), y);
        if constexpr (C == 16) {
          float v1[ell];
          tmem_ld_cols<ell>(tmem + lane_addr + (uint32_t)kTmemY + rb * colYB + (uint32_t)((g_lo + 1) * ell), v1);
          // lanes 16..31 belong to the warp's second plane
#pragma unroll
          for (int j = 0; j < ell; ++j) y[j] = lane >= 16 ? v1[j] : y[j];
        }
#pragma unroll
        for (int j = 0; j < ell; ++j) yacc[j] += y[j];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(TMR_EMPTY + rb));
      if (!KRY && ++ytiles == kYTiles) {
        flush_Y();
        ytiles = 0;
      }
    }
    if (!KRY && ok && cur_tl >= 0 && !*abort_flag) flush_L(cur_kL0, cur_nA, lf);
    if (ok && !*abort_flag && ytiles > 0) flush_Y();
    if constexpr (KRY) {
      // S_1 rows i_1: the lane's sums over every run of the CTA
      if (ok && !*abort_flag) {
        const SkTc& sk1 = s_col[0];
        const float* s1p = reinterpret_cast<const float*>(sm + kOffS1);
        for (int h1 = 0; h1 < g.H1; ++h1)
#pragma unroll
          for (int j = 0; j < ell; ++j)
            atomicAdd(g.ws + sk1.off + h1 * 128 + lrow + sk1.rows * j, (double)s1p[(h1 * ell + j) * 128 + lrow]);
      }
    }

  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
  }
}

// Staged R_3 blocks (dense test matrices): block (h, kL, kR) holds the 128
// rows 128 h + k + n_1 (kL + WL kR) of Psi_3 as the K-major core-matrix
// image the MMA reads (BF16 or FP16), kR fastest.
__global__ void slab_ytab_kernel(const SlabArgs g) {
  const SkTc sk = g.row[1];
  const int qps = g.ell / 4;
  const int64_t blkB = (int64_t)(g.ell / 8) * kS4;
  const int64_t nblk = (int64_t)g.H1 * g.WL * g.WR;
  const int64_t total = nblk * 16 * qps * 8;
  char* tab = reinterpret_cast<char*>(g.ws) + g.ytab;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r8 = (int)(e & 7);
    int64_t rest = e >> 3;
    const int q = (int)(rest % qps);
    rest /= qps;
    const int kg = (int)(rest & 15);
    const int64_t blk = rest >> 4;  // (h WL + kL) WR + kR
    const int64_t kR = blk % g.WR, hl = blk / g.WR;
    const int64_t kL = hl % g.WL, h = hl / g.WL;
    const int64_t k = 128 * h + 8 * kg + r8;
    const float4 z = normals4_f32(g.seed, (uint32_t)sk.sid, (uint64_t)(k + g.n1 * (kL + g.WL * kR)), (uint32_t)q);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    char* bp = tab + blk * blkB;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * q + u;
      *reinterpret_cast<uint16_t*>(bp + kg * kS1 + (j >> 3) * kS4 + (j & 7) * 16 + r8 * 2) =
          g.f16 ? op16_bits<true>(zz[u]) : op16_bits<false>(zz[u]);
    }
  }
}

constexpr int kFoldEvery = 16;  // slab launches between folds of S_2's FP32 staging

// S_2 += the launch's FP32 staging (row-major, l floats a row), which is
// cleared for the next launch; four columns of a row a thread, consecutive
// threads on consecutive rows (coalesced FP64 columns).
__global__ void s2_fold_kernel(double* __restrict__ s2, float* __restrict__ stage, int64_t rows, int ell) {
  const int qpr = ell / 4;
  float4* f = reinterpret_cast<float4*>(stage);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * qpr; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % rows;
    const int q = (int)(e / rows);
    const float4 v = f[r * qpr + q];
    double* d = s2 + r + rows * (4 * q);
    d[0] += (double)v.x;
    d[rows] += (double)v.y;
    d[2 * rows] += (double)v.z;
    d[3 * rows] += (double)v.w;
    f[r * qpr + q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Staged R_2 blocks: block (v, h) holds the 128 rows 128 h + k + n_1 v of the
// test matrix (v = kL) as the K-major core-matrix image the MMA reads (BF16
// or FP16).
__global__ void slab_table_kernel(const SlabArgs g, int64_t nv) {
  const SkTc sk = g.row[0];
  const int qps = g.ell / 4;
  const int64_t blkB = (int64_t)(g.ell / 8) * kS4;
  const int64_t total = nv * g.H1 * 16 * qps * 8;
  char* tab = reinterpret_cast<char*>(g.ws) + sk.tab;
  const DevSketch* kr = kr_of(g.ws, sk.kr);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r8 = (int)(e & 7);
    int64_t rest = e >> 3;
    const int q = (int)(rest % qps);
    rest /= qps;
    const int kg = (int)(rest & 15);
    rest >>= 4;
    const int h = (int)(rest % g.H1);
    const int64_t v = rest / g.H1;
    const int64_t k = 128 * h + 8 * kg + r8;
    const float4 z = tm_quad_f32(g.ws, kr, g.seed, (uint32_t)sk.sid, (uint64_t)(k + g.n1 * v), (uint32_t)q);
    const float zz[4] = {z.x, z.y, z.z, z.w};
    char* blk = tab + (v * g.H1 + h) * blkB;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * q + u;
      *reinterpret_cast<uint16_t*>(blk + kg * kS1 + (j >> 3) * kS4 + (j & 7) * 16 + r8 * 2) =
          g.f16 ? op16_bits<true>(zz[u]) : op16_bits<false>(zz[u]);
    }
  }
}

}  // namespace slab

// Shape rules of the slab kernel; fills the launch arguments when it applies.
bool plan_slab(const Plan& P, int item, int64_t count, slab::SlabArgs* out) {
  const DevItem& it = plan_items_host(&P)[item];
  if ((it.prec != TT_PREC_BF16 && it.prec != TT_PREC_FP16) || it.x_f64 || it.sided1 || it.passes != 1) return false;
  if (it.d != 4 || it.nsk != 4) return false;
  if (it.n[0] != 128 && it.n[0] != 256) return false;
  if (count != 16 && count != 32 && count != 64) return false;
  const int G = (int)(128 / count);
  const DevSketch* sks = plan_sketches_host(&P);
  const DevSketch &s1 = sks[it.sk0], &s2 = sks[it.sk0 + 1], &r2 = sks[it.sk0 + 2], &r3 = sks[it.sk0 + 3];
  if (s1.type != SK_COL || s1.k != 1 || s2.type != SK_COL || s2.k != 2 || r2.type != SK_ROW || r2.k != 2 ||
      r3.type != SK_ROW || r3.k != 3)
    return false;
  const int ell = s1.width;
  if ((ell != 8 && ell != 16) || s2.width != ell || r2.width != ell || r3.width != ell) return false;
  if (it.s2stage_doubles * 2 < s2.rows * s2.width) return false;  // the FP32 staging of S_2
  slab::SlabArgs g;
  memset(&g, 0, sizeof(g));
  g.n1 = it.n[0];
  g.W = it.W;
  g.WL = it.n[1];
  g.WR = it.n[2];
  if (g.WR % G) return false;
  g.WRg = g.WR / G;
  g.Nd1 = it.N[3];
  g.H1 = (int)(it.n[0] / 128);
  g.ell = ell;
  g.c = (int)count;
  g.lc = count == 16 ? 4 : count == 32 ? 5 : 6;
  g.G = G;
  // tensor memory, dense test matrices: D_Y (two buffers of G l columns, one
  // a tile), L slots (T2 H1 x 2l: S_1 | S_2), R_2 (two buffers of T3 l, one a
  // tile); every accumulator sees at most 256 MMAs (a tile's D_Y T2 T3 H1 x
  // 16, an R_2 slot T2 H1 x 16).  Khatri-Rao: D_Y and R_2 (l columns each)
  // in two buffers, one a super-plane (H1 x 16 MMAs), and the L slots.
  g.kry = r3.kr_nm ? 1 : 0;
  const int ycols = g.kry ? ell : G * ell;
  auto fits = [&](int t2, int t3) {
    if (g.kry) return 2 * ycols + t2 * g.H1 * 2 * ell + 2 * ell <= 512 && t2 * g.H1 * 16 <= kMaxChainL;
    return 2 * ycols + t2 * g.H1 * 2 * ell + 2 * t3 * ell <= 512 && t2 * g.H1 * 16 <= kMaxChainL &&
           t2 * t3 * g.H1 * 16 <= kMaxChainL;
  };
  // Each CTA takes a contiguous run of tiles, so the launch lasts as long as
  // the CTA with the most super-planes: pick the shape that minimises that,
  // weighted by the per-tile cost; ties: the larger T2.  Dense: the R_2 flush
  // traffic (2048 FP64 atomics per kR group and tile, about 1 / T2 of a
  // super-plane's own cost).  Khatri-Rao: R_2 is drained per super-plane
  // whatever the shape, and a tile costs about 0.14 of a super-plane
  // (measured on 1 GiB slabs of the 256^4 tensor: T2 = 5, 7 and 2 gave 0.754,
  // 0.746 and 0.689 of HBM); below four kL values a tile the L slots' drain
  // at every run change stalls the MMAs, so those shapes are left out.
  const int64_t sms = device_sm_count();
  int T2 = 0, T3 = 0;
  double best = 1e300;
  for (int t2 = 1; t2 <= 8; ++t2)
    for (int t3 = 1; t3 <= 8; ++t3) {
      if (t2 > g.WL || t3 > g.WRg || !fits(t2, t3)) continue;
      if (g.kry && t2 < std::min<int64_t>(4, g.WL)) continue;
      const int64_t tiles = ((g.WL + t2 - 1) / t2) * ((g.WRg + t3 - 1) / t3);
      const double cost = (double)((tiles + sms - 1) / sms * t2 * t3) * (1.0 + (g.kry ? 0.14 : 0.5) / t2);
      if (cost < best || (cost == best && t2 > T2)) {
        best = cost;
        T2 = t2;
        T3 = t3;
      }
    }
  if (T2 == 0) return false;
  g.T2 = T2;
  g.T3 = T3;
  g.colL = 2 * ycols;
  g.colR = g.colL + T2 * g.H1 * 2 * ell;
  g.tilesL = (g.WL + T2 - 1) / T2;
  g.tilesR = (g.WRg + T3 - 1) / T3;
  // L slots: accumulating MMAs per slot and tile T3 x 16 (T3 super-planes x
  // 8 k-steps x hi, lo); TT_FLAG_SHORT_CHAINS: runs of kMaxChainS MMAs keep
  // S_2's FP32 chains short (its accumulation error enters the middle core
  // directly)
  g.runL = std::max<int64_t>(1, (it.short_chains ? kMaxChainS : kMaxChainL) / (T3 * 16));
  g.col[0] = SkTc{s1.rows, s1.off, s1.wdiv, s1.hstride, -1, s1.stream_id, s1.kr_nm ? it.sk0 : -1};
  g.col[1] = SkTc{s2.rows, s2.off, s2.wdiv, s2.hstride, -1, s2.stream_id, s2.kr_nm ? it.sk0 + 1 : -1};
  g.row[0] = SkTc{r2.rows, r2.off, r2.wdiv, r2.hstride, -1, r2.stream_id, r2.kr_nm ? it.sk0 + 2 : -1};
  g.row[1] = SkTc{r3.rows, r3.off, r3.wdiv, r3.hstride, -1, r3.stream_id, r3.kr_nm ? it.sk0 + 3 : -1};
  // the staged R_2 blocks live in the plane kernel's staging area (one 128-row
  // block per kL and half of i_1)
  const int64_t blk = (int64_t)(ell / 8) * kS4;
  if (it.tctab_doubles * 8 < g.WL * g.H1 * blk) return false;
  g.row[0].tab = it.off_tctab * 8;
  g.tab_tx = (uint32_t)(g.H1 * blk);
  g.seed = it.seed;
  g.f16 = it.prec == TT_PREC_FP16 ? 1 : 0;
  g.xscale = g.f16 ? it.xscale : 1.0f;
  *out = g;
  return true;
}

static bool slab_kernel_launchable() {
  static int ok = -1;
  if (ok < 0) {
    cudaFuncAttributes fa, fb;
    int dev = 0, smem_optin = 0;
    ok = cudaFuncGetAttributes(&fa, slab::sketch_slab_kernel<16, 16, false, false>) == cudaSuccess &&
         cudaFuncGetAttributes(&fb, slab::sketch_slab_kernel<8, 16, true, false>) == cudaSuccess &&
         cudaGetDevice(&dev) == cudaSuccess &&
         fa.maxThreadsPerBlock >= slab::Roles<false>::threads && fb.maxThreadsPerBlock >= slab::Roles<true>::threads &&
         cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
         smem_optin >= slab::kSmemBytes;
  }
  return ok == 1;
}

}  // namespace tc

bool use_slab_kernel(const Plan& P, int item, int64_t count) { return slab_chunk(P, item, count) > 0; }

// Slices per slab-kernel launch for an accumulate of `count` slices: count
// itself (16, 32 or 64), or 64 for a Khatri-Rao plan's longer slabs (a
// multiple of 64: those shapes would otherwise go to the plane kernel, which
// does not take Khatri-Rao test matrices); 0 when the slab kernel does not apply.
int64_t slab_chunk(const Plan& P, int item, int64_t count) {
  tc::slab::SlabArgs g;
  if (tc::plan_slab(P, item, count, &g)) return count;
  if (count > 64 && count % 64 == 0 && tc::plan_slab(P, item, 64, &g) && g.kry) return 64;
  return 0;
}

static cudaError_t launch_slab_one(const Plan& P, int item, const void* X, int64_t first, int64_t count, void* ws,
                                   cudaStream_t st);

cudaError_t launch_sketch_slab(const Plan& P, int item, const void* X, int64_t first, int64_t count, void* ws,
                               cudaStream_t st) {
  const int64_t chunk = slab_chunk(P, item, count);
  if (chunk <= 0) return cudaErrorNotSupported;
  const int64_t nd1 = plan_items_host(&P)[item].N[3];
  for (int64_t a = 0; a < count; a += chunk) {
    const cudaError_t e =
        launch_slab_one(P, item, reinterpret_cast<const float*>(X) + a * nd1, first + a, chunk, ws, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t launch_slab_one(const Plan& P, int item, const void* X, int64_t first, int64_t count, void* ws,
                                   cudaStream_t st) {
  tc::slab::SlabArgs g;
  if (!tc::plan_slab(P, item, count, &g)) return cudaErrorNotSupported;
  if (!tc::slab_kernel_launchable()) return cudaErrorNotSupported;
  g.X = (const float*)X;
  g.ws = (double*)ws;
  g.status = reinterpret_cast<int*>((char*)ws + kStatusOff);
  g.first = first;
  const DevItem& it = plan_items_host(&P)[item];
  g.s2stage = reinterpret_cast<float*>((double*)ws + it.off_s2stage);
  g.ytab = (!g.kry && it.ytab_doubles > 0) ? it.off_ytab * 8 : -1;
  using KernelFn = void (*)(tc::slab::SlabArgs);
  using namespace tc::slab;
#define TT_SLAB_K(E, F)                                                                                        \
  {{sketch_slab_kernel<E, 16, false, F>, sketch_slab_kernel<E, 32, false, F>, sketch_slab_kernel<E, 64, false, F>}, \
   {sketch_slab_kernel<E, 16, true, F>, sketch_slab_kernel<E, 32, true, F>, sketch_slab_kernel<E, 64, true, F>}}
  const KernelFn kernels[2][2][2][3] = {{TT_SLAB_K(8, false), TT_SLAB_K(16, false)},
                                        {TT_SLAB_K(8, true), TT_SLAB_K(16, true)}};
#undef TT_SLAB_K
  static bool attr_set = false;
  if (!attr_set) {
    for (int f = 0; f < 2; ++f)
      for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 2; ++k)
          for (int j = 0; j < 3; ++j) {
            const cudaError_t e = cudaFuncSetAttribute(kernels[f][i][k][j],
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
            if (e != cudaSuccess) return e;
          }
    attr_set = true;
  }
  // the R_2 blocks (rows i_1 + n_1 kL) are the same for every slab: staged by
  // the first launch of a decomposition
  bool& ready = plan_stream_tables(const_cast<Plan&>(P));
  if (!ready) {
    const int64_t total = g.WL * g.H1 * 16 * (g.ell / 4) * 8;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8LL * device_sm_count());
    count_launch();
    tc::slab::slab_table_kernel<<<blocks, 256, 0, st>>>(g, g.WL);
    // the R_3 blocks of dense test matrices, likewise once per decomposition
    if (g.ytab >= 0) {
      count_launch();
      tc::slab::slab_ytab_kernel<<<(unsigned)(8 * device_sm_count()), 256, 0, st>>>(g);
    }
    ready = true;
  }
  const int64_t ntiles = g.tilesL * g.tilesR;
  const int grid = (int)std::min<int64_t>(ntiles, device_sm_count());
  count_launch();
  const KernelFn k = kernels[g.f16][g.ell == 16 ? 1 : 0][g.kry][g.c == 16 ? 0 : g.c == 32 ? 1 : 2];
  const int threads = g.kry ? tc::slab::Roles<true>::threads : tc::slab::Roles<false>::threads;
  k<<<grid, threads, tc::slab::kSmemBytes, st>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // S_2's FP32 staging is added into the FP64 sketch every kFoldEvery
  // launches (each adds about four CTA partials an entry, so the staged sums
  // hold at most ~64 FP32 terms: under 3e-7 relative, measured no change in
  // the 256^4 result) and before anything reads S_2
  if (++plan_pending_folds(const_cast<Plan&>(P)) >= tc::slab::kFoldEvery) return fold_s2_staging(P, item, ws, st);
  return cudaSuccess;
}

// S_2 += its FP32 staging, staging cleared (a no-op when nothing is pending).
cudaError_t fold_s2_staging(const Plan& P, int item, void* ws, cudaStream_t st) {
  int& pending = plan_pending_folds(const_cast<Plan&>(P));
  if (pending == 0) return cudaSuccess;
  const DevItem& it = plan_items_host(&P)[item];
  if (it.s2stage_doubles <= 0) {
    pending = 0;
    return cudaSuccess;
  }
  const DevSketch& s2 = plan_sketches_host(&P)[it.sk0 + 1];
  const int64_t n2 = s2.rows * s2.width;
  count_launch();
  tc::slab::s2_fold_kernel<<<(unsigned)std::min<int64_t>((n2 / 4 + 255) / 256, 8LL * device_sm_count()), 256, 0,
                             st>>>((double*)ws + s2.off, reinterpret_cast<float*>((double*)ws + it.off_s2stage),
                                   s2.rows, s2.width);
  pending = 0;
  return cudaGetLastError();
}

}  // namespace tts
