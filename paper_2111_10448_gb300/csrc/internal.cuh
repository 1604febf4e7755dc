// Internal declarations shared by the translation units of libttsketch.
//
// Notation follows the paper (Sec. 2.1, 3.2): X is column-major, N_k =
// n_1..n_k, M_k = n_{k+1}..n_d, d* = ceil(d/2).  Column sketches S_k = X_k
// Omega_k (k < d*, and k = d* in one-pass mode) and row sketches
// R_k = X_k^T Psi_k (k = d*..d-1).
//
// The sketch kernels see X as a stack of "planes" X(:, w, :) of size
// n_1 x n_d, w = (i_2..i_{d-1}) in [0, W), W = N_{d-1}/n_1.  For every
// sketch, the contribution of one plane is a plain product:
//   column sketch k: S_k[a + n_1 wlo, j] += sum_b X(a, w, b) Omega_k[whi + hs b, j]
//   row sketch k:    R_k[whi + hs b, j]  += sum_a X(a, w, b) Psi_k[a + n_1 wlo, j]
// with wlo = w mod (N_k/n_1), whi = w div (N_k/n_1), hs = N_{d-1}/N_k and b the
// global index of the last mode.  (For k = 1 the column sketch has wlo = 0;
// for k = d-1 the row sketch has whi = 0: these two collect every plane.)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/ttsketch.h"
#include <nvtx3/nvToolsExt.h>

namespace tts {

// Host-side NVTX range named after the C-ABI call that opens it, so that a
// timeline profiler shows plan building, sketching, finalisation and the
// backward as named spans (a few nanoseconds when no profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

constexpr int kMaxLev = 12;       // TSQR tree depth limit
constexpr int64_t kTsqrSmemMax = 200 * 1024;  // dynamic shared memory of a TSQR level block
constexpr int kTcGroupBytes = 2304;  // plane kernel: one 8-column group of a 128-row BF16 block image
constexpr int kMaxSk = TT_MAXD;   // sketches per item (d of them at most)

enum SkType : int { SK_COL = 0, SK_ROW = 1 };

// Status bits written on the device (workspace word 0).
enum : int { ST_RANK_CAP = 1, ST_RANK_DEFICIENT = 2, ST_TIMEOUT = 4, ST_NONFINITE = 8 };

struct DevSketch {
  int64_t rows;        // N_k (column) or M_k (row)
  int64_t off;         // FP64 sketch, column-major rows x width, element offset in ws
  int64_t wdiv;        // N_k / n_1
  int64_t hstride;     // N_{d-1} / N_k
  int type;            // SK_COL / SK_ROW
  int k;               // unfolding index, 1-based
  int width;           // l of this sketch
  int stream_id;       // Philox stream (k or 64 + k)
  int basis;           // 1: QR'd into an orthonormal basis; 0: one-pass middle sketch
  int item;            // owning item
  // ---- basis sketches: TSQR tree (level 0 is the sketch itself)
  int nlev;            // number of levels; level nlev-1 is the root (one block)
  int bl;              // rows per block at every level
  int rpad;            // padded rank (columns of the basis)
  int rank_slot;       // index into the rank array of this sketch's rank r_k
  int target_rank;     // fixed-rank mode target (already clamped)
  int rcap;            // min(N_k, M_k)
  int64_t lev_rows[kMaxLev];
  int64_t lev_nblk[kMaxLev];
  int64_t lev_mat[kMaxLev];   // level matrix (rows x width) offset; lev_mat[0] = off
  int64_t lev_beta[kMaxLev];  // nblk * width Householder scalars
  int64_t lev_z[kMaxLev];     // rows x rpad expansion buffer; lev_z[0] = the basis Q_k / P_k
  int64_t off_rt;      // CPQR R factor of the root R (width x width)
  int64_t off_q2;      // CPQR Q factor (width x width)
  int64_t off_piv;     // pivots (width ints, stored as int in a double slot area)
  int64_t gen_tab;     // generic tile kernel: byte offset (in the item's table area) of
                       // this sketch's staged test-matrix rows, -1: regenerated per tile
  int64_t sp_tab;      // small-plane kernel: byte offset of this sketch's staged
                       // test-matrix rows (BF16), -1 when it is generated per plane
  // ---- Khatri-Rao test matrix (TT_FLAG_KR; kr_nm = 0: dense Gaussian).  The
  // test-matrix row runs over kr_nm modes (kr_mode0, kr_mode0 + 1, ...; the
  // first fastest, kr_stride[t] = product of the sizes of the faster ones);
  // its entry is the product of one row of each mode's Gaussian factor,
  // staged per call in the workspace: factor t is kr_n[t] x kr_lp elements
  // (FP64 for FP64 plans, FP32 otherwise) at byte offset kr_tab + kr_off[t] *
  // element size.  The factors are multiplied in increasing mode order for a
  // column sketch and in decreasing order for a row sketch (kr_dec), so that
  // the mode a plane's rows vary in (the last for a column sketch, the first
  // for a row sketch) is always the final factor.
  int kr_nm, kr_mode0, kr_lp, kr_dec;
  // 1: the row sketch of X_{d-1} on a TF32 / BF16 path, evaluated mode by
  // mode (eq. (sketch_orig)): its entry is round(F_1(i_1, j)) times
  // round(F_{d-1}(i_{d-1}, j) ... F_2(i_2, j)), the rounded mode-1 factor in the
  // tensor-core product and the rounded product of the other rows as a
  // column scale of the partial sums
  int kr_mbm, kr_pad2_;
  int64_t kr_tab;
  int64_t kr_n[TT_MAXD];
  int64_t kr_off[TT_MAXD];
  int64_t kr_stride[TT_MAXD];
};

struct DevItem {
  int d, ds, passes, prec, x_f64, nsk, eps_mode;
  int sk0;                 // first sketch index in the sketch table
  int mid_sk;              // index of the one-pass middle sketch (-1 in two-pass)
  // The one-pass least-squares core: B = V^T G (V the basis of bond mbk, G the
  // test matrix of stream mstream), H = S_mid B^+, and core mcore takes H.
  // Two-sided: mbk = mcore = ds, mstream = ds (Omega_{d*}), S_mid = S_{d*};
  // one-sided (sided1): ds = d-1, mbk = d-1, mstream = 64 + d-1 (Psi_{d-1}),
  // S_mid = T_{d-1}^T, mcore = d.
  int sided1, mbk, mstream, mcore;
  int basis_of_k[TT_MAXD + 1];  // sketch index of the basis of unfolding k (1..d-1)
  int64_t n[TT_MAXD];
  int64_t N[TT_MAXD + 1];
  int64_t W;               // planes: N_{d-1} / n_1
  double eps;
  int rmax, p;
  uint64_t seed;
  int rpad[TT_MAXD + 1];
  int64_t core_off[TT_MAXD + 1];
  int64_t rank_off;        // first entry of this item's d+1 ranks in the rank array
  // one-pass middle core
  int64_t off_B, off_QB, off_RB, off_H;
  int lmid;
  // reconstruction interfaces
  int64_t off_L[TT_MAXD + 1];   // L_k, N_k x rpad_k (k = 1..ds)
  int64_t off_Rt[TT_MAXD + 2];  // Rt_k, rpad_{k-1} x M_{k-1} (k = ds+1..d)
  // backward
  int64_t off_bar;          // start of the backward scratch of this item
  int64_t off_sbar[TT_MAXD + 1];  // adjoint of each sketch (same layout as the sketch)
  int64_t off_qbar[TT_MAXD + 1];  // adjoint of each basis Q_k / P_k
  int64_t off_hbar;         // adjoint of H
  int64_t off_bbar;         // adjoint of B
  int64_t off_rr[TT_MAXD + 1];    // leading r x r block of the basis R factor (rpad x rpad)
  int64_t off_small;        // 4 x TT_MAXL^2 doubles of backward scratch (single-item plans)
  int diff;                 // TT_FLAG_DIFF: full interface chain reserved
  int64_t off_Lall[TT_MAXD + 1];  // left interfaces L_k, k = 1..d-1 (N_k x rpad_k)
  int64_t off_Rall[TT_MAXD + 2];  // right interfaces Rt_k, k = 2..d (rpad_{k-1} x M_{k-1})
  int64_t off_Y;            // max_k N_k x rpad_k
  int64_t off_tctab;        // plane kernel: staged test-matrix blocks shared by many planes
  int64_t tctab_doubles;    // its size (0 when the plane kernel cannot serve the item)
  int64_t off_sptab;        // small-plane kernel: staged test-matrix rows of the sketches
  int64_t sptab_doubles;    // its size (0 when the small-plane kernel cannot serve the item)
  int64_t off_gentab;       // generic tile kernel: staged test-matrix rows of the sketches whose
  int64_t gentab_doubles;   // rows repeat across planes (0: none)
  int64_t off_adjtab;       // tensor-core sketch adjoint: the sketch adjoints split into hi + lo in
  int64_t adjtab_doubles;   // the MMA type, every sketch's rows x lpad (0: that kernel does not apply)
  int64_t off_s2stage;      // slab kernel: FP32 staging of the mid sketch S_2 (rows x l floats), added
  int64_t s2stage_doubles;  // into S_2 after every launch (0: the slab kernel cannot serve the item)
  int64_t off_ytab;         // slab kernel, dense test matrices: Psi_3's 128-row blocks for every
  int64_t ytab_doubles;     // (half of i_1, kL, kR), generated once per decomposition (0: per quarter)
  int short_chains;         // TT_FLAG_SHORT_CHAINS: tcgen05 column-sketch accumulators flushed every
                            // kMaxChainS MMAs
  int x_scale_log2;         // FP16: s, the sketch kernels split X 2^s (0 for other precisions)
  float xscale;             // 2^s
};

struct Task {               // one block of one TSQR level (finalize)
  int sk;                   // sketch index
  int blk;                  // block index
  int lev;                  // level within the sketch's own tree (the launches are aligned
                            // so that every tree's root is in the last one)
};

// Device-resident tables, stored at the start of the workspace.
struct DevTables {
  int nitems, nsk;
  int64_t off_items, off_sketches;   // byte offsets from ws base
  int64_t off_tasks[kMaxLev];        // byte offsets of per-level task arrays
  int ntasks[kMaxLev];
  // batched sketch: item visiting order (largest first), the first tile of
  // each item in that order (nitems + 1, written per call) and the work counter
  int64_t off_border, off_bprefix, off_bcounter;
};

// Batched sketch launch: the workspace and one tensor pointer per item (by
// value, so that a captured launch needs nothing uploaded).
constexpr int kMaxBatchItems = 2048;
struct BatchLaunch {
  char* wsb;
  int64_t chunk;                       // tiles taken from the counter at a time
  int t3max;                           // small-plane kernel: largest kR values per block
  const void* X[kMaxBatchItems];
};
// Launch shape of the batched sketch (chosen by tt_plan_autotune).
struct BatchCfg {
  int ta;            // tile rows along i_1: 32 or 64
  int chunk;         // tiles per counter grab
  int ctas_per_sm;   // persistent CTAs per SM
};

// Byte offset of the status word inside the workspace, and of a copy of the
// ranks of item 0 (d+1 ints) that the backward reads.
constexpr int64_t kStatusOff = 0;
constexpr int64_t kRankCopyOff = 64;

// ---------------------------------------------------------------- host side
struct Plan;
const DevItem* plan_items_host(const Plan* p);
int plan_num_items(const Plan* p);
bool& plan_stream_tables(Plan& P);
int& plan_pending_folds(Plan& P);   // slab launches whose S_2 partials are still in the FP32 staging
cudaError_t fold_s2_staging(const Plan& P, int item, void* ws, cudaStream_t st);

// Kernel launchers (defined in the .cu files).
cudaError_t launch_sketch_f64(const Plan& P, int item, const void* X, int64_t first, int64_t count,
                              void* ws, cudaStream_t st);
cudaError_t launch_sketch_mixed(const Plan& P, int item, const void* X, int64_t first,
                                int64_t count, void* ws, cudaStream_t st);
bool mixed_tc_supported(const Plan& P, int item, int64_t count);
bool use_tc_kernel(const Plan& P, int item, int64_t count);
bool use_sp_kernel(const Plan& P, int item, int64_t count);
bool use_slab_kernel(const Plan& P, int item, int64_t count);
int64_t slab_chunk(const Plan& P, int item, int64_t count);
cudaError_t launch_sketch_slab(const Plan& P, int item, const void* X, int64_t first, int64_t count, void* ws,
                               cudaStream_t st);
// Fill the staged test-matrix rows of one sketch: entry (key, r, j), r < nr,
// j < lpad, at element (key nr + r) lpad + j of tab (BF16 or FP16, or FP32
// rounded to TF32, by prec), rows as the sketch's test matrix numbers them for
// the slab starting at `first` (column side) or for plane key (row side).
cudaError_t launch_rows_table(const DevSketch& d, int gsk, const char* wsb, uint64_t seed, int64_t first, int64_t n1,
                              int nr, int lpad, int64_t nkeys, char* tab, int prec, cudaStream_t st);
cudaError_t launch_sketch_sp(const Plan& P, int item, const void* X, int64_t first, int64_t count, void* ws,
                             cudaStream_t st);
bool sp_batched_eligible(const Plan& P, size_t* smem_out, int* lpad_out, int t3max = 4);
cudaError_t launch_sketch_sp_batched(const Plan& P, const void* const* X, const BatchCfg& cfg, void* ws,
                                     cudaStream_t st);
cudaError_t launch_finalize(const Plan& P, void* ws, double* cores, int* ranks, cudaStream_t st);
cudaError_t launch_reconstruct(const Plan& P, int item, const double* cores, void* Xt, int x_f64,
                               const void* Xcmp, int cmp_f64, double* out2, void* ws,
                               cudaStream_t st);
cudaError_t launch_reconstruct_backward(const Plan& P, int item, const double* cores,
                                        const void* dXt, int dx_f64, double* dcores, void* ws,
                                        cudaStream_t st);
cudaError_t launch_backward(const Plan& P, int item, const double* dcores, void* dX, void* ws,
                            cudaStream_t st);
cudaError_t launch_sketch_batched(const Plan& P, const void* const* X, const BatchCfg& cfg, void* ws,
                                  cudaStream_t st);
cudaError_t launch_sketch_f64_batched(const BatchLaunch& b, const BatchCfg& cfg, int lmax, cudaStream_t st);
cudaError_t launch_sketch_mma_batched(const BatchLaunch& b, const BatchCfg& cfg, bool f16, cudaStream_t st);
int64_t batched_tiles_f64(int64_t W, int64_t n1, int64_t cnt, int ta);
int64_t batched_tiles_mma(int64_t W, int64_t n1, int64_t cnt, int ta);
cudaError_t launch_finalize_mid_batched(const Plan& P, void* ws, const int* ranks, cudaStream_t st);
cudaError_t launch_batch_zero(const Plan& P, void* ws, cudaStream_t st);
cudaError_t launch_kr_tables(const Plan& P, int item, void* ws, cudaStream_t st);
// Terms of the MMA type that each FP64 sketch adjoint is split into for the
// tensor-core sketch adjoint: three capture the FP32 value (8 + 8 + 8 bits
// in BF16, 11 + 11 + 2 in TF32), so the products are as exact as the FP32
// accumulation.
constexpr int kAdjParts = 3;
bool adjoint_sp_eligible(const Plan& P, int item);
cudaError_t launch_adjoint_sp(const Plan& P, int item, void* dX, void* ws, cudaStream_t st);
cudaError_t launch_mid_b_mixed_batched(const Plan& P, void* ws, const int* ranks, cudaStream_t st);

int device_sm_count();
void count_launch(int n = 1);

}  // namespace tts
