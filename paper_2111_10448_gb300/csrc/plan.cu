// Host plan, workspace layout and the C ABI entry points of libttsketch.
//
// The plan follows the paper's PSTT2 (Sec. 3.2): split d* = ceil(d/2);
// column bases Q_k of X_k for k < d*, row bases P_k of X_k for k = d*..d-1
// (reading A1 of the design notes); in one-pass mode one extra column sketch
// S_{d*} = X_{d*} Omega_{d*} whose pseudo-inverse solve gives the middle core
// (eq. (3.3) applied to the middle unfolding; readings A2, A3).  Sketch
// widths are l_k = r_k + p (fixed ranks) or rmax + p (tolerance mode).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace tts {

struct Plan {
  std::vector<tt_problem> probs;
  std::vector<DevItem> items;
  std::vector<DevSketch> sketches;
  std::vector<Task> tasks[kMaxLev];
  int max_lev = 0;
  int64_t ws_doubles = 0;      // total workspace in doubles
  int64_t core_entries = 0;
  int rank_entries = 0;
  std::vector<unsigned char> blob;  // device tables (uploaded to ws + kTableOff)
  uint64_t id = 0;                  // process-unique plan id (workspace registry key)
  // streaming bookkeeping (single-item plans)
  std::vector<char> slab_seen;
  bool begun = false;
  bool stream_tables = false;        // staged tables of the slab kernel valid for this decomposition
  int pending_folds = 0;             // slab launches not yet folded from S_2's FP32 staging
  const void* stream_ws = nullptr;   // workspace of the streaming decomposition begun last
  const void* forward_ws = nullptr;  // workspace of the last completed forward call
  BatchCfg bcfg{64, 4, 4};  // batched sketch launch shape (tt_plan_autotune)
};

static constexpr int64_t kTableOff = 256;  // bytes

// Host log (TT_LOG set to anything but "0" in the environment): plan layouts
// and the sketch kernel of every accumulate, one line each on stderr.
static bool log_on() {
  static const int on = [] {
    const char* v = std::getenv("TT_LOG");
    return (v && *v && std::strcmp(v, "0") != 0) ? 1 : 0;
  }();
  return on != 0;
}
#define TT_LOGF(...)                               \
  do {                                             \
    if (log_on()) {                                \
      std::fprintf(stderr, "ttsketch: " __VA_ARGS__); \
      std::fputc('\n', stderr);                    \
    }                                              \
  } while (0)

// Workspace registry: for every workspace address a plan has used, which plan's
// tables it holds and whether it holds that plan's saved forward state (the
// state the backward reads).  A call of plan P on workspace W re-sends P's
// tables whenever W last held another plan's (or none), so plans can share a
// workspace in any order; a workspace that is freed and reallocated at the
// same address must be released first (tt_workspace_release).
namespace {
struct WsEntry {
  uint64_t plan_id;
  bool forward_valid;
};
std::mutex g_ws_mu;
std::unordered_map<const void*, WsEntry> g_ws;
std::atomic<uint64_t> g_next_plan_id{1};
}  // namespace

void plan_mark_forward(Plan* p, const void* ws, bool valid) {
  std::lock_guard<std::mutex> lock(g_ws_mu);
  auto it = g_ws.find(ws);
  if (it != g_ws.end() && it->second.plan_id == p->id) it->second.forward_valid = valid;
  p->forward_ws = valid ? ws : nullptr;
}


const DevItem* plan_items_host(const Plan* p) { return p->items.data(); }
const DevSketch* plan_sketches_host(const Plan* p) { return p->sketches.data(); }
int plan_num_items(const Plan* p) { return (int)p->items.size(); }
int plan_max_lev(const Plan* p) { return p->max_lev; }
int plan_ntasks(const Plan* p, int lev) { return lev < kMaxLev ? (int)p->tasks[lev].size() : 0; }
cudaError_t launch_twopass_mid(const Plan& P, const void* X, void* ws, double* cores, const int* ranks,
                               cudaStream_t st);

static int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Allocate `count` doubles in the workspace (256-byte aligned).
struct WsAlloc {
  int64_t top;  // in doubles
  int64_t take(int64_t count) {
    top = align_up(top, 32);
    const int64_t o = top;
    top += std::max<int64_t>(count, 1);
    return o;
  }
};

static tt_status validate(const tt_problem& q) {
  if (q.d < 2 || q.d > TT_MAXD) return TT_ERR_INVALID_ARG;
  for (int k = 0; k < q.d; ++k)
    if (q.n[k] < 1) return TT_ERR_INVALID_ARG;
  if (q.p < 1) return TT_ERR_INVALID_ARG;
  if (q.passes != 1 && q.passes != 2) return TT_ERR_INVALID_ARG;
  if (!(q.eps >= 0.0)) return TT_ERR_INVALID_ARG;
  if (q.x_dtype != TT_F32 && q.x_dtype != TT_F64) return TT_ERR_INVALID_ARG;
  if (q.prec != TT_PREC_FP64 && q.prec != TT_PREC_TF32 && q.prec != TT_PREC_BF16 && q.prec != TT_PREC_FP16)
    return TT_ERR_INVALID_ARG;
  if (q.prec == TT_PREC_FP16 && (q.x_scale_log2 < -100 || q.x_scale_log2 > 100)) return TT_ERR_INVALID_ARG;
  if (q.prec != TT_PREC_FP64 && q.x_dtype != TT_F32) return TT_ERR_UNSUPPORTED;
  if (q.eps > 0.0) {
    if (q.rmax < 1 || q.rmax + q.p > TT_MAXL) return TT_ERR_INVALID_ARG;
  } else {
    if (q.ranks[0] != 1 || q.ranks[q.d] != 1) return TT_ERR_INVALID_ARG;
    for (int k = 1; k < q.d; ++k)
      if (q.ranks[k] < 1) return TT_ERR_INVALID_ARG;
  }
  // total size must fit int64 comfortably
  double tot = 1.0;
  for (int k = 0; k < q.d; ++k) tot *= (double)q.n[k];
  if (tot > 9.0e15) return TT_ERR_INVALID_ARG;
  return TT_OK;
}

// Build the item (tables + workspace layout) of one problem.
static tt_status build_item(Plan& P, const tt_problem& q0, WsAlloc& ws, int64_t& core_top,
                            int& rank_top, bool single) {
  tt_problem q = q0;
  DevItem it;
  std::memset(&it, 0, sizeof(it));
  const int d = q.d;
  it.d = d;
  it.sided1 = (q.flags & TT_FLAG_ONESIDED) ? 1 : 0;
  if (it.sided1 && ((q.flags & TT_FLAG_DIFF) || !single)) return TT_ERR_UNSUPPORTED;
  const bool kr = (q.flags & TT_FLAG_KR) != 0;
  if (kr && !single) return TT_ERR_UNSUPPORTED;
  // split: d* = ceil(d/2) (two-sided); one-sided puts every basis on the column side
  it.ds = it.sided1 ? d - 1 : (d + 1) / 2;
  it.mbk = it.ds;
  it.mstream = it.sided1 ? 64 + d - 1 : it.ds;
  it.mcore = it.sided1 ? d : it.ds;
  it.passes = q.passes;
  it.prec = q.prec;
  it.x_scale_log2 = q.prec == TT_PREC_FP16 ? q.x_scale_log2 : 0;
  it.xscale = std::ldexp(1.0f, it.x_scale_log2);
  it.x_f64 = q.x_dtype == TT_F64;
  it.eps_mode = q.eps > 0.0;
  it.eps = q.eps;
  it.rmax = q.rmax;
  it.p = q.p;
  it.seed = q.seed;
  it.N[0] = 1;
  for (int k = 0; k < d; ++k) {
    it.n[k] = q.n[k];
    it.N[k + 1] = it.N[k] * q.n[k];
  }
  it.W = it.N[d - 1] / it.n[0];
  const int ds = it.ds;
  // ranks, padded ranks and widths
  int width[TT_MAXD + 1] = {0};
  it.rpad[0] = it.rpad[d] = 1;
  for (int k = 1; k < d; ++k) {
    const int64_t rcap = std::min(it.N[k], it.N[d] / it.N[k]);
    if (it.eps_mode) {
      it.rpad[k] = (int)std::min<int64_t>(q.rmax, rcap);
      width[k] = q.rmax + q.p;
    } else {
      const int r = (int)std::min<int64_t>(q.ranks[k], rcap);
      q.ranks[k] = r;
      it.rpad[k] = r;
      width[k] = r + q.p;
    }
    if (width[k] > TT_MAXL) return TT_ERR_INVALID_ARG;
  }
  it.lmid = width[it.mbk];
  P.probs.push_back(q);

  // sketches
  it.sk0 = (int)P.sketches.size();
  it.mid_sk = -1;
  auto add = [&](int type, int k, int basis) {
    DevSketch s;
    std::memset(&s, 0, sizeof(s));
    s.type = type;
    s.k = k;
    s.basis = basis;
    s.item = (int)P.items.size();
    s.width = width[k];
    s.rows = type == SK_COL ? it.N[k] : it.N[d] / it.N[k];
    s.wdiv = it.N[k] / it.n[0];
    s.hstride = it.N[d - 1] / it.N[k];
    s.stream_id = type == SK_COL ? k : 64 + k;
    s.off = ws.take(s.rows * s.width);
    s.rpad = basis ? it.rpad[k] : 0;
    s.target_rank = it.eps_mode ? it.rpad[k] : q.ranks[k];
    s.rcap = (int)std::min(it.N[k], it.N[d] / it.N[k]);
    s.rank_slot = k;
    P.sketches.push_back(s);
    return (int)P.sketches.size() - 1;
  };
  if (it.sided1) {
    for (int k = 1; k < d; ++k) it.basis_of_k[k] = add(SK_COL, k, 1);
    if (q.passes == 1) it.mid_sk = add(SK_ROW, d - 1, 0);  // T_{d-1}^T = X_{d-1}^T Psi_{d-1}
  } else {
    for (int k = 1; k < ds; ++k) it.basis_of_k[k] = add(SK_COL, k, 1);
    if (q.passes == 1) it.mid_sk = add(SK_COL, ds, 0);
    for (int k = ds; k < d; ++k) it.basis_of_k[k] = add(SK_ROW, k, 1);
  }
  it.nsk = (int)P.sketches.size() - it.sk0;
  // Khatri-Rao test matrices: one Gaussian factor per mode of each sketch's
  // rows (column sketch k: modes k+1..d; row sketch k: modes 1..k).  Factor
  // rows are padded to the widest sketch of the item rounded up to 16, the
  // widest column range any kernel reads (entries past a sketch's width are
  // zero).
  int kr_lp = 0;
  for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) kr_lp = std::max(kr_lp, (P.sketches[si].width + 15) / 16 * 16);
  for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) {
    DevSketch& s = P.sketches[si];
    s.kr_nm = 0;
    if (!kr) continue;
    s.kr_mode0 = s.type == SK_COL ? s.k + 1 : 1;
    s.kr_nm = s.type == SK_COL ? d - s.k : s.k;
    s.kr_lp = kr_lp;
    s.kr_dec = s.type == SK_ROW ? 1 : 0;
    s.kr_mbm = (q.prec != TT_PREC_FP64 && s.type == SK_ROW && s.k == d - 1 && s.k >= 2) ? 1 : 0;
    int64_t elems = 0, stride = 1;
    for (int t = 0; t < s.kr_nm; ++t) {
      s.kr_n[t] = it.n[s.kr_mode0 - 1 + t];
      s.kr_off[t] = elems;
      s.kr_stride[t] = stride;
      stride *= s.kr_n[t];
      elems += s.kr_n[t] * s.kr_lp;
    }
    const int64_t esz = q.prec == TT_PREC_FP64 ? 8 : 4;
    s.kr_tab = ws.take((elems * esz + 7) / 8) * 8;
  }

  // TSQR trees of the basis sketches
  for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) {
    DevSketch& s = P.sketches[si];
    if (!s.basis) continue;
    const int w = s.width;
    // Row blocks of 128 rows, or 4 l when that is more (a multiple of 32,
    // capped at 192 so that a root block and its l x l work matrices fit in
    // shared memory for l <= 64): each tree level shrinks the rows 3-8x, and a
    // block's QR -- a chain of FP64 steps on one SM -- stays short.  Widths up
    // to 16 take 256-row blocks: a level costs about its chain whatever the
    // rows, so fewer levels win (a 65536-row sketch of width 16: 256 leaf
    // blocks and three levels, 46 us less a 256^4 step than 128-row blocks'
    // four).
    const int bl = w <= 16 ? 256 : std::min(192, std::max(128, (4 * w + 31) / 32 * 32));
    if (8 * ((int64_t)(bl + 1) * w + 32 + 2 * TT_MAXL + 3LL * w * w) > kTsqrSmemMax) return TT_ERR_UNSUPPORTED;
    s.bl = bl;
    int64_t m = s.rows;
    int L = 0;
    while (true) {
      if (L >= kMaxLev) return TT_ERR_UNSUPPORTED;
      s.lev_rows[L] = m;
      s.lev_nblk[L] = (m + bl - 1) / bl;
      s.lev_mat[L] = (L == 0) ? s.off : ws.take(m * w);
      s.lev_beta[L] = ws.take(s.lev_nblk[L] * w);
      s.lev_z[L] = ws.take(m * s.rpad);
      if (s.lev_nblk[L] == 1) break;
      m = s.lev_nblk[L] * w;
      ++L;
    }
    s.nlev = L + 1;
    s.off_rt = ws.take((int64_t)w * w);
    s.off_q2 = ws.take((int64_t)w * w);
    s.off_piv = ws.take(w);
    P.max_lev = std::max(P.max_lev, s.nlev);
  }
  // cores and ranks
  for (int k = 1; k <= d; ++k) {
    it.core_off[k] = core_top;
    core_top += (int64_t)it.rpad[k - 1] * it.n[k - 1] * it.rpad[k];
  }
  it.rank_off = rank_top;
  rank_top += d + 1;
  // one-pass middle core
  if (q.passes == 1) {
    const int r = it.rpad[it.mbk];
    it.off_B = ws.take((int64_t)r * it.lmid);
    it.off_QB = ws.take((int64_t)it.lmid * r);
    it.off_RB = ws.take((int64_t)r * r);
    it.off_H = ws.take(P.sketches[it.mid_sk].rows * r);
  }
  // Staging area of the BF16 / FP16 plane kernel: test-matrix blocks whose
  // rows do not depend on the plane (column sketches with wdiv > 1, row
  // sketches with wdiv < W), one 128-row block image per distinct value and
  // half.
  const bool op16 = q.prec == TT_PREC_BF16 || q.prec == TT_PREC_FP16;
  it.tctab_doubles = 0;
  if (op16 && q.x_dtype == TT_F32 && (d == 3 || d == 4) &&
      (q.n[0] == 128 || q.n[0] == 256)) {
    int64_t bytes = 0;
    const int64_t hd = (std::min<int64_t>(q.n[d - 1], 256) + 127) / 128, h1 = q.n[0] / 128;
    for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) {
      const DevSketch& s = P.sketches[si];
      const int64_t blk = (int64_t)((s.width + 7) / 8) * kTcGroupBytes;
      if (s.type == SK_COL && s.wdiv > 1) bytes += (it.W / s.wdiv) * hd * blk;
      if (s.type == SK_ROW && s.wdiv < it.W) bytes += s.wdiv * h1 * blk;
    }
    it.tctab_doubles = (bytes + 7) / 8;
  }
  it.off_tctab = it.tctab_doubles ? ws.take(it.tctab_doubles) : 0;
  // FP32 staging of S_2 for the slab kernel (d = 4, BF16 / FP16, n_1 in {128, 256},
  // single-problem two-sided one-pass plans): its L-slot flush adds FP32
  // partials there, and one pass after each launch adds them into the FP64
  // sketch.
  it.s2stage_doubles = 0;
  if (it.tctab_doubles > 0 && d == 4 && single && !it.sided1 && q.passes == 1 && it.nsk == 4) {
    const DevSketch& s2 = P.sketches[it.sk0 + 1];
    if (s2.type == SK_COL && s2.k == 2) it.s2stage_doubles = (s2.rows * s2.width + 1) / 2;
  }
  it.off_s2stage = it.s2stage_doubles ? ws.take(it.s2stage_doubles) : 0;
  // Dense Gaussian slab streaming: R_3's test-matrix rows (i_1 + n_1 w) belong
  // to one plane each, so a slab of c slices draws l / c normals per entry of
  // X to regenerate them; every slab needs the same rows, so they are
  // generated once per decomposition (at its first slab launch) as 16-bit block
  // images, one per (half of i_1, kL, kR), kR fastest (2 (n_1 / 128) n_2 n_3 l
  // bytes up to padding: 604 MB at 256^4, capped at 1 GiB), and not kept
  // after it.
  it.ytab_doubles = 0;
  if (it.s2stage_doubles > 0 && !kr) {
    const DevSketch& r3 = P.sketches[it.sk0 + 3];
    if (r3.type == SK_ROW && r3.k == 3 && (r3.width == 8 || r3.width == 16)) {
      const int64_t bytes = (q.n[0] / 128) * q.n[1] * q.n[2] * (int64_t)(r3.width / 8) * kTcGroupBytes;
      if (bytes <= (1LL << 30)) it.ytab_doubles = (bytes + 7) / 8;
    }
  }
  it.off_ytab = it.ytab_doubles ? ws.take(it.ytab_doubles) : 0;
  // Staging area of the small-plane kernel (BF16, FP16 or TF32, n_1 and n_d <=
  // 32, one width l <= 32): the rows of every test matrix that many planes
  // share (column sketches with wdiv > 1: W/wdiv keys x n_d rows; row sketches
  // with wdiv < W: wdiv keys x n_1 rows), rounded to the MMA type, lpad
  // elements of 2 (BF16, FP16) or 4 (TF32) bytes per row.
  // A sketch whose table would exceed 512 MB is generated per plane instead.
  it.sptab_doubles = 0;
  {
    bool ok = (op16 || q.prec == TT_PREC_TF32) && q.x_dtype == TT_F32 && q.n[0] <= 32 &&
              q.n[d - 1] <= 32;
    const int64_t esz = q.prec == TT_PREC_TF32 ? 4 : 2;
    // sketch widths may differ (fixed ranks); the tables share the padding of
    // the widest one, which the small-plane launch uses for every sketch
    int lmax = 0;
    for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) lmax = std::max(lmax, P.sketches[si].width);
    ok = ok && lmax <= 32;
    int64_t bytes = 0;
    for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) {
      DevSketch& s = P.sketches[si];
      s.sp_tab = -1;
      if (!ok) continue;
      const int64_t lpad = lmax <= 16 ? 16 : 32;
      int64_t tb = 0;
      if (s.type == SK_COL && s.wdiv > 1) tb = (it.W / s.wdiv) * q.n[d - 1] * lpad * esz;
      if (s.type == SK_ROW && s.wdiv < it.W) tb = s.wdiv * q.n[0] * lpad * esz;
      if (tb > 0 && tb <= (512LL << 20)) {
        s.sp_tab = bytes;
        bytes += (tb + 255) / 256 * 256;
      }
    }
    it.sptab_doubles = ok ? std::max<int64_t>(1, (bytes + 7) / 8) : 0;
  }
  it.off_sptab = it.sptab_doubles ? ws.take(it.sptab_doubles) : 0;
  // The tensor-core sketch adjoint of the backward (single-problem, two-sided,
  // dense Gaussian TF32 / BF16 plans whose planes the small-plane kernel
  // serves): each sketch adjoint split into kAdjParts terms of the MMA type,
  // row-major rows x lpad (lpad = 16 or 32 elements of 2 or 4 bytes).
  it.adjtab_doubles = 0;
  if (single && it.sptab_doubles > 0 && !it.sided1 && !kr && q.passes == 1 && q.prec != TT_PREC_FP16) {
    int lmax = 0;
    for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) lmax = std::max(lmax, P.sketches[si].width);
    const int64_t lpad = lmax <= 16 ? 16 : 32, esz = q.prec == TT_PREC_TF32 ? 4 : 2;
    int64_t bytes = 0;
    for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) bytes += P.sketches[si].rows * lpad * esz * kAdjParts;
    it.adjtab_doubles = (bytes + 7) / 8;
  }
  it.off_adjtab = it.adjtab_doubles ? ws.take(it.adjtab_doubles) : 0;
  // Staging area of the generic tile kernel (single-problem plans whose item
  // neither the plane kernel nor the small-plane kernel serves; the batched
  // kernel draws its rows per tile): the test-matrix rows of each
  // sketch whose rows the tiles would otherwise draw more than once.  A
  // column-side row (key w / wdiv, i_d) is drawn by wdiv planes times the
  // 64-row tiles of i_1; a row-side row (key w % wdiv, i_1) by W / wdiv planes
  // times the 32-column tiles of i_d.  Rows for the whole last mode (column
  // side) or n_1 (row side), padded width round16(l); up to 256 MB a sketch
  // and 1 GB an item, sketches past that draw their rows per tile.  The
  // planes that share a column-side key are neighbours in the tile order, so
  // those rows stay in L2; the planes that share a row-side key lie wdiv
  // planes apart, so a row-side table is read from HBM once a plane unless it
  // fits in L2 (16 MB here): it is kept only then or when at least four
  // column tiles of the plane share the fetch.
  it.gentab_doubles = 0;
  {
    const bool ok = single && (op16 || q.prec == TT_PREC_TF32) && q.x_dtype == TT_F32 &&
                    it.tctab_doubles == 0 && it.sptab_doubles == 0;
    const int64_t esz = q.prec == TT_PREC_TF32 ? 4 : 2;
    const int64_t tilesA = (q.n[0] + 63) / 64, tilesB = (q.n[d - 1] + 31) / 32;
    int64_t bytes = 0;
    for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) {
      DevSketch& s = P.sketches[si];
      s.gen_tab = -1;
      if (!ok) continue;
      const int64_t lpad = (s.width + 15) / 16 * 16;
      int64_t tb = 0;
      if (s.type == SK_COL && s.wdiv * tilesA >= 2) tb = (it.W / s.wdiv) * q.n[d - 1] * lpad * esz;
      if (s.type == SK_ROW && (it.W / s.wdiv) * tilesB >= 2) {
        tb = s.wdiv * q.n[0] * lpad * esz;
        if (tilesB < 4 && tb > (16LL << 20)) tb = 0;
      }
      // a mode-by-mode Khatri-Rao sketch reads one factor row per tile row: nothing to stage
      if (tb > 0 && tb <= (256LL << 20) && bytes + tb <= (1LL << 30) && !s.kr_mbm) {
        s.gen_tab = bytes;
        bytes += (tb + 255) / 256 * 256;
      }
    }
    it.gentab_doubles = (bytes + 7) / 8;
  }
  it.off_gentab = it.gentab_doubles ? ws.take(it.gentab_doubles) : 0;
  // reconstruction interfaces
  for (int k = 1; k <= ds; ++k) it.off_L[k] = ws.take(it.N[k] * it.rpad[k]);
  for (int k = ds + 1; k <= d; ++k) it.off_Rt[k] = ws.take((int64_t)it.rpad[k - 1] * (it.N[d] / it.N[k - 1]));
  // backward scratch
  for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) {
    const DevSketch& s = P.sketches[si];
    it.off_sbar[si - it.sk0] = ws.take(s.rows * s.width);
  }
  for (int k = 1; k < d; ++k) {
    const DevSketch& s = P.sketches[it.basis_of_k[k]];
    it.off_qbar[k] = ws.take(s.rows * s.rpad);
    it.off_rr[k] = ws.take((int64_t)s.rpad * s.rpad);
  }
  if (q.passes == 1) {
    it.off_hbar = ws.take(it.N[ds] * it.rpad[ds]);
    it.off_bbar = ws.take((int64_t)it.rpad[ds] * it.lmid);
  }
  if (single) it.off_small = ws.take(4LL * TT_MAXL * TT_MAXL);
  it.diff = (q.flags & TT_FLAG_DIFF) ? 1 : 0;
  it.short_chains = (q.flags & TT_FLAG_SHORT_CHAINS) ? 1 : 0;
  if (it.diff) {
    int64_t ymax = 1;
    for (int k = 1; k < d; ++k) it.off_Lall[k] = ws.take(it.N[k] * it.rpad[k]);
    for (int k = 2; k <= d; ++k) it.off_Rall[k] = ws.take((int64_t)it.rpad[k - 1] * (it.N[d] / it.N[k - 1]));
    for (int k = 1; k <= d; ++k) ymax = std::max<int64_t>(ymax, it.N[k] * it.rpad[k]);
    it.off_Y = ws.take(ymax);
  }
  P.items.push_back(it);
  return TT_OK;
}

static void build_blob(Plan& P) {
  for (int L = 0; L < kMaxLev; ++L) P.tasks[L].clear();
  for (int si = 0; si < (int)P.sketches.size(); ++si) {
    const DevSketch& s = P.sketches[si];
    if (!s.basis) continue;
    for (int L = 0; L < s.nlev; ++L)
      for (int64_t b = 0; b < s.lev_nblk[L]; ++b)
        P.tasks[L + P.max_lev - s.nlev].push_back(Task{si, (int)b, L});
  }
  DevTables t;
  std::memset(&t, 0, sizeof(t));
  t.nitems = (int)P.items.size();
  t.nsk = (int)P.sketches.size();
  int64_t off = kTableOff + (int64_t)align_up(sizeof(DevTables), 64);
  t.off_items = off;
  off += align_up((int64_t)(sizeof(DevItem) * P.items.size()), 64);
  t.off_sketches = off;
  off += align_up((int64_t)(sizeof(DevSketch) * P.sketches.size()), 64);
  for (int L = 0; L < kMaxLev; ++L) {
    t.off_tasks[L] = off;
    t.ntasks[L] = (int)P.tasks[L].size();
    off += align_up((int64_t)(sizeof(Task) * P.tasks[L].size()), 64);
  }
  // batched sketch: items largest first (entries x sketches; ties by index)
  std::vector<int> order(P.items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const DevItem &A = P.items[(size_t)a], &B = P.items[(size_t)b];
    return A.N[A.d] * A.nsk > B.N[B.d] * B.nsk;
  });
  t.off_border = off;
  off += align_up((int64_t)(sizeof(int) * order.size()), 64);
  t.off_bprefix = off;
  off += align_up((int64_t)(sizeof(int64_t) * (order.size() + 1)), 64);
  t.off_bcounter = off;
  off += 64;
  P.blob.assign((size_t)(off - kTableOff), 0);
  auto put = [&](int64_t at, const void* src, size_t n) {
    if (n) std::memcpy(P.blob.data() + (at - kTableOff), src, n);
  };
  put(kTableOff, &t, sizeof(t));
  put(t.off_items, P.items.data(), sizeof(DevItem) * P.items.size());
  put(t.off_sketches, P.sketches.data(), sizeof(DevSketch) * P.sketches.size());
  for (int L = 0; L < kMaxLev; ++L) put(t.off_tasks[L], P.tasks[L].data(), sizeof(Task) * P.tasks[L].size());
  put(t.off_border, order.data(), sizeof(int) * order.size());
}

static tt_status build_all(Plan& P, const tt_problem* probs, int count, int64_t base_doubles) {
  WsAlloc ws{base_doubles};
  int64_t core_top = 0;
  int rank_top = 0;
  for (int i = 0; i < count; ++i) {
    tt_status st = validate(probs[i]);
    if (st == TT_OK) st = build_item(P, probs[i], ws, core_top, rank_top, count == 1);
    if (st != TT_OK) return st;
  }
  build_blob(P);
  P.ws_doubles = align_up(ws.top, 32);
  P.core_entries = core_top;
  P.rank_entries = rank_top;
  return TT_OK;
}

static tt_status make_plan(const tt_problem* probs, int count, tt_plan_t* out) {
  if (!out) return TT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!probs || count < 1) return TT_ERR_INVALID_ARG;
  // Pass 1 sizes the device tables (they depend on the TSQR trees); pass 2
  // lays the data out after them.
  int64_t table_end = 0;
  {
    Plan tmp;
    tt_status st = build_all(tmp, probs, count, 0);
    if (st != TT_OK) return st;
    table_end = kTableOff + (int64_t)tmp.blob.size();
  }
  Plan* P = new (std::nothrow) Plan();
  if (!P) return TT_ERR_INVALID_ARG;
  tt_status st = build_all(*P, probs, count, align_up(table_end, 256) / 8);
  if (st != TT_OK || kTableOff + (int64_t)P->blob.size() > table_end) {
    delete P;
    return st != TT_OK ? st : TT_ERR_INVALID_ARG;
  }
  if (count == 1) P->slab_seen.assign((size_t)P->items[0].n[P->items[0].d - 1], 0);
  P->id = g_next_plan_id.fetch_add(1);
  // batched default: tiles as tall as the largest n_1 needs (32 or 64 rows)
  int64_t n1max = 1;
  for (const DevItem& it : P->items) n1max = std::max(n1max, it.n[0]);
  P->bcfg = BatchCfg{n1max <= 32 ? 32 : 64, 4, 4};
  if (log_on()) {
    static const char* kPrec[] = {"fp64", "tf32", "bf16", "fp16"};
    for (size_t i = 0; i < P->items.size() && i < 8; ++i) {
      const DevItem& it = P->items[i];
      char dims[160] = {0};
      int o = 0;
      for (int k = 0; k < it.d && o < 140; ++k) o += std::snprintf(dims + o, sizeof(dims) - o, k ? "x%lld" : "%lld", (long long)it.n[k]);
      TT_LOGF("plan %llu item %zu: %s %s, %d sketches, %s, passes %d", (unsigned long long)P->id, i, dims,
              kPrec[it.prec & 3], it.nsk, it.eps_mode ? "tolerance" : "fixed ranks", it.passes);
    }
    TT_LOGF("plan %llu: %zu item(s), workspace %.1f MB, %lld core entries", (unsigned long long)P->id,
            P->items.size(), P->ws_doubles * 8.0 / 1e6, (long long)P->core_entries);
  }
  *out = reinterpret_cast<tt_plan_t>(P);
  return TT_OK;
}

static Plan* as_plan(tt_plan_t p) { return reinterpret_cast<Plan*>(p); }

static bool plan_owns(const Plan* p, const void* ws) {
  std::lock_guard<std::mutex> lock(g_ws_mu);
  auto it = g_ws.find(ws);
  return it != g_ws.end() && it->second.plan_id == p->id;
}

static bool plan_forward_valid(const Plan* p, const void* ws) {
  if (p->forward_ws != ws) return false;
  std::lock_guard<std::mutex> lock(g_ws_mu);
  auto it = g_ws.find(ws);
  return it != g_ws.end() && it->second.plan_id == p->id && it->second.forward_valid;
}

static void plan_release_all(const Plan* p) {
  std::lock_guard<std::mutex> lock(g_ws_mu);
  for (auto it = g_ws.begin(); it != g_ws.end();) {
    if (it->second.plan_id == p->id) it = g_ws.erase(it);
    else ++it;
  }
}

static tt_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TT_OK;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return TT_ERR_NO_DEVICE;
  return TT_ERR_CUDA;
}

static tt_status ensure_uploaded(Plan& P, void* ws, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_ws_mu);
  auto it = g_ws.find(ws);
  if (it != g_ws.end() && it->second.plan_id == P.id) return TT_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return TT_ERR_STATE;  // first use of a workspace by a plan must happen outside capture
  // the workspace no longer holds any plan's tables until the copy has landed
  if (it != g_ws.end()) g_ws.erase(it);
  cudaError_t e = cudaMemcpyAsync((char*)ws + kTableOff, P.blob.data(), P.blob.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaStreamSynchronize(st);  // the host blob must stay unchanged until copied
  if (e != cudaSuccess) return cuda_status(e);
  g_ws[ws] = WsEntry{P.id, false};
  return TT_OK;
}

static std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int device_sm_count() {
  static int cached = -1;
  if (cached > 0) return cached;
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  cached = n;
  return n;
}

// The staged tables of the slab kernel that do not depend on the slab are
// generated by the first accumulate of a decomposition and reused by the
// others (begin / tt_pstt2 clear the flag).
bool& plan_stream_tables(Plan& P) { return P.stream_tables; }
int& plan_pending_folds(Plan& P) { return P.pending_folds; }

// Start of a decomposition: clear the status word (so that a bit raised by
// the sketch kernels survives until tt_query_status) and the sketches.
static tt_status zero_sketches(Plan& P, int item, void* ws, cudaStream_t st) {
  const DevItem& it = P.items[item];
  double* base = (double*)ws;
  if (item == 0) {
    cudaError_t e = cudaMemsetAsync((char*)ws + kStatusOff, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) {
    const DevSketch& s = P.sketches[si];
    cudaError_t e = cudaMemsetAsync(base + s.off, 0, sizeof(double) * s.rows * s.width, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (it.s2stage_doubles > 0) {
    cudaError_t e = cudaMemsetAsync(base + it.off_s2stage, 0, sizeof(double) * it.s2stage_doubles, st);
    if (e != cudaSuccess) return cuda_status(e);
    P.pending_folds = 0;
  }
  // Khatri-Rao factors of the call (every later kernel of the call reads them)
  return cuda_status(launch_kr_tables(P, item, ws, st));
}

static tt_status accumulate(Plan& P, int item, const void* X, int64_t first, int64_t count, void* ws,
                            cudaStream_t st) {
  const DevItem& it = P.items[item];
  cudaError_t e;
  if (it.prec != TT_PREC_FP64 && !mixed_tc_supported(P, item, count)) return TT_ERR_UNSUPPORTED;
  if (it.prec == TT_PREC_FP64) {
    e = launch_sketch_f64(P, item, X, first, count, ws, st);
  } else {
    e = launch_sketch_mixed(P, item, X, first, count, ws, st);
  }
  return cuda_status(e);
}

}  // namespace tts

using namespace tts;

extern "C" {

tt_status tt_sketch_plan(const tt_problem* prob, tt_plan_t* out) {
  NvtxRange nvtx("tt_sketch_plan");
  return make_plan(prob, 1, out);
}

tt_status tt_sketch_plan_batched(const tt_problem* probs, int count, tt_plan_t* out) {
  NvtxRange nvtx("tt_sketch_plan_batched");
  return make_plan(probs, count, out);
}

void tt_plan_destroy(tt_plan_t plan) {
  Plan* P = as_plan(plan);
  if (!P) return;
  plan_release_all(P);
  delete P;
}

void tt_workspace_release(const void* ws) {
  std::lock_guard<std::mutex> lock(g_ws_mu);
  g_ws.erase(ws);
}

tt_status tt_plan_sizes(tt_plan_t plan, size_t* workspace_bytes, int64_t* core_entries,
                        int* rank_entries) {
  Plan* P = as_plan(plan);
  if (!P) return TT_ERR_INVALID_ARG;
  if (workspace_bytes) *workspace_bytes = (size_t)P->ws_doubles * 8;
  if (core_entries) *core_entries = P->core_entries;
  if (rank_entries) *rank_entries = P->rank_entries;
  return TT_OK;
}

tt_status tt_plan_core_layout(tt_plan_t plan, int item, int64_t* core_off, int* rpad) {
  Plan* P = as_plan(plan);
  if (!P || item < 0 || item >= (int)P->items.size()) return TT_ERR_INVALID_ARG;
  const DevItem& it = P->items[item];
  for (int k = 0; k <= TT_MAXD; ++k) {
    if (core_off) core_off[k] = (k >= 1 && k <= it.d) ? it.core_off[k] : 0;
    if (rpad) rpad[k] = k <= it.d ? it.rpad[k] : 0;
  }
  return TT_OK;
}

tt_status tt_plan_sketch_info(tt_plan_t plan, int item, int index, int* type, int* k, int64_t* rows,
                              int* width, int64_t* byte_off) {
  Plan* P = as_plan(plan);
  if (!P || item < 0 || item >= (int)P->items.size()) return TT_ERR_INVALID_ARG;
  const DevItem& it = P->items[item];
  if (index < 0 || index >= it.nsk) return TT_ERR_INVALID_ARG;
  const DevSketch& s = P->sketches[it.sk0 + index];
  if (type) *type = s.type;
  if (k) *k = s.k;
  if (rows) *rows = s.rows;
  if (width) *width = s.width;
  if (byte_off) *byte_off = s.off * 8;
  return TT_OK;
}

int tt_sketch_kernel_kind(tt_plan_t plan, int64_t count_last) {
  Plan* P = as_plan(plan);
  if (!P || P->items.empty()) return -1;
  if (P->items[0].prec == TT_PREC_FP64) return 0;
  if (use_tc_kernel(*P, 0, count_last) || use_slab_kernel(*P, 0, count_last)) return 2;
  return use_sp_kernel(*P, 0, count_last) ? 3 : 1;
}

tt_status tt_plan_problem(tt_plan_t plan, int item, tt_problem* out) {
  Plan* P = as_plan(plan);
  if (!P || !out || item < 0 || item >= (int)P->probs.size()) return TT_ERR_INVALID_ARG;
  *out = P->probs[item];
  return TT_OK;
}

tt_status tt_pstt2_begin(tt_plan_t plan, void* ws, tt_stream_t stream) {
  NvtxRange nvtx("tt_pstt2_begin");
  Plan* P = as_plan(plan);
  if (!P || !ws || P->items.size() != 1) return TT_ERR_INVALID_ARG;
  if (P->items[0].passes != 1) return TT_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  tt_status s = ensure_uploaded(*P, ws, st);
  if (s != TT_OK) return s;
  s = zero_sketches(*P, 0, ws, st);
  if (s != TT_OK) return s;
  std::fill(P->slab_seen.begin(), P->slab_seen.end(), 0);
  P->begun = true;
  P->stream_tables = false;
  P->stream_ws = ws;
  plan_mark_forward(P, ws, false);
  return TT_OK;
}

tt_status tt_pstt2_accumulate(tt_plan_t plan, const void* slab, int64_t first_last,
                              int64_t count_last, void* ws, tt_stream_t stream) {
  NvtxRange nvtx("tt_pstt2_accumulate");
  Plan* P = as_plan(plan);
  if (!P || !ws || !slab || P->items.size() != 1) return TT_ERR_INVALID_ARG;
  const DevItem& it = P->items[0];
  // the decomposition begun on this workspace, whose tables and sketches no
  // other plan has replaced since
  if (!P->begun || P->stream_ws != ws || !plan_owns(P, ws)) return TT_ERR_STATE;
  if (first_last < 0 || count_last < 1 || first_last + count_last > it.n[it.d - 1])
    return TT_ERR_INVALID_ARG;
  for (int64_t i = first_last; i < first_last + count_last; ++i)
    if (P->slab_seen[(size_t)i]) return TT_ERR_STATE;
  if (log_on()) {
    static const char* kKind[] = {"FP64 SIMT", "generic mma.sync tile", "tcgen05", "small-plane mma.sync"};
    const int kind = tt_sketch_kernel_kind(plan, count_last);
    TT_LOGF("plan %llu accumulate slices [%lld, %lld): %s kernel", (unsigned long long)P->id, (long long)first_last,
            (long long)(first_last + count_last), kKind[kind & 3]);
  }
  tt_status s = accumulate(*P, 0, slab, first_last, count_last, ws, (cudaStream_t)stream);
  if (s != TT_OK) return s;
  for (int64_t i = first_last; i < first_last + count_last; ++i) P->slab_seen[(size_t)i] = 1;
  return TT_OK;
}

// ------------------------------------------------ streaming state export
// Layout: StateHead, the slab bitmap (n_d bytes, padded to 8), then every
// sketch of the item (FP64, rows x width, column-major) in plan order.
namespace {
struct StateHead {
  char magic[8];
  int32_t d, passes, x_dtype, prec, flags, x_scale_log2, rmax, p, status_word, nsk;
  int64_t n[TT_MAXD];
  int32_t ranks[TT_MAXD + 1];
  int32_t pad_;
  double eps;
  uint64_t seed;
  int64_t sketch_doubles;
};
const char kStateMagic[8] = {'T', 'T', 'S', 'K', 'S', 'T', '0', '1'};

void state_head(const Plan& P, StateHead& h) {
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kStateMagic, 8);
  const tt_problem& q = P.probs[0];
  const DevItem& it = P.items[0];
  h.d = q.d;
  h.passes = q.passes;
  h.x_dtype = q.x_dtype;
  h.prec = q.prec;
  h.flags = q.flags;
  h.x_scale_log2 = it.x_scale_log2;
  h.rmax = q.eps > 0.0 ? q.rmax : 0;
  h.p = q.p;
  h.nsk = it.nsk;
  for (int k = 0; k < q.d; ++k) h.n[k] = q.n[k];
  if (!(q.eps > 0.0))
    for (int k = 0; k <= q.d; ++k) h.ranks[k] = q.ranks[k];
  h.eps = q.eps;
  h.seed = q.seed;
  for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) h.sketch_doubles += P.sketches[si].rows * P.sketches[si].width;
}
size_t state_bytes(const Plan& P) {
  StateHead h;
  state_head(P, h);
  const int64_t nd = P.items[0].n[P.items[0].d - 1];
  return sizeof(StateHead) + (size_t)((nd + 7) / 8 * 8) + sizeof(double) * (size_t)h.sketch_doubles;
}
bool state_usable(const Plan* P) { return P && P->items.size() == 1 && P->items[0].passes == 1; }
}  // namespace

tt_status tt_pstt2_sync(tt_plan_t plan, void* ws, tt_stream_t stream) {
  Plan* P = as_plan(plan);
  if (!P || !ws) return TT_ERR_INVALID_ARG;
  if (P->items.size() != 1 || !P->begun || P->stream_ws != ws || !plan_owns(P, ws)) return TT_OK;
  return cuda_status(fold_s2_staging(*P, 0, ws, (cudaStream_t)stream));
}

tt_status tt_pstt2_state_size(tt_plan_t plan, size_t* bytes) {
  Plan* P = as_plan(plan);
  if (!P || !bytes) return TT_ERR_INVALID_ARG;
  if (!state_usable(P)) return TT_ERR_UNSUPPORTED;
  *bytes = state_bytes(*P);
  return TT_OK;
}

tt_status tt_pstt2_export_state(tt_plan_t plan, const void* ws, void* host, size_t bytes, tt_stream_t stream) {
  NvtxRange nvtx("tt_pstt2_export_state");
  Plan* P = as_plan(plan);
  if (!P || !ws || !host) return TT_ERR_INVALID_ARG;
  if (!state_usable(P)) return TT_ERR_UNSUPPORTED;
  if (bytes < state_bytes(*P)) return TT_ERR_INVALID_ARG;
  if (!P->begun || P->stream_ws != ws || !plan_owns(P, ws)) return TT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  tt_status fs = cuda_status(fold_s2_staging(*P, 0, const_cast<void*>(ws), st));
  if (fs != TT_OK) return fs;
  StateHead h;
  state_head(*P, h);
  char* out = static_cast<char*>(host);
  const int64_t nd = P->items[0].n[P->items[0].d - 1];
  char* bitmap = out + sizeof(StateHead);
  double* dst = reinterpret_cast<double*>(bitmap + (nd + 7) / 8 * 8);
  std::memset(bitmap, 0, (size_t)((nd + 7) / 8 * 8));
  for (int64_t i = 0; i < nd; ++i) bitmap[i] = P->slab_seen[(size_t)i] ? 1 : 0;
  int word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, (const char*)ws + kStatusOff, sizeof(int), cudaMemcpyDeviceToHost, st);
  const DevItem& it = P->items[0];
  for (int si = it.sk0; si < it.sk0 + it.nsk && e == cudaSuccess; ++si) {
    const DevSketch& d = P->sketches[si];
    e = cudaMemcpyAsync(dst, (const double*)ws + d.off, sizeof(double) * d.rows * d.width, cudaMemcpyDeviceToHost, st);
    dst += d.rows * d.width;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  h.status_word = word;
  std::memcpy(out, &h, sizeof(h));
  return TT_OK;
}

tt_status tt_pstt2_import_state(tt_plan_t plan, void* ws, const void* host, size_t bytes, tt_stream_t stream) {
  NvtxRange nvtx("tt_pstt2_import_state");
  Plan* P = as_plan(plan);
  if (!P || !ws || !host) return TT_ERR_INVALID_ARG;
  if (!state_usable(P)) return TT_ERR_UNSUPPORTED;
  if (bytes < state_bytes(*P)) return TT_ERR_INVALID_ARG;
  StateHead mine, theirs;
  state_head(*P, mine);
  std::memcpy(&theirs, host, sizeof(theirs));
  mine.status_word = theirs.status_word;  // the only field that is not the problem's
  if (std::memcmp(&mine, &theirs, sizeof(mine)) != 0) return TT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  tt_status s = ensure_uploaded(*P, ws, st);
  if (s != TT_OK) return s;
  s = zero_sketches(*P, 0, ws, st);  // also the status word and the Khatri-Rao factors
  if (s != TT_OK) return s;
  const char* in = static_cast<const char*>(host);
  const int64_t nd = P->items[0].n[P->items[0].d - 1];
  const char* bitmap = in + sizeof(StateHead);
  const double* src = reinterpret_cast<const double*>(bitmap + (nd + 7) / 8 * 8);
  cudaError_t e = cudaMemcpyAsync((char*)ws + kStatusOff, &theirs.status_word, sizeof(int), cudaMemcpyHostToDevice, st);
  const DevItem& it = P->items[0];
  for (int si = it.sk0; si < it.sk0 + it.nsk && e == cudaSuccess; ++si) {
    const DevSketch& d = P->sketches[si];
    e = cudaMemcpyAsync((double*)ws + d.off, src, sizeof(double) * d.rows * d.width, cudaMemcpyHostToDevice, st);
    src += d.rows * d.width;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host buffer may go away after the call
  if (e != cudaSuccess) return cuda_status(e);
  for (int64_t i = 0; i < nd; ++i) P->slab_seen[(size_t)i] = bitmap[i] ? 1 : 0;
  P->begun = true;
  P->stream_tables = false;
  P->stream_ws = ws;
  plan_mark_forward(P, ws, false);
  return TT_OK;
}

tt_status tt_pstt2_finalize(tt_plan_t plan, void* ws, double* cores, int* ranks,
                            tt_stream_t stream) {
  NvtxRange nvtx("tt_pstt2_finalize");
  Plan* P = as_plan(plan);
  if (!P || !ws || !cores || !ranks || P->items.size() != 1) return TT_ERR_INVALID_ARG;
  if (!P->begun || P->stream_ws != ws || !plan_owns(P, ws)) return TT_ERR_STATE;
  for (char c : P->slab_seen)
    if (!c) return TT_ERR_STATE;
  tt_status s = cuda_status(launch_finalize(*P, ws, cores, ranks, (cudaStream_t)stream));
  if (s != TT_OK) return s;
  P->begun = false;
  plan_mark_forward(P, ws, true);
  return TT_OK;
}

tt_status tt_pstt2(tt_plan_t plan, const void* X, void* ws, double* cores, int* ranks,
                   tt_stream_t stream) {
  NvtxRange nvtx("tt_pstt2");
  Plan* P = as_plan(plan);
  if (!P || !X || !ws || !cores || !ranks || P->items.size() != 1) return TT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const DevItem& it = P->items[0];
  tt_status s = ensure_uploaded(*P, ws, st);
  if (s != TT_OK) return s;
  s = zero_sketches(*P, 0, ws, st);
  if (s != TT_OK) return s;
  P->stream_tables = false;
  s = accumulate(*P, 0, X, 0, it.n[it.d - 1], ws, st);
  if (s != TT_OK) return s;
  if (it.passes == 2) {
    s = cuda_status(launch_finalize(*P, ws, cores, ranks, st));  // bases + outer cores
    if (s != TT_OK) return s;
    s = cuda_status(launch_twopass_mid(*P, X, ws, cores, ranks, st));  // second pass over X
  } else {
    s = cuda_status(launch_finalize(*P, ws, cores, ranks, st));
  }
  if (s != TT_OK) return s;
  P->begun = false;
  plan_mark_forward(P, ws, true);
  return TT_OK;
}

static tt_status batched_check(const Plan* P, const void* const* X_ptrs) {
  const DevItem& i0 = P->items[0];
  if (P->items.size() > (size_t)kMaxBatchItems) return TT_ERR_UNSUPPORTED;
  for (size_t i = 0; i < P->items.size(); ++i) {
    const DevItem& it = P->items[i];
    if (it.passes != 1 || it.prec != i0.prec) return TT_ERR_UNSUPPORTED;
    if (it.prec != TT_PREC_FP64 && it.x_f64) return TT_ERR_UNSUPPORTED;
    if (!X_ptrs[i]) return TT_ERR_INVALID_ARG;
  }
  return TT_OK;
}

static tt_status batched_run(Plan& P, const void* const* X_ptrs, const BatchCfg& cfg, void* ws, double* cores,
                             int* ranks, cudaStream_t st) {
  tt_status s = ensure_uploaded(P, ws, st);
  if (s != TT_OK) return s;
  s = cuda_status(launch_batch_zero(P, ws, st));
  if (s != TT_OK) return s;
  s = cuda_status(launch_sketch_batched(P, X_ptrs, cfg, ws, st));
  if (s != TT_OK) return s;
  return cuda_status(launch_finalize(P, ws, cores, ranks, st));
}

tt_status tt_pstt2_batched(tt_plan_t plan, const void* const* X_ptrs, void* ws, double* cores,
                           int* ranks, tt_stream_t stream) {
  NvtxRange nvtx("tt_pstt2_batched");
  Plan* P = as_plan(plan);
  if (!P || !X_ptrs || !ws || !cores || !ranks) return TT_ERR_INVALID_ARG;
  tt_status s = batched_check(P, X_ptrs);
  if (s != TT_OK) return s;
  s = batched_run(*P, X_ptrs, P->bcfg, ws, cores, ranks, (cudaStream_t)stream);
  if (s != TT_OK) return s;
  plan_mark_forward(P, ws, true);
  return TT_OK;
}

// Autotuner cache (TT_TUNE_CACHE = path of a text file): one line "key ta
// chunk ctas_per_sm" per tuned batch; the key hashes the device (SM count,
// compute capability) and every item's precision, shape and sketch widths.
static std::string tune_key(const Plan& P) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](int64_t v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xFF);
      h *= 1099511628211ull;
    }
  };
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  mix(device_sm_count());
  mix(major * 10 + minor);
  mix((int64_t)P.items.size());
  for (const DevItem& it : P.items) {
    mix(it.prec);
    mix(it.d);
    for (int k = 0; k < it.d; ++k) mix(it.n[k]);
    for (int si = it.sk0; si < it.sk0 + it.nsk; ++si) mix(P.sketches[si].width);
  }
  char buf[24];
  std::snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
  return buf;
}

static bool tune_cache_find(const char* path, const std::string& key, BatchCfg& out) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char k[64];
  int ta, chunk, cps;
  bool found = false;
  while (std::fscanf(f, "%63s %d %d %d", k, &ta, &chunk, &cps) == 4)
    if (key == k) {
      out = BatchCfg{ta, chunk, cps};
      found = true;  // the last entry for a key wins
    }
  std::fclose(f);
  return found;
}

tt_status tt_plan_autotune(tt_plan_t plan, const void* const* X_ptrs, void* ws, double* cores, int* ranks,
                           tt_stream_t stream, int* best_out) {
  NvtxRange nvtx("tt_plan_autotune");
  Plan* P = as_plan(plan);
  if (!P || !X_ptrs || !ws || !cores || !ranks) return TT_ERR_INVALID_ARG;
  tt_status s = batched_check(P, X_ptrs);
  if (s != TT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return TT_ERR_STATE;
  s = batched_run(*P, X_ptrs, P->bcfg, ws, cores, ranks, st);  // warm-up (uploads the tables)
  if (s != TT_OK) return s;
  const bool f64 = P->items[0].prec == TT_PREC_FP64;
  std::vector<BatchCfg> cands;
  if (!f64 && sp_batched_eligible(*P, nullptr, nullptr)) {
    // small-plane batched kernel (one CTA per SM): the block shape (ta = the
    // largest number of kR values in a 16-plane block) and the units per grab
    for (int t3 : {1, 2, 4, 8})
      if (sp_batched_eligible(*P, nullptr, nullptr, t3))
        for (int chunk : {1, 4, 8}) cands.push_back(BatchCfg{t3, chunk, 1});
  } else {
    for (int ta : {32, 64}) {
      if (!f64 && ta == 32) continue;
      for (int chunk : {1, 4, 16})
        for (int cps : {2, 4, 8}) cands.push_back(BatchCfg{ta, chunk, cps});
    }
  }
  const char* cache = std::getenv("TT_TUNE_CACHE");
  const std::string key = (cache && *cache) ? tune_key(*P) : std::string();
  BatchCfg cached{0, 0, 0};
  if (!key.empty() && tune_cache_find(cache, key, cached)) {
    for (const BatchCfg& c : cands)
      if (c.ta == cached.ta && c.chunk == cached.chunk && c.ctas_per_sm == cached.ctas_per_sm) {
        TT_LOGF("plan %llu autotune: cached shape %d %d %d (%s)", (unsigned long long)P->id, c.ta, c.chunk,
                c.ctas_per_sm, key.c_str());
        P->bcfg = c;
        if (best_out) {
          best_out[0] = c.ta;
          best_out[1] = c.chunk;
          best_out[2] = c.ctas_per_sm;
        }
        s = batched_run(*P, X_ptrs, P->bcfg, ws, cores, ranks, st);
        if (s == TT_OK) plan_mark_forward(P, ws, true);
        return s;
      }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return TT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TT_ERR_CUDA;
  }
  float best = 1e30f;
  int best_i = -1;
  for (size_t c = 0; c < cands.size() && s == TT_OK; ++c) {
    float acc = 0.0f;
    for (int rep = 0; rep < 2 && s == TT_OK; ++rep) {
      s = cuda_status(launch_batch_zero(*P, ws, st));
      if (s == TT_OK) s = cuda_status(cudaEventRecord(e0, st));
      if (s == TT_OK) s = cuda_status(launch_sketch_batched(*P, X_ptrs, cands[c], ws, st));
      if (s == TT_OK) s = cuda_status(cudaEventRecord(e1, st));
      if (s == TT_OK) s = cuda_status(cudaEventSynchronize(e1));
      float ms = 0.0f;
      if (s == TT_OK) s = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
      if (rep == 1) acc = ms;  // the second run (the first warms the launch shape)
    }
    if (s == TT_OK && acc < best) {
      best = acc;
      best_i = (int)c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != TT_OK) return s;
  P->bcfg = cands[(size_t)best_i];
  TT_LOGF("plan %llu autotune: best shape %d %d %d, %.3f ms", (unsigned long long)P->id, P->bcfg.ta, P->bcfg.chunk,
          P->bcfg.ctas_per_sm, best);
  if (!key.empty()) {
    if (FILE* f = std::fopen(cache, "a")) {
      std::fprintf(f, "%s %d %d %d\n", key.c_str(), P->bcfg.ta, P->bcfg.chunk, P->bcfg.ctas_per_sm);
      std::fclose(f);
    }
  }
  if (best_out) {
    best_out[0] = P->bcfg.ta;
    best_out[1] = P->bcfg.chunk;
    best_out[2] = P->bcfg.ctas_per_sm;
  }
  // leave a complete decomposition with the chosen shape in the buffers
  s = batched_run(*P, X_ptrs, P->bcfg, ws, cores, ranks, st);
  if (s == TT_OK) plan_mark_forward(P, ws, true);
  return s;
}

tt_status tt_plan_batch_config(tt_plan_t plan, int ta, int chunk, int ctas_per_sm) {
  Plan* P = as_plan(plan);
  if (!P || (ta != 32 && ta != 64 && ta != 1 && ta != 2 && ta != 4 && ta != 8) || chunk < 1 || ctas_per_sm < 1 ||
      ctas_per_sm > 32)
    return TT_ERR_INVALID_ARG;
  P->bcfg = BatchCfg{ta, chunk, ctas_per_sm};
  return TT_OK;
}

tt_status tt_pstt2_backward(tt_plan_t plan, void* ws, const double* dcores, void* dX,
                            tt_stream_t stream) {
  NvtxRange nvtx("tt_pstt2_backward");
  Plan* P = as_plan(plan);
  if (!P || !ws || !dcores || !dX || P->items.size() != 1) return TT_ERR_INVALID_ARG;
  // the saved state of this plan's last forward call must still be in ws
  if (!plan_forward_valid(P, ws)) return TT_ERR_STATE;
  if (P->items[0].passes != 1) return TT_ERR_UNSUPPORTED;
  return cuda_status(launch_backward(*P, 0, dcores, dX, ws, (cudaStream_t)stream));
}

tt_status tt_reconstruct(tt_plan_t plan, const double* cores, void* Xt, tt_dtype dtype, void* ws,
                         tt_stream_t stream) {
  NvtxRange nvtx("tt_reconstruct");
  Plan* P = as_plan(plan);
  if (!P || !cores || !Xt || !ws || P->items.size() != 1) return TT_ERR_INVALID_ARG;
  if (dtype != TT_F32 && dtype != TT_F64) return TT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  tt_status s = ensure_uploaded(*P, ws, st);
  if (s != TT_OK) return s;
  return cuda_status(launch_reconstruct(*P, 0, cores, Xt, dtype == TT_F64, nullptr, 0, nullptr, ws, st));
}

tt_status tt_reconstruct_error(tt_plan_t plan, const double* cores, const void* X, double* out2,
                               void* ws, tt_stream_t stream) {
  NvtxRange nvtx("tt_reconstruct_error");
  Plan* P = as_plan(plan);
  if (!P || !cores || !X || !out2 || !ws || P->items.size() != 1) return TT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  tt_status s = ensure_uploaded(*P, ws, st);
  if (s != TT_OK) return s;
  return cuda_status(launch_reconstruct(*P, 0, cores, nullptr, 0, X, P->items[0].x_f64, out2, ws, st));
}

tt_status tt_reconstruct_backward(tt_plan_t plan, const double* cores, const void* dXt,
                                  tt_dtype dtype, double* dcores, void* ws, tt_stream_t stream) {
  NvtxRange nvtx("tt_reconstruct_backward");
  Plan* P = as_plan(plan);
  if (!P || !cores || !dXt || !dcores || !ws || P->items.size() != 1) return TT_ERR_INVALID_ARG;
  if (dtype != TT_F32 && dtype != TT_F64) return TT_ERR_INVALID_ARG;
  if (!P->items[0].diff) return TT_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  tt_status s = ensure_uploaded(*P, ws, st);
  if (s != TT_OK) return s;
  return cuda_status(launch_reconstruct_backward(*P, 0, cores, dXt, dtype == TT_F64, dcores, ws, st));
}

tt_status tt_query_status(tt_plan_t plan, const void* ws, const int* ranks, int* status_host,
                          int* ranks_host, tt_stream_t stream) {
  Plan* P = as_plan(plan);
  if (!P || !ws) return TT_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  int word = 0;
  e = cudaMemcpy(&word, (const char*)ws + kStatusOff, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (status_host) {
    int s = TT_OK;
    if (word & ST_RANK_CAP) s = TT_WARN_RANK_CAP;
    if (word & ST_TIMEOUT) s = TT_ERR_TIMEOUT;
    if (word & ST_RANK_DEFICIENT) s = TT_ERR_RANK_DEFICIENT;
    if (word & ST_NONFINITE) s = TT_ERR_NONFINITE;
    *status_host = s;
  }
  if (ranks_host) {
    if (!ranks) return TT_ERR_INVALID_ARG;
    e = cudaMemcpy(ranks_host, ranks, sizeof(int) * P->rank_entries, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return TT_OK;
}

const char* tt_status_string(tt_status s) {
  switch (s) {
    case TT_OK: return "ok";
    case TT_ERR_INVALID_ARG: return "invalid argument";
    case TT_ERR_UNSUPPORTED: return "unsupported";
    case TT_ERR_CUDA: return "CUDA runtime error";
    case TT_ERR_STATE: return "calls out of order";
    case TT_ERR_RANK_DEFICIENT: return "rank-deficient least-squares matrix";
    case TT_ERR_TIMEOUT: return "device wait timed out";
    case TT_WARN_RANK_CAP: return "tolerance not met at rmax";
    case TT_ERR_NO_DEVICE: return "no CUDA device";
    case TT_ERR_NONFINITE: return "non-finite sketch entry (X, or FP16 range)";
  }
  return "unknown status";
}

int64_t tt_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* tt_version(void) { return "ttsketch-gb300 sm_103a " __DATE__; }

}  // extern "C"
