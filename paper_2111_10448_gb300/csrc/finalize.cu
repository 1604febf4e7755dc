// FP64 finalize: orthonormal bases, ranks, the one-pass middle core and the
// core products (Sec. 3.2; Algorithm 2 steps 4-8; eq. (3.1) and its row-space
// mirror; eq. (3.3) for the middle core).
//
// Bases.  The paper takes a CPQR of each sketch and keeps Q(:, 1:r_k); it
// forms the ON bases of the distributed sketches with a skinny (TSQR) QR
// (Sec. 4.2, Benson et al.).  Here every basis sketch Y (m x l, m up to
// n^{ceil(d/2)}) is reduced by a TSQR tree of Householder QRs of row blocks;
// the CPQR is taken on the l x l root factor R, which has the same column
// norms and inner products as Y (Y = Q_1 R), so it selects the same pivots:
// R Pi = Q_2 Rt.  Then Q_k = Q_1 Q_2(:, 1:r_k), formed top-down through the
// tree.  Signs are normalised so that diag(Rt) >= 0.
//
// Ranks.  Fixed-rank mode keeps the (clamped) target.  Tolerance mode takes
// the smallest r with ||Rt(r:, r:)||_F <= eps/sqrt(d-1) ||Y||_F (the per-
// unfolding split of Theorem 3.2), capped at rmax; the cap is flagged.  Ranks
// stay on the device; later kernels read them from there.
#include <algorithm>

#include "internal.cuh"
#include "philox.cuh"
#include "testmat.cuh"

namespace tts {

const DevSketch* plan_sketches_host(const Plan* p);
int plan_num_items(const Plan* p);
int plan_max_lev(const Plan* p);
int plan_ntasks(const Plan* p, int lev);

namespace {

constexpr int kThreads = 256;
constexpr int64_t kTableOffB = 256;

__device__ __forceinline__ const DevTables& tables(const char* wsb) {
  return *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
}
__device__ __forceinline__ const DevSketch* dsk(const char* wsb) {
  return reinterpret_cast<const DevSketch*>(wsb + tables(wsb).off_sketches);
}
__device__ __forceinline__ const DevItem* ditems(const char* wsb) {
  return reinterpret_cast<const DevItem*>(wsb + tables(wsb).off_items);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (all threads get the result).  Uses red[32].
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// Sums over the 32 lanes of two or four per-lane values at once (halving
// butterflies: 5 or 6 additions instead of 2 x 5 or 4 x 5).  warp_sum2: lane
// L returns the sum of p[(L >> 4) & 1]; warp_sum4: of p[(L >> 3) & 3].
__device__ __forceinline__ double warp_sum2(double p0, double p1) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16;
  double k = h16 ? p1 : p0;
  k += __shfl_xor_sync(0xffffffffu, h16 ? p0 : p1, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  return k;
}
__device__ __forceinline__ double warp_sum4(double p0, double p1, double p2, double p3) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  double k0 = h16 ? p2 : p0, k1 = h16 ? p3 : p1;
  k0 += __shfl_xor_sync(0xffffffffu, h16 ? p0 : p2, 16);
  k1 += __shfl_xor_sync(0xffffffffu, h16 ? p1 : p3, 16);
  double k = h8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

// FP64 instructions on this GPU hold their sub-partition's FP64 pipe for 64
// cycles each, and guarding one with a run-time condition costs several times
// that even when the guard is false.  So the per-warp column groups below are
// templates on their column count NC (1..4), dispatched by a switch, and
// their FP64 arithmetic is unconditional.

// Gram row entries g_c = sum_{r >= i} A(r, i) A(r, c) of the NC columns
// c = cb + nw j, written to gram[c]; the group holding column i also forms the
// reflector of step i (beta, R(i, i), head v0).
template <int NC>
__device__ __forceinline__ void gram_group(const double* A, int lda, int nr, int i, int cb, int nw,
                                           double* gram, double* beta, double* rdiag, double* v0s) {
  const int lane = threadIdx.x & 31;
  double p[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r = i + lane; r < nr; r += 32) {
    const double a = A[r + lda * i];
#pragma unroll
    for (int j = 0; j < NC; ++j) p[j] = fma(a, A[r + lda * (cb + nw * j)], p[j]);
  }
  double g;
  int q;
  bool wr;
  if (NC == 1) {
    g = warp_sum(p[0]), q = 0, wr = lane == 0;
  } else if (NC == 2) {
    g = warp_sum2(p[0], p[1]), q = lane >> 4, wr = (lane & 15) == 0;
  } else {
    g = warp_sum4(p[0], p[1], p[2], p[3]), q = lane >> 3, wr = (lane & 7) == 0 && q < NC;
  }
  if (wr) gram[cb + nw * q] = g;
  if (cb == i && lane == 0) {
    const double x0 = A[i + lda * i];
    const double nx = sqrt(g);
    double alpha = 0.0, b = 0.0;
    if (nx > 0.0) {
      alpha = -copysign(nx, x0);
      const double v0 = x0 - alpha;
      const double vn2 = g - x0 * x0 + v0 * v0;
      b = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
    }
    beta[i] = b;
    rdiag[i] = alpha;
    *v0s = nx > 0.0 ? x0 - alpha : 0.0;
  }
}

// A(i:, c) -= b v (v^T A(i:, c)) for the NC columns c = cb + nw j, with
// v^T A(i:, c) = g_c - alpha A(i, c) and v = (v0, A(i+1:, i)).
template <int NC>
__device__ __forceinline__ void update_group(double* A, int lda, int nr, int i, int cb, int nw,
                                             const double* gram, double b, double alpha, double v0) {
  const int lane = threadIdx.x & 31;
  double coef[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const int c = cb + nw * j;
    coef[j] = b * fma(-alpha, A[i + lda * c], gram[c]);
  }
  __syncwarp();
  for (int r = i + lane; r < nr; r += 32) {
    const double v = r == i ? v0 : A[r + lda * i];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      double* e = A + r + lda * (cb + nw * j);
      *e = fma(-coef[j], v, *e);
    }
  }
}

// In-shared-memory Householder QR of an nr x w block A (ld = lda), nr >= 1.
// On exit column i holds v_i in rows i..nr-1 (v_i(0) at the diagonal), beta[i]
// = 2 / (v_i^T v_i) (0 for a zero column), rdiag[i] = R(i, i); the strict
// upper triangle holds R.
//
// Step i works from the Gram row g_c = sum_{r >= i} A(r, i) A(r, c), c >= i:
// g_i is the squared norm of the pivot column, and with v = A(i:, i) - alpha
// e_1 the reflector products are v^T A(i:, c) = g_c - alpha A(i, c).  So a
// step is one reduction pass (every column's dot at once; the warp owning
// columns c, c+8, c+16, c+24 sums them with one butterfly) and one update
// pass, two barriers in all.
__device__ __forceinline__ void house_qr(double* A, int lda, int nr, int w, double* beta, double* rdiag) {
  const int kmax = min(nr, w);
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double v0s;
  __shared__ double gram[TT_MAXL];
  for (int i = 0; i < kmax; ++i) {
    for (int cb = i + wid; cb < w; cb += 4 * nw) {
      switch (min(4, (w - 1 - cb) / nw + 1)) {
        case 1: gram_group<1>(A, lda, nr, i, cb, nw, gram, beta, rdiag, &v0s); break;
        case 2: gram_group<2>(A, lda, nr, i, cb, nw, gram, beta, rdiag, &v0s); break;
        case 3: gram_group<3>(A, lda, nr, i, cb, nw, gram, beta, rdiag, &v0s); break;
        default: gram_group<4>(A, lda, nr, i, cb, nw, gram, beta, rdiag, &v0s); break;
      }
    }
    __syncthreads();
    const double b = beta[i], alpha = rdiag[i], v0 = v0s;
    if (b != 0.0) {
      for (int cb = i + 1 + wid; cb < w; cb += 4 * nw) {
        switch (min(4, (w - 1 - cb) / nw + 1)) {
          case 1: update_group<1>(A, lda, nr, i, cb, nw, gram, b, alpha, v0); break;
          case 2: update_group<2>(A, lda, nr, i, cb, nw, gram, b, alpha, v0); break;
          case 3: update_group<3>(A, lda, nr, i, cb, nw, gram, b, alpha, v0); break;
          default: update_group<4>(A, lda, nr, i, cb, nw, gram, b, alpha, v0); break;
        }
      }
    }
    if (threadIdx.x == 0) A[i + lda * i] = v0;
    __syncthreads();
  }
  for (int i = kmax + threadIdx.x; i < w; i += blockDim.x) {
    beta[i] = 0.0;
    rdiag[i] = 0.0;
  }
  __syncthreads();
}

// Apply the reflectors of a block (V: nr x w in global or shared, ld = ldv,
// beta) to Z (nr x ncol, ld = ldz):  Z <- H_0 ... H_{k-1} Z.
__device__ void apply_q(const double* V, int64_t ldv, const double* beta, int nr, int w, double* Z,
                        int64_t ldz, int ncol) {
  const int kmax = min(nr, w);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = kmax - 1; i >= 0; --i) {
    const double b = beta[i];
    if (b != 0.0) {
      for (int c = wid; c < ncol; c += nw) {
        double dot = 0.0;
        for (int r = i + lane; r < nr; r += 32) dot += V[r + ldv * i] * Z[r + ldz * c];
        dot = warp_sum(dot) * b;
        for (int r = i + lane; r < nr; r += 32) Z[r + ldz * c] -= dot * V[r + ldv * i];
      }
    }
    __syncthreads();
  }
}

// Z(:, c) = H_0 ... H_{kmax-1} [Z0(0:kmax, c); 0] for the nr-row block of
// reflectors V (ld ldv, heads v_i(0) on the diagonal) and beta, columns c <
// ncol; columns ncol..npad-1 of Z are zero.  Z0 = Zin (ld ldzin).  A warp
// keeps NC columns c = cb + nw j in registers through all reflectors (no
// barrier between reflectors; one butterfly per reflector for the NC dots;
// NC > 1 only for blocks of at most 64 rows); NT = ceil(nr / 32) rows per
// lane, nr <= 256.
constexpr int kRowsPerLane = 8;
template <int NC>
__device__ __forceinline__ void warp_sums(const double (&p)[4], double (&d)[4]) {
  if (NC == 1) {
    d[0] = warp_sum(p[0]);
  } else if (NC == 2) {
    const double g = warp_sum2(p[0], p[1]);
    d[0] = __shfl_sync(0xffffffffu, g, 0);
    d[1] = __shfl_sync(0xffffffffu, g, 16);
  } else {
    const double g = warp_sum4(p[0], p[1], p[2], p[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = __shfl_sync(0xffffffffu, g, 8 * j);
  }
}
template <int NT, int NC>
__device__ __forceinline__ void expand_group(const double* V, int64_t ldv, const double* beta, int nr, int kmax,
                                             const double* Zin, int64_t ldzin, int cb, int nw, double* Z,
                                             int64_t ldz) {
  const int lane = threadIdx.x & 31;
  double z[NC][NT];
#pragma unroll
  for (int j = 0; j < NC; ++j)
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int r = lane + 32 * t;
      z[j][t] = r < kmax ? Zin[r + ldzin * (cb + nw * j)] : 0.0;
    }
  for (int i = kmax - 1; i >= 0; --i) {
    const double b = beta[i];
    if (b == 0.0) continue;
    double v[NT];
    double p[4] = {0.0, 0.0, 0.0, 0.0}, d[4];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int r = lane + 32 * t;
      v[t] = (r >= i && r < nr) ? V[r + ldv * i] : 0.0;
#pragma unroll
      for (int j = 0; j < NC; ++j) p[j] = fma(v[t], z[j][t], p[j]);
    }
    warp_sums<NC>(p, d);
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const double s = d[j] * b;
#pragma unroll
      for (int t = 0; t < NT; ++t) z[j][t] = fma(-s, v[t], z[j][t]);
    }
  }
#pragma unroll
  for (int j = 0; j < NC; ++j)
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int r = lane + 32 * t;
      if (r < nr) Z[r + ldz * (cb + nw * j)] = z[j][t];
    }
}
template <int NT>
__device__ __forceinline__ void expand_cols_nt(const double* V, int64_t ldv, const double* beta, int nr, int w,
                                               const double* Zin, int64_t ldzin, int ncol, int npad, double* Z,
                                               int64_t ldz) {
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int kmax = min(nr, w);
  if (NT > 2) {  // tall blocks: one column per warp keeps the registers in bounds
    for (int c = wid; c < ncol; c += nw) expand_group<NT, 1>(V, ldv, beta, nr, kmax, Zin, ldzin, c, nw, Z, ldz);
  } else {
    for (int cb = wid; cb < ncol; cb += 4 * nw) {
      switch (min(4, (ncol - 1 - cb) / nw + 1)) {
        case 1: expand_group<NT, 1>(V, ldv, beta, nr, kmax, Zin, ldzin, cb, nw, Z, ldz); break;
        case 2: expand_group<NT, 2>(V, ldv, beta, nr, kmax, Zin, ldzin, cb, nw, Z, ldz); break;
        case 3: expand_group<NT, 3>(V, ldv, beta, nr, kmax, Zin, ldzin, cb, nw, Z, ldz); break;
        default: expand_group<NT, 4>(V, ldv, beta, nr, kmax, Zin, ldzin, cb, nw, Z, ldz); break;
      }
    }
  }
  for (int o = threadIdx.x; o < nr * (npad - ncol); o += blockDim.x) Z[o % nr + ldz * (ncol + o / nr)] = 0.0;
}
__device__ __forceinline__ void expand_cols(const double* V, int64_t ldv, const double* beta, int nr, int w,
                                            const double* Zin, int64_t ldzin, int ncol, int npad, double* Z,
                                            int64_t ldz) {
  switch ((nr + 31) / 32) {
    case 1: expand_cols_nt<1>(V, ldv, beta, nr, w, Zin, ldzin, ncol, npad, Z, ldz); break;
    case 2: expand_cols_nt<2>(V, ldv, beta, nr, w, Zin, ldzin, ncol, npad, Z, ldz); break;
    case 3: expand_cols_nt<3>(V, ldv, beta, nr, w, Zin, ldzin, ncol, npad, Z, ldz); break;
    case 4: expand_cols_nt<4>(V, ldv, beta, nr, w, Zin, ldzin, ncol, npad, Z, ldz); break;
    case 5: expand_cols_nt<5>(V, ldv, beta, nr, w, Zin, ldzin, ncol, npad, Z, ldz); break;
    case 6: expand_cols_nt<6>(V, ldv, beta, nr, w, Zin, ldzin, ncol, npad, Z, ldz); break;
    case 7: expand_cols_nt<7>(V, ldv, beta, nr, w, Zin, ldzin, ncol, npad, Z, ldz); break;
    default: expand_cols_nt<kRowsPerLane>(V, ldv, beta, nr, w, Zin, ldzin, ncol, npad, Z, ldz); break;
  }
}

// One pivoted-QR step's update of the NC root columns c = cb + nw j > i by
// reflector i (v = Rs(i:, i), beta b), and their trailing norms over rows > i.
template <int NC>
__device__ __forceinline__ void cpqr_group(double* Rs, int w, int i, int cb, int nw, double b, double* nrm) {
  const int lane = threadIdx.x & 31;
  double p[4] = {0.0, 0.0, 0.0, 0.0}, d[4];
  for (int r = i + lane; r < w; r += 32) {
    const double v = Rs[r + w * i];
#pragma unroll
    for (int j = 0; j < NC; ++j) p[j] = fma(v, Rs[r + w * (cb + nw * j)], p[j]);
  }
  warp_sums<NC>(p, d);
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r = i + lane; r < w; r += 32) {
    const double v = Rs[r + w * i];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      double* e = Rs + r + w * (cb + nw * j);
      const double x = fma(-d[j] * b, v, *e);
      *e = x;
      const double xt = r > i ? x : 0.0;
      t[j] = fma(xt, xt, t[j]);
    }
  }
  warp_sums<NC>(t, d);
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < NC; ++j) nrm[cb + nw * j] = d[j];
}

// Copies an nr x w column-major block (leading dimension ldy) into shared
// memory (leading dimension lda); eight independent loads per thread are in
// flight at a time.
__device__ void load_block(double* A, int lda, const double* Y, int64_t ldy, int nr, int w) {
  for (int c0 = 0; c0 < w; c0 += 8)
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = (c0 + u < w) ? Y[r + ldy * (c0 + u)] : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (c0 + u < w) A[r + lda * (c0 + u)] = v[u];
    }
}

__device__ __forceinline__ void flag_status(char* wsb, int bits) {
  atomicOr(reinterpret_cast<int*>(wsb + kStatusOff), bits);
}

// FP16 plans: the sketch kernels split X 2^s (s = x_scale_log2), so every
// sketch holds 2^s times its value.  Scale the sketches of item item0 +
// blockIdx.y back by 2^-s (exact in FP64) and flag a non-finite entry (an
// inf or NaN in X, or |X| 2^s past the FP16 range), which is replaced by
// zero so that the finalize runs on finite values (its result is then
// meaningless; the status word says so).
__global__ void __launch_bounds__(kThreads) sketch_unscale_kernel(char* wsb, int item0) {
  const DevItem& it = ditems(wsb)[item0 + (int)blockIdx.y];
  if (it.prec != TT_PREC_FP16) return;
  const DevSketch* sks = dsk(wsb);
  double* ws = reinterpret_cast<double*>(wsb);
  const double f = ldexp(1.0, -it.x_scale_log2);
  int bad = 0;
  auto scale = [&](double& x) {
    const double v = x * f;
    const bool fin = isfinite(v);
    bad |= fin ? 0 : 1;
    x = fin ? v : 0.0;
  };
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& d = sks[it.sk0 + s];
    double* p = ws + d.off;  // 16-byte aligned (workspace regions are)
    const int64_t n = d.rows * d.width;
    double2* p2 = reinterpret_cast<double2*>(p);
    for (int64_t e = tid; e < n / 2; e += nthr) {
      double2 v = p2[e];
      scale(v.x);
      scale(v.y);
      p2[e] = v;
    }
    if ((n & 1) && tid == 0) scale(p[n - 1]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) flag_status(wsb, ST_NONFINITE);
}

// ------------------------------------------------------------------ TSQR up
// One task = one row block of level L of one basis sketch (launch Lg holds
// the tasks whose tree has Lg - L more levels above them than the deepest
// tree, so that every root runs in the last launch).  Non-root blocks write
// their R into the next level's matrix; the root block also does the CPQR of
// R, the rank decision and the first expansion step.
__global__ void __launch_bounds__(kThreads, 4) tsqr_level_kernel(char* wsb, int Lg, int* ranks) {
  extern __shared__ double sm[];
  const DevTables& T = tables(wsb);
  const Task task = reinterpret_cast<const Task*>(wsb + T.off_tasks[Lg])[blockIdx.x];
  const int L = task.lev;
  const DevSketch& s = dsk(wsb)[task.sk];
  const DevItem& it = ditems(wsb)[s.item];
  double* ws = reinterpret_cast<double*>(wsb);
  const int w = s.width;
  const int64_t m = s.lev_rows[L];
  const int64_t r0 = (int64_t)task.blk * s.bl;
  const int nr = (int)imin64(s.bl, m - r0);
  const int lda = nr + 1;
  double* A = sm;                         // lda x w
  double* red = A + (size_t)lda * w;      // 32
  double* beta = red + 32;                // w
  double* rdiag = beta + TT_MAXL;         // w
  double* Rs = rdiag + TT_MAXL;           // w x w (root only)
  double* Q2 = Rs + w * w;                // w x w (root only), then w x w of rank sums
  __shared__ int piv[TT_MAXL];
  __shared__ int s_rank;
  double* Y = ws + s.lev_mat[L];
  load_block(A, lda, Y + r0, m, nr, w);
  __syncthreads();
  house_qr(A, lda, nr, w, beta, rdiag);
  const int kmax = min(nr, w);
  // Householder vectors back in place, scalars to the level's beta array
  for (int o = threadIdx.x; o < nr * w; o += blockDim.x) {
    const int r = o % nr, c = o / nr;
    Y[r0 + r + m * c] = A[r + lda * c];
  }
  for (int i = threadIdx.x; i < w; i += blockDim.x) ws[s.lev_beta[L] + (int64_t)task.blk * w + i] = beta[i];
  auto rval = [&](int i, int c) -> double {
    if (i >= kmax || c < i) return 0.0;
    return c == i ? rdiag[i] : A[i + lda * c];
  };
  const bool root = (s.lev_nblk[L] == 1);
  if (!root) {
    const int64_t m1 = s.lev_rows[L + 1];
    double* Yn = ws + s.lev_mat[L + 1];
    for (int o = threadIdx.x; o < w * w; o += blockDim.x) {
      const int i = o % w, c = o / w;
      Yn[(int64_t)task.blk * w + i + m1 * c] = rval(i, c);
    }
    return;
  }
  // ---- root: CPQR of R (w x w) in shared memory.  Per step: warp 0 picks
  // the pivot (largest recomputed trailing norm, lowest index on ties), swaps
  // it into place and forms the reflector; then each warp applies it to its
  // own columns and recomputes their trailing norms for the next step.
  for (int o = threadIdx.x; o < w * w; o += blockDim.x) {
    const int i = o % w, c = o / w;
    Rs[i + w * c] = rval(i, c);
  }
  for (int c = threadIdx.x; c < w; c += blockDim.x) piv[c] = c;
  __syncthreads();
  __shared__ double nrm[TT_MAXL];
  __shared__ double qb[TT_MAXL], qd[TT_MAXL];
  double total2 = 0.0;
  for (int o = threadIdx.x; o < w * w; o += blockDim.x) total2 += Rs[o] * Rs[o];
  total2 = block_sum(total2, red);
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = wid; c < w; c += nw) {  // trailing norms of step 0
      double t = 0.0;
      for (int r = lane; r < w; r += 32) t = fma(Rs[r + w * c], Rs[r + w * c], t);
      t = warp_sum(t);
      if (lane == 0) nrm[c] = t;
    }
    __syncthreads();
    for (int i = 0; i < w; ++i) {
      if (wid == 0) {
        // argmax over c >= i; norms are >= 0, so their bit patterns order like them
        long long key = -1;
        int arg = w;
        for (int c = i + lane; c < w; c += 32) {
          const long long k2 = __double_as_longlong(nrm[c]);
          if (k2 > key) key = k2, arg = c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
          const int a2 = __shfl_xor_sync(0xffffffffu, arg, o);
          if (k2 > key || (k2 == key && a2 < arg)) key = k2, arg = a2;
        }
        // no key above -1 (every trailing norm a NaN with the sign bit set):
        // keep column i, so that the swap stays inside the block
        const int j = arg < w ? arg : i;
        if (j != i) {
          for (int r = lane; r < w; r += 32) {
            const double t = Rs[r + w * i];
            Rs[r + w * i] = Rs[r + w * j];
            Rs[r + w * j] = t;
          }
          if (lane == 0) {
            const int t = piv[i];
            piv[i] = piv[j];
            piv[j] = t;
            const double tn = nrm[i];
            nrm[i] = nrm[j];
            nrm[j] = tn;
          }
        }
        __syncwarp();
        if (lane == 0) {  // Householder on column i, rows i..w-1
          const double nsq = nrm[i];
          const double x0 = Rs[i + w * i];
          const double nx = sqrt(nsq);
          double alpha = 0.0, b = 0.0;
          if (nx > 0.0) {
            alpha = -copysign(nx, x0);
            const double v0 = x0 - alpha;
            const double vn2 = nsq - x0 * x0 + v0 * v0;
            b = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
          }
          Rs[i + w * i] = nx > 0.0 ? x0 - alpha : 0.0;
          qb[i] = b;
          qd[i] = alpha;
        }
      }
      __syncthreads();
      const double b = qb[i];
      for (int cb = i + 1 + wid; cb < w; cb += 4 * nw) {
        switch (min(4, (w - 1 - cb) / nw + 1)) {
          case 1: cpqr_group<1>(Rs, w, i, cb, nw, b, nrm); break;
          case 2: cpqr_group<2>(Rs, w, i, cb, nw, b, nrm); break;
          case 3: cpqr_group<3>(Rs, w, i, cb, nw, b, nrm); break;
          default: cpqr_group<4>(Rs, w, i, cb, nw, b, nrm); break;
        }
      }
      __syncthreads();
    }
  }
  // Q2 = H_0 ... H_{w-1} I
  for (int o = threadIdx.x; o < w * w; o += blockDim.x) Q2[o] = (o % w == o / w) ? 1.0 : 0.0;
  __syncthreads();
  expand_cols(Rs, w, qb, w, w, Q2, w, w, w, Q2, w);
  __syncthreads();
  // Rt with signs normalised (diag >= 0), Q2 columns likewise
  double* Rt = ws + s.off_rt;
  for (int o = threadIdx.x; o < w * w; o += blockDim.x) {
    const int i = o % w, c = o / w;
    const double sg = qd[i] < 0.0 ? -1.0 : 1.0;
    double v = 0.0;
    if (c > i) v = Rs[i + w * c];
    else if (c == i) v = qd[i];
    Rt[o] = sg * v;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < w * w; o += blockDim.x) {
    const int c = o / w;
    const double sg = qd[c] < 0.0 ? -1.0 : 1.0;
    Q2[o] *= sg;
    ws[s.off_q2 + o] = Q2[o];
  }
  for (int c = threadIdx.x; c < w; c += blockDim.x) reinterpret_cast<int*>(ws + s.off_piv)[c] = piv[c];
  __syncthreads();
  // rank decision.  tail(r) = ||Rt(r:, r:)||_F^2 = sum_{c >= r} t_c(r) with
  // t_c(r) = sum_{i = r..c} Rt(i, c)^2; thread c forms t_c(.) by a running sum
  // from the diagonal up, then tail(r) is summed over the columns.
  double* tcol = Q2 + w * w;  // t_c(r) at [r + w c] (r <= c), w x w
  __shared__ double tails[TT_MAXL + 1];
  for (int c = threadIdx.x; c < w; c += blockDim.x) {
    double run = 0.0;
    for (int i2 = c; i2 >= 0; --i2) {
      run += Rt[i2 + w * c] * Rt[i2 + w * c];
      tcol[i2 + w * c] = run;
    }
  }
  __syncthreads();
  for (int cand = threadIdx.x; cand <= w; cand += blockDim.x) {
    double tail = 0.0;
    for (int c = cand; c < w; ++c) tail += tcol[cand + w * c];
    tails[cand] = tail;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int limit = min(s.rpad, w);
    int r = s.target_rank;
    if (it.eps_mode) {
      const double thr = it.eps / sqrt((double)max(it.d - 1, 1)) * sqrt(total2);
      r = limit;
      bool met = false;
      for (int cand = 1; cand <= limit; ++cand) {
        if (sqrt(tails[cand]) <= thr) {
          r = cand;
          met = true;
          break;
        }
      }
      if (!met) flag_status(wsb, ST_RANK_CAP);
    }
    r = max(1, min(r, limit));
    s_rank = r;
    int* rk = ranks + it.rank_off;
    rk[s.k] = r;
    if (s.k == 1) rk[0] = 1;
    if (s.k == it.d - 1) rk[it.d] = 1;
    if (it.rank_off == 0) {  // copy for the backward of a single-item plan
      int* cp = reinterpret_cast<int*>(wsb + kRankCopyOff);
      cp[s.k] = r;
      if (s.k == 1) cp[0] = 1;
      if (s.k == it.d - 1) cp[it.d] = 1;
    }
  }
  __syncthreads();
  const int r = s_rank;
  // leading r x r block of Rt for the backward pass (rpad x rpad, zero padded)
  for (int o = threadIdx.x; o < s.rpad * s.rpad; o += blockDim.x) {
    const int i = o % s.rpad, c = o / s.rpad;
    ws[it.off_rr[s.k] + o] = (i < r && c < r) ? Rt[i + w * c] : 0.0;
  }
  // Z_root = Q_root [Q2(:, 1:r); 0]  (m x rpad, columns >= r are zero)
  expand_cols(A, lda, beta, nr, w, Q2, w, r, s.rpad, ws + s.lev_z[L], m);
}

// ---------------------------------------------------------------- TSQR down
// Z_L(block) = Q_block [Z_{L+1}(rows of this block's R); 0].
__global__ void __launch_bounds__(kThreads) tsqr_expand_kernel(char* wsb, int Lg, const int* ranks) {
  extern __shared__ double sm[];
  const DevTables& T = tables(wsb);
  const Task task = reinterpret_cast<const Task*>(wsb + T.off_tasks[Lg])[blockIdx.x];
  const int L = task.lev;
  const DevSketch& s = dsk(wsb)[task.sk];
  if (s.nlev - 1 <= L) return;  // root of this tree, already expanded
  const DevItem& it = ditems(wsb)[s.item];
  double* ws = reinterpret_cast<double*>(wsb);
  const int w = s.width;
  const int r = ranks[it.rank_off + s.k];
  const int64_t m = s.lev_rows[L];
  const int64_t r0 = (int64_t)task.blk * s.bl;
  const int nr = (int)imin64(s.bl, m - r0);
  const int lda = nr + 1;
  double* V = sm;
  double* beta = V + (size_t)lda * w;
  const double* Y = ws + s.lev_mat[L];
  load_block(V, lda, Y + r0, m, nr, w);
  for (int i = threadIdx.x; i < w; i += blockDim.x) beta[i] = ws[s.lev_beta[L] + (int64_t)task.blk * w + i];
  const int64_t m1 = s.lev_rows[L + 1];
  __syncthreads();
  expand_cols(V, lda, beta, nr, w, ws + s.lev_z[L + 1] + (int64_t)task.blk * w, m1, r, s.rpad,
              ws + s.lev_z[L] + r0, m);
}

// --------------------------------------------------------- one-pass middle
// B = P_{d*}^T Omega_{d*}  (r x l), summed over row chunks with atomics.
// item < 0: batched launch, item = blockIdx.y
__global__ void __launch_bounds__(kThreads) mid_b_kernel_f64(char* wsb, int item_arg, const int* ranks) {
  const int item = item_arg >= 0 ? item_arg : (int)blockIdx.y;
  constexpr int CH = 32;
  __shared__ double Ps[CH * TT_MAXL];
  __shared__ double Gs[CH * (TT_MAXL + 1)];
  const DevItem& it = ditems(wsb)[item];
  const DevSketch& sp = dsk(wsb)[it.basis_of_k[it.mbk]];
  // the middle test matrix is the one the least-squares sketch used
  const DevSketch* kr_mid = dsk(wsb)[it.mid_sk].kr_nm ? &dsk(wsb)[it.mid_sk] : nullptr;
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
      double z[4];
      tm_quad_f64(wsb, kr_mid, it.seed, (uint32_t)it.mstream, (uint64_t)(v0 + v), (uint32_t)q, z);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < l) Gs[v + CH * (4 * q + t)] = z[t];
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

// QR of B^T (l x r) -> QB (l x r), RB (r x r); singular B is flagged.
// item < 0: batched launch, item = blockIdx.y
__global__ void __launch_bounds__(kThreads) mid_ls_kernel(char* wsb, int item_arg, const int* ranks) {
  const int item = item_arg >= 0 ? item_arg : (int)blockIdx.y;
  __shared__ double A[TT_MAXL * (TT_MAXL + 1)];
  __shared__ double beta[TT_MAXL], rdiag[TT_MAXL];
  const DevItem& it = ditems(wsb)[item];
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + it.mbk];
  const int l = it.lmid;
  const int rp = it.rpad[it.mbk];
  const int lda = l + 1;
  for (int o = threadIdx.x; o < l * r; o += blockDim.x) {
    const int j = o % l, c = o / l;
    A[j + lda * c] = ws[it.off_B + c + (int64_t)rp * j];  // B^T(j, c) = B(c, j)
  }
  __syncthreads();
  house_qr(A, lda, l, r, beta, rdiag);
  // RB (rp x rp) with diag >= 0; QB = H_0..H_{r-1} [I_r; 0] with matching signs
  double* RB = ws + it.off_RB;
  double* QB = ws + it.off_QB;
  __shared__ double sgn[TT_MAXL];
  __shared__ double rmax_abs;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < r; ++i) mx = fmax(mx, fabs(rdiag[i]));
    rmax_abs = mx;
  }
  for (int i = threadIdx.x; i < r; i += blockDim.x) sgn[i] = rdiag[i] < 0.0 ? -1.0 : 1.0;
  __syncthreads();
  for (int o = threadIdx.x; o < rp * rp; o += blockDim.x) {
    const int i = o % rp, c = o / rp;
    double v = 0.0;
    if (i < r && c < r && c >= i) v = sgn[i] * (c == i ? rdiag[i] : A[i + lda * c]);
    RB[o] = v;
  }
  if (threadIdx.x == 0) {
    bool sing = !(rmax_abs > 0.0);
    for (int i = 0; i < r; ++i)
      if (!(fabs(rdiag[i]) > 1e-13 * rmax_abs)) sing = true;
    if (sing) flag_status(wsb, ST_RANK_DEFICIENT);
  }
  for (int o = threadIdx.x; o < l * rp; o += blockDim.x) {
    const int j = o % l, c = o / l;
    QB[j + (int64_t)l * c] = (c < r && j == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  apply_q(A, lda, beta, l, r, QB, l, r);
  // M = QB RB^{-T}, stored over QB: row j solves m RB^T = QB(j, :) from the
  // last column (a zero diagonal of RB gives a zero column, as flagged above),
  // so that H = S_{d*} M is a plain product.
  __shared__ double rinv[TT_MAXL];
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    const double dg = RB[c + rp * c];
    rinv[c] = dg != 0.0 ? 1.0 / dg : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < l; j += blockDim.x) {
    for (int c = r - 1; c >= 0; --c) {
      double t = QB[j + (int64_t)l * c] * sgn[c];
      for (int c2 = c + 1; c2 < r; ++c2) t = fma(-QB[j + (int64_t)l * c2], RB[c + rp * c2], t);
      QB[j + (int64_t)l * c] = t * rinv[c];
    }
  }
}

// H = S_{d*} M  (N_{d*} x rpad, columns >= r zero), M = QB RB^{-T} (l x r)
// from mid_ls_kernel; one thread per entry of H.
// item < 0: batched launch, item = blockIdx.y
__global__ void __launch_bounds__(kThreads) mid_h_kernel(char* wsb, int item_arg, const int* ranks) {
  const int item = item_arg >= 0 ? item_arg : (int)blockIdx.y;
  __shared__ double Ms[TT_MAXL * TT_MAXL];
  const DevItem& it = ditems(wsb)[item];
  const DevSketch& sm_ = dsk(wsb)[it.mid_sk];
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + it.mbk];
  const int rp = it.rpad[it.mbk];
  const int l = it.lmid;
  for (int o = threadIdx.x; o < l * r; o += blockDim.x) Ms[o] = ws[it.off_QB + o];
  __syncthreads();
  const int64_t Nm = sm_.rows;
  const double* S = ws + sm_.off;
  double* H = ws + it.off_H;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < Nm * rp; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = o % Nm;
    const int c = (int)(o / Nm);
    double h = 0.0;
    if (c < r)
      for (int j = 0; j < l; ++j) h = fma(S[u + Nm * j], Ms[j + l * c], h);
    H[o] = h;
  }
}

// --------------------------------------------------------------- the cores
// Left type  (k <= d*): G(a,i,c) = sum_u A(u,a) B(u + N_{k-1} i, c),  A = Q_{k-1}
//            (identity 1x1 for k = 1), B = Q_k or H (middle core, one-pass).
// Right type (k > d*):  G(a,i,c) = sum_v A(i + n_k v, a) B(v, c),   A = P_{k-1},
//            B = P_k (identity 1x1 for k = d).
//
// Both are G(:, i, :) = A_i^T B_i (ra x rc) over a contraction of length
// `inner`: left A_i = A, B_i = rows [inner i, inner (i + 1)) of B; right A_i =
// rows {i + n_k v} of A, B_i = B; an absent factor is the 1 x 1 identity.  One
// block per (item, k, slice i): chunks of A_i and B_i are staged in shared
// memory and the threads split the (a, c) pairs and the contraction index, so
// the FP64 work is the plain multiply-adds with one short reduction per pair.
constexpr int kCoreChunk = 32;
__global__ void __launch_bounds__(kThreads) cores_kernel(char* wsb, double* cores, const int* ranks,
                                                         int item0, int nitems, int only_k, int dmax) {
  __shared__ double sA[kCoreChunk * TT_MAXL], sB[kCoreChunk * TT_MAXL];
  __shared__ double red[kThreads];
  const int item = item0 + (int)blockIdx.x / dmax;
  const int k = (int)blockIdx.x % dmax + 1;
  if (item >= item0 + nitems) return;
  const DevItem& it = ditems(wsb)[item];
  if (k > it.d) return;
  if (only_k > 0 && k != only_k) return;
  if (only_k == 0 && k == it.mcore && it.passes == 2) return;  // second pass computes it
  const DevSketch* S = dsk(wsb);
  const double* ws = reinterpret_cast<const double*>(wsb);
  const int* rk = ranks + it.rank_off;
  const int ra = rk[k - 1], rc = rk[k];
  const int rpa = it.rpad[k - 1], rpc = it.rpad[k];
  const int64_t nk = it.n[k - 1];
  double* G = cores + it.core_off[k];
  const bool left = k <= it.ds;
  const double* A = nullptr;
  const double* B = nullptr;
  int64_t lda = 0, ldb = 0, inner = 0;
  if (left) {
    inner = it.N[k - 1];
    if (k >= 2) {
      const DevSketch& sa = S[it.basis_of_k[k - 1]];
      A = ws + sa.lev_z[0];
      lda = sa.rows;
    }
    if (k == it.mcore) {
      B = ws + it.off_H;
      ldb = it.N[k];
    } else {
      const DevSketch& sb = S[it.basis_of_k[k]];
      B = ws + sb.lev_z[0];
      ldb = sb.rows;
    }
  } else {
    inner = it.N[it.d] / it.N[k];
    if (k == it.mcore) {  // one-sided last core: G_d(a, i, 0) = H(i, a)
      A = ws + it.off_H;
      lda = S[it.mid_sk].rows;
    } else {
      const DevSketch& sa = S[it.basis_of_k[k - 1]];
      A = ws + sa.lev_z[0];
      lda = sa.rows;
    }
    if (k < it.d) {
      const DevSketch& sb = S[it.basis_of_k[k]];
      B = ws + sb.lev_z[0];
      ldb = sb.rows;
    }
  }
  const int P = ra * rc;
  for (int64_t i = blockIdx.y; i < nk; i += gridDim.y) {
    double* Gi = G + rpa * i;  // G(a, i, c) = Gi[a + rpa nk c]
    for (int pg = 0; pg < P; pg += blockDim.x) {
      const int Pg = min(P - pg, (int)blockDim.x), nsplit = blockDim.x / Pg;
      const int p = pg + (int)threadIdx.x % Pg, sp = (int)threadIdx.x / Pg;
      const int a = p % ra, c = p / ra;
      double acc = 0.0;
      for (int64_t u0 = 0; u0 < inner; u0 += kCoreChunk) {
        const int uc = (int)imin64(kCoreChunk, inner - u0);
        __syncthreads();
        for (int o = threadIdx.x; o < uc * ra; o += blockDim.x) {
          const int u = o % uc, aa = o / uc;
          sA[u + kCoreChunk * aa] = left ? (A ? A[u0 + u + lda * aa] : 1.0) : A[i + nk * (u0 + u) + lda * aa];
        }
        for (int o = threadIdx.x; o < uc * rc; o += blockDim.x) {
          const int u = o % uc, cc = o / uc;
          sB[u + kCoreChunk * cc] = left ? B[u0 + u + inner * i + ldb * cc] : (B ? B[u0 + u + ldb * cc] : 1.0);
        }
        __syncthreads();
        if (sp < nsplit)
          for (int u = sp; u < uc; u += nsplit) acc = fma(sA[u + kCoreChunk * a], sB[u + kCoreChunk * c], acc);
      }
      red[threadIdx.x] = sp < nsplit ? acc : 0.0;
      __syncthreads();
      if ((int)threadIdx.x < Pg) {
        double t = 0.0;
        for (int q = 0; q < nsplit; ++q) t += red[threadIdx.x + Pg * q];
        Gi[a + rpa * nk * c] = t;
      }
      __syncthreads();
    }
    for (int o = threadIdx.x; o < rpa * rpc; o += blockDim.x) {
      const int a = o % rpa, c = o / rpa;
      if (a >= ra || c >= rc) Gi[a + rpa * nk * c] = 0.0;
    }
  }
}

// Two-pass middle core, eq. (3.5): G_{d*}(a, i, c) =
//   sum_{u, v} Q_{d*-1}(u, a) X(u + N_{d*-1} i + N_{d*} v) P_{d*}(v, c).
// One block per (i, chunk of v): y(v, a) = sum_u Q(u, a) X(...), then the
// block adds sum_v y(v, a) P(v, c) into the (zeroed) core with atomics.
__global__ void __launch_bounds__(kThreads) twopass_mid_kernel(char* wsb, const void* X, double* cores,
                                                               const int* ranks) {
  constexpr int CH = 64;
  __shared__ double Ys[CH * TT_MAXL];
  const DevItem& it = ditems(wsb)[0];
  const DevSketch* S = dsk(wsb);
  const double* ws = reinterpret_cast<const double*>(wsb);
  const int ds = it.ds;
  const int* rk = ranks + it.rank_off;
  const int ra = rk[ds - 1], rc = rk[ds];
  const int rpa = it.rpad[ds - 1];
  const int64_t Np = it.N[ds - 1], nk = it.n[ds - 1], Nm = it.N[ds];
  const int64_t Mm = it.N[it.d] / Nm;
  const double* Q = nullptr;
  int64_t ldq = 1;
  if (ds >= 2) {
    Q = ws + S[it.basis_of_k[ds - 1]].lev_z[0];
    ldq = S[it.basis_of_k[ds - 1]].rows;
  }
  const DevSketch& sp = S[it.basis_of_k[ds]];
  const double* Pm = ws + sp.lev_z[0];
  double* G = cores + it.core_off[ds];
  const int64_t nchunks = (Mm + CH - 1) / CH;
  for (int64_t job = blockIdx.x; job < nk * nchunks; job += gridDim.x) {
    const int64_t i = job % nk, v0 = (job / nk) * CH;
    const int nv = (int)imin64(CH, Mm - v0);
    __syncthreads();
    for (int o = threadIdx.x; o < CH * ra; o += blockDim.x) {
      const int v = o % CH, a = o / CH;
      double acc = 0.0;
      if (v < nv) {
        const int64_t base = Np * i + Nm * (v0 + v);
        for (int64_t u = 0; u < Np; ++u) {
          const double x = it.x_f64 ? ((const double*)X)[base + u] : (double)((const float*)X)[base + u];
          acc += (Q ? Q[u + ldq * a] : 1.0) * x;
        }
      }
      Ys[v + CH * a] = acc;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < ra * rc; o += blockDim.x) {
      const int a = o % ra, c = o / ra;
      double acc = 0.0;
      for (int v = 0; v < nv; ++v) acc += Ys[v + CH * a] * Pm[v0 + v + sp.rows * c];
      atomicAdd(G + a + rpa * (i + nk * c), acc);
    }
  }
}

// One-sided two-pass last core (Algorithm 2): G_d(a, i, 0) = sum_u
// Q_{d-1}(u, a) X(u + N_{d-1} i).  Block (i, row chunk): the threads stride
// over the chunk's rows (coalesced in X and in each column of Q), eight
// columns a at a time with unconditional FMAs (columns past r_{d-1} read
// column r_{d-1} - 1 and are dropped), then a block sum and one atomic per a.
__global__ void __launch_bounds__(kThreads) twopass_last_kernel(char* wsb, const void* X, double* cores,
                                                                const int* ranks, int64_t chunk) {
  __shared__ double red[32];
  const DevItem& it = ditems(wsb)[0];
  const DevSketch& sq = dsk(wsb)[it.basis_of_k[it.d - 1]];
  const double* ws = reinterpret_cast<const double*>(wsb);
  const double* Q = ws + sq.lev_z[0];
  const int64_t ldq = sq.rows;
  const int ra = ranks[it.rank_off + it.d - 1];
  const int rpa = it.rpad[it.d - 1];
  const int64_t Np = it.N[it.d - 1];
  const int64_t i = blockIdx.x;
  const int64_t u0 = (int64_t)blockIdx.y * chunk, u1 = imin64(Np, u0 + chunk);
  double* G = cores + it.core_off[it.d];
  for (int a0 = 0; a0 < ra; a0 += 8) {
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const double* qc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) qc[j] = Q + ldq * min(a0 + j, ra - 1);
    for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
      const int64_t e = u + Np * i;
      const double x = it.x_f64 ? reinterpret_cast<const double*>(X)[e] : (double)reinterpret_cast<const float*>(X)[e];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = fma(qc[j][u], x, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const double t = block_sum(acc[j], red);
      if (threadIdx.x == 0 && a0 + j < ra) atomicAdd(G + (a0 + j) + (int64_t)rpa * i, t);
    }
  }
}

}  // namespace

cudaError_t launch_mid_b_mixed(const Plan& P, int item, void* ws, const int* ranks, cudaStream_t st);

// Middle cores of every item of a batched plan; B was zeroed with the sketches.
cudaError_t launch_finalize_mid_batched(const Plan& P, void* ws, const int* ranks, cudaStream_t st) {
  char* wsb = (char*)ws;
  const int nitems = plan_num_items(&P);
  const DevSketch* sks = plan_sketches_host(&P);
  int64_t Mmax = 1, Nmax = 1;
  for (int i = 0; i < nitems; ++i) {
    const DevItem& it = plan_items_host(&P)[i];
    Mmax = std::max(Mmax, sks[it.basis_of_k[it.mbk]].rows);
    Nmax = std::max(Nmax, sks[it.mid_sk].rows);
  }
  cudaError_t e;
  if (plan_items_host(&P)[0].prec == TT_PREC_FP64) {
    const unsigned gx = (unsigned)std::min<int64_t>((Mmax + 31) / 32, 64);
    count_launch();
    mid_b_kernel_f64<<<dim3(gx, (unsigned)nitems), kThreads, 0, st>>>(wsb, -1, ranks);
    e = cudaGetLastError();
  } else {
    e = launch_mid_b_mixed_batched(P, ws, ranks, st);
  }
  if (e != cudaSuccess) return e;
  count_launch();
  mid_ls_kernel<<<dim3(1, (unsigned)nitems), kThreads, 0, st>>>(wsb, -1, ranks);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned gx = (unsigned)std::min<int64_t>((Nmax * TT_MAXL + kThreads - 1) / kThreads, 64);
  count_launch();
  mid_h_kernel<<<dim3(gx, (unsigned)nitems), kThreads, 0, st>>>(wsb, -1, ranks);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Plan& P, void* ws, double* cores, int* ranks, cudaStream_t st) {
  char* wsb = (char*)ws;
  const int max_lev = plan_max_lev(&P);
  const DevSketch* sks = plan_sketches_host(&P);
  const int nitems = plan_num_items(&P);
  cudaError_t e;
  if (nitems == 1) {  // the slab kernel's staged S_2 partials not yet folded
    e = fold_s2_staging(P, 0, ws, st);
    if (e != cudaSuccess) return e;
  }
  static bool attr = false;
  if (!attr) {
    e = cudaFuncSetAttribute(tsqr_level_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTsqrSmemMax);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tsqr_expand_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTsqrSmemMax);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // FP16 items: sketches back to the scale of X, and the range check
  {
    bool any16 = false;
    for (int i = 0; i < nitems; ++i) any16 = any16 || plan_items_host(&P)[i].prec == TT_PREC_FP16;
    if (any16) {
      count_launch();
      sketch_unscale_kernel<<<dim3((unsigned)(4 * device_sm_count()), (unsigned)nitems), kThreads, 0, st>>>(wsb, 0);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  // smem: block (bl+1) x w + scalars + two w x w matrices (root)
  int maxw = 1, maxbl = 1;
  for (int i = 0, n = 0; i < nitems; ++i) {
    const DevItem& it = plan_items_host(&P)[i];
    for (int s = 0; s < it.nsk; ++s) {
      const DevSketch& d = sks[it.sk0 + s];
      if (!d.basis) continue;
      maxw = std::max(maxw, d.width);
      maxbl = std::max(maxbl, d.bl);
      ++n;
    }
  }
  size_t smem_up = 0;
  for (int i = 0; i < nitems; ++i) {
    const DevItem& it = plan_items_host(&P)[i];
    for (int s = 0; s < it.nsk; ++s) {
      const DevSketch& d = sks[it.sk0 + s];
      if (!d.basis) continue;
      const size_t need = sizeof(double) * ((size_t)(d.bl + 1) * d.width + 32 + 2 * TT_MAXL +
                                            3 * (size_t)d.width * d.width);
      smem_up = std::max(smem_up, need);
    }
  }
  for (int L = 0; L < max_lev; ++L) {
    const int nt = plan_ntasks(&P, L);
    if (nt == 0) continue;
    count_launch();
    tsqr_level_kernel<<<nt, kThreads, smem_up, st>>>(wsb, L, ranks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  for (int L = max_lev - 2; L >= 0; --L) {
    const int nt = plan_ntasks(&P, L);
    if (nt == 0) continue;
    const size_t smem = sizeof(double) * ((size_t)(maxbl + 1) * maxw + TT_MAXL);
    count_launch();
    tsqr_expand_kernel<<<nt, kThreads, smem, st>>>(wsb, L, ranks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // one-pass middle cores (one launch per step over all items when batched)
  if (nitems > 1) {
    e = launch_finalize_mid_batched(P, ws, ranks, st);
    if (e != cudaSuccess) return e;
  }
  for (int i = 0; i < nitems && nitems == 1; ++i) {
    const DevItem& it = plan_items_host(&P)[i];
    if (it.passes != 1) continue;
    const int rp = it.rpad[it.mbk];
    e = cudaMemsetAsync((double*)ws + it.off_B, 0, sizeof(double) * rp * it.lmid, st);
    if (e != cudaSuccess) return e;
    if (it.prec == TT_PREC_FP64) {
      const int64_t M = sks[it.basis_of_k[it.mbk]].rows;
      const int grid = (int)std::min<int64_t>((M + 31) / 32, 2LL * device_sm_count());
      count_launch();
      mid_b_kernel_f64<<<grid, kThreads, 0, st>>>(wsb, i, ranks);
      e = cudaGetLastError();
    } else {
      e = launch_mid_b_mixed(P, i, ws, ranks, st);
    }
    if (e != cudaSuccess) return e;
    count_launch();
    mid_ls_kernel<<<1, kThreads, 0, st>>>(wsb, i, ranks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t Nm = sks[it.mid_sk].rows;
    const int grid = (int)std::min<int64_t>((Nm * it.rpad[it.mbk] + kThreads - 1) / kThreads, 8LL * device_sm_count());
    count_launch();
    mid_h_kernel<<<grid, kThreads, 0, st>>>(wsb, i, ranks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  int dmax = 1;
  int64_t nmax = 1;
  for (int i = 0; i < nitems; ++i) {
    const DevItem& it = plan_items_host(&P)[i];
    dmax = std::max(dmax, it.d);
    for (int k = 0; k < it.d; ++k) nmax = std::max(nmax, it.n[k]);
  }
  const int64_t gy = std::min<int64_t>(nmax, std::max<int64_t>(1, 2048 / ((int64_t)nitems * dmax)));
  dim3 grid((unsigned)(nitems * dmax), (unsigned)gy);
  count_launch();
  cores_kernel<<<grid, kThreads, 0, st>>>(wsb, cores, ranks, 0, nitems, 0, dmax);
  return cudaGetLastError();
}

// Cores of one item only (k = only_k), used by the two-pass middle core.
cudaError_t launch_cores_one(const Plan& P, int item, int only_k, void* ws, double* cores,
                             const int* ranks, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  dim3 grid((unsigned)it.d, (unsigned)std::min<int64_t>(it.n[only_k - 1], 512));
  count_launch();
  cores_kernel<<<grid, kThreads, 0, st>>>((char*)ws, cores, ranks, item, 1, only_k, it.d);
  return cudaGetLastError();
}

}  // namespace tts

namespace tts {
cudaError_t launch_twopass_mid(const Plan& P, const void* X, void* ws, double* cores, const int* ranks,
                               cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[0];
  if (it.sided1) {  // the last core G_d = Q_{d-1}^T X_{d-1}
    const int d = it.d;
    cudaError_t e = cudaMemsetAsync(cores + it.core_off[d], 0, sizeof(double) * it.rpad[d - 1] * it.n[d - 1], st);
    if (e != cudaSuccess) return e;
    const int64_t Np = it.N[d - 1], chunk = 65536;
    const dim3 grid((unsigned)it.n[d - 1], (unsigned)((Np + chunk - 1) / chunk));
    count_launch();
    twopass_last_kernel<<<grid, kThreads, 0, st>>>((char*)ws, X, cores, ranks, chunk);
    return cudaGetLastError();
  }
  const int ds = it.ds;
  cudaError_t e = cudaMemsetAsync(cores + it.core_off[ds], 0,
                                  sizeof(double) * it.rpad[ds - 1] * it.n[ds - 1] * it.rpad[ds], st);
  if (e != cudaSuccess) return e;
  const int64_t Mm = it.N[it.d] / it.N[ds];
  const int64_t jobs = it.n[ds - 1] * ((Mm + 63) / 64);
  const int grid = (int)std::min<int64_t>(jobs, 8LL * device_sm_count());
  count_launch();
  twopass_mid_kernel<<<grid, kThreads, 0, st>>>((char*)ws, X, cores, ranks);
  return cudaGetLastError();
}
}  // namespace tts
