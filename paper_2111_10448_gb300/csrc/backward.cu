// Backward (adjoint) of the one-pass PSTT2 map X -> cores, pivots and ranks
// frozen at the forward call, and of the reconstruction cores -> X~.
//
// X enters the one-pass map only through the sketches (Sec. 3.2), so
//   dX = sum_{k<=d*} Sbar_k Omega_k^T + sum_{k>=d*} Psi_k Rbar_k^T
// (each term read as a tensor through the unfolding X_k).  The adjoints of
// the sketches come from the small FP64 steps, in reverse order:
//  1. core products (eq. (3.1) and its row mirror)  -> Qbar_k, Pbar_k, Hbar
//  2. middle least squares H = S B^T (B B^T)^{-1}, B = P^T Omega (eq. (3.3)):
//       Sbar = Hbar C B,  Bbar = C Hbar^T (S - H B) - H^T Hbar C B,
//       Pbar += Omega Bbar^T,  C = (B B^T)^{-1} = RB^{-1} RB^{-T}
//  3. QR of the selected pivot columns A = Y(:, piv(1:r)) = Q R:
//       Abar = [Qbar - Q sym(Q^T Qbar)] R^{-T},  sym(W) = triu(W) + triu(W,1)^T,
//     scattered back into the pivot columns of Ybar (other columns get 0).
//  4. the write-once sketch adjoint over X (in the test-matrix TU).
#include <algorithm>

#include "internal.cuh"

namespace tts {

const DevSketch* plan_sketches_host(const Plan* p);

namespace {

constexpr int kThreads = 256;

int grid_for(int64_t n, int per = 16) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)per * device_sm_count()));
}

struct Ctx {
  const double* ws;
  const DevItem* it;
  const DevSketch* sk;
};

__device__ __forceinline__ const DevItem& item_of(const char* wsb, int item) {
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + 256);
  return reinterpret_cast<const DevItem*>(wsb + T.off_items)[item];
}
__device__ __forceinline__ const DevSketch* sketches_of(const char* wsb) {
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + 256);
  return reinterpret_cast<const DevSketch*>(wsb + T.off_sketches);
}

// 1. Qbar_k / Pbar_k from the core adjoints (gather form: one thread per entry).
__global__ void qbar_kernel(char* wsb, int item, int k, const double* dG, const int* ranks) {
  const DevItem& it = item_of(wsb, item);
  const DevSketch* S = sketches_of(wsb);
  const DevSketch& sb = S[it.basis_of_k[k]];
  double* ws = reinterpret_cast<double*>(wsb);
  const int* rk = ranks + it.rank_off;
  const int d = it.d, ds = it.ds;
  const int64_t rows = sb.rows;
  const int rp = sb.rpad;
  double* out = ws + it.off_qbar[k];
  auto G = [&](int kk, int a, int64_t i, int c) -> double {
    return dG[it.core_off[kk] + a + (int64_t)it.rpad[kk - 1] * (i + it.n[kk - 1] * c)];
  };
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * rp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e % rows;
    const int c = (int)(e / rows);
    double val = 0.0;
    if (c < rk[k]) {
      if (k < ds) {
        // B side of core k
        if (k == 1) {
          val += G(1, 0, row, c);
        } else {
          const DevSketch& sa = S[it.basis_of_k[k - 1]];
          const int64_t Np = it.N[k - 1];
          const int64_t u = row % Np, i = row / Np;
          for (int a = 0; a < rk[k - 1]; ++a) val += ws[sa.lev_z[0] + u + sa.rows * a] * G(k, a, i, c);
        }
        // A side of core k+1
        const int64_t nk1 = it.n[k], Nk = it.N[k];
        const double* Bm;
        int64_t ldb;
        if (k + 1 == ds) {
          Bm = ws + it.off_H;
          ldb = it.N[ds];
        } else {
          const DevSketch& s2 = S[it.basis_of_k[k + 1]];
          Bm = ws + s2.lev_z[0];
          ldb = s2.rows;
        }
        for (int64_t i2 = 0; i2 < nk1; ++i2)
          for (int c2 = 0; c2 < rk[k + 1]; ++c2) val += G(k + 1, c, i2, c2) * Bm[row + Nk * i2 + ldb * c2];
      } else {
        // A side of core k+1: P_k(i + n_{k+1} v, a)
        const int64_t nk1 = it.n[k];
        const int64_t i = row % nk1, v = row / nk1;
        if (k + 1 == d) {
          val += G(d, c, i, 0);
        } else {
          const DevSketch& s2 = S[it.basis_of_k[k + 1]];
          for (int c2 = 0; c2 < rk[k + 1]; ++c2) val += G(k + 1, c, i, c2) * ws[s2.lev_z[0] + v + s2.rows * c2];
        }
        // B side of core k (k > d*): P_k(v, c)
        if (k > ds) {
          const DevSketch& sa = S[it.basis_of_k[k - 1]];
          const int64_t nk = it.n[k - 1];
          for (int a = 0; a < rk[k - 1]; ++a)
            for (int64_t i2 = 0; i2 < nk; ++i2) val += ws[sa.lev_z[0] + i2 + nk * row + sa.rows * a] * G(k, a, i2, c);
        }
      }
    }
    out[row + rows * c] = val;
  }
}

// Hbar(u + N_{d*-1} i, c) = sum_a Q_{d*-1}(u, a) dG_{d*}(a, i, c).
__global__ void hbar_kernel(char* wsb, int item, const double* dG, const int* ranks) {
  const DevItem& it = item_of(wsb, item);
  const DevSketch* S = sketches_of(wsb);
  double* ws = reinterpret_cast<double*>(wsb);
  const int* rk = ranks + it.rank_off;
  const int ds = it.ds;
  const int64_t rows = it.N[ds];
  const int rp = it.rpad[ds];
  const int64_t Np = it.N[ds - 1];
  double* out = ws + it.off_hbar;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * rp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e % rows;
    const int c = (int)(e / rows);
    double val = 0.0;
    if (c < rk[ds]) {
      const int64_t u = row % Np, i = row / Np;
      auto G = [&](int a) { return dG[it.core_off[ds] + a + (int64_t)it.rpad[ds - 1] * (i + it.n[ds - 1] * c)]; };
      if (ds == 1) {
        val = G(0);
      } else {
        const DevSketch& sa = S[it.basis_of_k[ds - 1]];
        for (int a = 0; a < rk[ds - 1]; ++a) val += ws[sa.lev_z[0] + u + sa.rows * a] * G(a);
      }
    }
    out[row + rows * c] = val;
  }
}

// E = S_{d*} - H B (residual of the least squares), written into Sbar_{d*}.
__global__ void resid_kernel(char* wsb, int item, const int* ranks) {
  const DevItem& it = item_of(wsb, item);
  const DevSketch& sm = sketches_of(wsb)[it.mid_sk];
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + it.ds];
  const int rp = it.rpad[it.ds];
  const int l = it.lmid;
  const int64_t rows = sm.rows;
  double* E = ws + it.off_sbar[it.mid_sk - it.sk0];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * l;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = e % rows;
    const int j = (int)(e / rows);
    double v = ws[sm.off + u + rows * j];
    for (int c = 0; c < r; ++c) v -= ws[it.off_H + u + rows * c] * ws[it.off_B + c + (int64_t)rp * j];
    E[e] = v;
  }
}

// C (p x q, ld ldc) += A^T B over all rows, A: rows x p (ld lda), B: rows x q.
__global__ void gram_kernel(const double* A, int64_t lda, const double* Bm, int64_t ldb, int64_t rows, int p, int q,
                            double* C, int ldc) {
  constexpr int CH = 32;
  __shared__ double As[CH * TT_MAXL];
  __shared__ double Bs[CH * TT_MAXL];
  for (int64_t r0 = (int64_t)blockIdx.x * CH; r0 < rows; r0 += (int64_t)gridDim.x * CH) {
    const int nr = (int)imin64(CH, rows - r0);
    __syncthreads();
    for (int o = threadIdx.x; o < CH * p; o += blockDim.x) {
      const int u = o % CH, c = o / CH;
      As[u + CH * c] = u < nr ? A[r0 + u + lda * c] : 0.0;
    }
    for (int o = threadIdx.x; o < CH * q; o += blockDim.x) {
      const int u = o % CH, c = o / CH;
      Bs[u + CH * c] = u < nr ? Bm[r0 + u + ldb * c] : 0.0;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < p * q; o += blockDim.x) {
      const int i = o % p, j = o / p;
      double acc = 0.0;
      for (int u = 0; u < nr; ++u) acc += As[u + CH * i] * Bs[u + CH * j];
      atomicAdd(C + i + (int64_t)ldc * j, acc);
    }
  }
}

// C = RB^{-1} RB^{-T};  Bbar = C T1 - T2 C B;  CB = C B   (one block)
__global__ void ls_small_kernel(char* wsb, int item, const int* ranks, double* small) {
  __shared__ double Ri[TT_MAXL * TT_MAXL];
  __shared__ double Cm[TT_MAXL * TT_MAXL];
  __shared__ double CBs[TT_MAXL * TT_MAXL];
  const DevItem& it = item_of(wsb, item);
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + it.ds];
  const int rp = it.rpad[it.ds];
  const int l = it.lmid;
  const double* RB = ws + it.off_RB;
  const double* B = ws + it.off_B;
  const double* T1 = small;                   // rp x l
  const double* T2 = small + TT_MAXL * TT_MAXL;  // rp x rp
  double* CB = small + 2 * TT_MAXL * TT_MAXL;    // rp x l
  // inverse of the upper triangular RB, column by column (one thread per column)
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    for (int i = r - 1; i >= 0; --i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int k2 = i + 1; k2 <= j; ++k2) v -= RB[i + rp * k2] * Ri[k2 + TT_MAXL * j];
      Ri[i + TT_MAXL * j] = (i <= j) ? v / RB[i + rp * i] : 0.0;
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < r * r; o += blockDim.x) {
    const int i = o % r, j = o / r;
    double v = 0.0;
    for (int k2 = 0; k2 < r; ++k2) v += Ri[i + TT_MAXL * k2] * Ri[j + TT_MAXL * k2];
    Cm[i + TT_MAXL * j] = v;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < r * l; o += blockDim.x) {
    const int i = o % r, j = o / r;
    double v = 0.0;
    for (int k2 = 0; k2 < r; ++k2) v += Cm[i + TT_MAXL * k2] * B[k2 + rp * j];
    CBs[i + TT_MAXL * j] = v;
    CB[i + rp * j] = v;
  }
  __syncthreads();
  double* Bbar = ws + it.off_bbar;
  for (int o = threadIdx.x; o < rp * l; o += blockDim.x) {
    const int i = o % rp, j = o / rp;
    double v = 0.0;
    if (i < r) {
      for (int k2 = 0; k2 < r; ++k2) v += Cm[i + TT_MAXL * k2] * T1[k2 + rp * j];
      for (int k2 = 0; k2 < r; ++k2) v -= T2[i + rp * k2] * CBs[k2 + TT_MAXL * j];
    }
    Bbar[i + (int64_t)rp * j] = v;
  }
}

// Sbar_{d*}(u, j) = sum_c Hbar(u, c) CB(c, j)
__global__ void sbar_mid_kernel(char* wsb, int item, const int* ranks, const double* small) {
  const DevItem& it = item_of(wsb, item);
  const DevSketch& sm = sketches_of(wsb)[it.mid_sk];
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + it.ds];
  const int rp = it.rpad[it.ds];
  const int l = it.lmid;
  const int64_t rows = sm.rows;
  const double* CB = small + 2 * TT_MAXL * TT_MAXL;
  double* out = ws + it.off_sbar[it.mid_sk - it.sk0];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * l;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = e % rows;
    const int j = (int)(e / rows);
    double v = 0.0;
    for (int c = 0; c < r; ++c) v += ws[it.off_hbar + u + rows * c] * CB[c + rp * j];
    out[e] = v;
  }
}

// 3. Ybar(u, piv(c)) = y_c, y = [Qbar(u,:) - Q(u,:) sym(W)] R^{-T}; other columns 0.
__global__ void qr_abar_kernel(char* wsb, int item, int k, const int* ranks, const double* W) {
  const DevItem& it = item_of(wsb, item);
  const DevSketch* S = sketches_of(wsb);
  const int si = it.basis_of_k[k];
  const DevSketch& sb = S[si];
  double* ws = reinterpret_cast<double*>(wsb);
  const int r = ranks[it.rank_off + k];
  const int rp = sb.rpad;
  const int l = sb.width;
  const int64_t rows = sb.rows;
  const double* Q = ws + sb.lev_z[0];
  const double* Qb = ws + it.off_qbar[k];
  const double* R = ws + it.off_rr[k];
  const int* piv = reinterpret_cast<const int*>(ws + sb.off_piv);
  double* Yb = ws + it.off_sbar[si - it.sk0];
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < rows; u += (int64_t)gridDim.x * blockDim.x) {
    double z[TT_MAXL];
    for (int c = 0; c < r; ++c) {
      double v = Qb[u + rows * c];
      for (int c2 = 0; c2 < r; ++c2) {
        const double sw = (c2 <= c) ? W[c2 + rp * c] : W[c + rp * c2];
        v -= Q[u + rows * c2] * sw;
      }
      z[c] = v;
    }
    for (int c = r - 1; c >= 0; --c) {
      double v = z[c];
      for (int c2 = c + 1; c2 < r; ++c2) v -= z[c2] * R[c + rp * c2];
      z[c] = v / R[c + rp * c];
    }
    for (int j = 0; j < l; ++j) Yb[u + rows * j] = 0.0;
    for (int c = 0; c < r; ++c) Yb[u + rows * piv[c]] = z[c];
  }
}

}  // namespace

cudaError_t launch_pbar_ls(const Plan& P, int item, void* ws, const int* ranks, cudaStream_t st);
cudaError_t launch_sketch_adjoint(const Plan& P, int item, void* dX, void* ws, cudaStream_t st);

cudaError_t launch_backward(const Plan& P, int item, const double* dcores, void* dX, void* ws, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  const DevSketch* sks = plan_sketches_host(&P);
  char* wsb = (char*)ws;
  double* W = (double*)ws;
  cudaError_t e;
  // ranks of the forward call: the finalize keeps a copy of item 0's in ws
  const int* ranks_dev = reinterpret_cast<const int*>(wsb + kRankCopyOff);
  double* small = W + it.off_small;
  const int d = it.d, ds = it.ds;
  // 1. core adjoints
  for (int k = 1; k < d; ++k) {
    const int64_t n = sks[it.basis_of_k[k]].rows * sks[it.basis_of_k[k]].rpad;
    count_launch();
    qbar_kernel<<<grid_for(n), kThreads, 0, st>>>(wsb, item, k, dcores, ranks_dev);
  }
  count_launch();
  hbar_kernel<<<grid_for(it.N[ds] * it.rpad[ds]), kThreads, 0, st>>>(wsb, item, dcores, ranks_dev);
  // 2. least squares
  const DevSketch& sm = sks[it.mid_sk];
  count_launch();
  resid_kernel<<<grid_for(sm.rows * it.lmid), kThreads, 0, st>>>(wsb, item, ranks_dev);
  e = cudaMemsetAsync(small, 0, sizeof(double) * 3 * TT_MAXL * TT_MAXL, st);
  if (e != cudaSuccess) return e;
  const int rp = it.rpad[ds];
  const int gg = (int)std::min<int64_t>((sm.rows + 31) / 32, 4LL * device_sm_count());
  count_launch();
  gram_kernel<<<gg, kThreads, 0, st>>>(W + it.off_hbar, sm.rows, W + it.off_sbar[it.mid_sk - it.sk0], sm.rows, sm.rows,
                                        rp, it.lmid, small, rp);                       // T1 = Hbar^T E
  count_launch();
  gram_kernel<<<gg, kThreads, 0, st>>>(W + it.off_H, sm.rows, W + it.off_hbar, sm.rows, sm.rows, rp, rp,
                                        small + TT_MAXL * TT_MAXL, rp);                // T2 = H^T Hbar
  count_launch();
  ls_small_kernel<<<1, kThreads, 0, st>>>(wsb, item, ranks_dev, small);
  e = launch_pbar_ls(P, item, ws, ranks_dev, st);                                     // Pbar_{d*} += Omega Bbar^T
  if (e != cudaSuccess) return e;
  count_launch();
  sbar_mid_kernel<<<grid_for(sm.rows * it.lmid), kThreads, 0, st>>>(wsb, item, ranks_dev, small);
  // 3. QR adjoints of every basis
  for (int k = 1; k < d; ++k) {
    const DevSketch& sb = sks[it.basis_of_k[k]];
    double* Wk = small + 3 * TT_MAXL * TT_MAXL;
    e = cudaMemsetAsync(Wk, 0, sizeof(double) * TT_MAXL * TT_MAXL, st);
    if (e != cudaSuccess) return e;
    const int g2 = (int)std::min<int64_t>((sb.rows + 31) / 32, 4LL * device_sm_count());
    count_launch();
    gram_kernel<<<g2, kThreads, 0, st>>>(W + sb.lev_z[0], sb.rows, W + it.off_qbar[k], sb.rows, sb.rows, sb.rpad,
                                          sb.rpad, Wk, sb.rpad);
    count_launch();
    qr_abar_kernel<<<grid_for(sb.rows, 8), 128, 0, st>>>(wsb, item, k, ranks_dev, Wk);
  }
  // 4. dX
  return launch_sketch_adjoint(P, item, dX, ws, st);
}

}  // namespace tts
