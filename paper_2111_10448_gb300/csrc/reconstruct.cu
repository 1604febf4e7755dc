// Reconstruction X~(i_1..i_d) = G_1(:, i_1, :) ... G_d(:, i_d, :) (Sec. 2.2)
// and its fused relative-error form (eq. (1.1)).
//
// The cores are contracted into a left interface L_{d*} (N_{d*} x r_{d*}) and a
// right interface Rt_{d*+1} (r_{d*} x M_{d*}); then X~ = L_{d*} Rt_{d*+1} seen as
// the middle unfolding, one thread per entry (FP64).
#include <algorithm>

#include "internal.cuh"

namespace tts {
namespace {

constexpr int kThreads = 256;

// L_k(u + N_{k-1} i, c) = sum_a L_{k-1}(u, a) G_k(a, i, c);  L_0 = [1].
__global__ void iface_left_kernel(const double* Lp, int64_t Np, int rpp, const double* G, int64_t nk,
                                  int rpk, double* Lo) {
  const int64_t Nk = Np * nk;
  const int64_t total = Nk * rpk;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e % Nk;
    const int c = (int)(e / Nk);
    const int64_t u = row % Np, i = row / Np;
    double acc = 0.0;
    if (Lp == nullptr) {
      acc = G[0 + rpp * (i + nk * c)];
    } else {
      for (int a = 0; a < rpp; ++a) acc += Lp[u + Np * a] * G[a + rpp * (i + nk * c)];
    }
    Lo[row + Nk * c] = acc;
  }
}

// Rt_k(a, i + n_k v) = sum_c G_k(a, i, c) Rt_{k+1}(c, v);  Rt_{d+1} = [1].
__global__ void iface_right_kernel(const double* Rn, int64_t Mn, int rpn, const double* G, int64_t nk,
                                   int rpa, double* Ro) {
  const int64_t Mk = nk * Mn;
  const int64_t total = (int64_t)rpa * Mk;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e % rpa);
    const int64_t col = e / rpa;
    const int64_t i = col % nk, v = col / nk;
    double acc = 0.0;
    if (Rn == nullptr) {
      acc = G[a + rpa * (i + nk * 0)];
    } else {
      for (int c = 0; c < rpn; ++c) acc += G[a + rpa * (i + nk * c)] * Rn[c + rpn * v];
    }
    Ro[a + (int64_t)rpa * col] = acc;
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// X~(u + Nm v) = sum_c L(u, c) Rt(c, v); optionally store it and/or accumulate
// [sum (X - X~)^2, sum X^2].
__global__ void __launch_bounds__(kThreads) dense_kernel(const double* L, const double* Rt, int64_t Nm,
                                                         int64_t Mm, int rp, void* out, int out_f64,
                                                         const void* Xc, int xc_f64, double* out2) {
  double e2 = 0.0, x2 = 0.0;
  const int64_t total = Nm * Mm;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = e % Nm, v = e / Nm;
    double acc = 0.0;
    for (int c = 0; c < rp; ++c) acc += L[u + Nm * c] * Rt[c + (int64_t)rp * v];
    if (out) {
      if (out_f64) ((double*)out)[e] = acc;
      else ((float*)out)[e] = (float)acc;
    }
    if (Xc) {
      const double x = xc_f64 ? ((const double*)Xc)[e] : (double)((const float*)Xc)[e];
      e2 += (x - acc) * (x - acc);
      x2 += x * x;
    }
  }
  if (out2) {
    __shared__ double red[2][32];
    e2 = warp_sum(e2);
    x2 = warp_sum(x2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][wid] = e2;
      red[1][wid] = x2;
    }
    __syncthreads();
    if (wid == 0) {
      double a = lane < (int)(blockDim.x >> 5) ? red[0][lane] : 0.0;
      double b = lane < (int)(blockDim.x >> 5) ? red[1][lane] : 0.0;
      a = warp_sum(a);
      b = warp_sum(b);
      if (lane == 0) {
        atomicAdd(out2, a);
        atomicAdd(out2 + 1, b);
      }
    }
  }
}

// Y(row, c) += sum_v dX(row + Nk v) Rt(c, v)   (Rt: rp x Mk, ld rp; Rt = null: 1).
// A job is 32 consecutive rows (the lanes) x vc consecutive v; the four warps
// of a block take consecutive jobs of the same rows, add their partial sums in
// shared memory and the block adds them into Y (FP64 atomics).  RP >= rp is a
// compile-time bound so that the accumulators stay in registers.
template <int RP>
__global__ void __launch_bounds__(128) ygram_kernel(const void* dX, int dx_f64, int64_t Nk, int64_t Mk,
                                                    const double* Rt, int rp, double* Y, int64_t vc) {
  extern __shared__ double part[];  // 4 x RP x 32
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nrb = (Nk + 31) / 32, nvc = (Mk + vc - 1) / vc;
  const int64_t nvg = (nvc + 3) / 4;  // groups of four v chunks, one per warp
  for (int64_t job = blockIdx.x; job < nrb * nvg; job += gridDim.x) {
    const int64_t rb = job % nrb, vg = job / nrb;
    const int64_t row = rb * 32 + lane;
    const int64_t v0 = (vg * 4 + warp) * vc, v1 = imin64(Mk, v0 + vc);
    double acc[RP];
#pragma unroll
    for (int c = 0; c < RP; ++c) acc[c] = 0.0;
    if (row < Nk) {
      for (int64_t v = v0; v < v1; ++v) {
        const int64_t idx = row + Nk * v;
        const double x = dx_f64 ? __ldg((const double*)dX + idx) : (double)__ldg((const float*)dX + idx);
#pragma unroll
        for (int c = 0; c < RP; ++c)
          if (c < rp) acc[c] += x * (Rt ? __ldg(Rt + c + (int64_t)rp * v) : 1.0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < RP; ++c) part[(warp * RP + c) * 32 + lane] = acc[c];
    __syncthreads();
    for (int e = threadIdx.x; e < rp * 32; e += blockDim.x) {
      const int c = e >> 5, l = e & 31;
      const int64_t r = rb * 32 + l;
      if (r < Nk) {
        const double sum = part[(0 * RP + c) * 32 + l] + part[(1 * RP + c) * 32 + l] +
                           part[(2 * RP + c) * 32 + l] + part[(3 * RP + c) * 32 + l];
        atomicAdd(Y + r + Nk * c, sum);
      }
    }
  }
}

// dG_k(a, i, c) = sum_u L_{k-1}(u, a) Y_k(u + N_{k-1} i, c);  L_0 = [1].
// dG is zeroed first; a warp takes one entry and one chunk of u (lanes split
// the chunk) and adds its sum with an atomic.
__global__ void dcore_kernel(const double* Lp, int64_t Np, int rpa, const double* Y, int64_t nk, int rpc,
                             double* dG, int64_t uc) {
  const int64_t total = (int64_t)rpa * nk * rpc;
  const int64_t Nk = Np * nk;
  if (Lp == nullptr) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = (e / rpa) % nk;
      const int c = (int)(e / (rpa * nk));
      dG[e] = Y[i + Nk * c];
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const int64_t nuc = (Np + uc - 1) / uc;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t job = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); job < total * nuc; job += nwarps) {
    const int64_t e = job % total, ch = job / total;
    const int a = (int)(e % rpa);
    const int64_t i = (e / rpa) % nk;
    const int c = (int)(e / (rpa * nk));
    const int64_t u0 = ch * uc, u1 = imin64(Np, u0 + uc);
    double acc = 0.0;
    for (int64_t u = u0 + lane; u < u1; u += 32) acc += Lp[u + Np * a] * Y[u + Np * i + Nk * c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicAdd(dG + e, acc);
  }
}

int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 16LL * device_sm_count()));
}

}  // namespace

cudaError_t build_interfaces(const Plan& P, int item, const double* cores, void* ws, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  double* W = (double*)ws;
  const int d = it.d, ds = it.ds;
  for (int k = 1; k <= ds; ++k) {
    const double* Lp = k == 1 ? nullptr : W + it.off_L[k - 1];
    const int64_t n = it.N[k] * it.rpad[k];
    count_launch();
    iface_left_kernel<<<grid_for(n), kThreads, 0, st>>>(Lp, it.N[k - 1], it.rpad[k - 1],
                                                        cores + it.core_off[k], it.n[k - 1],
                                                        it.rpad[k], W + it.off_L[k]);
  }
  for (int k = d; k >= ds + 1; --k) {
    const double* Rn = k == d ? nullptr : W + it.off_Rt[k + 1];
    const int64_t Mn = it.N[d] / it.N[k];
    const int64_t n = (int64_t)it.rpad[k - 1] * it.n[k - 1] * Mn;
    count_launch();
    iface_right_kernel<<<grid_for(n), kThreads, 0, st>>>(Rn, Mn, it.rpad[k], cores + it.core_off[k],
                                                         it.n[k - 1], it.rpad[k - 1], W + it.off_Rt[k]);
  }
  return cudaGetLastError();
}

cudaError_t launch_reconstruct(const Plan& P, int item, const double* cores, void* Xt, int x_f64,
                               const void* Xcmp, int cmp_f64, double* out2, void* ws,
                               cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  cudaError_t e = build_interfaces(P, item, cores, ws, st);
  if (e != cudaSuccess) return e;
  if (out2) {
    e = cudaMemsetAsync(out2, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
  }
  double* W = (double*)ws;
  const int ds = it.ds;
  const int64_t Nm = it.N[ds], Mm = it.N[it.d] / it.N[ds];
  count_launch();
  dense_kernel<<<grid_for(Nm * Mm), kThreads, 0, st>>>(W + it.off_L[ds], W + it.off_Rt[ds + 1], Nm, Mm,
                                                       it.rpad[ds], Xt, x_f64, Xcmp, cmp_f64, out2);
  return cudaGetLastError();
}

// Adjoint of the reconstruction: for every core k,
//   dG_k(a, i, c) = sum_{u, v} L_{k-1}(u, a) dX(u + N_{k-1} i + N_k v) Rt_{k+1}(c, v)
// with the left / right interfaces of the train (all of them: TT_FLAG_DIFF).
cudaError_t launch_reconstruct_backward(const Plan& P, int item, const double* cores, const void* dXt,
                                        int dx_f64, double* dcores, void* ws, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  double* W = (double*)ws;
  const int d = it.d;
  for (int k = 1; k < d; ++k) {
    const double* Lp = k == 1 ? nullptr : W + it.off_Lall[k - 1];
    count_launch();
    iface_left_kernel<<<grid_for(it.N[k] * it.rpad[k]), kThreads, 0, st>>>(
        Lp, it.N[k - 1], it.rpad[k - 1], cores + it.core_off[k], it.n[k - 1], it.rpad[k], W + it.off_Lall[k]);
  }
  for (int k = d; k >= 2; --k) {
    const double* Rn = k == d ? nullptr : W + it.off_Rall[k + 1];
    const int64_t Mn = it.N[d] / it.N[k];
    count_launch();
    iface_right_kernel<<<grid_for((int64_t)it.rpad[k - 1] * it.n[k - 1] * Mn), kThreads, 0, st>>>(
        Rn, Mn, it.rpad[k], cores + it.core_off[k], it.n[k - 1], it.rpad[k - 1], W + it.off_Rall[k]);
  }
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(ygram_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         4 * 64 * 32 * (int)sizeof(double));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  for (int k = 1; k <= d; ++k) {
    const int64_t Nk = it.N[k], Mk = it.N[d] / it.N[k];
    const int rpk = it.rpad[k];
    cudaError_t e = cudaMemsetAsync(W + it.off_Y, 0, sizeof(double) * Nk * rpk, st);
    if (e != cudaSuccess) return e;
    // v chunks sized so that about 32k warp jobs cover the entries
    const int64_t vc = std::max<int64_t>(16, (Nk * Mk) / (32LL * 32768));
    const int64_t nrb = (Nk + 31) / 32, nvg = ((Mk + vc - 1) / vc + 3) / 4;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(nrb * nvg, 16LL * device_sm_count()));
    const double* Rt = k == d ? nullptr : W + it.off_Rall[k + 1];
    count_launch();
    if (rpk <= 8)
      ygram_kernel<8><<<g, 128, 4 * 8 * 32 * sizeof(double), st>>>(dXt, dx_f64, Nk, Mk, Rt, rpk, W + it.off_Y, vc);
    else if (rpk <= 16)
      ygram_kernel<16><<<g, 128, 4 * 16 * 32 * sizeof(double), st>>>(dXt, dx_f64, Nk, Mk, Rt, rpk, W + it.off_Y, vc);
    else if (rpk <= 32)
      ygram_kernel<32><<<g, 128, 4 * 32 * 32 * sizeof(double), st>>>(dXt, dx_f64, Nk, Mk, Rt, rpk, W + it.off_Y, vc);
    else
      ygram_kernel<64><<<g, 128, 4 * 64 * 32 * sizeof(double), st>>>(dXt, dx_f64, Nk, Mk, Rt, rpk, W + it.off_Y, vc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nout = (int64_t)it.rpad[k - 1] * it.n[k - 1] * rpk;
    e = cudaMemsetAsync(dcores + it.core_off[k], 0, sizeof(double) * nout, st);
    if (e != cudaSuccess) return e;
    const int64_t Np = it.N[k - 1];
    const int64_t uc = std::max<int64_t>(256, (nout * Np) / 32768);
    count_launch();
    dcore_kernel<<<grid_for(nout * ((Np + uc - 1) / uc) * 32), kThreads, 0, st>>>(
        k == 1 ? nullptr : W + it.off_Lall[k - 1], Np, it.rpad[k - 1], W + it.off_Y, it.n[k - 1], rpk,
        dcores + it.core_off[k], uc);
  }
  return cudaGetLastError();
}

}  // namespace tts
