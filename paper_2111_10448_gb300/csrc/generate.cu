// Synthetic inputs and raw access to the Gaussian stream (test and benchmark
// helpers of the C ABI).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"
#include "philox.cuh"

namespace tts {
namespace {

struct Dims {
  int d;
  int64_t n[TT_MAXD];
};

// Hilbert-type tensor 1 / (x_{i_1} + ... + x_{i_d}), x_i = 1 + i/(n-1)
// (the large streaming workload); slab [first, first + count) of the last mode.
__global__ void hilbert_type_kernel(Dims D, int64_t first, int64_t count, void* out, int f64) {
  int64_t inner = 1;
  for (int k = 0; k < D.d - 1; ++k) inner *= D.n[k];
  const int64_t total = inner * count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = e;
    double s = 0.0;
    for (int k = 0; k < D.d; ++k) {
      int64_t i;
      if (k < D.d - 1) {
        i = rem % D.n[k];
        rem /= D.n[k];
      } else {
        i = rem + first;
      }
      const double x = 1.0 + (double)i / (double)(D.n[k] > 1 ? D.n[k] - 1 : 1);
      s = (k == 0) ? x : s + x;
    }
    const double v = 1.0 / s;
    if (f64) ((double*)out)[e] = v;
    else ((float*)out)[e] = (float)v;
  }
}

// The paper's Hilbert tensor 1 / (1 - d + i_1 + ... + i_d) with 1-based
// indices (Sec. 4.3), i.e. 1 / (1 + sum of the 0-based indices): an exact
// integer sum and one FP64 division, rounded to the output dtype.
__global__ void hilbert_paper_kernel(Dims D, int64_t first, int64_t count, void* out, int f64) {
  int64_t inner = 1;
  for (int k = 0; k < D.d - 1; ++k) inner *= D.n[k];
  const int64_t total = inner * count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = e, s = 1;
    for (int k = 0; k < D.d - 1; ++k) {
      s += rem % D.n[k];
      rem /= D.n[k];
    }
    s += rem + first;
    const double v = 1.0 / (double)s;
    if (f64) ((double*)out)[e] = v;
    else ((float*)out)[e] = (float)v;
  }
}

// Gaussian bumps (Sec. 4.4): X(i) = sum_j prod_k E_k[j][i_k] with the factor
// tables E_k[j][i] = exp(-gamma (x_i - c_{j,k})^2), x_i = 2 i / n_k - 1 (one
// table entry per mode, bump and index: the exponential of the sum is the
// product of the exponentials).  Tables: tab + toff[k] + n_k j + i.
__global__ void bumps_table_kernel(Dims D, int nb, double gamma, const double* centres, const int64_t* toff,
                                   double* tab) {
  for (int k = 0; k < D.d; ++k) {
    const int64_t n = D.n[k];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * nb;
         e += (int64_t)gridDim.x * blockDim.x) {
      const int64_t i = e % n;
      const int j = (int)(e / n);
      const double x = 2.0 * (double)i / (double)n - 1.0;
      const double t = x - centres[(int64_t)j * D.d + k];
      tab[toff[k] + e] = exp(-gamma * (t * t));
    }
  }
}
__global__ void bumps_kernel(Dims D, int nb, const int64_t* toff, const double* tab, int64_t first,
                             int64_t count, void* out, int f64) {
  int64_t inner = 1;
  for (int k = 0; k < D.d - 1; ++k) inner *= D.n[k];
  const int64_t total = inner * count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx[TT_MAXD];
    int64_t rem = e;
    for (int k = 0; k < D.d - 1; ++k) {
      idx[k] = rem % D.n[k];
      rem /= D.n[k];
    }
    idx[D.d - 1] = rem + first;
    double v = 0.0;
    for (int j = 0; j < nb; ++j) {
      double f = 1.0;
      for (int k = 0; k < D.d; ++k) f *= tab[toff[k] + D.n[k] * j + idx[k]];
      v += f;
    }
    if (f64) ((double*)out)[e] = v;
    else ((float*)out)[e] = (float)v;
  }
}

__global__ void test_matrix_f64_kernel(uint64_t seed, int sid, int64_t row0, int64_t nrows, int ncols,
                                       double* out) {
  const int nq = (ncols + 3) / 4;
  const int64_t total = nrows * nq;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % nrows;
    const int q = (int)(e / nrows);
    double z[4];
    normals4_f64(seed, (uint32_t)sid, (uint64_t)(row0 + r), (uint32_t)q, z);
    for (int t = 0; t < 4; ++t)
      if (4 * q + t < ncols) out[r + nrows * (4 * q + t)] = z[t];
  }
}

__global__ void philox_kernel(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                              int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c0 = ctr[4 * e], c1 = ctr[4 * e + 1], c2 = ctr[4 * e + 2], c3 = ctr[4 * e + 3];
    philox4x32_10(c0, c1, c2, c3, k0, k1);
    out[4 * e] = c0;
    out[4 * e + 1] = c1;
    out[4 * e + 2] = c2;
    out[4 * e + 3] = c3;
  }
}

int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16LL * device_sm_count()));
}

// max |X| as the bit pattern of an FP64 value (non-negative FP64 values order
// like their bit patterns; an inf or NaN gives a pattern >= that of inf).
__global__ void absmax_kernel(const void* x, int f64, int64_t n, unsigned long long* out) {
  unsigned long long m = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = f64 ? reinterpret_cast<const double*>(x)[e] : (double)reinterpret_cast<const float*>(x)[e];
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(v));
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

}  // namespace

cudaError_t launch_test_matrix_mixed(uint64_t seed, int sid, int64_t row0, int64_t nrows, int ncols,
                                     int prec, double* out, cudaStream_t st);

}  // namespace tts

using namespace tts;

extern "C" {

tt_status tt_generate_hilbert_type(int d, const int64_t* n, int64_t first_last, int64_t count_last,
                                   void* out, tt_dtype dtype, tt_stream_t stream) {
  if (d < 1 || d > TT_MAXD || !n || !out || first_last < 0 || count_last < 0) return TT_ERR_INVALID_ARG;
  if (dtype != TT_F32 && dtype != TT_F64) return TT_ERR_INVALID_ARG;
  Dims D;
  D.d = d;
  int64_t inner = 1;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1) return TT_ERR_INVALID_ARG;
    D.n[k] = n[k];
    if (k < d - 1) inner *= n[k];
  }
  if (first_last + count_last > n[d - 1]) return TT_ERR_INVALID_ARG;
  if (count_last == 0) return TT_OK;
  count_launch();
  hilbert_type_kernel<<<grid_for(inner * count_last), 256, 0, (cudaStream_t)stream>>>(
      D, first_last, count_last, out, dtype == TT_F64);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

tt_status tt_generate_hilbert(int d, const int64_t* n, int64_t first_last, int64_t count_last, void* out,
                              tt_dtype dtype, tt_stream_t stream) {
  if (d < 1 || d > TT_MAXD || !n || !out || first_last < 0 || count_last < 0) return TT_ERR_INVALID_ARG;
  if (dtype != TT_F32 && dtype != TT_F64) return TT_ERR_INVALID_ARG;
  Dims D;
  D.d = d;
  int64_t inner = 1;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1) return TT_ERR_INVALID_ARG;
    D.n[k] = n[k];
    if (k < d - 1) inner *= n[k];
  }
  if (first_last + count_last > n[d - 1]) return TT_ERR_INVALID_ARG;
  if (count_last == 0) return TT_OK;
  count_launch();
  hilbert_paper_kernel<<<grid_for(inner * count_last), 256, 0, (cudaStream_t)stream>>>(
      D, first_last, count_last, out, dtype == TT_F64);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

tt_status tt_generate_gaussian_bumps(int d, const int64_t* n, int nbumps, double gamma, const double* centres,
                                     int64_t first_last, int64_t count_last, void* out, tt_dtype dtype,
                                     tt_stream_t stream) {
  if (d < 1 || d > TT_MAXD || !n || !out || !centres || nbumps < 1 || !(gamma >= 0.0) || first_last < 0 ||
      count_last < 0)
    return TT_ERR_INVALID_ARG;
  if (dtype != TT_F32 && dtype != TT_F64) return TT_ERR_INVALID_ARG;
  Dims D;
  D.d = d;
  int64_t inner = 1, toff[TT_MAXD], tsz = 0;
  for (int k = 0; k < d; ++k) {
    if (n[k] < 1) return TT_ERR_INVALID_ARG;
    D.n[k] = n[k];
    if (k < d - 1) inner *= n[k];
    toff[k] = tsz;
    tsz += n[k] * nbumps;
  }
  if (first_last + count_last > n[d - 1]) return TT_ERR_INVALID_ARG;
  if (count_last == 0) return TT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // scratch: centres, table offsets and the factor tables (stream-ordered, freed on return)
  const size_t cbytes = sizeof(double) * (size_t)nbumps * d, obytes = sizeof(int64_t) * TT_MAXD;
  char* scratch = nullptr;
  if (cudaMallocAsync(&scratch, cbytes + obytes + sizeof(double) * (size_t)tsz, st) != cudaSuccess) {
    cudaGetLastError();
    return TT_ERR_CUDA;
  }
  double* dc = reinterpret_cast<double*>(scratch);
  int64_t* dto = reinterpret_cast<int64_t*>(scratch + cbytes);
  double* tab = reinterpret_cast<double*>(scratch + cbytes + obytes);
  cudaError_t e = cudaMemcpyAsync(dc, centres, cbytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dto, toff, sizeof(int64_t) * d, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    count_launch();
    bumps_table_kernel<<<grid_for(tsz / d + 1), 256, 0, st>>>(D, nbumps, gamma, dc, dto, tab);
    count_launch();
    bumps_kernel<<<grid_for(inner * count_last), 256, 0, st>>>(D, nbumps, dto, tab, first_last, count_last, out,
                                                              dtype == TT_F64);
    e = cudaGetLastError();
  }
  // the host copies read pageable memory: finish them before returning
  const cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFreeAsync(scratch, st);
  if (e == cudaSuccess) e = e2;
  return e == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

tt_status tt_test_matrix(uint64_t seed, int stream_id, int64_t row0, int64_t nrows, int ncols,
                         tt_prec prec, double* out, tt_stream_t stream) {
  if (!out || nrows < 0 || row0 < 0 || ncols < 0 || ncols > TT_MAXL) return TT_ERR_INVALID_ARG;
  if (nrows == 0 || ncols == 0) return TT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == TT_PREC_FP64) {
    count_launch();
    test_matrix_f64_kernel<<<grid_for(nrows * ((ncols + 3) / 4)), 256, 0, st>>>(seed, stream_id, row0, nrows,
                                                                                ncols, out);
    return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
  }
  if (prec != TT_PREC_TF32 && prec != TT_PREC_BF16 && prec != TT_PREC_FP16) return TT_ERR_INVALID_ARG;
  return launch_test_matrix_mixed(seed, stream_id, row0, nrows, ncols, prec, out, st) == cudaSuccess
             ? TT_OK
             : TT_ERR_CUDA;
}

tt_status tt_x_scale_log2(const void* X, tt_dtype dtype, int64_t count, int* s_out, tt_stream_t stream) {
  if (!X || !s_out || count < 0 || (dtype != TT_F32 && dtype != TT_F64)) return TT_ERR_INVALID_ARG;
  if (count == 0) {
    *s_out = 0;
    return TT_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* d = nullptr;
  if (cudaMallocAsync(&d, sizeof(unsigned long long), st) != cudaSuccess) return TT_ERR_CUDA;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    count_launch();
    absmax_kernel<<<(unsigned)std::min<int64_t>((count + 255) / 256, 4LL * device_sm_count()), 256, 0, st>>>(
        X, dtype == TT_F64 ? 1 : 0, count, d);
    e = cudaGetLastError();
  }
  unsigned long long bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return TT_ERR_CUDA;
  // |v| as FP64 bits: the largest finite pattern is below that of infinity
  if (bits >= 0x7FF0000000000000ull) return TT_ERR_NONFINITE;
  double mx = 0.0;
  std::memcpy(&mx, &bits, sizeof(mx));
  if (mx == 0.0) {
    *s_out = 0;
    return TT_OK;
  }
  int ex = 0;
  std::frexp(mx, &ex);  // 2^(ex-1) <= mx < 2^ex
  *s_out = std::max(-100, std::min(100, 15 - ex));
  return TT_OK;
}

tt_status tt_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, uint32_t* out,
                           int64_t count, tt_stream_t stream) {
  if (!ctr || !out || count < 0) return TT_ERR_INVALID_ARG;
  if (count == 0) return TT_OK;
  count_launch();
  philox_kernel<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(ctr, key0, key1, out, count);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

}  // extern "C"
