// Tucker2TT (Algorithm 3), its second step: every TT core of the Tucker
// core's train multiplied along its middle mode by the Tucker factor,
// T = H x_2 A, T(a, i, c) = sum_s A(i, s) H(a, s, c); and the layout step of
// TT2Tucker (Algorithm 4): a core's mode-2 matricization and its inverse.
#include <algorithm>

#include "internal.cuh"

namespace tts {
namespace {

// One thread per entry of T (r0 x n x r1, column-major); the s loop reads a row
// of A (stride n) and a column of H's middle mode (stride r0).
__global__ void core_mode2_kernel(const double* H, int r0, int64_t s, int r1, const double* A, int64_t n,
                                  double* T) {
  const int64_t total = (int64_t)r0 * n * r1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e % r0, i = (e / r0) % n, c = e / (r0 * n);
    const double* h = H + a + (int64_t)r0 * s * c;
    double acc = 0.0;
    for (int64_t k = 0; k < s; ++k) acc = fma(A[i + n * k], h[r0 * k], acc);
    T[e] = acc;
  }
}

// out(j, i, k) = in(i, j, k) for column-major in (n0 x n1 x n2): the mode-2
// matricization of a TT core (n0 = r_{k-1}, n1 = n_k) and its inverse.
__global__ void swap12_kernel(const double* in, int64_t n0, int64_t n1, int64_t n2, double* out) {
  const int64_t total = n0 * n1 * n2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e % n1, i = (e / n1) % n0, k = e / (n0 * n1);  // e indexes out (n1 x n0 x n2)
    out[e] = in[i + n0 * (j + n1 * k)];
  }
}

}  // namespace
}  // namespace tts

using namespace tts;

extern "C" tt_status tt_swap12(const double* in, int64_t n0, int64_t n1, int64_t n2, double* out, tt_stream_t stream) {
  if (!in || !out || n0 < 1 || n1 < 1 || n2 < 1 || in == out) return TT_ERR_INVALID_ARG;
  const int64_t total = n0 * n1 * n2;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * device_sm_count()));
  count_launch();
  swap12_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(in, n0, n1, n2, out);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}

extern "C" tt_status tt_core_mode2(const double* H, int r0, int64_t s, int r1, const double* A, int64_t n, double* T,
                                   tt_stream_t stream) {
  if (!H || !A || !T || r0 < 1 || r1 < 1 || s < 1 || n < 1) return TT_ERR_INVALID_ARG;
  const int64_t total = (int64_t)r0 * n * r1;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * device_sm_count()));
  count_launch();
  core_mode2_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(H, r0, s, r1, A, n, T);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ERR_CUDA;
}
