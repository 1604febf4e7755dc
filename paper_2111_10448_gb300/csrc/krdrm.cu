// Khatri-Rao test matrices (TT_FLAG_KR): staging of the per-mode Gaussian
// factors of every sketch of an item (Sec. 3.2, eq. (sketch_orig): the test
// matrix of X_j is a Khatri-Rao product of n_k x l Gaussian factors).
//
// Factor t of sketch s is kr_n[t] x kr_lp: row i holds the normals of row
// i + (2^31 + mode) 2^32 of the sketch's stream (columns >= l are zero).  The
// FP64 path stores the FP64 normals, the TF32 / BF16 paths the FP32 normals
// of the mixed generator; the kernels form products of them (testmat.cuh).
#include <algorithm>

#include "internal.cuh"
#include "philox.cuh"

namespace tts {

const DevSketch* plan_sketches_host(const Plan* p);

namespace {

constexpr int64_t kTableOffB = 256;

// blockIdx.y = the (sketch, factor) pair, in plan order
__global__ void kr_factor_kernel(char* wsb, int item) {
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
  const DevItem& it = reinterpret_cast<const DevItem*>(wsb + T.off_items)[item];
  const DevSketch* sks = reinterpret_cast<const DevSketch*>(wsb + T.off_sketches);
  const bool f64 = it.prec == TT_PREC_FP64;
  int pair = 0;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& sk = sks[it.sk0 + s];
    if (sk.kr_nm == 0) continue;
    const int qpr = sk.kr_lp / 4;
    for (int t = 0; t < sk.kr_nm; ++t, ++pair) {
      if (pair != (int)blockIdx.y) continue;
      const uint64_t base = (uint64_t)(0x80000000u + (uint32_t)(sk.kr_mode0 + t)) << 32;
      const int64_t total = sk.kr_n[t] * qpr;
      for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
           e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / qpr;
        const int q = (int)(e - i * qpr);
        const int64_t el = sk.kr_off[t] + i * sk.kr_lp + 4 * q;
        double z[4];
        if (f64) {
          normals4_f64(it.seed, (uint32_t)sk.stream_id, base + (uint64_t)i, (uint32_t)q, z);
        } else {
          const float4 f = normals4_f32(it.seed, (uint32_t)sk.stream_id, base + (uint64_t)i, (uint32_t)q);
          z[0] = f.x; z[1] = f.y; z[2] = f.z; z[3] = f.w;
        }
        for (int u = 0; u < 4; ++u) {
          const double v = 4 * q + u < sk.width ? z[u] : 0.0;
          if (f64) reinterpret_cast<double*>(wsb + sk.kr_tab)[el + u] = v;
          else reinterpret_cast<float*>(wsb + sk.kr_tab)[el + u] = (float)v;
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_kr_tables(const Plan& P, int item, void* ws, cudaStream_t st) {
  const DevItem& it = plan_items_host(&P)[item];
  const DevSketch* sks = plan_sketches_host(&P);
  int64_t most = 0;
  bool any = false;
  for (int s = 0; s < it.nsk; ++s) {
    const DevSketch& sk = sks[it.sk0 + s];
    if (!sk.kr_nm) continue;
    any = true;
    for (int t = 0; t < sk.kr_nm; ++t) most = std::max<int64_t>(most, sk.kr_n[t] * (sk.kr_lp / 4));
  }
  if (!any) return cudaSuccess;
  int pairs = 0;
  for (int s = 0; s < it.nsk; ++s) pairs += sks[it.sk0 + s].kr_nm;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((most + 255) / 256, 4LL * device_sm_count()));
  count_launch();
  kr_factor_kernel<<<dim3((unsigned)grid, (unsigned)pairs), 256, 0, st>>>((char*)ws, item);
  return cudaGetLastError();
}

}  // namespace tts
