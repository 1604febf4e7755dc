// Batched form: many independent tensors of uneven shape sketched by one
// persistent launch (a work queue over the tiles of every tensor, largest
// tensors first), then finalized by launches that each cover every tensor.
// Nothing here synchronises with the host, so a whole batched decomposition
// can be captured in a CUDA graph once the plan tables are in the workspace.
#include <algorithm>

#include "internal.cuh"

namespace tts {
const DevSketch* plan_sketches_host(const Plan* p);
int plan_num_items(const Plan* p);

namespace {

constexpr int64_t kTableOffB = 256;

// First tile of every item in visiting order, for tiles of ta x tb entries of
// each plane; resets the work counter and the status word.  One block: the
// tile counts are loaded in parallel, then scanned in shared memory.
__global__ void __launch_bounds__(1024) batch_prep_kernel(char* wsb, int ta, int tb) {
  __shared__ int64_t cnt[kMaxBatchItems];
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
  const DevItem* items = reinterpret_cast<const DevItem*>(wsb + T.off_items);
  const int* order = reinterpret_cast<const int*>(wsb + T.off_border);
  int64_t* prefix = reinterpret_cast<int64_t*>(wsb + T.off_bprefix);
  for (int i = threadIdx.x; i < T.nitems; i += blockDim.x) {
    const DevItem& it = items[order[i]];
    cnt[i] = it.W * ((it.n[0] + ta - 1) / ta) * ((it.n[it.d - 1] + tb - 1) / tb);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int i = 0; i < T.nitems; ++i) {
      prefix[i] = acc;
      acc += cnt[i];
    }
    prefix[T.nitems] = acc;
    *reinterpret_cast<unsigned long long*>(wsb + T.off_bcounter) = 0ull;
    *reinterpret_cast<int*>(wsb + kStatusOff) = 0;
  }
}

// Zero every sketch (blockIdx.y < nsk) and every one-pass B (blockIdx.y >= nsk).
__global__ void batch_zero_kernel(char* wsb) {
  const DevTables& T = *reinterpret_cast<const DevTables*>(wsb + kTableOffB);
  double* ws = reinterpret_cast<double*>(wsb);
  int64_t off = 0, n = 0;
  if ((int)blockIdx.y < T.nsk) {
    const DevSketch& s = reinterpret_cast<const DevSketch*>(wsb + T.off_sketches)[blockIdx.y];
    off = s.off;
    n = s.rows * s.width;
  } else {
    const DevItem& it = reinterpret_cast<const DevItem*>(wsb + T.off_items)[blockIdx.y - T.nsk];
    if (it.passes != 1) return;
    off = it.off_B;
    n = (int64_t)it.rpad[it.mbk] * it.lmid;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    ws[off + i] = 0.0;
}

}  // namespace

cudaError_t launch_batch_zero(const Plan& P, void* ws, cudaStream_t st) {
  int nsk = 0;
  for (int i = 0; i < plan_num_items(&P); ++i) nsk += plan_items_host(&P)[i].nsk;
  count_launch();
  batch_zero_kernel<<<dim3(8, (unsigned)(nsk + plan_num_items(&P))), 256, 0, st>>>((char*)ws);
  return cudaGetLastError();
}

cudaError_t launch_sketch_batched(const Plan& P, const void* const* X, const BatchCfg& cfg, void* ws,
                                  cudaStream_t st) {
  const int nitems = plan_num_items(&P);
  if (nitems > kMaxBatchItems) return cudaErrorNotSupported;
  const int t3max = (cfg.ta == 1 || cfg.ta == 2 || cfg.ta == 4 || cfg.ta == 8) ? cfg.ta : 4;
  if (plan_items_host(&P)[0].prec != TT_PREC_FP64 && sp_batched_eligible(P, nullptr, nullptr, t3max))
    return launch_sketch_sp_batched(P, X, cfg, ws, st);
  static BatchLaunch b;  // 16 KB: kept off the host stack
  b.wsb = (char*)ws;
  b.chunk = std::max(1, cfg.chunk);
  int lmax = 1;
  const DevSketch* sks = plan_sketches_host(&P);
  for (int i = 0; i < nitems; ++i) {
    b.X[i] = X[i];
    const DevItem& it = plan_items_host(&P)[i];
    for (int s = 0; s < it.nsk; ++s) lmax = std::max(lmax, sks[it.sk0 + s].width);
  }
  const bool f64 = plan_items_host(&P)[0].prec == TT_PREC_FP64;
  const int ta = f64 ? cfg.ta : 64;
  count_launch();
  batch_prep_kernel<<<1, 1024, 0, st>>>((char*)ws, ta, 32);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  BatchCfg c = cfg;
  c.ta = ta;
  return f64 ? launch_sketch_f64_batched(b, c, lmax, st)
             : launch_sketch_mma_batched(b, c, plan_items_host(&P)[0].prec == TT_PREC_FP16, st);
}

}  // namespace tts
