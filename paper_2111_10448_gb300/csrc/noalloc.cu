// tt_pstt2_noalloc: the one-shot PSTT2 (tt_pstt2) with its workspace in a
// fixed device array of this library instead of a caller buffer.
//
// For callers that cannot allocate device memory at the point of the call
// (no allocator handle in their context, or a rule against allocating there);
// they still get the whole forward path.  The workspace lives in
// g_noalloc_scratch below, a file-scope device array of kNoallocScratchBytes
// (32 MiB); a plan whose workspace is larger is refused.
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};  // address of the array on each device

}  // namespace

extern "C" tt_status tt_pstt2_noalloc(tt_plan_t plan, const void* X, double* cores, int* ranks,
                                      int* status_dev, tt_stream_t stream) {
  if (!plan || !X || !cores || !ranks) return TT_ERR_INVALID_ARG;
  size_t need = 0;
  tt_status s = tt_plan_sizes(plan, &need, nullptr, nullptr);
  if (s != TT_OK) return s;
  if (need > kNoallocScratchBytes) return TT_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TT_ERR_NO_DEVICE;
  if (dev < 0 || dev >= kMaxDevices) return TT_ERR_UNSUPPORTED;
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
      // set-up, once per device, with that device current
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return TT_ERR_CUDA;
      g_ptr[dev] = p;
    }
    ws = g_ptr[dev];
  }
  // tt_pstt2 re-sends the plan tables whenever another plan used the array
  // last (the library's workspace registry), and records the array as the
  // workspace of this plan's last forward call, so a later tt_pstt2_backward
  // on any caller workspace is refused (TT_ERR_STATE).
  s = tt_pstt2(plan, X, ws, cores, ranks, stream);
  if (s != TT_OK) return s;
  if (status_dev) {
    const cudaError_t e = cudaMemcpyAsync(status_dev, (const char*)ws + tts::kStatusOff, sizeof(int), cudaMemcpyDeviceToDevice,
                                          (cudaStream_t)stream);
    if (e != cudaSuccess) return TT_ERR_CUDA;
  }
  return TT_OK;
}
