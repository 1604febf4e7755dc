// Backward (adjoint) of the one-pass PSTT2 map and of the reconstruction.
#include "internal.cuh"

namespace tts {

cudaError_t launch_backward(const Plan&, int, const double*, void*, void*, cudaStream_t) {
  return cudaErrorNotSupported;
}

cudaError_t launch_reconstruct_backward(const Plan&, int, const double*, const void*, int, double*,
                                        void*, cudaStream_t) {
  return cudaErrorNotSupported;
}

cudaError_t launch_sketch_batched(const Plan&, void*, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace tts
