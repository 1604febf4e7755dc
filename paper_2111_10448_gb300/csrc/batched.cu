// Batched form: many independent tensors of uneven shape in one persistent launch.
#include "internal.cuh"

namespace tts {

cudaError_t launch_sketch_batched(const Plan&, void*, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace tts
