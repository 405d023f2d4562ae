// Batched encode launcher: stripes of one geometry anywhere in memory,
// addressed through per-stripe pointer arrays (kernels in encode_kernels.cuh).
#include "encode_kernels.cuh"

namespace mojette {

int launch_encode_batched(const EncodeArgs &a, cudaStream_t st) { return launch_encode_impl<true>(a, st); }

}  // namespace mojette
