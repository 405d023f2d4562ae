// Plain encode launcher: S stripes back to back (kernels in encode_kernels.cuh).
#include "encode_kernels.cuh"

namespace mojette {

int launch_encode(const EncodeArgs &a, cudaStream_t st) { return launch_encode_impl<false>(a, st); }

}  // namespace mojette
