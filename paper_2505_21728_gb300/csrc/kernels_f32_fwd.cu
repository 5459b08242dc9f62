// Instantiates the persistent HyGT kernels of one kind for N = 2..256.
#include "hygt_launch.cuh"

namespace hygt {
cudaError_t launch_f32_fwd(int log2n, const Params& p, cudaStream_t stream) {
  return launch_kind<2>(log2n, p, stream);
}
}  // namespace hygt
