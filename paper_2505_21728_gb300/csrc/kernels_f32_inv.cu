// Instantiates the persistent HyGT kernels of one kind for N = 2..256.
#include "hygt_launch.cuh"

namespace hygt {
cudaError_t launch_f32_inv(int log2n, const Params& p, cudaStream_t stream) {
  return launch_kind<3>(log2n, p, stream);
}
}  // namespace hygt
