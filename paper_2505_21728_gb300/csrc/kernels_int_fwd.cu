// Instantiates the persistent HyGT kernels of one kind for N = 2..256.
#include "hygt_launch.cuh"

namespace hygt {
cudaError_t launch_int_fwd(int log2n, const Params& p, cudaStream_t stream) {
  return launch_kind<0>(log2n, p, stream);
}
}  // namespace hygt
