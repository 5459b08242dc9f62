// batch_fwd.cu -- forward launchers of the set-bucketed kernels (the
// instantiations of hygt_batch_launch.cuh for the forward direction).
#include "hygt_batch_launch.cuh"

namespace hygt {

cudaError_t launch_batch_fwd(int log2n, const BatchParams& p, cudaStream_t stream,
                             const BatchTune& tune) {
  return launch_batch<0>(log2n, p, stream, tune);
}

cudaError_t launch_batch_primary_fwd(int log2n, const BatchParams& p, cudaStream_t stream,
                                     const BatchTune& tune) {
  if (log2n == 4) return launch_primary_sized<4, 0>(p, stream, tune);
  if (log2n == 6) return launch_primary_sized<6, 0>(p, stream, tune);
  return cudaErrorInvalidValue;
}

}  // namespace hygt
