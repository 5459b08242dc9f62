// batch_inv.cu -- inverse launchers of the set-bucketed kernels (the
// instantiations of hygt_batch_launch.cuh for the inverse direction).
#include "hygt_batch_launch.cuh"

namespace hygt {

cudaError_t launch_batch_inv(int log2n, const BatchParams& p, cudaStream_t stream,
                             const BatchTune& tune) {
  return launch_batch<1>(log2n, p, stream, tune);
}

cudaError_t launch_batch_primary_inv(int log2n, const BatchParams& p, cudaStream_t stream,
                                     const BatchTune& tune) {
  if (log2n == 4) return launch_primary_sized<4, 1>(p, stream, tune);
  if (log2n == 6) return launch_primary_sized<6, 1>(p, stream, tune);
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch_primary(int log2n, int inverse, const BatchParams& p,
                                 cudaStream_t stream, const BatchTune& tune) {
  return inverse ? launch_batch_primary_inv(log2n, p, stream, tune)
                 : launch_batch_primary_fwd(log2n, p, stream, tune);
}

}  // namespace hygt
