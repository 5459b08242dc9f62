// batch_fwd.cu -- forward launchers of the set-bucketed kernels: dispatch on
// the block size to the per-size launchers of batch_n*.cu.
#include "hygt_batch.cuh"

namespace hygt {

cudaError_t launch_batch_fwd(int log2n, const BatchParams& p, cudaStream_t stream,
                             const BatchTune& tune) {
  switch (log2n) {
    case 1: return launch_batch_n<1, 0>(p, stream, tune);
    case 2: return launch_batch_n<2, 0>(p, stream, tune);
    case 3: return launch_batch_n<3, 0>(p, stream, tune);
    case 4: return launch_batch_n<4, 0>(p, stream, tune);
    case 5: return launch_batch_n<5, 0>(p, stream, tune);
    case 6: return launch_batch_n<6, 0>(p, stream, tune);
    case 7: return launch_batch_n<7, 0>(p, stream, tune);
    case 8: return launch_batch_n<8, 0>(p, stream, tune);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_primary_fwd(int log2n, const BatchParams& p, cudaStream_t stream,
                                     const BatchTune& tune) {
  if (log2n == 4) return launch_primary_n<4, 0>(p, stream, tune);
  if (log2n == 6) return launch_primary_n<6, 0>(p, stream, tune);
  return cudaErrorInvalidValue;
}

}  // namespace hygt
