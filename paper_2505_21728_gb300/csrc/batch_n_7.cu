// batch_n_7.cu -- bucketed kernels for 128-value blocks, both directions.
#include "hygt_batch_launch.cuh"

namespace hygt {

template cudaError_t launch_batch_n<7, 0>(const BatchParams&, cudaStream_t, const BatchTune&);
template cudaError_t launch_batch_n<7, 1>(const BatchParams&, cudaStream_t, const BatchTune&);

}  // namespace hygt
