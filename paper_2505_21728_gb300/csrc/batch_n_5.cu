// batch_n_5.cu -- bucketed kernels for 32-value blocks, both directions.
#include "hygt_batch_launch.cuh"

namespace hygt {

template cudaError_t launch_batch_n<5, 0>(const BatchParams&, cudaStream_t, const BatchTune&);
template cudaError_t launch_batch_n<5, 1>(const BatchParams&, cudaStream_t, const BatchTune&);

}  // namespace hygt
