// batch_n_small.cu -- bucketed kernels for 2-, 4- and 8-value blocks, both directions.
#include "hygt_batch_launch.cuh"

namespace hygt {

template cudaError_t launch_batch_n<1, 0>(const BatchParams&, cudaStream_t, const BatchTune&);
template cudaError_t launch_batch_n<1, 1>(const BatchParams&, cudaStream_t, const BatchTune&);
template cudaError_t launch_batch_n<2, 0>(const BatchParams&, cudaStream_t, const BatchTune&);
template cudaError_t launch_batch_n<2, 1>(const BatchParams&, cudaStream_t, const BatchTune&);
template cudaError_t launch_batch_n<3, 0>(const BatchParams&, cudaStream_t, const BatchTune&);
template cudaError_t launch_batch_n<3, 1>(const BatchParams&, cudaStream_t, const BatchTune&);

}  // namespace hygt
