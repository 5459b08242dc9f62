// batch_n_8_fwd.cu -- bucketed forward kernels for 16x16 blocks.
#include "hygt_batch_launch.cuh"

namespace hygt {

template cudaError_t launch_batch_n<8, 0>(const BatchParams&, cudaStream_t, const BatchTune&);

}  // namespace hygt
