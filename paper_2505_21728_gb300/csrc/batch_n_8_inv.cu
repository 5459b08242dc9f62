// batch_n_8_inv.cu -- bucketed inverse kernels for 16x16 blocks.
#include "hygt_batch_launch.cuh"

namespace hygt {

template cudaError_t launch_batch_n<8, 1>(const BatchParams&, cudaStream_t, const BatchTune&);

}  // namespace hygt
