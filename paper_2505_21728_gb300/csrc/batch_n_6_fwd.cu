// batch_n_6_fwd.cu -- bucketed forward kernels for 8x8 blocks (with the fused DCT-II primary).
#include "hygt_batch_launch.cuh"

namespace hygt {

template cudaError_t launch_batch_n<6, 0>(const BatchParams&, cudaStream_t, const BatchTune&);
template cudaError_t launch_primary_n<6, 0>(const BatchParams&, cudaStream_t, const BatchTune&);

}  // namespace hygt
