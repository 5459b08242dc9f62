// dyn_8_fwd.cu -- the bucketed forward kernels with a dynamic tail, 16x16 blocks.
#include "hygt_batch_dyn.cuh"

namespace hygt {

template cudaError_t launch_dyn_n<8, 0>(const BatchParams&, void*, int, cudaStream_t,
                                        const BatchTune&);

}  // namespace hygt
