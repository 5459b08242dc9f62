// dyn_6_fwd.cu -- the bucketed forward kernels with a dynamic tail, 8x8 blocks.
#include "hygt_batch_dyn.cuh"

namespace hygt {

template cudaError_t launch_dyn_n<6, 0>(const BatchParams&, void*, int, cudaStream_t,
                                        const BatchTune&);

}  // namespace hygt
