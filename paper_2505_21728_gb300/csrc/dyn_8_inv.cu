// dyn_8_inv.cu -- the bucketed inverse kernels with a dynamic tail, 16x16 blocks.
#include "hygt_batch_dyn.cuh"

namespace hygt {

template cudaError_t launch_dyn_n<8, 1>(const BatchParams&, void*, int, cudaStream_t,
                                        const BatchTune&);

}  // namespace hygt
