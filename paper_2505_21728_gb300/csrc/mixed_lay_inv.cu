// mixed_lay_inv.cu -- the layout-aware persistent mixed launch, inverse.
#include "hygt_mixed_lay.cuh"

namespace hygt {

template cudaError_t launch_mixed_lay<1>(MixedParams, cudaStream_t);

}  // namespace hygt
