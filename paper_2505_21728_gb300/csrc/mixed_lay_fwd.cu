// mixed_lay_fwd.cu -- the layout-aware persistent mixed launch, forward.
#include "hygt_mixed_lay.cuh"

namespace hygt {

template cudaError_t launch_mixed_lay<0>(MixedParams, cudaStream_t);

}  // namespace hygt
