// hygt_mixed.cuh -- parameters of the mixed-size persistent launch.
#pragma once

#include "hygt_batch.cuh"

namespace hygt {

constexpr int kMaxMixedClasses = 3;

struct MixedParams {
  BatchParams cls[kMaxMixedClasses];
  int log2n[kMaxMixedClasses];
  int cta_begin[kMaxMixedClasses + 1];  // class c runs on CTAs [cta_begin[c], cta_begin[c + 1])
  int nclasses;
};

// CTAs of one mixed launch (one CTA per SM).
int mixed_grid_ctas();
// kind 0: forward, 1: inverse.
cudaError_t launch_mixed(int kind, const MixedParams& mp, cudaStream_t stream);

}  // namespace hygt
