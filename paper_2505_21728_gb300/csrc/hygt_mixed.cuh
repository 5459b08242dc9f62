// hygt_mixed.cuh -- parameters of the mixed-size persistent launch.
#pragma once

#include "hygt_batch.cuh"

namespace hygt {

constexpr int kMaxMixedClasses = 3;

// Classes are stored by block size, slot k holding N = 2^(4 + 2k) (16, 64,
// 256), so the kernel reads every class's parameters at fixed offsets.
struct MixedParams {
  BatchParams cls[kMaxMixedClasses];
  int present[kMaxMixedClasses];
  // concurrent: slot k runs on CTAs [cta_begin[k], cta_begin[k + 1]);
  // sequential: every CTA runs every present slot in turn.  The grid is
  // cta_begin[kMaxMixedClasses].
  int cta_begin[kMaxMixedClasses + 1];
  int sequential;
};

__host__ __device__ constexpr int mixed_slot_log2n(int k) { return 4 + 2 * k; }

// CTAs of one mixed launch (one CTA per SM).
int mixed_grid_ctas();
// kind 0: forward, 1: inverse.
cudaError_t launch_mixed(int kind, const MixedParams& mp, cudaStream_t stream);

}  // namespace hygt
