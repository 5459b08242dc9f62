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
  // per slot, the entry of mixed_variant the class runs in; all 0 (layout 0
  // with its default staging) runs the first kernel, anything else the
  // layout-aware one
  int variant[kMaxMixedClasses];
};

__host__ __device__ constexpr int mixed_slot_log2n(int k) { return 4 + 2 * k; }

// Staging and register layout of a class in the layout-aware persistent
// kernel (the batch kernel's tuning fields, BatchTune::stage and ::layout).
// The kernel carries a short menu per block size, the pairs the batch
// autotuner picks for frame-sized batches: a whole BatchTune space per class
// would multiply one kernel's code by the product of three spaces.  Entry 0
// is layout 0 with its default staging; stage -1 marks the end of a menu.
// The bulk stage (3) is left out: its per-warp mbarrier lives in the shared
// memory that the next class of a sequential launch reuses.
struct MixedVariant {
  int stage;
  int layout;
};
constexpr int kMixedVariants = 4;
constexpr int kMixedLayThreads = 384;  // CTA of the layout-aware kernel
__host__ __device__ constexpr MixedVariant mixed_variant(int log2n, int v) {
  return log2n == 4   ? (v == 0   ? MixedVariant{0, 0}
                         : v == 1 ? MixedVariant{0, 2}
                         : v == 2 ? MixedVariant{1, 2}
                                  : MixedVariant{-1, -1})
         : log2n == 6 ? (v == 0   ? MixedVariant{1, 0}
                         : v == 1 ? MixedVariant{0, 3}
                         : v == 2 ? MixedVariant{2, 3}
                                  : MixedVariant{-1, -1})
         : log2n == 8 ? (v == 0   ? MixedVariant{0, 0}
                         : v == 1 ? MixedVariant{0, 5}
                         : v == 2 ? MixedVariant{1, 5}
                         : v == 3 ? MixedVariant{0, 4}
                                  : MixedVariant{-1, -1})
                      : MixedVariant{-1, -1};
}
static_assert(mixed_variant(4, 0).stage == (batch_staged(4, 0) ? 1 : 0) &&
                  mixed_variant(6, 0).stage == (batch_staged(6, 0) ? 1 : 0) &&
                  mixed_variant(8, 0).stage == (batch_staged(8, 0) ? 1 : 0),
              "entry 0 is the first kernel's staging");

// The menu entry for a class tuned to (stage, layout), stage -1 meaning the
// layout's default: the same pair when the menu has it, else the layout's
// first entry, else entry 0.
__host__ inline int mixed_variant_of(int log2n, int stage, int layout) {
  if (stage < 0) stage = (layout == 0 && batch_staged(log2n, 0)) ? 1 : 0;
  int first = -1;
  for (int v = 0; v < kMixedVariants; ++v) {
    const MixedVariant mv = mixed_variant(log2n, v);
    if (mv.stage < 0 || mv.layout != layout) continue;
    if (mv.stage == stage) return v;
    if (first < 0) first = v;
  }
  return first < 0 ? 0 : first;
}

// CTAs of one mixed launch (one CTA per SM).
int mixed_grid_ctas();
// kind 0: forward, 1: inverse.
cudaError_t launch_mixed(int kind, const MixedParams& mp, cudaStream_t stream);
// The layout-aware kernel (mixed_lay_fwd.cu, mixed_lay_inv.cu).
template <int KIND>
cudaError_t launch_mixed_lay(MixedParams mp, cudaStream_t stream);

}  // namespace hygt
