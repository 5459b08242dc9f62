// mixed_int.cu -- one persistent launch over a mixed batch of block sizes.
//
// A frame tiled into 4x4, 8x8 and 16x16 blocks gives one bucketed batch per
// block size (each with its own plan and schedule).  The mixed kernel runs
// all of them in a single launch, in one of two ways: sequential -- every
// CTA works on class 0 exactly like the batch kernel of that block size,
// then on class 1, ... (a CTA that finishes its share of a class goes on to
// the next without waiting for the others); or concurrent -- CTAs
// [begin[c], begin[c + 1]) work on class c only, so the classes proceed on
// disjoint SMs.  Which, and the split, is a launch parameter (chosen by the
// autotuner).  This kernel runs every class in layout 0 with its default
// staging; when a class's tuning names another entry of its menu
// (mixed_variant), the launch goes to the layout-aware kernel of
// hygt_mixed_lay.cuh instead.
#include <algorithm>

#include "hygt_batch.cuh"
#include "hygt_launch.cuh"
#include "hygt_mixed.cuh"

namespace hygt {

template <int KIND>
__global__ void __launch_bounds__(batch_threads(6, KIND), 1) hygt_mixed_kernel(MixedParams mp) {
  extern __shared__ __align__(16) int32_t msmem[];
  if (mp.sequential) {
    // every CTA works through the classes in turn; shared memory is reused
    if (mp.present[0]) {
      batch_cta<4, KIND>(mp.cls[0], blockIdx.x, gridDim.x, msmem);
      __syncthreads();
    }
    if (mp.present[1]) {
      batch_cta<6, KIND>(mp.cls[1], blockIdx.x, gridDim.x, msmem);
      __syncthreads();
    }
    if (mp.present[2]) batch_cta<8, KIND>(mp.cls[2], blockIdx.x, gridDim.x, msmem);
    return;
  }
  const int b = (int)blockIdx.x;
  if (b < mp.cta_begin[1])
    batch_cta<4, KIND>(mp.cls[0], b, mp.cta_begin[1], msmem);
  else if (b < mp.cta_begin[2])
    batch_cta<6, KIND>(mp.cls[1], b - mp.cta_begin[1], mp.cta_begin[2] - mp.cta_begin[1], msmem);
  else
    batch_cta<8, KIND>(mp.cls[2], b - mp.cta_begin[2], mp.cta_begin[3] - mp.cta_begin[2], msmem);
}

template <int KIND>
static size_t pbuf_for(int log2n) {
  switch (log2n) {
    case 4: return batch_pbuf_bytes<4, KIND>(batch_threads(6, KIND));
    case 6: return batch_pbuf_bytes<6, KIND>(batch_threads(6, KIND));
    case 8: return batch_pbuf_bytes<8, KIND>(batch_threads(6, KIND));
    default: return 0;
  }
}

int mixed_grid_ctas() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  return device_info(dev).sms;  // one CTA per SM
}

template <int KIND>
static cudaError_t launch_mixed_kind(MixedParams mp, cudaStream_t stream) {
  auto kern = hygt_mixed_kernel<KIND>;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  // one shared-memory size for the launch: the largest any present class asks for
  size_t smem = 0;
  for (int k = 0; k < kMaxMixedClasses; ++k) {
    if (!mp.present[k]) continue;
    const size_t pbuf = pbuf_for<KIND>(mixed_slot_log2n(k));
    const size_t set_bytes = (size_t)mp.cls[k].set_words * 4;
    const int fit = batch_cached_sets((size_t)info.max_smem_optin, pbuf, set_bytes,
                                      mp.cls[k].num_sets, info.sms);
    mp.cls[k].max_cached_sets = fit;
    smem = std::max(smem, pbuf + (size_t)fit * set_bytes);
  }
  if (smem == 0) return cudaSuccess;
  static std::atomic<int> attr_set{0};
  if ((int)smem > attr_set.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set.store((int)smem);
  }
  const int grid = mp.cta_begin[kMaxMixedClasses];
  if (grid < 1) return cudaSuccess;
  kern<<<grid, batch_threads(6, KIND), smem, stream>>>(mp);
  return cudaGetLastError();
}

cudaError_t launch_mixed(int kind, const MixedParams& mp, cudaStream_t stream) {
  bool tuned = false;  // a class in another layout or staging than layout 0's default
  for (int k = 0; k < kMaxMixedClasses; ++k) tuned |= mp.present[k] && mp.variant[k] != 0;
  if (tuned) return kind == 0 ? launch_mixed_lay<0>(mp, stream) : launch_mixed_lay<1>(mp, stream);
  return kind == 0 ? launch_mixed_kind<0>(mp, stream) : launch_mixed_kind<1>(mp, stream);
}

}  // namespace hygt
