// hygt_mixed_lay.cuh -- the layout-aware persistent launch over a mixed
// batch: as the kernel of mixed_int.cu (sequential or concurrent classes),
// with each class in the staging and register layout that its entry of
// mixed_variant names, so that a class runs the code the batch autotuner
// picked for it instead of layout 0.  Instantiated per direction in
// mixed_lay_fwd.cu and mixed_lay_inv.cu.
#pragma once

#include <algorithm>
#include <atomic>

#include "hygt_batch.cuh"
#include "hygt_launch.cuh"
#include "hygt_mixed.cuh"

namespace hygt {

template <int LOG2N, int KIND, int V>
__device__ __forceinline__ void mixed_variant_cta(const BatchParams& p, long long cta,
                                                  long long ncta, int32_t* smem) {
  constexpr MixedVariant mv = mixed_variant(LOG2N, V);
  if constexpr (mv.stage >= 0)
    batch_cta<LOG2N, KIND, mv.stage == 1, false, mv.stage == 2, false, mv.layout>(p, cta, ncta,
                                                                                 smem);
}

template <int LOG2N, int KIND>
__device__ __forceinline__ void mixed_class_cta(const BatchParams& p, int v, long long cta,
                                                long long ncta, int32_t* smem) {
  switch (v) {  // block-uniform
    case 1: mixed_variant_cta<LOG2N, KIND, 1>(p, cta, ncta, smem); break;
    case 2: mixed_variant_cta<LOG2N, KIND, 2>(p, cta, ncta, smem); break;
    case 3: mixed_variant_cta<LOG2N, KIND, 3>(p, cta, ncta, smem); break;
    default: mixed_variant_cta<LOG2N, KIND, 0>(p, cta, ncta, smem); break;
  }
}

template <int KIND>
__global__ void __launch_bounds__(kMixedLayThreads, 1) hygt_mixed_lay_kernel(MixedParams mp) {
  extern __shared__ __align__(16) int32_t lsmem[];
  if (mp.sequential) {
    if (mp.present[0]) {
      mixed_class_cta<4, KIND>(mp.cls[0], mp.variant[0], blockIdx.x, gridDim.x, lsmem);
      __syncthreads();
    }
    if (mp.present[1]) {
      mixed_class_cta<6, KIND>(mp.cls[1], mp.variant[1], blockIdx.x, gridDim.x, lsmem);
      __syncthreads();
    }
    if (mp.present[2])
      mixed_class_cta<8, KIND>(mp.cls[2], mp.variant[2], blockIdx.x, gridDim.x, lsmem);
    return;
  }
  const int b = (int)blockIdx.x;
  if (b < mp.cta_begin[1])
    mixed_class_cta<4, KIND>(mp.cls[0], mp.variant[0], b, mp.cta_begin[1], lsmem);
  else if (b < mp.cta_begin[2])
    mixed_class_cta<6, KIND>(mp.cls[1], mp.variant[1], b - mp.cta_begin[1],
                             mp.cta_begin[2] - mp.cta_begin[1], lsmem);
  else
    mixed_class_cta<8, KIND>(mp.cls[2], mp.variant[2], b - mp.cta_begin[2],
                             mp.cta_begin[3] - mp.cta_begin[2], lsmem);
}

// Per-warp shared memory of a menu entry (0 past the end of the menu).
template <int LOG2N, int KIND, int V>
inline size_t mixed_variant_pbuf(int threads) {
  constexpr MixedVariant mv = mixed_variant(LOG2N, V);
  if constexpr (mv.stage >= 0)
    return batch_pbuf_bytes<LOG2N, KIND, mv.stage == 1, false, mv.layout>(threads);
  else
    return 0;
}

template <int LOG2N, int KIND>
inline size_t mixed_class_pbuf(int v, int threads) {
  switch (v) {
    case 1: return mixed_variant_pbuf<LOG2N, KIND, 1>(threads);
    case 2: return mixed_variant_pbuf<LOG2N, KIND, 2>(threads);
    case 3: return mixed_variant_pbuf<LOG2N, KIND, 3>(threads);
    default: return mixed_variant_pbuf<LOG2N, KIND, 0>(threads);
  }
}

template <int KIND>
cudaError_t launch_mixed_lay(MixedParams mp, cudaStream_t stream) {
  auto kern = hygt_mixed_lay_kernel<KIND>;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  size_t smem = 0;
  for (int k = 0; k < kMaxMixedClasses; ++k) {
    if (!mp.present[k]) continue;
    const int log2n = mixed_slot_log2n(k);
    const int v = mp.variant[k];
    if (v < 0 || v >= kMixedVariants) return cudaErrorInvalidConfiguration;
    const MixedVariant mv = mixed_variant(log2n, v);
    if (mv.stage < 0) return cudaErrorInvalidConfiguration;
    BatchParams& c = mp.cls[k];
    if (mv.layout != 0) {  // the layout's own set tables
      if (!c.ktabs[mv.layout]) return cudaErrorInvalidConfiguration;
      c.ktab = c.ktabs[mv.layout];
      c.set_words = c.set_words_of[mv.layout];
    }
    const size_t pbuf = log2n == 4   ? mixed_class_pbuf<4, KIND>(v, kMixedLayThreads)
                        : log2n == 6 ? mixed_class_pbuf<6, KIND>(v, kMixedLayThreads)
                                     : mixed_class_pbuf<8, KIND>(v, kMixedLayThreads);
    const size_t set_bytes = (size_t)c.set_words * 4;
    const int fit =
        batch_cached_sets((size_t)info.max_smem_optin, pbuf, set_bytes, c.num_sets, info.sms);
    if (fit < 0 || pbuf > (size_t)info.max_smem_optin) return cudaErrorInvalidConfiguration;
    c.max_cached_sets = fit;
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
  kern<<<grid, kMixedLayThreads, smem, stream>>>(mp);
  return cudaGetLastError();
}

}  // namespace hygt
