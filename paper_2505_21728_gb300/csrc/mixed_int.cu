// mixed_int.cu -- one persistent launch over a mixed batch of block sizes.
//
// A frame tiled into 4x4, 8x8 and 16x16 blocks gives one bucketed batch per
// block size (each with its own plan and schedule).  The mixed kernel runs
// all of them in a single launch: CTAs [begin[c], begin[c + 1]) work on
// class c exactly like the batch kernel of that block size, so the classes
// proceed concurrently on disjoint SMs.  The split of CTAs among the classes
// is a launch parameter (chosen by the autotuner, or proportional to an
// estimate of each class's cost).
#include "hygt_batch.cuh"
#include "hygt_launch.cuh"
#include "hygt_mixed.cuh"

namespace hygt {

template <int KIND>
__global__ void __launch_bounds__(kBatchThreads, 1) hygt_mixed_kernel(MixedParams mp) {
  extern __shared__ __align__(16) int32_t msmem[];
  int c = 0;
  while (c + 1 < mp.nclasses && (int)blockIdx.x >= mp.cta_begin[c + 1]) ++c;
  const long long cta = (long long)blockIdx.x - mp.cta_begin[c];
  const long long ncta = (long long)mp.cta_begin[c + 1] - mp.cta_begin[c];
  if (ncta <= 0) return;
  switch (mp.log2n[c]) {
    case 4: batch_cta<4, KIND>(mp.cls[c], cta, ncta, msmem); break;
    case 6: batch_cta<6, KIND>(mp.cls[c], cta, ncta, msmem); break;
    case 8: batch_cta<8, KIND>(mp.cls[c], cta, ncta, msmem); break;
    default: break;
  }
}

template <int KIND>
static size_t pbuf_for(int log2n) {
  switch (log2n) {
    case 4: return batch_pbuf_bytes<4, KIND>(kBatchThreads);
    case 6: return batch_pbuf_bytes<6, KIND>(kBatchThreads);
    case 8: return batch_pbuf_bytes<8, KIND>(kBatchThreads);
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
  const size_t smem = (size_t)info.max_smem_optin;
  for (int c = 0; c < mp.nclasses; ++c) {
    const size_t pbuf = pbuf_for<KIND>(mp.log2n[c]);
    const size_t set_bytes = (size_t)mp.cls[c].set_words * 4;
    long long fit = ((long long)smem - (long long)pbuf) / (long long)set_bytes;
    if (fit > 64) fit = 64;
    if (fit < 0) fit = 0;
    mp.cls[c].max_cached_sets = (int)fit;
  }
  static std::atomic<int> attr_set{0};
  if ((int)smem > attr_set.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set.store((int)smem);
  }
  const int grid = mp.cta_begin[mp.nclasses];
  if (grid < 1) return cudaSuccess;
  kern<<<grid, kBatchThreads, smem, stream>>>(mp);
  return cudaGetLastError();
}

cudaError_t launch_mixed(int kind, const MixedParams& mp, cudaStream_t stream) {
  return kind == 0 ? launch_mixed_kind<0>(mp, stream) : launch_mixed_kind<1>(mp, stream);
}

}  // namespace hygt
