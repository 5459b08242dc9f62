// batch_int.cu -- the bucketing kernels of the set-bucketed integer HyGT (counting sort of
// the block ids by transform set; see hygt_batch.cuh).  The transform launchers are in
// batch_fwd.cu and batch_inv.cu.
#include "hygt_batch.cuh"
#include "hygt_launch.cuh"

namespace hygt {

__device__ __forceinline__ int bucket_of(unsigned set, int num_sets) {
  if (set == 0xFFFFu) return num_sets;   // skip: identity
  if (set >= (unsigned)num_sets) return num_sets + 1;  // bad set index
  return (int)set;
}

// Pass 1: per-bucket counts (shared-memory histogram per CTA when it fits).
__global__ void __launch_bounds__(kBucketThreads) batch_count(const uint16_t* __restrict__ set,
                                                              long long nblocks, int num_sets,
                                                              int* __restrict__ counts) {
  extern __shared__ int hist[];
  const int nb = num_sets + 2;
  const bool local = nb <= 4096;
  if (local)
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < nblocks; b += stride) {
    const int k = bucket_of(set ? __ldg(set + b) : 0u, num_sets);
    if (local)
      atomicAdd(&hist[k], 1);
    else
      atomicAdd(&counts[k], 1);
  }
  __syncthreads();
  if (local)
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
      if (hist[i]) atomicAdd(&counts[i], hist[i]);
}

// Pass 2 (one CTA): exclusive scan of the counts, each padded to a multiple
// of the task size `group`, into the bucket starts and scatter cursors;
// writes -1 into the padding slots.
__global__ void __launch_bounds__(1024) batch_scan(const int* __restrict__ counts, int num_sets,
                                                  long long nblocks, int group,
                                                  int* __restrict__ starts,
                                                  int* __restrict__ cursor, int* __restrict__ meta,
                                                  int* __restrict__ order) {
  __shared__ long long part[1024];
  __shared__ long long carry;
  const int nb = num_sets + 2;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const long long padded =
        (k < nb) ? (long long)((counts[k] + group - 1) / group) * group : 0;
    part[threadIdx.x] = padded;
    __syncthreads();
    for (int d = 1; d < (int)blockDim.x; d <<= 1) {  // inclusive Hillis-Steele scan
      const long long t = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
      __syncthreads();
      part[threadIdx.x] += t;
      __syncthreads();
    }
    const long long start = carry + part[threadIdx.x] - padded;
    if (k < nb) {
      starts[k] = (int)start;
      cursor[k] = (int)start;
      const int c = counts[k];
      for (long long s = start + c; s < start + padded; ++s) order[s] = -1;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    meta[0] = (int)(carry / group);
    meta[1] = (int)nblocks;
    meta[2] = num_sets;
    meta[3] = group;
    starts[nb] = (int)carry;
  }
}

// Pass 3: scatter block ids into their buckets.  Each CTA ranks a tile of
// blocks in shared memory and reserves one range per bucket with a single
// global atomic.
__global__ void __launch_bounds__(kBucketThreads) batch_scatter(const uint16_t* __restrict__ set,
                                                                long long nblocks, int num_sets,
                                                                int* __restrict__ cursor,
                                                                int* __restrict__ order) {
  extern __shared__ int sh[];
  const int nb = num_sets + 2;
  const bool local = nb <= 4096;
  int* cnt = sh;
  int* base = sh + (local ? nb : 0);
  constexpr int PER = kBucketTile / kBucketThreads;
  for (long long tile = (long long)blockIdx.x * kBucketTile; tile < nblocks;
       tile += (long long)gridDim.x * kBucketTile) {
    if (local) {
      for (int i = threadIdx.x; i < nb; i += blockDim.x) cnt[i] = 0;
      __syncthreads();
    }
    int bk[PER], rk[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const long long b = tile + (long long)u * blockDim.x + threadIdx.x;
      bk[u] = -1;
      rk[u] = 0;
      if (b < nblocks) {
        bk[u] = bucket_of(set ? __ldg(set + b) : 0u, num_sets);
        rk[u] = local ? atomicAdd(&cnt[bk[u]], 1) : atomicAdd(&cursor[bk[u]], 1);
      }
    }
    if (local) {
      __syncthreads();
      for (int i = threadIdx.x; i < nb; i += blockDim.x)
        base[i] = cnt[i] ? atomicAdd(&cursor[i], cnt[i]) : 0;
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const long long b = tile + (long long)u * blockDim.x + threadIdx.x;
      if (bk[u] >= 0) order[(local ? base[bk[u]] : 0) + rk[u]] = (int)b;
    }
    if (local) __syncthreads();
  }
}

cudaError_t batch_build(const uint16_t* d_set, long long nblocks, int num_sets, int group,
                        void* d_work, cudaStream_t stream) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  const BatchLayout L = batch_layout(num_sets, nblocks, group);
  char* w = static_cast<char*>(d_work);
  int* counts = reinterpret_cast<int*>(w + L.counts);
  int* starts = reinterpret_cast<int*>(w + L.starts);
  int* cursor = reinterpret_cast<int*>(w + L.cursor);
  int* meta = reinterpret_cast<int*>(w + L.meta);
  int* order = reinterpret_cast<int*>(w + L.order);
  err = cudaMemsetAsync(counts, 0, 4 * (size_t)L.nb, stream);
  if (err != cudaSuccess) return err;
  const bool local = L.nb <= 4096;
  long long g1 = (nblocks + kBucketThreads - 1) / kBucketThreads;
  if (g1 > 4LL * info.sms) g1 = 4LL * info.sms;
  if (g1 < 1) g1 = 1;
  batch_count<<<(unsigned)g1, kBucketThreads, local ? 4 * L.nb : 0, stream>>>(d_set, nblocks,
                                                                            num_sets, counts);
  batch_scan<<<1, 1024, 0, stream>>>(counts, num_sets, nblocks, group, starts, cursor, meta,
                                     order);
  long long g3 = (nblocks + kBucketTile - 1) / kBucketTile;
  if (g3 > 4LL * info.sms) g3 = 4LL * info.sms;
  if (g3 < 1) g3 = 1;
  batch_scatter<<<(unsigned)g3, kBucketThreads, local ? 8 * L.nb : 0, stream>>>(
      d_set, nblocks, num_sets, cursor, order);
  return cudaGetLastError();
}

}  // namespace hygt
