// f32b.cu -- the set-bucketed FP32 kernels and their launcher (see
// hygt_f32b.cuh).
#include <atomic>

#include "hygt_f32b.cuh"
#include "hygt_launch.cuh"

namespace hygt {

template <int LOG2N, bool INV>
__global__ void __launch_bounds__(kF32bThreads) hygt_f32b_kernel(F32bParams p) {
  using M = GradMap<LOG2N>;
  constexpr int G = M::G;
  extern __shared__ __align__(16) unsigned char fbs[];
  // the schedule must have been built for this batch
  if (p.meta[1] != (int)p.nblocks || p.meta[2] != p.num_sets || p.meta[3] != p.group_sched) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && p.status) atomicCAS(p.status, 0, 1);
    return;
  }
  const long long ntasks = max(0LL, min((long long)p.meta[0], p.tmax)) * (p.group_sched / G);
  const int wpc = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const long long warps_total = (long long)gridDim.x * wpc;
  const long long chunk = (ntasks + warps_total - 1) / warps_total;
  const long long t0 = min(ntasks, ((long long)blockIdx.x * wpc + warp) * chunk);
  const long long t1 = min(ntasks, t0 + chunk);
  // sets spanned by this CTA's tasks (consecutive in the sorted order)
  const long long c0 = min(ntasks, (long long)blockIdx.x * wpc * chunk);
  const long long c1 = min(ntasks, c0 + (long long)wpc * chunk);
  int set_lo = 0, ncache = 0;
  if (c1 > c0) {
    const int lo = bucket_of_slot(p.starts, p.num_sets, (int)(c0 * G));
    const int hi = bucket_of_slot(p.starts, p.num_sets, (int)(c1 * G - 1));
    set_lo = min(lo, p.num_sets);
    const int set_hi = min(hi, p.num_sets - 1);
    ncache = set_hi >= set_lo ? set_hi - set_lo + 1 : 0;
  }
  const bool cached = ncache <= p.max_cached_sets;
  if (cached && ncache > 0) f32b_copy_sets<LOG2N>(p, set_lo, ncache, fbs);
  __syncthreads();
  const int lane32 = threadIdx.x & 31;
  float* pb = reinterpret_cast<float*>(fbs + (size_t)p.max_cached_sets * f32b_set_bytes<LOG2N>(p.rounds)) +
              (size_t)warp * M::GROUPS * M::RW + (lane32 / M::L) * M::RW;
  if (cached)
    f32b_tasks<LOG2N, INV, true>(p, t0, t1, fbs, set_lo, pb);
  else
    f32b_tasks<LOG2N, INV, false>(p, t0, t1, fbs, set_lo, pb);
}

template <int LOG2N, bool INV>
static cudaError_t launch_sized(F32bParams p, cudaStream_t stream) {
  using M = GradMap<LOG2N>;
  if (p.group_sched % M::G != 0) return cudaErrorInvalidConfiguration;
  auto kern = hygt_f32b_kernel<LOG2N, INV>;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  const size_t per_set = f32b_set_bytes<LOG2N>(p.rounds);
  const size_t fixed = f32b_smem_bytes<LOG2N>(kF32bThreads, p.rounds, 0);
  // the sets a CTA's share of the sorted order usually spans (at least 4)
  long long cap = 2 + (p.num_sets + info.sms - 1) / info.sms;
  if (cap < 4) cap = 4;
  const size_t budget = (size_t)info.max_smem_optin / 2;  // leave room for a second CTA
  long long fit = budget > fixed ? (long long)((budget - fixed) / per_set) : 0;
  p.max_cached_sets = (int)(fit < cap ? fit : cap);
  const size_t smem = fixed + (size_t)p.max_cached_sets * per_set;
  static std::atomic<int> attr_set{0};
  if ((int)smem > attr_set.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set.store((int)smem);
  }
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kF32bThreads, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) occ = 1;
  kern<<<(unsigned)(occ * info.sms), kF32bThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_f32b(int log2n, int kind, const F32bParams& p, cudaStream_t stream) {
  const bool inv = kind == 1;
  switch (log2n) {
#define HYGT_F32B_CASE(n) \
  case n: return inv ? launch_sized<n, true>(p, stream) : launch_sized<n, false>(p, stream);
    HYGT_F32B_CASE(4)
    HYGT_F32B_CASE(5)
    HYGT_F32B_CASE(6)
    HYGT_F32B_CASE(7)
    HYGT_F32B_CASE(8)
#undef HYGT_F32B_CASE
    default: return cudaErrorInvalidConfiguration;
  }
}

}  // namespace hygt
