// hygt_batch_il.cuh -- the set-interleaved order of the bucketed kernels.
//
// The bucketed kernels give each warp one contiguous range of the sorted
// order, so the warps of one set sweep that set's blocks from the start of
// the batch to its end over the whole launch, and the warps of another set
// reach the same region of memory at another time.  For blocks smaller than
// a 128-byte line (N = 16: 32 bytes of int16 input, 64 bytes of int32
// coefficients) the neighbours of a block in a line belong to other sets,
// so a line is fetched from DRAM once per set that reads it.  Here all
// warps advance through the sets together instead: round r of the
// round-robin order holds task r of every set's bucket and an even share of
// the skip and bad-set buckets' tasks, and warp w takes entries w, w + W,
// w + 2W, ... of the rounds laid end to end.  Within a bucket the blocks
// follow the scatter's tile order, which is nearly the same for every
// bucket, so task t of every set covers about the same region of memory: a
// line's blocks are read within one sweep of the warps, while the line is
// still in L2.  A CTA keeps the
// tables of all sets in shared memory (N = 16: 1,152 bytes a set in layout
// 2) or reads them from global memory, by the launch tuning.  The
// arithmetic is batch_tasks', one task per call, without staging.
#pragma once

#include <atomic>

#include "hygt_batch.cuh"
#include "hygt_launch.cuh"

namespace hygt {

// batch_il.cu: block sizes and layouts with the interleaved order, and its
// launcher (kind 0 forward, 1 inverse).
bool batch_il_ok(int log2n, int layout);
cudaError_t launch_batch_il(int kind, int log2n, const BatchParams& p, cudaStream_t stream,
                            const BatchTune& tune);

template <int LOG2N, int KIND, bool CACHED, int LAY>
__global__ void __launch_bounds__(batch_threads(LOG2N, KIND, LAY), 1)
    hygt_batch_il_kernel(BatchParams p) {
  extern __shared__ __align__(16) int32_t ismem[];
  __shared__ int s_rounds;
  constexpr int GS = batch_group(LOG2N);
  constexpr int G = batch_task_group(LOG2N, KIND == 1, LAY);
  // The schedule must have been built for this block count, set count and G.
  if (p.meta[1] != (int)p.nblocks || p.meta[2] != p.num_sets || p.meta[3] != GS) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && p.status) atomicCAS(p.status, 0, 1);
    return;
  }
  const int S = p.num_sets;
  const long long ntasks = max(0LL, min((long long)p.meta[0], p.tmax)) * (GS / G);
  // Rounds of the interleave: T = the largest set bucket's task count.  A
  // round holds task r of every set bucket, then Q tasks of the skip bucket
  // and Qb of the bad-set bucket (their tasks spread evenly over the rounds,
  // so that they too keep pace with the sets).
  if (threadIdx.x < 32) {
    int m = 0;
    for (int b = threadIdx.x; b < S; b += 32)
      m = max(m, (__ldg(p.starts + b + 1) - __ldg(p.starts + b)) / G);
#pragma unroll
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) s_rounds = max(m, 1);
  }
  if constexpr (CACHED) {
    const int4* src = reinterpret_cast<const int4*>(p.ktab);
    int4* dst = reinterpret_cast<int4*>(ismem);
    const int n4 = S * p.set_words / 4;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  const int T = s_rounds;
  const int n_skip = (__ldg(p.starts + S + 1) - __ldg(p.starts + S)) / G;
  const int n_bad = (__ldg(p.starts + S + 2) - __ldg(p.starts + S + 1)) / G;
  const int Q = (n_skip + T - 1) / T;
  const int Qb = (n_bad + T - 1) / T;
  const int P = S + Q + Qb;  // entries per round
  const long long entries = (long long)T * P;
  const int wpc = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const long long W = (long long)gridDim.x * wpc;
  int32_t* pbuf = ismem + (CACHED ? (size_t)S * p.set_words : 0);
  int32_t* wbuf = pbuf + (size_t)warp * (batch_warp_bytes<LOG2N, KIND, false, false, LAY>() / 4);
  for (long long e = (long long)blockIdx.x * wpc + warp; e < entries; e += W) {
    const int r = (int)(e / P);
    const int j = (int)(e - (long long)r * P);
    int b, t, n;  // bucket, its task, its task count (warp-uniform)
    if (j < S) {
      b = j;
      t = r;
      n = (__ldg(p.starts + b + 1) - __ldg(p.starts + b)) / G;
    } else if (j < S + Q) {
      b = S;
      t = r * Q + (j - S);
      n = n_skip;
    } else {
      b = S + 1;
      t = r * Qb + (j - S - Q);
      n = n_bad;
    }
    if (t >= n) continue;
    const long long task = __ldg(p.starts + b) / G + t;
    if (task >= ntasks) continue;
    batch_tasks<LOG2N, KIND, CACHED, false, false, false, false, LAY>(p, task, task + 1, ismem,
                                                                       0, wbuf);
  }
}

template <int LOG2N, int KIND, bool CACHED, int LAY>
inline cudaError_t launch_il_kernel(const BatchParams& p, int threads, size_t smem, int want,
                                    int sms, cudaStream_t stream) {
  auto kern = hygt_batch_il_kernel<LOG2N, KIND, CACHED, LAY>;
  static std::atomic<int> attr_set{0};
  cudaError_t err;
  if ((int)smem > attr_set.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set.store((int)smem);
  }
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) occ = 1;
  if (want > 0 && want < occ) occ = want;
  kern<<<(unsigned)((long long)occ * sms), threads, smem, stream>>>(p);
  return cudaGetLastError();
}

// One launch in the interleaved order, warps per CTA from `tune`.  CTAs per
// SM 0: as many as the registers allow, the set tables read from global
// memory (through L1; without a stage, this order wants many warps to hide
// its load latency); k >= 1: at most k, each holding the tables of all sets
// in shared memory when they fit in its share.
template <int LOG2N, int KIND, int LAY>
inline cudaError_t launch_il_variant(BatchParams p, cudaStream_t stream, const BatchTune& tune) {
  if constexpr (LAY != 0) {
    if (!p.ktabs[LAY]) return cudaErrorInvalidConfiguration;
    p.ktab = p.ktabs[LAY];
    p.set_words = p.set_words_of[LAY];
  }
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  constexpr int kMaxWarps = batch_threads(LOG2N, KIND, LAY) / 32;
  const int warps = tune.warps > 0 && tune.warps < kMaxWarps ? tune.warps : kMaxWarps;
  const int threads = warps * 32;
  const size_t pbuf = batch_pbuf_bytes<LOG2N, KIND, false, false, LAY>(threads);
  p.max_cached_sets = 0;
  if (tune.ctas_per_sm == 0) {
    if (pbuf > (size_t)info.max_smem_optin) return cudaErrorInvalidConfiguration;
    return launch_il_kernel<LOG2N, KIND, false, LAY>(p, threads, pbuf, 0, info.sms, stream);
  }
  const int want = tune.ctas_per_sm;
  const size_t budget = (size_t)info.max_smem_optin / want - (want > 1 ? 1024 : 0);
  if (pbuf > budget) return cudaErrorInvalidConfiguration;
  const size_t tables = (size_t)p.num_sets * p.set_words * 4;
  if (pbuf + tables <= budget)
    return launch_il_kernel<LOG2N, KIND, true, LAY>(p, threads, pbuf + tables, tune.ctas_per_sm,
                                                    info.sms, stream);
  return launch_il_kernel<LOG2N, KIND, false, LAY>(p, threads, pbuf, tune.ctas_per_sm, info.sms,
                                                   stream);
}

}  // namespace hygt
