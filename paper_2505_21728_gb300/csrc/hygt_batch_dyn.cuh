// hygt_batch_dyn.cuh -- the bucketed kernels with a dynamic tail.
//
// The batch kernel splits the sorted order into one contiguous range per
// warp, fixed at launch, so each SM's share of the work is fixed too: SMs
// whose tasks run slower (set tables read from global memory, the DRAM
// parts they land on) finish late, and in a short launch -- about a dozen
// tasks per warp -- a quarter of the warps' time goes to the launch's ramp,
// its tail and that imbalance.  Here the first (64 - tail) / 64 of the
// order is split into contiguous warp ranges that differ by at most one
// task (each CTA caching the tables of the sets its range spans), and the
// last tail / 64 is handed out one task at a time by an atomic counter to
// the warps that finish their range, so the SMs that are done early take
// the rest.  The tail of the sorted order is the last
// sets, the skip bucket and the bad-set bucket; its tasks read their tables
// from global memory and run without a stage.  The counter sits in the 16
// bytes after the schedule (BatchLayout::total), which the schedule build
// zeroes; the last warp to finish puts it back to zero, so forward and
// inverse launches may repeat without a rebuild.
#pragma once

#include <atomic>

#include "hygt_batch.cuh"
#include "hygt_launch.cuh"

namespace hygt {

// Bytes after BatchLayout::total: the claimed-task counter (64-bit) and the
// count of warps that are done (32-bit).
constexpr size_t kDynCounterBytes = 16;

// dyn.cu: block sizes, layouts and stages with a dynamic tail, and the
// launcher (kind 0 forward, 1 inverse; tail_64ths 1 .. 32).
bool batch_dyn_ok(int log2n, int layout, int stage);
cudaError_t launch_batch_dyn(int kind, int log2n, const BatchParams& p, void* counters,
                             int tail_64ths, cudaStream_t stream, const BatchTune& tune);

template <int LOG2N, int KIND, bool STAGED, bool PF, bool BULK, int LAY>
__global__ void __launch_bounds__(batch_threads(LOG2N, KIND, LAY), 1)
    hygt_batch_dyn_kernel(BatchParams p, unsigned long long* counters, int tail_64ths) {
  extern __shared__ __align__(16) int32_t dsmem[];
  constexpr int GS = batch_group(LOG2N);
  constexpr int G = batch_task_group(LOG2N, KIND == 1, LAY);
  // The schedule must have been built for this block count, set count and G.
  if (p.meta[1] != (int)p.nblocks || p.meta[2] != p.num_sets || p.meta[3] != GS) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && p.status) atomicCAS(p.status, 0, 1);
    return;
  }
  const long long ntasks = max(0LL, min((long long)p.meta[0], p.tmax)) * (GS / G);
  const long long ntail = ntasks * tail_64ths / 64;
  const long long nstatic = ntasks - ntail;
  const long long cta = blockIdx.x, ncta = gridDim.x;

  // the static part over [0, nstatic): warp gw takes tasks
  // [gw nstatic / W, (gw + 1) nstatic / W), so that shares differ by at most
  // one task (whole chunks of ceil(nstatic / W) would leave the last CTAs
  // short or empty), and each CTA caches the sets of its warps' ranges
  const int wpc = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const long long warps_total = ncta * wpc;
  const long long gw = cta * wpc + warp;
  const long long t0 = gw * nstatic / warps_total;
  const long long t1 = (gw + 1) * nstatic / warps_total;
  const long long c0 = cta * wpc * nstatic / warps_total;
  const long long c1 = (cta + 1) * wpc * nstatic / warps_total;
  int set_lo = 0, ncache = 0;
  if (c1 > c0) {
    const int bk_lo = bucket_of_slot(p.starts, p.num_sets, (int)(c0 * G));
    const int bk_hi = bucket_of_slot(p.starts, p.num_sets, (int)(c1 * G - 1));
    set_lo = min(bk_lo, p.num_sets);
    const int set_hi = min(bk_hi, p.num_sets - 1);
    ncache = set_hi >= set_lo ? set_hi - set_lo + 1 : 0;
  }
  const bool cached = ncache <= p.max_cached_sets;
  int32_t* cache = dsmem;
  int32_t* pbuf = dsmem + (size_t)p.max_cached_sets * p.set_words;
  if (cached && ncache > 0) {
    const int4* src = reinterpret_cast<const int4*>(p.ktab + (size_t)set_lo * p.set_words);
    int4* dst = reinterpret_cast<int4*>(cache);
    const int n4 = ncache * p.set_words / 4;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  int32_t* wbuf =
      pbuf + (size_t)warp * (batch_warp_bytes<LOG2N, KIND, STAGED, BULK, LAY>() / 4);
  if (cached)
    batch_tasks<LOG2N, KIND, true, STAGED, false, PF, BULK, LAY>(p, t0, t1, cache, set_lo, wbuf);
  else
    batch_tasks<LOG2N, KIND, false, STAGED, false, PF, BULK, LAY>(p, t0, t1, cache, set_lo, wbuf);

  // the tail, one task per claim (the permutation buffer is the start of
  // the warp's region in every staging variant)
  const int lane32 = threadIdx.x & 31;
  for (;;) {
    unsigned long long t = 0;
    if (lane32 == 0) t = atomicAdd(counters, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if ((long long)t >= ntail) break;
    const long long task = nstatic + (long long)t;
    batch_tasks<LOG2N, KIND, false, false, false, false, false, LAY>(p, task, task + 1, nullptr,
                                                                     0, wbuf);
  }
  if (lane32 == 0) {  // the last warp done resets the counters for the next launch
    unsigned* done = reinterpret_cast<unsigned*>(counters + 1);
    if (atomicAdd(done, 1u) == (unsigned)warps_total - 1u) {
      atomicExch(counters, 0ull);
      atomicExch(done, 0u);
    }
  }
}

template <int LOG2N, int KIND, bool STAGED, bool PF, bool BULK, int LAY>
inline cudaError_t launch_dyn_variant(BatchParams p, void* counters, int tail_64ths,
                                      cudaStream_t stream, const BatchTune& tune) {
  auto kern = hygt_batch_dyn_kernel<LOG2N, KIND, STAGED, PF, BULK, LAY>;
  if constexpr (LAY != 0) {  // the layout's own set tables
    if (!p.ktabs[LAY]) return cudaErrorInvalidConfiguration;
    p.ktab = p.ktabs[LAY];
    p.set_words = p.set_words_of[LAY];
  }
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  constexpr int G = batch_task_group(LOG2N, KIND == 1, LAY);
  constexpr int kMaxWarps = batch_threads(LOG2N, KIND, LAY) / 32;
  const int warps = tune.warps > 0 && tune.warps < kMaxWarps ? tune.warps : kMaxWarps;
  const int threads = warps * 32;
  const size_t pbuf = batch_pbuf_bytes<LOG2N, KIND, STAGED, BULK, LAY>(threads);
  const size_t set_bytes = (size_t)p.set_words * 4;
  const int want = tune.ctas_per_sm > 0 ? tune.ctas_per_sm : 1;
  const size_t budget = (size_t)info.max_smem_optin / want - (want > 1 ? 1024 : 0);
  const int fit = batch_cached_sets(budget, pbuf, set_bytes, p.num_sets, info.sms * want);
  if (fit < 0 || pbuf > budget) return cudaErrorInvalidConfiguration;
  p.max_cached_sets = fit;
  const size_t smem = pbuf + (size_t)fit * set_bytes;
  static std::atomic<int> attr_set{0};
  if ((int)smem > attr_set.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set.store((int)smem);
  }
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) occ = 1;
  if (tune.ctas_per_sm > 0 && tune.ctas_per_sm < occ) occ = tune.ctas_per_sm;
  const long long per_cta = (long long)warps * G;
  long long need = (p.nblocks + per_cta - 1) / per_cta + 1;
  long long grid = (long long)occ * info.sms;
  if (need < grid) grid = need;
  kern<<<(unsigned)grid, threads, smem, stream>>>(
      p, static_cast<unsigned long long*>(counters), tail_64ths);
  return cudaGetLastError();
}

// The variants of one block size and direction (stage as BatchTune::stage:
// -1 the default, 0 none, 1 cp.async, 2 L2 prefetch, 3 bulk copies (layout 0)).
template <int LOG2N, int KIND, int LAY>
inline cudaError_t launch_dyn_layout(const BatchParams& p, void* counters, int tail_64ths,
                                     cudaStream_t stream, const BatchTune& tune) {
  int stage = tune.stage < 0 ? (LAY == 0 && batch_staged(LOG2N, KIND) ? 1 : 0) : tune.stage;
  if (stage == 3 && (reinterpret_cast<uintptr_t>(p.in) & 15) != 0) stage = 0;
  if (stage == 1)
    return launch_dyn_variant<LOG2N, KIND, true, false, false, LAY>(p, counters, tail_64ths,
                                                                    stream, tune);
  if (stage == 2)
    return launch_dyn_variant<LOG2N, KIND, false, true, false, LAY>(p, counters, tail_64ths,
                                                                    stream, tune);
  if constexpr (LAY == 0) {
    if (stage == 3)
      return launch_dyn_variant<LOG2N, KIND, false, false, true, LAY>(p, counters, tail_64ths,
                                                                      stream, tune);
  }
  if (stage == 0)
    return launch_dyn_variant<LOG2N, KIND, false, false, false, LAY>(p, counters, tail_64ths,
                                                                     stream, tune);
  return cudaErrorInvalidConfiguration;
}

// Layouts with a dynamic tail: 8x8 blocks in layouts 0 and 3, 16x16 blocks
// in layouts 0, 4 and 5 (instantiated in dyn_6_fwd.cu ... dyn_8_inv.cu).
template <int LOG2N, int KIND>
cudaError_t launch_dyn_n(const BatchParams& p, void* counters, int tail_64ths,
                         cudaStream_t stream, const BatchTune& tune) {
  if constexpr (LOG2N == 6) {
    if (tune.layout == 3)
      return launch_dyn_layout<6, KIND, 3>(p, counters, tail_64ths, stream, tune);
    if (tune.layout == 0)
      return launch_dyn_layout<6, KIND, 0>(p, counters, tail_64ths, stream, tune);
  } else if constexpr (LOG2N == 8) {
    if (tune.layout == 5)
      return launch_dyn_layout<8, KIND, 5>(p, counters, tail_64ths, stream, tune);
    if (tune.layout == 4)
      return launch_dyn_layout<8, KIND, 4>(p, counters, tail_64ths, stream, tune);
    if (tune.layout == 0)
      return launch_dyn_layout<8, KIND, 0>(p, counters, tail_64ths, stream, tune);
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace hygt
