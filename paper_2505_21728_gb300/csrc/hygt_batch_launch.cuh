// hygt_batch_launch.cuh -- launch templates of the set-bucketed kernels,
// included by the per-direction translation units (batch_fwd.cu,
// batch_inv.cu) so that their many instantiations compile in parallel.
#pragma once

#include <atomic>

#include "hygt_batch.cuh"
#include "hygt_launch.cuh"

namespace hygt {

template <int LOG2N, int KIND, bool STAGED, bool PRIM = false, bool PF = false,
          bool BULK = false, int LAY = 0>
inline cudaError_t launch_variant(BatchParams p, cudaStream_t stream, const BatchTune& tune) {
  auto kern = hygt_batch_kernel<LOG2N, KIND, STAGED, PRIM, PF, BULK, LAY>;
  if constexpr (LAY == 1) {  // the layout's own set tables
    if (!p.ktab1) return cudaErrorInvalidConfiguration;
    p.ktab = p.ktab1;
    p.set_words = p.set_words1;
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
  // with several CTAs per SM each gets its share of the shared memory
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
  kern<<<(unsigned)grid, threads, smem, stream>>>(p);
  return cudaGetLastError();
}

// The staging choice of a launch: the tuned one, else the measured default;
// bulk copies need a 16-byte aligned input (whole blocks are copied), else
// no stage.
template <int LOG2N, int KIND>
inline int batch_stage_of(const BatchParams& p, const BatchTune& tune) {
  const int stage = tune.stage < 0 ? (batch_staged(LOG2N, KIND) ? 1 : 0) : tune.stage;
  if (stage == 3 && (reinterpret_cast<uintptr_t>(p.in) & 15) != 0) return 0;
  return stage;
}

// Staging exists as a tuning choice for N >= 16; smaller blocks keep the
// measured default (no stage).
template <int LOG2N, int KIND>
inline cudaError_t launch_batch_sized(const BatchParams& p, cudaStream_t stream,
                                      const BatchTune& tune) {
  constexpr bool kDefault = batch_staged(LOG2N, KIND);
  if constexpr (batch_layout_ok(LOG2N, 1)) {
    if (tune.layout == 1) {
      const int stage = tune.stage < 0 ? 0 : tune.stage;
      if (stage == 2) return launch_variant<LOG2N, KIND, false, false, true, false, 1>(p, stream, tune);
      if (stage == 1) return launch_variant<LOG2N, KIND, true, false, false, false, 1>(p, stream, tune);
      if (stage == 0) return launch_variant<LOG2N, KIND, false, false, false, false, 1>(p, stream, tune);
      return cudaErrorInvalidConfiguration;
    }
  }
  if (tune.layout != 0) return cudaErrorInvalidConfiguration;
  if constexpr (LOG2N >= 4) {
    const int stage = batch_stage_of<LOG2N, KIND>(p, tune);
    if (stage == 3)
      return launch_variant<LOG2N, KIND, false, false, false, true>(p, stream, tune);
    if (stage == 2) return launch_variant<LOG2N, KIND, false, false, true>(p, stream, tune);
    return stage == 1 ? launch_variant<LOG2N, KIND, true>(p, stream, tune)
                      : launch_variant<LOG2N, KIND, false>(p, stream, tune);
  } else {
    return launch_variant<LOG2N, KIND, kDefault>(p, stream, tune);
  }
}

template <int KIND>
inline cudaError_t launch_batch(int log2n, const BatchParams& p, cudaStream_t stream,
                                const BatchTune& tune) {
  switch (log2n) {
    case 1: return launch_batch_sized<1, KIND>(p, stream, tune);
    case 2: return launch_batch_sized<2, KIND>(p, stream, tune);
    case 3: return launch_batch_sized<3, KIND>(p, stream, tune);
    case 4: return launch_batch_sized<4, KIND>(p, stream, tune);
    case 5: return launch_batch_sized<5, KIND>(p, stream, tune);
    case 6: return launch_batch_sized<6, KIND>(p, stream, tune);
    case 7: return launch_batch_sized<7, KIND>(p, stream, tune);
    case 8: return launch_batch_sized<8, KIND>(p, stream, tune);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOG2N, int KIND>
inline cudaError_t launch_primary_sized(const BatchParams& p, cudaStream_t stream,
                                        const BatchTune& tune) {
  const int stage = batch_stage_of<LOG2N, KIND>(p, tune);
  if (stage == 3) return launch_variant<LOG2N, KIND, false, true, false, true>(p, stream, tune);
  if (stage == 2) return launch_variant<LOG2N, KIND, false, true, true>(p, stream, tune);
  return stage == 1 ? launch_variant<LOG2N, KIND, true, true>(p, stream, tune)
                    : launch_variant<LOG2N, KIND, false, true>(p, stream, tune);
}

}  // namespace hygt
