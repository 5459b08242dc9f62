// hygt_batch_launch.cuh -- launch templates of the set-bucketed kernels,
// instantiated per block size and direction by the batch_n*.cu translation
// units, so that their many kernels compile in parallel.
#pragma once

#include <atomic>

#include "hygt_batch.cuh"
#include "hygt_launch.cuh"

namespace hygt {

template <int LOG2N, int KIND, bool STAGED, bool PRIM = false, bool PF = false,
          bool BULK = false, int LAY = 0>
inline cudaError_t launch_variant(BatchParams p, cudaStream_t stream, const BatchTune& tune) {
  auto kern = hygt_batch_kernel<LOG2N, KIND, STAGED, PRIM, PF, BULK, LAY>;
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

// A register layout other than the default: stages 0 (default), 1 and 2.
template <int LOG2N, int KIND, int LAY>
inline cudaError_t launch_layout(const BatchParams& p, cudaStream_t stream, const BatchTune& tune) {
  const int stage = tune.stage < 0 ? 0 : tune.stage;
  if (stage == 2) return launch_variant<LOG2N, KIND, false, false, true, false, LAY>(p, stream, tune);
  if (stage == 1) return launch_variant<LOG2N, KIND, true, false, false, false, LAY>(p, stream, tune);
  if (stage == 0) return launch_variant<LOG2N, KIND, false, false, false, false, LAY>(p, stream, tune);
  return cudaErrorInvalidConfiguration;
}

// Staging exists as a tuning choice for N >= 16; smaller blocks keep the
// measured default (no stage).
template <int LOG2N, int KIND>
inline cudaError_t launch_batch_sized(const BatchParams& p, cudaStream_t stream,
                                      const BatchTune& tune) {
  constexpr bool kDefault = batch_staged(LOG2N, KIND);
  if constexpr (batch_layout_ok(LOG2N, 1)) {
    if (tune.layout == 1) return launch_layout<LOG2N, KIND, 1>(p, stream, tune);
  }
  if constexpr (batch_layout_ok(LOG2N, 2)) {
    if (tune.layout == 2) return launch_layout<LOG2N, KIND, 2>(p, stream, tune);
  }
  if constexpr (batch_layout_ok(LOG2N, 3)) {
    if (tune.layout == 3) return launch_layout<LOG2N, KIND, 3>(p, stream, tune);
  }
  if constexpr (batch_layout_ok(LOG2N, 4)) {
    if (tune.layout == 4) return launch_layout<LOG2N, KIND, 4>(p, stream, tune);
  }
  if constexpr (batch_layout_ok(LOG2N, 5)) {
    if (tune.layout == 5) return launch_layout<LOG2N, KIND, 5>(p, stream, tune);
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

template <int LOG2N, int KIND>
cudaError_t launch_batch_n(const BatchParams& p, cudaStream_t stream, const BatchTune& tune) {
  return launch_batch_sized<LOG2N, KIND>(p, stream, tune);
}

template <int LOG2N, int KIND>
cudaError_t launch_primary_n(const BatchParams& p, cudaStream_t stream, const BatchTune& tune) {
  const int stage = batch_stage_of<LOG2N, KIND>(p, tune);
  if (stage == 3) return launch_variant<LOG2N, KIND, false, true, false, true>(p, stream, tune);
  if (stage == 2) return launch_variant<LOG2N, KIND, false, true, true>(p, stream, tune);
  return stage == 1 ? launch_variant<LOG2N, KIND, true, true>(p, stream, tune)
                    : launch_variant<LOG2N, KIND, false, true>(p, stream, tune);
}

}  // namespace hygt
