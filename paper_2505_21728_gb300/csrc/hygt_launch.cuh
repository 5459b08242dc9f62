// hygt_launch.cuh -- launch helpers shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "hygt_device.cuh"

namespace hygt {

struct DeviceInfo {
  int sms = 0;
  int max_smem_optin = 0;
};

// Cached per device (host side).
DeviceInfo device_info(int device);

// Elements per lane chosen for each block size (LOG2E).
constexpr int lane_log2e(int log2n) { return log2n < 3 ? log2n : 3; }

// Launch the persistent kernel for one block size and kind.  Stages the
// tables in shared memory when tab + perm + scratch fit; sizes the grid to
// (resident CTAs per SM) x SMs, capped by the work.
template <int LOG2N, int KIND>
cudaError_t launch_sized(Params p, cudaStream_t stream) {
  constexpr int LOG2E = lane_log2e(LOG2N);
  constexpr int E = 1 << LOG2E;
  constexpr int N = 1 << LOG2N;
  constexpr int G = 32 / (N / E);
  auto kern = hygt_kernel<LOG2N, LOG2E, KIND>;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  const size_t scratch = (size_t)(kThreads / 32) * 32 * E * 4;
  size_t smem = scratch;
  const size_t staged = (size_t)p.tab_bytes + (size_t)p.perm_bytes + scratch;
  p.stage = (p.tab_bytes > 0 && staged <= (size_t)info.max_smem_optin) ? 1 : 0;
  if (p.stage) smem = staged;
  static std::atomic<int> attr_set{0};
  if ((int)smem > attr_set.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set.store((int)smem);
  }
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) occ = 1;
  const long long per_cta = (long long)(kThreads / 32) * G;
  long long need = (p.nblocks + per_cta - 1) / per_cta;
  long long grid = (long long)occ * info.sms;
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_kind(int log2n, const Params& p, cudaStream_t stream) {
  switch (log2n) {
    case 1: return launch_sized<1, KIND>(p, stream);
    case 2: return launch_sized<2, KIND>(p, stream);
    case 3: return launch_sized<3, KIND>(p, stream);
    case 4: return launch_sized<4, KIND>(p, stream);
    case 5: return launch_sized<5, KIND>(p, stream);
    case 6: return launch_sized<6, KIND>(p, stream);
    case 7: return launch_sized<7, KIND>(p, stream);
    case 8: return launch_sized<8, KIND>(p, stream);
    default: return cudaErrorInvalidValue;
  }
}

// Defined in one translation unit each (parallel compilation).
cudaError_t launch_int_fwd(int log2n, const Params& p, cudaStream_t stream);
cudaError_t launch_int_inv(int log2n, const Params& p, cudaStream_t stream);
cudaError_t launch_f32_fwd(int log2n, const Params& p, cudaStream_t stream);
cudaError_t launch_f32_inv(int log2n, const Params& p, cudaStream_t stream);

}  // namespace hygt
