// f32u.cu -- launchers of the one-set FP32 kernels (see hygt_f32u.cuh).
#include <atomic>

#include "hygt_f32u.cuh"
#include "hygt_launch.cuh"

namespace hygt {

template <int LOG2N, bool INV>
static cudaError_t launch_sized(const F32uParams& p, cudaStream_t stream) {
  using M = GradMap<LOG2N>;
  auto kern = hygt_f32u_kernel<LOG2N, INV>;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  const size_t smem = f32u_smem_bytes<LOG2N>(kF32uThreads, p.rounds);
  if (smem > (size_t)info.max_smem_optin) return cudaErrorInvalidConfiguration;
  static std::atomic<int> attr_set{0};
  if ((int)smem > attr_set.load()) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    attr_set.store((int)smem);
  }
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kF32uThreads, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) occ = 1;
  const long long per_cta = (long long)(kF32uThreads / 32) * M::G;
  long long grid = (long long)occ * info.sms;
  const long long need = (p.nblocks + per_cta - 1) / per_cta;
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kF32uThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_f32u(int log2n, int kind, const F32uParams& p, cudaStream_t stream) {
  const bool inv = kind == 1;
  switch (log2n) {
#define HYGT_F32U_CASE(n) \
  case n: return inv ? launch_sized<n, true>(p, stream) : launch_sized<n, false>(p, stream);
    HYGT_F32U_CASE(1)
    HYGT_F32U_CASE(2)
    HYGT_F32U_CASE(3)
    HYGT_F32U_CASE(4)
    HYGT_F32U_CASE(5)
    HYGT_F32U_CASE(6)
    HYGT_F32U_CASE(7)
    HYGT_F32U_CASE(8)
#undef HYGT_F32U_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hygt
