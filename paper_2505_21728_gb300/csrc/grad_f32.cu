// grad_f32.cu -- launchers of the FP32 HyGT backward (see hygt_grad.cuh).
#include "hygt_grad.cuh"
#include "hygt_launch.cuh"

namespace hygt {

__global__ void hygt_grad_reduce(const double* __restrict__ partials, int nparts, int angles,
                                 double* __restrict__ gtheta) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= angles) return;
  double s = 0.0;
  for (int c = 0; c < nparts; ++c) s += partials[(size_t)c * angles + a];
  gtheta[a] = s;
}

__global__ void hygt_theta_to_table(const float* __restrict__ theta, float2* __restrict__ tab,
                                    long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s, c;
  sincosf(theta[i], &s, &c);
  tab[i] = make_float2(c, s);
}

template <int LOG2N>
static void config_sized(int angles, long long nblocks, int* threads, int* grid, size_t* smem) {
  int dev = 0;
  cudaGetDevice(&dev);
  const DeviceInfo info = device_info(dev);
  // up to two CTAs per SM; each warp needs its accumulators and scratch
  const size_t per_warp = grad_smem_bytes<LOG2N>(1, angles);
  const size_t budget2 = (size_t)info.max_smem_optin / 2;
  int warps = (int)(budget2 / per_warp);
  if (warps > kGradThreadsMax / 32) warps = kGradThreadsMax / 32;
  if (warps < 1) warps = per_warp <= (size_t)info.max_smem_optin ? 1 : 0;
  *threads = warps * 32;
  *smem = grad_smem_bytes<LOG2N>(warps, angles);
  if (warps == 0) {
    *grid = 0;
    return;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hygt_grad_kernel<LOG2N>, *threads, *smem);
  if (occ < 1) occ = 1;
  const long long per_cta = (long long)warps * GradMap<LOG2N>::G;
  long long need = (nblocks + per_cta - 1) / per_cta;
  long long g = (long long)occ * info.sms;
  if (need < g) g = need;
  if (g < 1) g = 1;
  *grid = (int)g;
}

void grad_config(int log2n, int angles, long long nblocks, int* threads, int* grid, size_t* smem) {
  switch (log2n) {
    case 1: config_sized<1>(angles, nblocks, threads, grid, smem); break;
    case 2: config_sized<2>(angles, nblocks, threads, grid, smem); break;
    case 3: config_sized<3>(angles, nblocks, threads, grid, smem); break;
    case 4: config_sized<4>(angles, nblocks, threads, grid, smem); break;
    case 5: config_sized<5>(angles, nblocks, threads, grid, smem); break;
    case 6: config_sized<6>(angles, nblocks, threads, grid, smem); break;
    case 7: config_sized<7>(angles, nblocks, threads, grid, smem); break;
    case 8: config_sized<8>(angles, nblocks, threads, grid, smem); break;
    default: *threads = 0; *grid = 0; *smem = 0;
  }
}

template <int LOG2N>
static cudaError_t launch_sized(GradLaunch& gl, cudaStream_t stream) {
  auto kern = hygt_grad_kernel<LOG2N>;
  static std::atomic<int> attr_set{0};
  if ((int)gl.smem > attr_set.load()) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)gl.smem);
    if (err != cudaSuccess) return err;
    attr_set.store((int)gl.smem);
  }
  kern<<<gl.grid, gl.threads, gl.smem, stream>>>(gl.p);
  return cudaGetLastError();
}

cudaError_t launch_grad(GradLaunch& gl, double* gtheta, cudaStream_t stream) {
  cudaError_t err = cudaSuccess;
  switch (gl.log2n) {
    case 1: err = launch_sized<1>(gl, stream); break;
    case 2: err = launch_sized<2>(gl, stream); break;
    case 3: err = launch_sized<3>(gl, stream); break;
    case 4: err = launch_sized<4>(gl, stream); break;
    case 5: err = launch_sized<5>(gl, stream); break;
    case 6: err = launch_sized<6>(gl, stream); break;
    case 7: err = launch_sized<7>(gl, stream); break;
    case 8: err = launch_sized<8>(gl, stream); break;
    default: return cudaErrorInvalidValue;
  }
  if (err != cudaSuccess) return err;
  const int a = gl.p.angles;
  hygt_grad_reduce<<<(a + 255) / 256, 256, 0, stream>>>(gl.p.partials, gl.grid, a, gtheta);
  return cudaGetLastError();
}

}  // namespace hygt
