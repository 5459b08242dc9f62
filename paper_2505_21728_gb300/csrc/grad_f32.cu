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
static void config_sized(int num_sets, int rounds, long long nblocks, int* threads, int* grid,
                         size_t* smem, int* cache_tables, int* group) {
  using M = GradMap<LOG2N>;
  int dev = 0;
  cudaGetDevice(&dev);
  const DeviceInfo info = device_info(dev);
  const int angles = num_sets * rounds * LOG2N * (M::N / 2);
  const size_t per_warp = grad_warp_bytes<LOG2N>(angles);
  const size_t tables = grad_table_bytes<LOG2N>(num_sets, rounds);
  const size_t budget = (size_t)info.max_smem_optin;
  *group = M::G;
  // one CTA per SM: as many warps as fit next to the tables (up to 12)
  *cache_tables = tables + per_warp <= budget && tables <= budget / 4 ? 1 : 0;
  const size_t avail = budget - (*cache_tables ? tables : 0);
  int warps = (int)(avail / per_warp);
  if (warps > kGradThreads / 32) warps = kGradThreads / 32;
  if (warps < 1) {
    *threads = 0;
    *grid = 0;
    *smem = 0;
    return;
  }
  *threads = warps * 32;
  *smem = (*cache_tables ? tables : 0) + (size_t)warps * per_warp;
  const long long tasks = (nblocks + M::G - 1) / M::G + num_sets + 2;
  long long g = info.sms;
  if (tasks < g * warps) g = (tasks + warps - 1) / warps;
  if (g < 1) g = 1;
  *grid = (int)g;
}

void grad_config(int log2n, int num_sets, int rounds, long long nblocks, int* threads, int* grid,
                 size_t* smem, int* cache_tables, int* group) {
  switch (log2n) {
#define HYGT_GRAD_CASE(n)                                                                  \
  case n:                                                                                  \
    config_sized<n>(num_sets, rounds, nblocks, threads, grid, smem, cache_tables, group);  \
    break;
    HYGT_GRAD_CASE(1)
    HYGT_GRAD_CASE(2)
    HYGT_GRAD_CASE(3)
    HYGT_GRAD_CASE(4)
    HYGT_GRAD_CASE(5)
    HYGT_GRAD_CASE(6)
    HYGT_GRAD_CASE(7)
    HYGT_GRAD_CASE(8)
#undef HYGT_GRAD_CASE
    default: *threads = 0; *grid = 0; *smem = 0; *cache_tables = 0; *group = 0;
  }
}

template <int LOG2N>
static cudaError_t launch_sized(GradLaunch& gl, cudaStream_t stream) {
  auto kern = gl.p.cache_tables ? hygt_grad_kernel<LOG2N, true> : hygt_grad_kernel<LOG2N, false>;
  static std::atomic<int> attr_set[2] = {{0}, {0}};
  std::atomic<int>& as = attr_set[gl.p.cache_tables ? 1 : 0];
  if ((int)gl.smem > as.load()) {
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)gl.smem);
    if (err != cudaSuccess) return err;
    as.store((int)gl.smem);
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
