// fit_f32.cu -- kernels of the coding-gain objective and the Adam step (see
// hygt_fit.cuh).
#include <math.h>

#include "hygt_fit.cuh"
#include "hygt_launch.cuh"

namespace hygt {

int moments_grid(long long n4) {
  int dev = 0;
  cudaGetDevice(&dev);
  const DeviceInfo info = device_info(dev);
  long long g = (long long)info.sms * 8;
  const long long need = (n4 + (long long)kMomentThreads * kMomentUnroll - 1) /
                         ((long long)kMomentThreads * kMomentUnroll);
  if (need < g) g = need;
  return (int)(g < 1 ? 1 : g);
}

__global__ void __launch_bounds__(kMomentThreads) hygt_moments_kernel(
    const float4* __restrict__ y, long long n4, int n, double* __restrict__ partials) {
  __shared__ double red[kMomentThreads][4];
  // every float4 this thread reads covers coefficients q .. q + 3 with
  // q = (4 * tid) mod n, because the stride (4 * threads of the grid) is a
  // multiple of n; kMomentUnroll independent loads are in flight per thread
  const long long stride = (long long)gridDim.x * blockDim.x;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; f + (kMomentUnroll - 1) * stride < n4; f += kMomentUnroll * stride) {
    float4 a[kMomentUnroll];
#pragma unroll
    for (int u = 0; u < kMomentUnroll; ++u) a[u] = __ldcs(y + f + u * stride);
    float run[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < kMomentUnroll; ++u) {
      run[0] = fmaf(a[u].x, a[u].x, run[0]);
      run[1] = fmaf(a[u].y, a[u].y, run[1]);
      run[2] = fmaf(a[u].z, a[u].z, run[2]);
      run[3] = fmaf(a[u].w, a[u].w, run[3]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += (double)run[j];
  }
  for (; f < n4; f += stride) {  // the tail, one float4 at a time
    const float4 a = __ldcs(y + f);
    acc[0] += (double)(a.x * a.x);
    acc[1] += (double)(a.y * a.y);
    acc[2] += (double)(a.z * a.z);
    acc[3] += (double)(a.w * a.w);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) red[threadIdx.x][j] = acc[j];
  __syncthreads();
  // coefficient i is held by the threads t with (4 t) mod n = i - i mod 4
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double sm = 0.0;
    for (int t = i / 4; t < (int)blockDim.x; t += n / 4) sm += red[t][i & 3];
    partials[(size_t)blockIdx.x * n + i] = sm;
  }
}

__global__ void hygt_coding_gain_finish(const double* __restrict__ partials, int nparts, int n,
                                        long long nblocks, double* __restrict__ v,
                                        float* __restrict__ w, double* __restrict__ J) {
  __shared__ double lg[256];
  const int i = threadIdx.x;
  if (i < n) {
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += partials[(size_t)c * n + i];
    const double vi = s / (double)nblocks;
    v[i] = vi;
    // dJ/dy_{b,i} = (1 / (2 N ln 2)) (1 / v_i) (2 y_{b,i} / B)
    w[i] = vi > 0.0 ? (float)(1.0 / ((double)n * M_LN2 * (double)nblocks * vi)) : 0.f;
    lg[i] = vi > 0.0 ? log2(vi) : -INFINITY;
  }
  __syncthreads();
  if (i == 0) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += lg[k];
    *J = s / (2.0 * n);
  }
}

__global__ void hygt_adam_kernel(float* __restrict__ theta, const double* __restrict__ g,
                                 float* __restrict__ m, float* __restrict__ v, long long n,
                                 float lr, float beta1, float beta2, float eps, float corr1,
                                 float corr2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = (float)g[i];
  const float mi = beta1 * m[i] + (1.f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / corr1) / (sqrtf(vi / corr2) + eps);
}

}  // namespace hygt
