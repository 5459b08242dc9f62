// hygt_fit.cuh -- the coding-gain objective of Sec. V on the GPU, and the
// optimiser step of the angle fit (sm_103a).
//
// For a batch y[B][N] of transform outputs (one class), the variance
// vector of Sec. V is estimated by the per-coefficient second moments
//     v_i = (1/B) sum_b y_{b,i}^2      (= diag(T Phi T^T) with Phi the
//                                        batch's correlation matrix)
// and the high-rate rate model R(D) = 1/2 log2(eps^2 sigma^2 / D) gives, up
// to terms that do not depend on the transform, the average rate
//     J = 1/(2N) sum_i log2 v_i.
// Its gradient with respect to the outputs is diagonal:
//     dJ/dy_{b,i} = w_i y_{b,i},   w_i = 1 / (N ln2 B v_i),
// so the backward kernel takes w and forms dL/dy in registers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hygt {

constexpr int kMomentThreads = 256;
constexpr int kMomentUnroll = 8;   // 16-byte loads in flight per thread

// Per-CTA second moments: partials[cta][i] = sum of y_{b,i}^2 over the
// float4s that CTA reads (FP32 within runs of 8 values, FP64 across them;
// fixed order).  n4 = B N / 4 float4s; N divides 4 * kMomentThreads.
__global__ void hygt_moments_kernel(const float4* __restrict__ y, long long n4, int n,
                                    double* __restrict__ partials);

// v, J and w from the partials of `nparts` CTAs (one CTA of n threads).
__global__ void hygt_coding_gain_finish(const double* __restrict__ partials, int nparts, int n,
                                        long long nblocks, double* __restrict__ v,
                                        float* __restrict__ w, double* __restrict__ J);

// One Adam step on FP32 parameters from an FP64 gradient.
__global__ void hygt_adam_kernel(float* __restrict__ theta, const double* __restrict__ g,
                                 float* __restrict__ m, float* __restrict__ v, long long n,
                                 float lr, float beta1, float beta2, float eps, float corr1,
                                 float corr2);

int moments_grid(long long n4);

}  // namespace hygt
