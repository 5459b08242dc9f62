// hygt_grad.cuh -- backward pass of the FP32 HyGT (sm_103a).
//
// For a rotation of the pair (a, b) by theta,
//     y_m = c a + s b,   y_n = -s a + c b        (c = cos theta, s = sin theta)
// the derivatives are dy_m/dtheta = y_n and dy_n/dtheta = -y_m, so with the
// output gradients (g_m, g_n):
//     dL/dtheta += g_m y_n - g_n y_m
//     (a, b)     = (c y_m - s y_n, s y_m + c y_n)       (inverse rotation)
//     (g_a, g_b) = (c g_m - s g_n, s g_m + c g_n)       (transpose)
// The kernel starts from the forward output y and its gradient, walks the
// passes in reverse (permutation slots undone by scatter), recomputing each
// pass's input instead of storing it, and ends with dL/dx.
//
// Mapping as in hygt_device.cuh: a block is held by L = N / 8 sub-warp lanes
// with 8 values each; cross-lane passes exchange y and g with
// __shfl_xor_sync.  dL/dtheta: every pair of a pass is owned by exactly one
// lane of the block (the lane that holds its m side), which adds the term to
// a private shared-memory accumulator of its (warp, block slot).  The
// accumulation order is fixed, so the result is deterministic.  At the end
// each CTA sums its accumulators in FP64 into one partial vector; a second
// kernel sums the partials of all CTAs in a fixed order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hygt_device.cuh"

namespace hygt {

constexpr int kGradThreadsMax = 256;

struct GradParams {
  const float* y;       // [B][N] forward output
  const float* gy;      // [B][N] dL/dy
  float* gx;            // [B][N] dL/dx
  const uint16_t* set;  // nullable
  long long nblocks;
  const float2* tab;    // (cos, sin) per pair, [S][R][k][N/2]
  const uint8_t* perm;  // [S][R][N] or nullptr
  unsigned perm_mask;
  int rounds;
  int num_sets;
  int angles;           // S * R * k * N/2
  double* partials;     // [gridDim.x][angles]
  int* status;
};

template <int LOG2N>
struct GradMap {
  static constexpr int N = 1 << LOG2N;
  static constexpr int LOG2E = LOG2N < 3 ? LOG2N : 3;
  static constexpr int E = 1 << LOG2E;
  static constexpr int L = N / E;
  static constexpr int G = 32 / L;
};

// Shared memory: accumulators [warps][G][angles + pad] floats, then the
// permutation scratch [warps][32 * E] (y) and [warps][32 * E] (g).  The
// accumulator stride is padded to an odd multiple of the 4-word lane step,
// so the G block slots of a warp, updating the same angle index, use
// different banks.
__host__ __device__ inline int grad_acc_stride(int angles) { return ((angles + 3) & ~3) + 4 + 1; }

template <int LOG2N>
__host__ __device__ inline size_t grad_smem_bytes(int warps, int angles) {
  return (size_t)warps * GradMap<LOG2N>::G * grad_acc_stride(angles) * 4 +
         (size_t)warps * 2 * 32 * GradMap<LOG2N>::E * 4;
}

template <int LOG2N, int P>
__device__ __forceinline__ void grad_pass(float (&v)[GradMap<LOG2N>::E],
                                          float (&g)[GradMap<LOG2N>::E], const float2* row,
                                          float* acc, int lane, bool counts) {
  using M = GradMap<LOG2N>;
  constexpr int E = M::E;
  if constexpr (P < M::LOG2E) {
#pragma unroll
    for (int jl = 0; jl < E / 2; ++jl) {
      const int im = ((jl >> P) << (P + 1)) | (jl & ((1 << P) - 1));
      const int in = im | (1 << P);
      const int j = lane * (E / 2) + jl;
      const float2 cs = row[j];
      const float ym = v[im], yn = v[in], gm = g[im], gn = g[in];
      if (counts) acc[j] += gm * yn - gn * ym;
      v[im] = cs.x * ym - cs.y * yn;
      v[in] = cs.y * ym + cs.x * yn;
      g[im] = cs.x * gm - cs.y * gn;
      g[in] = cs.y * gm + cs.x * gn;
    }
  } else {
    constexpr int Q = P - M::LOG2E;
    constexpr int D = 1 << Q;
    const bool upper = (lane >> Q) & 1;
    const int jbase = ((lane >> (Q + 1)) << P) + ((lane & (D - 1)) << M::LOG2E);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const float2 cs = row[jbase + i];
      const float yo = v[i], go = g[i];
      const float yp = __shfl_xor_sync(kFullMask, yo, D);
      const float gp = __shfl_xor_sync(kFullMask, go, D);
      if (counts && !upper) acc[jbase + i] += go * yp - gp * yo;  // m side owns the pair
      const float sp = upper ? cs.y : -cs.y;
      v[i] = cs.x * yo + sp * yp;
      g[i] = cs.x * go + sp * gp;
    }
  }
}

template <int LOG2N, int K>
__device__ __forceinline__ void grad_round(float (&v)[GradMap<LOG2N>::E],
                                           float (&g)[GradMap<LOG2N>::E], const float2* rtab,
                                           float* racc, int lane, bool counts) {
  constexpr int N = 1 << LOG2N;
  if constexpr (K < LOG2N) {
    constexpr int P = LOG2N - 1 - K;  // passes in reverse order
    grad_pass<LOG2N, P>(v, g, rtab + P * (N / 2), racc + P * (N / 2), lane, counts);
    grad_round<LOG2N, K + 1>(v, g, rtab, racc, lane, counts);
  }
}

template <int LOG2N>
__global__ void __launch_bounds__(kGradThreadsMax) hygt_grad_kernel(GradParams p) {
  using M = GradMap<LOG2N>;
  constexpr int N = M::N;
  constexpr int E = M::E;
  constexpr int L = M::L;
  constexpr int G = M::G;
  extern __shared__ __align__(16) float gsm[];

  const int warps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane32 = threadIdx.x & 31;
  const int sub = lane32 / L;
  const int lane = lane32 % L;
  const int stride = grad_acc_stride(p.angles);
  float* acc_all = gsm;
  float* acc = acc_all + (size_t)(warp * G + sub) * stride;
  float* ybuf = gsm + (size_t)warps * G * stride + (size_t)warp * 2 * 32 * E + sub * N;
  float* gbuf = ybuf + 32 * E;
  for (int i = threadIdx.x; i < warps * G * stride; i += blockDim.x) acc_all[i] = 0.f;
  __syncthreads();

  const long long warps_total = (long long)gridDim.x * warps;
  const long long gw = (long long)blockIdx.x * warps + warp;
  const int R = p.rounds;
  const int rowlen = LOG2N * (N / 2);  // angles per round

  for (long long base = gw * G; base < p.nblocks; base += warps_total * G) {
    const long long b = base + sub;
    const bool valid = b < p.nblocks;
    unsigned set = 0;
    if (valid && p.set) set = __ldg(p.set + b);
    const bool skip = set == 0xFFFFu;
    const bool bad = !skip && set >= (unsigned)p.num_sets;
    const unsigned cset = (skip || bad) ? 0u : set;
    float v[E], g[E];
    if (valid) {
      load_f32<E>(p.y + b * N + lane * E, v);
      load_f32<E>(p.gy + b * N + lane * E, g);
    } else {
#pragma unroll
      for (int i = 0; i < E; ++i) v[i] = g[i] = 0.f;
    }
    // skip, bad and tail blocks run the passes like set 0 (the warp stays
    // converged for the shuffles) but add nothing to dL/dtheta
    const bool counts = valid && !skip && !bad;
    float keep[E];
#pragma unroll
    for (int i = 0; i < E; ++i) keep[i] = g[i];
    for (int r = R - 1; r >= 0; --r) {
      if (p.perm && ((p.perm_mask >> r) & 1u)) {
        const uint8_t* prow = p.perm + ((size_t)cset * R + r) * N;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int d = prow[lane * E + i];
          ybuf[d] = v[i];
          gbuf[d] = g[i];
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < E; ++i) {
          v[i] = ybuf[lane * E + i];
          g[i] = gbuf[lane * E + i];
        }
        __syncwarp();
      }
      const size_t off = ((size_t)cset * R + r) * rowlen;
      grad_round<LOG2N, 0>(v, g, p.tab + off, acc + off, lane, counts);
    }
    if (skip) {
#pragma unroll
      for (int i = 0; i < E; ++i) g[i] = keep[i];
    } else if (bad) {
#pragma unroll
      for (int i = 0; i < E; ++i) g[i] = 0.f;
      if (valid && lane == 0 && p.status) atomicCAS(p.status, 0, 4);
    }
    if (valid) store_f32<E>(p.gx + b * N + lane * E, g);
  }
  __syncthreads();
  // CTA partial: sum of all (warp, block slot) accumulators, in FP64, fixed order
  for (int a = threadIdx.x; a < p.angles; a += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < warps * G; ++k) s += (double)acc_all[(size_t)k * stride + a];
    p.partials[(size_t)blockIdx.x * p.angles + a] = s;
  }
}

// dL/dtheta[a] = sum over CTAs of partials[cta][a], fixed order, FP64.
__global__ void hygt_grad_reduce(const double* __restrict__ partials, int nparts, int angles,
                                 double* __restrict__ gtheta);

// theta -> (cos, sin) table on the device.
__global__ void hygt_theta_to_table(const float* __restrict__ theta, float2* __restrict__ tab,
                                    long long n);

struct GradLaunch {
  int log2n;
  GradParams p;
  int threads;
  int grid;
  size_t smem;
};

cudaError_t launch_grad(GradLaunch& gl, double* gtheta, cudaStream_t stream);
// Grid, threads and shared memory of the backward launch (0 threads: too
// many angles for the shared-memory accumulators).
void grad_config(int log2n, int angles, long long nblocks, int* threads, int* grid, size_t* smem);

}  // namespace hygt
