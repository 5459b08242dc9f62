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
// Mapping.  A block is held by L = N / E lanes with E = 8 values each (a lane
// group); every lane group holds K = 4 blocks of the same set, so each
// (cos, sin) pair read from shared memory serves K rotations and the K
// contributions to a dL/dtheta entry are summed in a register before they
// reach the accumulators.  Cross-lane passes exchange y and g with
// __shfl_xor_sync.  A warp task is G = (32 / L) K blocks of one set: the
// blocks in order when no set indices are given, else the slots of the
// set-bucketed schedule (skip and bad-set buckets are whole tasks).
//
// dL/dtheta: every pair of a pass is owned by exactly one lane of the group
// (the lane that holds its m side), which adds the K-block sum to a private
// shared-memory accumulator row of its (warp, lane group).  The accumulation
// order within a row is fixed by the task order.  At the end each CTA sums
// its rows in FP64 into one partial vector; a second kernel sums the
// partials of all CTAs in a fixed order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hygt_batch.cuh"
#include "hygt_device.cuh"

namespace hygt {

constexpr int kGradThreads = 384;

struct GradParams {
  const float* y;       // [B][N] forward output
  const float* gy;      // [B][N] dL/dy, or nullptr: dL/dy = w * y (w below)
  const float* w;       // [N] per-coefficient weights when gy is nullptr
  float* gx;            // [B][N] dL/dx, or nullptr: not written
  long long nblocks;
  const float2* tab;    // (cos, sin) per pair, [S][R][k][N/2]
  const uint8_t* perm;  // [S][R][N] or nullptr
  unsigned perm_mask;
  int rounds;
  int num_sets;
  int angles;           // S * R * k * N/2
  // schedule (set-bucketed, task size G) or nullptr: blocks in order, set 0
  const int* order;
  const int* starts;
  const int* meta;
  long long tmax;
  int cache_tables;     // the tables of all sets are copied to shared memory
  double* partials;     // [gridDim.x][angles]
  int* status;
};

template <int LOG2N>
struct GradMap {
  static constexpr int N = 1 << LOG2N;
  static constexpr int LOG2E = LOG2N < 3 ? LOG2N : 3;
  static constexpr int E = 1 << LOG2E;
  static constexpr int L = N / E;
  static constexpr int GROUPS = 32 / L;
  static constexpr int K = 4;
  static constexpr int G = GROUPS * K;
  static constexpr int RW = N + L;  // words per block region of the permutation buffer
};

// (cos, sin) tables as the lane groups read them.  Register pass: lane l's
// E/2 pairs (jl = 0 .. E/2-1, pair j = l E/2 + jl) contiguous in a segment of
// SEG bytes; cross-lane pass: the E pairs jbase .. jbase + E - 1 that a lane
// pair reads, in a group of GRP bytes.  PADDED (the shared-memory copy)
// pads both by 16 bytes, which makes the distinct segments (groups) that the
// lanes of a group read at once start in distinct banks; unpadded, it is the
// plan's global layout [S][R][k][N/2] float2.
template <int LOG2N, bool PADDED>
struct GradTab {
  using M = GradMap<LOG2N>;
  static constexpr int SEG = 4 * M::E + (PADDED ? 16 : 0);
  static constexpr int GRP = 8 * M::E + (PADDED ? 16 : 0);
  static constexpr int REG_ROW = M::L * SEG;
  static constexpr int LANE_ROW = (M::N / 2 / M::E) * GRP;
  __host__ __device__ static constexpr int pass_off(int p) {
    return p < M::LOG2E ? p * REG_ROW : M::LOG2E * REG_ROW + (p - M::LOG2E) * LANE_ROW;
  }
  static constexpr int ROUND = M::LOG2E * REG_ROW + (LOG2N - M::LOG2E) * LANE_ROW;
  // byte offset of pair j of pass p within a round
  __host__ __device__ static constexpr int pair_off(int p, int j) {
    return p < M::LOG2E ? pass_off(p) + (j / (M::E / 2)) * SEG + (j % (M::E / 2)) * 8
                        : pass_off(p) + (j / M::E) * GRP + (j % M::E) * 8;
  }
};

// Shared memory (bytes): the tables of all sets when cached (padded layout,
// then the permutation bytes, 16-byte padded), then per warp GROUPS
// accumulator rows of grad_acc_stride(angles) floats and the permutation
// buffer (y and g regions of GROUPS blocks).  The row stride is odd, so the
// lane groups of a warp updating the same angle use different banks.
__host__ __device__ inline int grad_acc_stride(int angles) { return ((angles + 3) & ~3) + 4 + 1; }

template <int LOG2N>
__host__ __device__ inline size_t grad_table_bytes(int num_sets, int rounds) {
  using M = GradMap<LOG2N>;
  const size_t tab = (size_t)num_sets * rounds * GradTab<LOG2N, true>::ROUND;
  const size_t perm = ((size_t)num_sets * rounds * M::N + 15) & ~(size_t)15;
  return tab + perm;
}

// Copy the plan's (cos, sin) tables of `rows` rounds (all passes) into the
// padded shared-memory layout, then `pbytes` permutation bytes after them.
template <int LOG2N>
__device__ __forceinline__ void grad_copy_tables(const float2* tab, int rows, const uint8_t* perm,
                                                 int pbytes, unsigned char* dst) {
  using M = GradMap<LOG2N>;
  using T = GradTab<LOG2N, true>;
  constexpr int PAIRS = LOG2N * (M::N / 2);  // pairs per round
  for (int i = threadIdx.x; i < rows * PAIRS; i += blockDim.x) {
    const int r = i / PAIRS, q = i % PAIRS;
    const int pp = q / (M::N / 2), j = q % (M::N / 2);
    *reinterpret_cast<float2*>(dst + (size_t)r * T::ROUND + T::pair_off(pp, j)) = __ldg(tab + i);
  }
  if (perm) {
    uint8_t* pd = dst + (size_t)rows * T::ROUND;
    for (int i = threadIdx.x; i < pbytes; i += blockDim.x) pd[i] = __ldg(perm + i);
  }
}

template <int LOG2N>
__host__ __device__ inline size_t grad_warp_bytes(int angles) {
  using M = GradMap<LOG2N>;
  return (size_t)M::GROUPS * grad_acc_stride(angles) * 4 + (size_t)2 * M::GROUPS * M::RW * 4;
}

// word of element e in a block region: one padding word after each lane's E values
template <int LOG2N>
__device__ __forceinline__ int grad_word(int e) {
  return e + (e >> GradMap<LOG2N>::LOG2E);
}

template <int LOG2N, bool PADDED, int P>
__device__ __forceinline__ void grad_pass(float (&v)[GradMap<LOG2N>::K][GradMap<LOG2N>::E],
                                          float (&g)[GradMap<LOG2N>::K][GradMap<LOG2N>::E],
                                          const unsigned char* rtab, float* acc, int lane) {
  using M = GradMap<LOG2N>;
  using T = GradTab<LOG2N, PADDED>;
  constexpr int E = M::E;
  constexpr int K = M::K;
  if constexpr (P < M::LOG2E) {
    const float2* seg = reinterpret_cast<const float2*>(rtab + T::pass_off(P) + lane * T::SEG);
#pragma unroll
    for (int jl = 0; jl < E / 2; ++jl) {
      const int im = ((jl >> P) << (P + 1)) | (jl & ((1 << P) - 1));
      const int in = im | (1 << P);
      const int j = lane * (E / 2) + jl;
      const float2 cs = seg[jl];
      float sum = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float ym = v[k][im], yn = v[k][in], gm = g[k][im], gn = g[k][in];
        sum = fmaf(gm, yn, sum);
        sum = fmaf(-gn, ym, sum);
        v[k][im] = cs.x * ym - cs.y * yn;
        v[k][in] = cs.y * ym + cs.x * yn;
        g[k][im] = cs.x * gm - cs.y * gn;
        g[k][in] = cs.y * gm + cs.x * gn;
      }
      acc[j] += sum;
    }
  } else {
    constexpr int Q = P - M::LOG2E;
    constexpr int D = 1 << Q;
    const bool upper = (lane >> Q) & 1;
    const int jbase = ((lane >> (Q + 1)) << P) + ((lane & (D - 1)) << M::LOG2E);
    const float2* grp =
        reinterpret_cast<const float2*>(rtab + T::pass_off(P) + (jbase >> M::LOG2E) * T::GRP);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const float2 cs = grp[i];
      const float sp = upper ? cs.y : -cs.y;
      float sum = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float yo = v[k][i], go = g[k][i];
        const float yp = __shfl_xor_sync(kFullMask, yo, D);
        const float gp = __shfl_xor_sync(kFullMask, go, D);
        sum = fmaf(go, yp, sum);
        sum = fmaf(-gp, yo, sum);
        v[k][i] = cs.x * yo + sp * yp;
        g[k][i] = cs.x * go + sp * gp;
      }
      if (!upper) acc[jbase + i] += sum;  // the m side owns the pair
    }
  }
}

template <int LOG2N, bool PADDED, int J>
__device__ __forceinline__ void grad_round(float (&v)[GradMap<LOG2N>::K][GradMap<LOG2N>::E],
                                           float (&g)[GradMap<LOG2N>::K][GradMap<LOG2N>::E],
                                           const unsigned char* rtab, float* racc, int lane) {
  constexpr int N = 1 << LOG2N;
  if constexpr (J < LOG2N) {
    constexpr int P = LOG2N - 1 - J;  // passes in reverse order
    grad_pass<LOG2N, PADDED, P>(v, g, rtab, racc + P * (N / 2), lane);
    grad_round<LOG2N, PADDED, J + 1>(v, g, rtab, racc, lane);
  }
}

template <int LOG2N, bool CACHED>
__global__ void __launch_bounds__(kGradThreads, 1) hygt_grad_kernel(GradParams p) {
  using M = GradMap<LOG2N>;
  constexpr int N = M::N;
  constexpr int E = M::E;
  constexpr int L = M::L;
  constexpr int K = M::K;
  constexpr int GROUPS = M::GROUPS;
  constexpr int G = M::G;
  constexpr int RW = M::RW;
  extern __shared__ __align__(16) unsigned char gsm[];

  const int S = p.num_sets;
  const int R = p.rounds;
  const int rowlen = LOG2N * (N / 2);  // angles per round
  using T = GradTab<LOG2N, CACHED>;
  const unsigned char* tab = reinterpret_cast<const unsigned char*>(p.tab);
  const uint8_t* perm = p.perm;
  size_t off = 0;
  if constexpr (CACHED) {
    grad_copy_tables<LOG2N>(p.tab, S * R, p.perm, S * R * N, gsm);
    tab = gsm;
    if (p.perm) perm = gsm + (size_t)S * R * T::ROUND;
    off = grad_table_bytes<LOG2N>(S, R);
  }
  const int warps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane32 = threadIdx.x & 31;
  const int grp = lane32 / L;
  const int lane = lane32 % L;
  const int stride = grad_acc_stride(p.angles);
  float* acc_all = reinterpret_cast<float*>(gsm + off);
  float* acc = acc_all + (size_t)(warp * GROUPS + grp) * stride;
  float* ybuf = acc_all + (size_t)warps * GROUPS * stride + (size_t)warp * 2 * GROUPS * RW +
                grp * RW;
  float* gbuf = ybuf + GROUPS * RW;
  for (int i = threadIdx.x; i < warps * GROUPS * stride; i += blockDim.x) acc_all[i] = 0.f;
  __syncthreads();

  // this warp's contiguous range of tasks
  long long ntasks;
  if (p.order) {
    if (p.meta[1] != (int)p.nblocks || p.meta[2] != S || p.meta[3] != G) {
      if (threadIdx.x == 0 && blockIdx.x == 0 && p.status) atomicCAS(p.status, 0, 1);
      ntasks = 0;
    } else {
      ntasks = max(0LL, min((long long)p.meta[0], p.tmax));
    }
  } else {
    ntasks = (p.nblocks + G - 1) / G;
  }
  const long long warps_total = (long long)gridDim.x * warps;
  const long long chunk = (ntasks + warps_total - 1) / warps_total;
  const long long t0 = min(ntasks, ((long long)blockIdx.x * warps + warp) * chunk);
  const long long t1 = min(ntasks, t0 + chunk);

  // diagonal objective: this lane's E weights (dL/dy_e = w_e y_e)
  float wl[E];
#pragma unroll
  for (int i = 0; i < E; ++i) wl[i] = p.gy ? 0.f : __ldg(p.w + lane * E + i);

  int bucket = 0, bucket_end = 0;
  for (long long t = t0; t < t1; ++t) {
    const long long slot = t * G;
    if (!p.order && lane32 == 0 && t + 1 < t1) {
      // blocks in order: the next task's rows are contiguous; pull them into
      // L2 while this task computes (the sizes stay inside the buffers)
      const long long nb = min((long long)G, p.nblocks - (t + 1) * G);
      const uint32_t bytes = (uint32_t)(nb * N * 4);
      if (nb > 0 && (bytes & 15u) == 0) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p.y + (t + 1) * G * N),
                     "r"(bytes)
                     : "memory");
        if (p.gy)
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p.gy + (t + 1) * G * N),
                       "r"(bytes)
                       : "memory");
      }
    }
    if (p.order && slot >= bucket_end) {  // warp-uniform
      bucket = bucket_of_slot(p.starts, S, (int)slot);
      bucket_end = __ldg(p.starts + bucket + 1);
    }
    long long b[K];
    bool valid[K];
    float v[K][E], g[K][E];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const long long s = slot + k * GROUPS + grp;
      b[k] = p.order ? (long long)__ldg(p.order + s) : s;
      valid[k] = b[k] >= 0 && b[k] < p.nblocks;
      if (valid[k]) {
        load_f32<E>(p.y + b[k] * N + lane * E, v[k]);
        if (p.gy) {
          load_f32<E>(p.gy + b[k] * N + lane * E, g[k]);
        } else {
#pragma unroll
          for (int i = 0; i < E; ++i) g[k][i] = wl[i] * v[k][i];
        }
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i) v[k][i] = g[k][i] = 0.f;
      }
    }
    if (bucket < S) {
      for (int r = R - 1; r >= 0; --r) {
        if (perm && ((p.perm_mask >> r) & 1u)) {  // undo the gather: v_prev[perm[e]] = v[e]
          const uint8_t* prow = perm + ((size_t)bucket * R + r) * N + lane * E;
#pragma unroll
          for (int k = 0; k < K; ++k) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
              const int d = grad_word<LOG2N>(prow[i]);
              ybuf[d] = v[k][i];
              gbuf[d] = g[k][i];
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < E; ++i) {
              v[k][i] = ybuf[grad_word<LOG2N>(lane * E + i)];
              g[k][i] = gbuf[grad_word<LOG2N>(lane * E + i)];
            }
            __syncwarp();
          }
        }
        const size_t o = (size_t)bucket * R + r;
        grad_round<LOG2N, CACHED, 0>(v, g, tab + o * T::ROUND, acc + o * rowlen, lane);
      }
    } else if (bucket == S + 1) {  // bad set index: zero gradient, status
#pragma unroll
      for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int i = 0; i < E; ++i) g[k][i] = 0.f;
        if (valid[k] && lane == 0 && p.status) atomicCAS(p.status, 0, 4);
      }
    }  // skip bucket (S): identity, dL/dx = dL/dy
    if (p.gx) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (valid[k]) store_f32<E>(p.gx + b[k] * N + lane * E, g[k]);
    }
  }
  __syncthreads();
  // CTA partial: sum of all (warp, lane group) rows, in FP64, fixed order
  for (int a = threadIdx.x; a < p.angles; a += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < warps * GROUPS; ++k) s += (double)acc_all[(size_t)k * stride + a];
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
// Launch shape of the backward: threads, grid and shared memory (0 threads:
// too many angles for the shared-memory accumulators), whether the tables are
// cached, and the task size G of its schedule.
void grad_config(int log2n, int num_sets, int rounds, long long nblocks, int* threads, int* grid,
                 size_t* smem, int* cache_tables, int* group);

}  // namespace hygt
