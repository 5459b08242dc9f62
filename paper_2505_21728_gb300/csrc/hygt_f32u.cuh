// hygt_f32u.cuh -- FP32 HyGT forward / inverse for batches that use one
// transform set (no set indices), as in angle fitting (sm_103a).
//
// Same mapping as the backward (hygt_grad.cuh): a block is held by a lane
// group of L = N / 8 lanes with 8 values each, and every lane group holds
// K = 4 blocks, so each (cos, sin) pair read from shared memory serves four
// rotations.  Passes within a lane's values are register rotations,
// cross-lane passes exchange values with __shfl_xor_sync.  The set's
// (cos, sin) table and permutation slots are copied to shared memory once
// per CTA; a permutation slot goes through a per-warp buffer, one block per
// lane group at a time.
//   forward: y_m = c a + s b, y_n = c b - s a, passes p = 0 .. k-1, then the
//            gather of slot r;
//   inverse: the scatter of slot r, then passes p = k-1 .. 0 with (c, -s).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hygt_device.cuh"
#include "hygt_grad.cuh"

namespace hygt {

constexpr int kF32uThreads = 512;

struct F32uParams {
  const float* in;
  float* out;
  long long nblocks;
  const float2* tab;    // (cos, sin) of set 0, [R][k][N/2]
  const uint8_t* perm;  // permutation slots of set 0, [R][N], or nullptr
  unsigned perm_mask;
  int rounds;
};

// Shared memory: the set's table (padded layout of hygt_grad.cuh) and
// permutation bytes, then per warp GROUPS block regions of the permutation
// buffer.
template <int LOG2N>
__host__ __device__ inline size_t f32u_table_bytes(int rounds) {
  return grad_table_bytes<LOG2N>(1, rounds);
}
template <int LOG2N>
__host__ __device__ inline size_t f32u_smem_bytes(int threads, int rounds) {
  using M = GradMap<LOG2N>;
  return f32u_table_bytes<LOG2N>(rounds) + (size_t)(threads / 32) * M::GROUPS * M::RW * 4;
}

template <int LOG2N, bool INV, bool PADDED, int P>
__device__ __forceinline__ void f32u_pass(float (&v)[GradMap<LOG2N>::K][GradMap<LOG2N>::E],
                                          const unsigned char* rtab, int lane) {
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
      const float2 cs = seg[jl];
      const float s = INV ? -cs.y : cs.y;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float a = v[k][im], b = v[k][in];
        v[k][im] = cs.x * a + s * b;
        v[k][in] = cs.x * b - s * a;
      }
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
      // m side: c own + s partner; n side: c own - s partner (s -> -s inverse)
      const float sp = (upper != INV) ? -cs.y : cs.y;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float o = v[k][i];
        const float pt = __shfl_xor_sync(kFullMask, o, D);
        v[k][i] = cs.x * o + sp * pt;
      }
    }
  }
}

// All passes of one round; PADDED: the shared-memory table layout, else the
// plan's global layout [k][N/2] (hygt_grad.cuh, GradTab).
template <int LOG2N, bool INV, bool PADDED, int J>
__device__ __forceinline__ void f32u_round(float (&v)[GradMap<LOG2N>::K][GradMap<LOG2N>::E],
                                           const unsigned char* rtab, int lane) {
  if constexpr (J < LOG2N) {
    constexpr int P = INV ? LOG2N - 1 - J : J;
    f32u_pass<LOG2N, INV, PADDED, P>(v, rtab, lane);
    f32u_round<LOG2N, INV, PADDED, J + 1>(v, rtab, lane);
  }
}

template <int LOG2N, bool INV>
__global__ void __launch_bounds__(kF32uThreads, 1) hygt_f32u_kernel(F32uParams p) {
  using M = GradMap<LOG2N>;
  constexpr int N = M::N;
  constexpr int E = M::E;
  constexpr int L = M::L;
  constexpr int K = M::K;
  constexpr int GROUPS = M::GROUPS;
  constexpr int G = M::G;
  constexpr int RW = M::RW;
  extern __shared__ __align__(16) unsigned char fsm[];

  using T = GradTab<LOG2N, true>;
  const int R = p.rounds;
  grad_copy_tables<LOG2N>(p.tab, R, p.perm, R * N, fsm);
  const unsigned char* tab = fsm;
  const uint8_t* perm = fsm + (size_t)R * T::ROUND;
  const int warps = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5;
  const int lane32 = threadIdx.x & 31;
  const int grp = lane32 / L;
  const int lane = lane32 % L;
  float* pb = reinterpret_cast<float*>(fsm + f32u_table_bytes<LOG2N>(R)) +
              (size_t)warp * GROUPS * RW + grp * RW;
  __syncthreads();

  const long long ntasks = (p.nblocks + G - 1) / G;
  const long long warps_total = (long long)gridDim.x * warps;
  const long long chunk = (ntasks + warps_total - 1) / warps_total;
  const long long t0 = min(ntasks, ((long long)blockIdx.x * warps + warp) * chunk);
  const long long t1 = min(ntasks, t0 + chunk);

  for (long long t = t0; t < t1; ++t) {
    if (lane32 == 0 && t + 1 < t1) {
      // the next task's blocks are contiguous: pull them into L2 while this
      // task computes (the size stays inside the buffer)
      const long long nb = min((long long)G, p.nblocks - (t + 1) * G);
      const uint32_t bytes = (uint32_t)(nb * N * 4);
      if (nb > 0 && (bytes & 15u) == 0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p.in + (t + 1) * G * N),
                     "r"(bytes)
                     : "memory");
    }
    long long b[K];
    float v[K][E];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      b[k] = t * G + k * GROUPS + grp;
      if (b[k] < p.nblocks) {
        load_f32<E>(p.in + b[k] * N + lane * E, v[k]);
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i) v[k][i] = 0.f;
      }
    }
    for (int rr = 0; rr < R; ++rr) {
      const int r = INV ? R - 1 - rr : rr;
      const bool has_perm = p.perm && ((p.perm_mask >> r) & 1u);
      const uint8_t* prow = perm + (size_t)r * N + lane * E;
      if (INV && has_perm) {  // undo the gather: v_prev[perm[e]] = v[e]
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
          for (int i = 0; i < E; ++i) pb[grad_word<LOG2N>(prow[i])] = v[k][i];
          __syncwarp();
#pragma unroll
          for (int i = 0; i < E; ++i) v[k][i] = pb[grad_word<LOG2N>(lane * E + i)];
          __syncwarp();
        }
      }
      f32u_round<LOG2N, INV, true, 0>(v, tab + (size_t)r * T::ROUND, lane);
      if (!INV && has_perm) {  // gather: v'[e] = v[perm[e]]
#pragma unroll
        for (int k = 0; k < K; ++k) {
#pragma unroll
          for (int i = 0; i < E; ++i) pb[grad_word<LOG2N>(lane * E + i)] = v[k][i];
          __syncwarp();
#pragma unroll
          for (int i = 0; i < E; ++i) v[k][i] = pb[grad_word<LOG2N>(prow[i])];
          __syncwarp();
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (b[k] < p.nblocks) store_f32<E>(p.out + b[k] * N + lane * E, v[k]);
  }
}

// kind 0: forward, 1: inverse.  Returns cudaErrorInvalidConfiguration when
// the set's table does not fit in shared memory (the caller then uses the
// direct kernels).
cudaError_t launch_f32u(int log2n, int kind, const F32uParams& p, cudaStream_t stream);

}  // namespace hygt
