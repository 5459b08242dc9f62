// hygt_f32b.cuh -- set-bucketed FP32 HyGT forward / inverse (sm_103a).
//
// The FP32 counterpart of the bucketed integer kernels: the schedule that
// hygt_batch_build writes (block ids sorted by transform set, every bucket
// padded to the schedule group) makes every warp task G blocks of one set,
// so the lane groups read warp-uniform (cos, sin) pairs.  Arithmetic and
// lane mapping are those of the one-set FP32 kernel (hygt_f32u.cuh): a block
// is held by L = N / 8 lanes with 8 values each, K = 4 blocks per lane
// group, register rotations within a lane, __shfl_xor_sync across lanes.
// A CTA walks a contiguous range of tasks; when the sets that range spans
// fit, their tables are copied to shared memory once (padded layout), else
// the lanes read the plan's table [S][R][k][N/2] from global memory
// (L1-cached).  Skip blocks (0xFFFF) are copied through; bad set indices
// give zeros and HYGT_ERR_SET_INDEX (4) in the status word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hygt_batch.cuh"
#include "hygt_f32u.cuh"

namespace hygt {

constexpr int kF32bThreads = 512;

struct F32bParams {
  const float* in;
  float* out;
  long long nblocks;
  const float2* tab;    // (cos, sin), [S][R][k][N/2]
  const uint8_t* perm;  // [S][R][N] or nullptr
  unsigned perm_mask;
  int rounds, num_sets;
  const int* order;     // schedule of hygt_batch_build (group GS)
  const int* starts;
  const int* meta;
  long long tmax;
  int group_sched;      // GS; a multiple of the kernel's task size
  int max_cached_sets;
  int* status;
};

template <int LOG2N>
__host__ __device__ inline size_t f32b_set_bytes(int rounds) {
  return (size_t)rounds * GradTab<LOG2N, true>::ROUND +
         (((size_t)rounds * (1 << LOG2N) + 15) & ~(size_t)15);
}

template <int LOG2N>
__host__ __device__ inline size_t f32b_smem_bytes(int threads, int rounds, int cached) {
  using M = GradMap<LOG2N>;
  return (size_t)cached * f32b_set_bytes<LOG2N>(rounds) +
         (size_t)(threads / 32) * M::GROUPS * M::RW * 4;
}

// Copy the tables of sets [s0, s0 + n) into the padded shared-memory layout:
// per set R * ROUND bytes of (cos, sin), then its permutation bytes.
template <int LOG2N>
__device__ __forceinline__ void f32b_copy_sets(const F32bParams& p, int s0, int n,
                                               unsigned char* dst) {
  const size_t sb = f32b_set_bytes<LOG2N>(p.rounds);
  const int R = p.rounds, N = 1 << LOG2N;
  for (int k = 0; k < n; ++k) {
    grad_copy_tables<LOG2N>(p.tab + (size_t)(s0 + k) * R * LOG2N * (N / 2), R,
                            p.perm ? p.perm + (size_t)(s0 + k) * R * N : nullptr, R * N,
                            dst + k * sb);
  }
}

template <int LOG2N, bool INV, bool CACHED>
__device__ __forceinline__ void f32b_tasks(const F32bParams& p, long long t0, long long t1,
                                           const unsigned char* cache, int set_lo, float* pb) {
  using M = GradMap<LOG2N>;
  using T = GradTab<LOG2N, CACHED>;
  constexpr int N = M::N, E = M::E, L = M::L, K = M::K, GROUPS = M::GROUPS, G = M::G;
  const int lane32 = threadIdx.x & 31;
  const int grp = lane32 / L, lane = lane32 % L;
  const int R = p.rounds, S = p.num_sets;
  const size_t sb = f32b_set_bytes<LOG2N>(R);
  int bucket = 0, bucket_end = 0;
  for (long long t = t0; t < t1; ++t) {
    const int slot = (int)(t * G);
    if (slot >= bucket_end) {  // warp-uniform
      bucket = bucket_of_slot(p.starts, S, slot);
      bucket_end = __ldg(p.starts + bucket + 1);
    }
    int b[K];
    bool active[K];
    float v[K][E];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      b[k] = __ldg(p.order + slot + k * GROUPS + grp);
      active[k] = b[k] >= 0 && b[k] < p.nblocks;
      if (active[k]) {
        load_f32<E>(p.in + (long long)b[k] * N + lane * E, v[k]);
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i) v[k][i] = 0.f;
      }
    }
    if (bucket < S) {
      const unsigned char* stab;
      const uint8_t* sperm;
      if constexpr (CACHED) {
        stab = cache + (size_t)(bucket - set_lo) * sb;
        sperm = stab + (size_t)R * T::ROUND;
      } else {
        stab = reinterpret_cast<const unsigned char*>(p.tab + (size_t)bucket * R * LOG2N * (N / 2));
        sperm = p.perm ? p.perm + (size_t)bucket * R * N : nullptr;
      }
      for (int rr = 0; rr < R; ++rr) {
        const int r = INV ? R - 1 - rr : rr;
        const bool has_perm = p.perm && ((p.perm_mask >> r) & 1u);
        const uint8_t* prow = sperm + (size_t)r * N + lane * E;
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
        f32u_round<LOG2N, INV, CACHED, 0>(v, stab + (size_t)r * T::ROUND, lane);
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
    } else if (bucket == S + 1) {  // bad set index
#pragma unroll
      for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int i = 0; i < E; ++i) v[k][i] = 0.f;
        if (active[k] && lane == 0 && p.status) atomicCAS(p.status, 0, 4);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (active[k]) store_f32<E>(p.out + (long long)b[k] * N + lane * E, v[k]);
  }
}

cudaError_t launch_f32b(int log2n, int kind, const F32bParams& p, cudaStream_t stream);

}  // namespace hygt
