// hygt_batch.cuh -- set-bucketed integer HyGT (sm_103a).
//
// A batch is first bucketed by transform set (counting sort of block ids;
// every bucket padded to a multiple of 32 with id -1), so that each warp
// task is 32 blocks that share one set.  The multipliers of that set are
// then warp-uniform: every lane reads the same address (one broadcast
// transaction), and a thread holds a whole block (N <= 64) so every
// hypercube pass is a register butterfly.
//
// Butterfly.  The rotation of (a, b) by the integer multipliers (c, s) is
// computed with three multiplications instead of four:
//     k   = c (a + b) + 2^(f-1)
//     y_m = (k + (s - c) b) >> f        (= (c a + s b + 2^(f-1)) >> f)
//     y_n = (k - (c + s) a) >> f        (= (c b - s a + 2^(f-1)) >> f)
// The table stores (c, d1 = s - c, d2 = -(c + s)); the inverse rotation
// (c, -s) uses the same entries with d1 and d2 exchanged.  The arithmetic is
// done modulo 2^32: the sums equal the direct products modulo 2^32, so the
// result is exact whenever the direct formula fits in int32 (always, for
// int16 input; see the inverse precondition in hygt.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hygt_device.cuh"

namespace hygt {

constexpr int kBatchThreads = 512;   // threads per CTA of the batch transform
constexpr int kBucketThreads = 512;  // threads per CTA of the bucketing kernels
constexpr int kBucketTile = 8192;    // blocks per CTA tile in the scatter pass

// Workspace layout (all offsets in bytes, 16-byte aligned sections):
//   counts [nb]     int32  blocks per bucket (bucket S = skip, S + 1 = bad set)
//   starts [nb + 1] int32  first slot of each bucket (padded to 32); starts[nb] = total
//   cursor [nb]     int32  scatter cursor per bucket
//   meta   [4]      int32  warp tasks (total / 32), nblocks, num_sets
//   order  [32 * tmax] int32 block id per slot, -1 for padding
struct BatchLayout {
  int nb;           // buckets = S + 2
  long long tmax;   // max warp tasks
  size_t counts, starts, cursor, meta, order, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline BatchLayout batch_layout(int num_sets, long long nblocks) {
  BatchLayout L;
  L.nb = num_sets + 2;
  L.tmax = (nblocks + 31) / 32 + L.nb;
  size_t off = 0;
  L.counts = off; off = align16(off + 4 * (size_t)L.nb);
  L.starts = off; off = align16(off + 4 * (size_t)(L.nb + 1));
  L.cursor = off; off = align16(off + 4 * (size_t)L.nb);
  L.meta = off;   off = align16(off + 16);
  L.order = off;  off = align16(off + 4 * 32 * (size_t)L.tmax);
  L.total = off;
  return L;
}

// ---------------------------------------------------------------- transform
struct BatchParams {
  const void* in;
  void* out;
  const int* order;      // [32 * ntasks]
  const int* starts;     // [nb + 1] padded bucket starts
  const int* meta;       // meta[0] = ntasks, meta[1] = nblocks, meta[2] = num_sets
  long long nblocks;
  const int4* gtab;      // (c, d1, d2, s) per pair, [S][R][k][N/2]
  const int* poff;       // permutation gather indices as int32, [S][R][N], or nullptr
  unsigned perm_mask;
  int rounds;
  int num_sets;
  int frac_bits;
  int* status;
};

// Gauss butterfly, forward (INV = false) or inverse.
template <bool INV>
__device__ __forceinline__ void gbfly(int32_t& a, int32_t& b, const int4 w, uint32_t half, int f) {
  const uint32_t ua = (uint32_t)a, ub = (uint32_t)b;
  const uint32_t k = (uint32_t)w.x * (ua + ub) + half;
  const uint32_t d1 = (uint32_t)(INV ? w.z : w.y);
  const uint32_t d2 = (uint32_t)(INV ? w.y : w.z);
  a = (int32_t)(k + d1 * ub) >> f;
  b = (int32_t)(k + d2 * ua) >> f;
}

// One thread per block (E = N <= 64): every pass is a register pass.
template <int LOG2N, bool INV>
__device__ __forceinline__ void batch_round(int32_t (&v)[1 << LOG2N], const int4* row,
                                            uint32_t half, int f) {
  constexpr int N = 1 << LOG2N;
#pragma unroll
  for (int pp = 0; pp < LOG2N; ++pp) {
    const int p = INV ? (LOG2N - 1 - pp) : pp;
    const int4* prow = row + p * (N / 2);
#pragma unroll
    for (int j = 0; j < N / 2; ++j) {
      const int m = ((j >> p) << (p + 1)) | (j & ((1 << p) - 1));
      const int n = m | (1 << p);
      const int4 w = __ldg(prow + j);
      gbfly<INV>(v[m], v[n], w, half, f);
    }
  }
}

// KIND 0: int16 -> int32 forward; KIND 1: int32 -> int16 inverse.
template <int LOG2N, int KIND>
__global__ void __launch_bounds__(kBatchThreads) hygt_batch_kernel(BatchParams p) {
  constexpr int N = 1 << LOG2N;
  constexpr bool INV = (KIND == 1);
  static_assert(LOG2N <= 6, "one thread per block up to N = 64");
  extern __shared__ __align__(16) int32_t pscr[];  // [N][blockDim.x] permutation scratch

  // The schedule must have been built for this block count and set count.
  if (p.meta[1] != (int)p.nblocks || p.meta[2] != p.num_sets) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && p.status) atomicCAS(p.status, 0, 1);
    return;
  }
  const int ntasks = p.meta[0];
  const int lane = threadIdx.x & 31;
  const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long chunk = (ntasks + warps_total - 1) / warps_total;
  const long long t0 = gw * chunk;
  const long long t1 = min((long long)ntasks, t0 + chunk);
  const uint32_t half = 1u << (p.frac_bits - 1);
  const int f = p.frac_bits;
  const int R = p.rounds;
  const int S = p.num_sets;
  int32_t* col = pscr + threadIdx.x;
  const int T = blockDim.x;

  // Bucket of the first task: the largest k with starts[k] <= slot (empty
  // buckets share their start with the next one, so the largest is non-empty).
  int bucket = 0, bucket_end = 0;
  for (long long t = t0; t < t1; ++t) {
    const int slot = (int)(t * 32);
    if (slot >= bucket_end) {  // warp-uniform
      int lo = 0, hi = S + 1;  // search over buckets 0..S+1
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(p.starts + mid) <= slot) lo = mid; else hi = mid - 1;
      }
      bucket = lo;
      bucket_end = __ldg(p.starts + bucket + 1);
    }
    const int b = __ldg(p.order + t * 32 + lane);
    const bool active = b >= 0 && b < p.nblocks;
    int32_t v[N];
    if (active) {
      if constexpr (KIND == 0)
        load_i16<N>(static_cast<const int16_t*>(p.in) + (long long)b * N, v);
      else
        load_i32<N>(static_cast<const int32_t*>(p.in) + (long long)b * N, v);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = 0;
    }
    if (bucket < S) {
      const int4* tab = p.gtab + (size_t)bucket * R * LOG2N * (N / 2);
      const int* poff = p.poff ? p.poff + (size_t)bucket * R * N : nullptr;
      for (int rr = 0; rr < R; ++rr) {
        const int r = INV ? (R - 1 - rr) : rr;
        const bool has_perm = poff && ((p.perm_mask >> r) & 1u);
        if (INV && has_perm) {  // undo the gather of slot r: v_prev[perm[i]] = v[i]
#pragma unroll
          for (int i = 0; i < N; ++i) col[__ldg(poff + r * N + i) * T] = v[i];
#pragma unroll
          for (int i = 0; i < N; ++i) v[i] = col[i * T];
        }
        batch_round<LOG2N, INV>(v, tab + (size_t)r * LOG2N * (N / 2), half, f);
        if (!INV && has_perm) {  // gather: v'[i] = v[perm[i]]
#pragma unroll
          for (int i = 0; i < N; ++i) col[i * T] = v[i];
#pragma unroll
          for (int i = 0; i < N; ++i) v[i] = col[__ldg(poff + r * N + i) * T];
        }
      }
    } else if (bucket == S + 1) {  // bad set index: zeros, status
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = 0;
      if (active && p.status) atomicCAS(p.status, 0, 4);
    }
    if (active) {
      if constexpr (KIND == 0)
        store_i32<N>(static_cast<int32_t*>(p.out) + (long long)b * N, v);
      else
        store_i16_sat<N>(static_cast<int16_t*>(p.out) + (long long)b * N, v);
    }
  }
}

}  // namespace hygt

namespace hygt {
// Host launchers (batch_int.cu).
cudaError_t batch_build(const uint16_t* d_set, long long nblocks, int num_sets, void* d_work,
                        cudaStream_t stream);
cudaError_t launch_batch_fwd(int log2n, const BatchParams& p, bool perms, long long nblocks,
                             cudaStream_t stream);
cudaError_t launch_batch_inv(int log2n, const BatchParams& p, bool perms, long long nblocks,
                             cudaStream_t stream);
}  // namespace hygt
