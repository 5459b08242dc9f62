// hygt_device.cuh -- CUDA kernels (sm_103a) of the Hypercube-Givens Transform.
//
// Mapping.  One block (N = 2^LOG2N values) is held by a sub-warp of
// L = N / E lanes, E = 2^LOG2E consecutive values per lane (element
// e = lane * E + i lives in register i of sub-lane `lane`), so a lane's slice
// of the block is one contiguous, vector-aligned piece of global memory.
//   - Pass p < LOG2E pairs two registers of the same lane: a butterfly in
//     registers.
//   - Pass p >= LOG2E pairs lane l with lane l ^ 2^(p - LOG2E), same
//     register: each lane fetches its partner's value with __shfl_xor_sync
//     and computes its own output.
//   - The permutation slot after a round goes through a per-warp shared
//     memory buffer (write the slice, gather by the permutation).
// Per pass, the pairs a lane touches have consecutive pair indices j, so the
// lane reads its (c, s) multipliers as one vector from the table.
//
// Tables (built on the host from the plan): integer plans keep one 32-bit
// word per pair, c in the low and s in the high 16 bits; FP32 plans keep
// (cos, sin) as float2.  Layout [set][round][pass][pair], permutations as
// uint8 [set][round][N].  When they fit, the kernel stages them in shared
// memory once per CTA; otherwise it reads them through the read-only cache.
//
// The kernels are persistent: a grid of (SMs x resident CTAs) walks all
// blocks with a warp-granular stride.  Nothing waits on another CTA.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hygt {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kThreads = 1024;  // threads per CTA of the persistent kernels

struct Params {
  const void* in;
  void* out;
  const uint16_t* set;  // nullable: set 0 for all blocks
  long long nblocks;
  const void* tab;      // uint32 (integer) or float2 (FP32), [S][R][k][N/2]
  const uint8_t* perm;  // [S][R][N] or nullptr
  unsigned perm_mask;   // bit r set: slot r has a permutation
  int rounds;
  int num_sets;
  int frac_bits;
  int tab_bytes;        // bytes of tab, padded to 16 (staged in smem when stage != 0)
  int perm_bytes;       // bytes of perm, padded to 16
  int stage;            // 1: copy tab and perm to shared memory
  int* status;          // nullable
};

// ---------------------------------------------------------------- I/O
template <int WORDS>
__device__ __forceinline__ void load_words(const void* p, uint32_t (&w)[WORDS]) {
  static_assert(WORDS == 1 || WORDS == 2 || WORDS % 4 == 0, "vector width");
  if constexpr (WORDS % 4 == 0) {
#pragma unroll
    for (int k = 0; k < WORDS / 4; ++k) {
      uint4 t = __ldg(reinterpret_cast<const uint4*>(p) + k);
      w[4 * k] = t.x; w[4 * k + 1] = t.y; w[4 * k + 2] = t.z; w[4 * k + 3] = t.w;
    }
  } else if constexpr (WORDS == 2) {
    uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    w[0] = t.x; w[1] = t.y;
  } else {
    w[0] = __ldg(reinterpret_cast<const uint32_t*>(p));
  }
}

template <int WORDS>
__device__ __forceinline__ void store_words(void* p, const uint32_t (&w)[WORDS]) {
  static_assert(WORDS == 1 || WORDS == 2 || WORDS % 4 == 0, "vector width");
  if constexpr (WORDS % 4 == 0) {
#pragma unroll
    for (int k = 0; k < WORDS / 4; ++k)
      reinterpret_cast<uint4*>(p)[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
  } else if constexpr (WORDS == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  } else {
    *reinterpret_cast<uint32_t*>(p) = w[0];
  }
}

// Table words from shared memory or global memory (generic pointer: the
// staged copy is addressed through the same code path).
template <int WORDS>
__device__ __forceinline__ void load_tab(const uint32_t* p, uint32_t (&w)[WORDS]) {
  static_assert(WORDS == 1 || WORDS == 2 || WORDS % 4 == 0, "vector width");
  if constexpr (WORDS % 4 == 0) {
#pragma unroll
    for (int k = 0; k < WORDS / 4; ++k) {
      uint4 t = reinterpret_cast<const uint4*>(p)[k];
      w[4 * k] = t.x; w[4 * k + 1] = t.y; w[4 * k + 2] = t.z; w[4 * k + 3] = t.w;
    }
  } else if constexpr (WORDS == 2) {
    uint2 t = *reinterpret_cast<const uint2*>(p);
    w[0] = t.x; w[1] = t.y;
  } else {
    w[0] = *p;
  }
}

// ---------------------------------------------------------------- arithmetic
// Integer butterfly on (a, b) with packed multipliers w = (c | s << 16).
// Forward: (c a + s b, -s a + c b); inverse: (c a - s b, s a + c b); each
// output rounded half up: (u + 2^(f-1)) >> f (arithmetic shift = floor).
struct IntMath {
  using V = int32_t;
  static constexpr int kTabWordsPerPair = 1;
  int half, f;
  __device__ __forceinline__ static int cval(uint32_t w) { return (int)(int16_t)(w & 0xffffu); }
  __device__ __forceinline__ static int sval(uint32_t w) { return (int)w >> 16; }
  template <bool INV>
  __device__ __forceinline__ void bfly(V& a, V& b, const uint32_t* w) const {
    const int c = cval(w[0]);
    const int s = INV ? -sval(w[0]) : sval(w[0]);
    const int ym = (c * a + s * b + half) >> f;
    const int yn = (c * b - s * a + half) >> f;
    a = ym;
    b = yn;
  }
  // One output of a cross-lane pass: own * c + partner * (+/-s).
  __device__ __forceinline__ V rot(V own, V partner, const uint32_t* w, bool neg_s) const {
    const int c = cval(w[0]);
    const int s = neg_s ? -sval(w[0]) : sval(w[0]);
    return (c * own + s * partner + half) >> f;
  }
};

struct FloatMath {
  using V = float;
  static constexpr int kTabWordsPerPair = 2;
  template <bool INV>
  __device__ __forceinline__ void bfly(V& a, V& b, const uint32_t* w) const {
    const float c = __uint_as_float(w[0]);
    const float s = INV ? -__uint_as_float(w[1]) : __uint_as_float(w[1]);
    const float ym = fmaf(c, a, s * b);
    const float yn = fmaf(c, b, -(s * a));
    a = ym;
    b = yn;
  }
  __device__ __forceinline__ V rot(V own, V partner, const uint32_t* w, bool neg_s) const {
    const float c = __uint_as_float(w[0]);
    const float s = neg_s ? -__uint_as_float(w[1]) : __uint_as_float(w[1]);
    return fmaf(c, own, s * partner);
  }
};

// ---------------------------------------------------------------- block load / store
// Element types on the global side: forward integer reads int16 and writes
// int32; inverse integer reads int32 and writes int16 (saturated); FP32
// reads and writes float.
template <int E>
__device__ __forceinline__ void load_i16(const int16_t* p, int32_t (&v)[E]) {
  uint32_t w[E / 2];
  load_words<E / 2>(p, w);
#pragma unroll
  for (int k = 0; k < E / 2; ++k) {
    v[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
    v[2 * k + 1] = (int32_t)w[k] >> 16;
  }
}

template <int E>
__device__ __forceinline__ void load_i32(const int32_t* p, int32_t (&v)[E]) {
  uint32_t w[E];
  load_words<E>(p, w);
#pragma unroll
  for (int k = 0; k < E; ++k) v[k] = (int32_t)w[k];
}

template <int E>
__device__ __forceinline__ void load_f32(const float* p, float (&v)[E]) {
  uint32_t w[E];
  load_words<E>(p, w);
#pragma unroll
  for (int k = 0; k < E; ++k) v[k] = __uint_as_float(w[k]);
}

// Two int32 values saturated to int16 and packed, lo in the low half (one
// cvt.pack.sat instruction: its first source goes to the high half).
__device__ __forceinline__ uint32_t pack_sat16(int32_t lo, int32_t hi) {
  uint32_t d;
  asm("cvt.pack.sat.s16.s32 %0, %1, %2;" : "=r"(d) : "r"(hi), "r"(lo));
  return d;
}

template <int E>
__device__ __forceinline__ void store_i16_sat(int16_t* p, const int32_t (&v)[E]) {
  uint32_t w[E / 2];
#pragma unroll
  for (int k = 0; k < E / 2; ++k) w[k] = pack_sat16(v[2 * k], v[2 * k + 1]);
  store_words<E / 2>(p, w);
}

template <int E>
__device__ __forceinline__ void store_i32(int32_t* p, const int32_t (&v)[E]) {
  uint32_t w[E];
#pragma unroll
  for (int k = 0; k < E; ++k) w[k] = (uint32_t)v[k];
  store_words<E>(p, w);
}

template <int E>
__device__ __forceinline__ void store_f32(float* p, const float (&v)[E]) {
  uint32_t w[E];
#pragma unroll
  for (int k = 0; k < E; ++k) w[k] = __float_as_uint(v[k]);
  store_words<E>(p, w);
}

// ---------------------------------------------------------------- passes
// Register pass p (< LOG2E): the lane's E/2 pairs are j = lane*E/2 + jl.
template <int LOG2N, int LOG2E, int P, bool INV, class M>
__device__ __forceinline__ void reg_pass(const M& math, typename M::V (&v)[1 << LOG2E],
                                         const uint32_t* row, int lane) {
  constexpr int E = 1 << LOG2E;
  constexpr int WPP = M::kTabWordsPerPair;
  uint32_t w[(E / 2) * WPP];
  load_tab<(E / 2) * WPP>(row + lane * (E / 2) * WPP, w);
#pragma unroll
  for (int jl = 0; jl < E / 2; ++jl) {
    constexpr int lowmask = (1 << P) - 1;
    const int im = ((jl >> P) << (P + 1)) | (jl & lowmask);
    const int in = im | (1 << P);
    math.template bfly<INV>(v[im], v[in], &w[jl * WPP]);
  }
}

// Lane pass p (>= LOG2E): partner lane = lane ^ 2^(p - LOG2E).
template <int LOG2N, int LOG2E, int P, bool INV, class M>
__device__ __forceinline__ void lane_pass(const M& math, typename M::V (&v)[1 << LOG2E],
                                          const uint32_t* row, int lane) {
  constexpr int E = 1 << LOG2E;
  constexpr int Q = P - LOG2E;
  constexpr int D = 1 << Q;
  constexpr int WPP = M::kTabWordsPerPair;
  const bool upper = (lane >> Q) & 1;  // this lane holds the n side of its pairs
  const int jbase = ((lane >> (Q + 1)) << P) + ((lane & (D - 1)) << LOG2E);
  uint32_t w[E * WPP];
  load_tab<E * WPP>(row + jbase * WPP, w);
  // forward: m side uses +s, n side -s; inverse: the opposite
  const bool neg_s = upper ^ INV;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const typename M::V partner = __shfl_xor_sync(kFullMask, v[i], D);
    v[i] = math.rot(v[i], partner, &w[i * WPP], neg_s);
  }
}

template <int LOG2N, int LOG2E, int P, bool INV, class M>
__device__ __forceinline__ void one_pass(const M& math, typename M::V (&v)[1 << LOG2E],
                                         const uint32_t* tab, int row_base, int lane) {
  constexpr int WPP = M::kTabWordsPerPair;
  const uint32_t* row = tab + (size_t)(row_base + P) * ((1 << LOG2N) / 2) * WPP;
  if constexpr (P < LOG2E)
    reg_pass<LOG2N, LOG2E, P, INV>(math, v, row, lane);
  else
    lane_pass<LOG2N, LOG2E, P, INV>(math, v, row, lane);
}

template <int LOG2N, int LOG2E, int P, class M>
__device__ __forceinline__ void round_fwd(const M& math, typename M::V (&v)[1 << LOG2E],
                                          const uint32_t* tab, int row_base, int lane) {
  if constexpr (P < LOG2N) {
    one_pass<LOG2N, LOG2E, P, false>(math, v, tab, row_base, lane);
    round_fwd<LOG2N, LOG2E, P + 1>(math, v, tab, row_base, lane);
  }
}

template <int LOG2N, int LOG2E, int P, class M>
__device__ __forceinline__ void round_inv(const M& math, typename M::V (&v)[1 << LOG2E],
                                          const uint32_t* tab, int row_base, int lane) {
  if constexpr (P >= 0) {
    one_pass<LOG2N, LOG2E, P, true>(math, v, tab, row_base, lane);
    round_inv<LOG2N, LOG2E, P - 1>(math, v, tab, row_base, lane);
  }
}

// Permutation slot through the warp's shared buffer `buf` (this sub-warp's
// N values start at buf).  Forward gathers v'[i] = v[perm[i]]; the inverse
// scatters v[perm[i]] = v'[i].
template <int LOG2N, int LOG2E, bool INV, class V>
__device__ __forceinline__ void permute(V (&v)[1 << LOG2E], V* buf, const uint8_t* prow, int lane) {
  constexpr int E = 1 << LOG2E;
  uint8_t idx[E];
#pragma unroll
  for (int i = 0; i < E; ++i) idx[i] = prow[lane * E + i];
  if constexpr (!INV) {
#pragma unroll
    for (int i = 0; i < E; ++i) buf[lane * E + i] = v[i];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = buf[idx[i]];
  } else {
#pragma unroll
    for (int i = 0; i < E; ++i) buf[idx[i]] = v[i];
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = buf[lane * E + i];
  }
  __syncwarp();
}

// ---------------------------------------------------------------- kernel
// KIND: 0 = integer forward (int16 -> int32), 1 = integer inverse
// (int32 -> int16), 2 = FP32 forward, 3 = FP32 inverse.
template <int LOG2N, int LOG2E, int KIND>
__global__ void __launch_bounds__(kThreads) hygt_kernel(Params p) {
  constexpr int N = 1 << LOG2N;
  constexpr int E = 1 << LOG2E;
  constexpr int L = N / E;       // lanes per block
  constexpr int G = 32 / L;      // blocks per warp
  static_assert(L >= 1 && L <= 32, "sub-warp size");
  constexpr bool INV = (KIND == 1 || KIND == 3);
  constexpr bool FP = (KIND >= 2);
  using M = typename std::conditional<FP, FloatMath, IntMath>::type;
  using V = typename M::V;

  extern __shared__ __align__(16) unsigned char smem[];

  const uint32_t* tab = static_cast<const uint32_t*>(p.tab);
  const uint8_t* perm = p.perm;
  unsigned char* scratch = smem;
  if (p.stage) {
    const int4* src = static_cast<const int4*>(p.tab);
    int4* dst = reinterpret_cast<int4*>(smem);
    for (int i = threadIdx.x; i < p.tab_bytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    if (perm) {
      const int4* psrc = reinterpret_cast<const int4*>(p.perm);
      int4* pdst = reinterpret_cast<int4*>(smem + p.tab_bytes);
      for (int i = threadIdx.x; i < p.perm_bytes / 16; i += blockDim.x) pdst[i] = __ldg(psrc + i);
      perm = smem + p.tab_bytes;
    }
    tab = reinterpret_cast<const uint32_t*>(smem);
    scratch = smem + p.tab_bytes + p.perm_bytes;
    __syncthreads();
  }

  M math;
  if constexpr (!FP) {
    math.half = 1 << (p.frac_bits - 1);
    math.f = p.frac_bits;
  }

  const int warp = threadIdx.x >> 5;
  const int lane32 = threadIdx.x & 31;
  const int sub = lane32 / L;   // block slot within the warp
  const int lane = lane32 % L;  // lane within the block's sub-warp
  V* buf = reinterpret_cast<V*>(scratch) + (size_t)warp * 32 * E + sub * N;

  const long long warps_total = (long long)gridDim.x * (blockDim.x >> 5);
  const long long warp_global = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  const int rounds = p.rounds;

  for (long long base = warp_global * G; base < p.nblocks; base += warps_total * G) {
    const long long b = base + sub;
    const bool valid = b < p.nblocks;
    unsigned set = 0;
    if (valid && p.set) set = __ldg(p.set + b);
    const bool skip = (set == 0xFFFFu);
    const bool bad = !skip && set >= (unsigned)p.num_sets;
    const unsigned cset = (skip || bad) ? 0u : set;

    V v[E];
    if (valid) {
      if constexpr (KIND == 0) {
        load_i16<E>(static_cast<const int16_t*>(p.in) + b * N + lane * E, v);
      } else if constexpr (KIND == 1) {
        load_i32<E>(static_cast<const int32_t*>(p.in) + b * N + lane * E, v);
      } else {
        load_f32<E>(static_cast<const float*>(p.in) + b * N + lane * E, v);
      }
    } else {
#pragma unroll
      for (int i = 0; i < E; ++i) v[i] = V(0);
    }
    V keep[E];
#pragma unroll
    for (int i = 0; i < E; ++i) keep[i] = v[i];

    if constexpr (!INV) {
      for (int r = 0; r < rounds; ++r) {
        const int row_base = ((int)cset * rounds + r) * LOG2N;
        round_fwd<LOG2N, LOG2E, 0>(math, v, tab, row_base, lane);
        if (perm && ((p.perm_mask >> r) & 1u))
          permute<LOG2N, LOG2E, false>(v, buf, perm + ((size_t)cset * rounds + r) * N, lane);
      }
    } else {
      for (int r = rounds - 1; r >= 0; --r) {
        if (perm && ((p.perm_mask >> r) & 1u))
          permute<LOG2N, LOG2E, true>(v, buf, perm + ((size_t)cset * rounds + r) * N, lane);
        const int row_base = ((int)cset * rounds + r) * LOG2N;
        round_inv<LOG2N, LOG2E, LOG2N - 1>(math, v, tab, row_base, lane);
      }
    }

    if (skip) {
#pragma unroll
      for (int i = 0; i < E; ++i) v[i] = keep[i];
    } else if (bad) {
#pragma unroll
      for (int i = 0; i < E; ++i) v[i] = V(0);
      if (valid && lane == 0 && p.status) atomicCAS(p.status, 0, 4);
    }
    if (valid) {
      if constexpr (KIND == 0) {
        store_i32<E>(static_cast<int32_t*>(p.out) + b * N + lane * E, v);
      } else if constexpr (KIND == 1) {
        store_i16_sat<E>(static_cast<int16_t*>(p.out) + b * N + lane * E, v);
      } else {
        store_f32<E>(static_cast<float*>(p.out) + b * N + lane * E, v);
      }
    }
  }
}

}  // namespace hygt
