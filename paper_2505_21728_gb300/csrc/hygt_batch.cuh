// hygt_batch.cuh -- set-bucketed integer HyGT (sm_103a).
//
// A batch is first bucketed by transform set (counting sort of block ids;
// every bucket padded to a multiple of G blocks with id -1), so that every
// warp task is G blocks sharing one set.  The kernels then see warp-uniform
// multipliers.  Because the warps of a CTA walk consecutive tasks of the
// sorted order, a CTA's tasks span only a few sets: the CTA copies those
// sets' multipliers into shared memory once, and every lane reads them by
// broadcast.
//
// Mapping.  A block of N = 2^LOG2N values is held by a group of L = N / E
// lanes with E consecutive values per lane (element e = lane * E + i in
// register i), and every lane group holds K blocks of the same set at once:
// each multiplier loaded into a register serves K butterflies, and the K
// blocks are independent work for the scheduler.  A warp task is
// G = (32 / L) K blocks; block k of lane group g is the task's block
// k (32 / L) + g.
//   - Pass p < LOG2E pairs two registers of a lane (register butterfly).
//   - Pass p >= LOG2E pairs lane l with lane l ^ 2^(p - LOG2E): each lane
//     fetches its partner's value with __shfl_xor_sync and computes its own
//     output, y = c * own +/- s * partner.
//   - The permutation slot after a round goes through the block's region of
//     a shared-memory buffer.
//
// Register butterfly with three multiplications:
//     k   = c (a + b) + 2^(f-1)
//     y_m = (k + (s - c) b) >> f        (= (c a + s b + 2^(f-1)) >> f)
//     y_n = (k - (c + s) a) >> f        (= (c b - s a + 2^(f-1)) >> f)
// evaluated modulo 2^32, so it equals the direct formula whenever that fits
// in int32.  The inverse rotation (c, -s) uses the same entries with
// d1 = s - c and d2 = -(c + s) exchanged.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hygt_device.cuh"
#include "hygt_primary.cuh"

namespace hygt {

// Threads per CTA of the batch transform for block size 2^log2n (forward:
// KIND 0, inverse: KIND 1), measured: where a block spans several lanes the
// forward (more blocks per lane group) wants the registers of 384 threads,
// and so does the 16x16 inverse (four blocks per lane group); the inverse on
// 32-value blocks the warps of 640; otherwise 512.
//
// Other register layouts (launch-tuning choices, batch_log2e / batch_k):
// layout 1 holds a whole block in one lane (4x4, 8x8): every pass is a
// register pass, no shuffles, and a warp task's 32 K blocks share their
// multipliers by broadcast loads; layout 2 holds more values per lane with
// fewer blocks per lane group (8x8, 16x16: E = 32, K = 2) or fewer values
// with more blocks (4x4: E = 4, K = 8 / 4); layout 3 (4x4, 8x8) is layout 0
// with the forward's 8 blocks per lane group in the inverse too; layout 4
// (16x16) is layout 0 with the cross-lane passes replaced by register passes
// on the transposed block (a shared-memory transpose in the middle of each
// round, the transpose back folded into the permutation slot where there is
// one; 8x8 and 4x4 with K = 8 in both directions); layout 5 (16x16) is
// layout 4 with K = 2 (half-size warp tasks: a short batch ends with a
// smaller tail).  Their CTAs have 384 threads.
constexpr int kBatchLayouts = 6;
__host__ __device__ constexpr bool batch_layout_ok(int log2n, int lay) {
  return lay == 0 || (lay == 1 && (log2n == 4 || log2n == 6)) ||
         (lay == 2 && (log2n == 4 || log2n == 6 || log2n == 8)) ||
         (lay == 3 && (log2n == 4 || log2n == 6)) ||
         (lay == 4 && (log2n == 4 || log2n == 6 || log2n == 8)) || (lay == 5 && log2n == 8);
}
__host__ __device__ constexpr bool batch_layout_all_reg(int lay) { return lay == 4 || lay == 5; }
__host__ __device__ constexpr int batch_threads(int log2n, int kind, int lay = 0) {
  return lay != 0 ? 384
         : log2n <= 3 ? 512
         : (kind == 0 || log2n == 8) ? 384
                                     : (log2n == 5 ? 640 : 512);
}
constexpr int kBucketThreads = 512;  // threads per CTA of the bucketing kernels
constexpr int kBucketTile = 8192;    // blocks per CTA tile in the scatter pass

// Layout for block size 2^log2n: E = 2^batch_log2e values of a block per
// lane, L = N / E lanes per block (a lane group), K = batch_k blocks of the
// same set per lane group, so a warp task is (32 / L) K blocks.  K may differ
// between the directions; the schedule's group G = batch_group is a multiple
// of both task sizes, so one schedule serves the forward and the inverse.
// For 8x8 blocks E = 8 (L = 8 lanes, three cross-lane passes) with K = 8
// forward and 4 inverse: fewer multiplier bytes per block than E = 16 with
// K = 4 / 2 (measured 4-9% faster), for the same 64 value registers; for
// 16x16 blocks likewise E = 16 with K = 4 rather than E = 32 with K = 2
// (forward 16% faster), and K = 4 in the inverse too, on 384 threads (13%
// faster than K = 2 on 512, whose multiplier loads filled the L1 data pipe;
// the 8x8 inverse with K = 8 on 384 threads is 27% slower than K = 4 on
// 512); for 4x4 blocks E = 8 (two lanes) with K = 8 / 4 rather than one
// lane per block (forward 5% faster).
__host__ __device__ constexpr int batch_log2e(int log2n, int lay = 0) {
  if (lay == 1) return log2n;
  if (lay == 2) return log2n == 4 ? 2 : 5;
  if (lay == 3) return 3;
  if (lay == 4 || lay == 5) return log2n / 2;
  switch (log2n) {
    case 4: return 3;   // 4x4: 8 values per lane, 2 lanes
    case 5: return 4;
    case 6: return 3;   // 8x8: 8 values per lane, 8 lanes
    case 7: return 5;
    case 8: return 4;   // 16x16: 16 values per lane, 16 lanes
    default: return log2n;  // N <= 8: one lane per block
  }
}
__host__ __device__ constexpr int batch_k(int log2n, bool inv, int lay = 0) {
  if (lay == 1) return log2n == 4 ? (inv ? 2 : 4) : 1;
  if (lay == 2) return log2n == 4 ? (inv ? 4 : 8) : 2;
  if (lay == 3) return 8;
  if (lay == 4) return log2n == 8 ? 4 : 8;
  if (lay == 5) return 2;
  switch (log2n) {
    case 1: case 2: return 1;
    case 4: case 6: return inv ? 4 : 8;
    case 5: return inv ? 2 : 4;
    case 8: return 4;
    default: return 2;
  }
}
__host__ __device__ constexpr int batch_task_group(int log2n, bool inv, int lay = 0) {
  return (32 >> (log2n - batch_log2e(log2n, lay))) * batch_k(log2n, inv, lay);
}
__host__ __device__ constexpr int batch_group(int log2n) {
  return batch_task_group(log2n, false) > batch_task_group(log2n, true)
             ? batch_task_group(log2n, false)
             : batch_task_group(log2n, true);
}

// Workspace layout (all offsets in bytes, 16-byte aligned sections):
//   counts [nb]     int32  blocks per bucket (bucket S = skip, S + 1 = bad set)
//   starts [nb + 1] int32  first slot of each bucket (padded to G); starts[nb] = total
//   cursor [nb]     int32  scatter cursor per bucket
//   meta   [4]      int32  warp tasks (total / G), nblocks, num_sets, G
//   order  [G * tmax] int32 block id per slot, -1 for padding
struct BatchLayout {
  int nb;           // buckets = S + 2
  int group;        // G
  long long tmax;   // max warp tasks
  size_t counts, starts, cursor, meta, order, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline BatchLayout batch_layout(int num_sets, long long nblocks, int group) {
  BatchLayout L;
  L.nb = num_sets + 2;
  L.group = group;
  L.tmax = (nblocks + group - 1) / group + L.nb;
  size_t off = 0;
  L.counts = off; off = align16(off + 4 * (size_t)L.nb);
  L.starts = off; off = align16(off + 4 * (size_t)(L.nb + 1));
  L.cursor = off; off = align16(off + 4 * (size_t)L.nb);
  L.meta = off;   off = align16(off + 16);
  L.order = off;  off = align16(off + 4 * (size_t)group * (size_t)L.tmax);
  L.total = off;
  return L;
}

// ---------------------------------------------------------------- tables
// Per-set multiplier table of the batch kernels (int32 words), for block
// size 2^LOG2N, E = 2^log2e values per lane and L = N / E lanes per block:
//   for each round r, for each pass p:
//     p <  log2e: lane l's E/2 pairs (c, s - c, -(c + s)) (3 words each) in a
//                 segment of seg() words starting at l * seg();
//     p >= log2e: for each pair j, (c, s) for its m side and (c, -s) for its
//                 n side; 16-byte chunk c = 2 (j / 2) + side holds pairs
//                 j & ~1 and j | 1 of that side and is stored at chunk
//                 c + 2 (c / E);
//   then, if the plan permutes, for each round r: lane l's permutation
//   segment of perm_seg() words at l * perm_seg(): bytes [0, E) the words
//   of its elements l E + i in a block's permutation region, bytes [E, 2E)
//   the words of their gather sources perm[l E + i] (layout of the region
//   below).
// The segment strides are odd numbers of 16-byte chunks and the chunk skew
// spreads the (up to 8) lanes of a block over distinct bank groups.
// all_reg (the transposed layout, batch layout 4): every pass is stored as a
// register pass -- passes p >= log2e for a lane that holds the elements
// (i << log2e) + l of a transposed block (pairs over bit p - log2e of i) --
// and each round's permutation bytes are those of the transposing slot
// (own: the words of the lane's transposed elements; sources as above).
struct SetTableShape {
  int log2n, log2e, rounds, perms;
  bool all_reg = false;
  __host__ __device__ constexpr int n() const { return 1 << log2n; }
  __host__ __device__ constexpr int e() const { return 1 << log2e; }
  __host__ __device__ constexpr int lanes() const { return 1 << (log2n - log2e); }
  __host__ __device__ constexpr int seg() const {
    return e() >= 8 ? ((3 * e() / 2 + 3) / 4 | 1) * 4 : 3 * e() / 2;
  }
  __host__ __device__ constexpr int reg_row() const { return lanes() * seg(); }
  __host__ __device__ constexpr int lane_row() const { return 2 * n() + 4 * n() / e() - 8; }
  __host__ __device__ constexpr int perm_seg() const {
    // 2E bytes in whole 16-byte chunks, an odd number of them when a block
    // spans several lanes
    return 4 * (((2 * e() + 15) / 16) | (lanes() > 1 ? 1 : 0));
  }
  __host__ __device__ constexpr int pass_offset(int p) const {
    return all_reg ? reg_row() * p
                   : reg_row() * (p < log2e ? p : log2e) + lane_row() * (p < log2e ? 0 : p - log2e);
  }
  __host__ __device__ constexpr int round_words() const { return pass_offset(log2n); }
  __host__ __device__ constexpr int perm_offset(int r) const {
    return rounds * round_words() + r * lanes() * perm_seg();
  }
  __host__ __device__ constexpr int set_words() const {
    return rounds * round_words() + (perms ? rounds * lanes() * perm_seg() : 0);
  }
  // word of entry (c, s') of pair j on `side` in a lane-pass row
  __host__ __device__ constexpr int lane_word(int j, int side) const {
    return 4 * ((2 * (j / 2) + side) + 2 * ((2 * (j / 2) + side) / e())) + 2 * (j & 1);
  }
};

// Words per block region of the permutation buffer: N + L, so that with the
// regions of a warp task numbered k (32 / L) + g, region g starts at a bank
// offset of g L (mod 32).  Within a region, element x of the block sits at
// word L q(x) + c(x), where c is an L-colouring of the elements under which
// the L elements that one register index i covers -- the lanes' own
// elements l E + i (written in natural order) as well as their gather
// sources perm[l E + i] -- always have distinct colours.  Such a colouring
// exists for every permutation: it is a proper edge colouring with L colours
// of the L-regular bipartite multigraph joining, for every element, its
// natural group to its source group (Konig's theorem); the host finds it as
// L successive perfect matchings.  A warp's 32 lanes (GROUPS lane groups x L
// lanes) then reach 32 distinct banks in every permutation access.  q(x)
// numbers the elements of one colour in increasing order, so the words
// cover 0 .. N-1.
__host__ __device__ constexpr int perm_region_words(int log2n, int lay = 0) {
  return (1 << log2n) + (1 << (log2n - batch_log2e(log2n, lay)));
}

// ---------------------------------------------------------------- transform
struct BatchParams {
  const void* in;
  void* out;
  const int* order;      // [G * ntasks]
  const int* starts;     // [nb + 1] padded bucket starts (slots)
  const int* meta;       // tasks, nblocks, num_sets, G
  long long nblocks;
  long long tmax;        // capacity of order[] in warp tasks (bounds the task count)
  const int* ktab;       // per-set tables, [S][set_words]
  int set_words;
  const int* ktabs[kBatchLayouts];  // the same for each register layout (null: not built)
  int set_words_of[kBatchLayouts];
  unsigned perm_mask;
  int perms;
  int rounds;
  int num_sets;
  int frac_bits;
  int max_cached_sets;   // sets that fit in shared memory next to the permutation buffer
  int* status;
};

template <int LOG2N, bool INV, int LAY = 0>
struct BatchMath {
  static constexpr int N = 1 << LOG2N;
  static constexpr int LOG2E = batch_log2e(LOG2N, LAY);
  static constexpr int E = 1 << LOG2E;
  static constexpr int L = N / E;
  static constexpr int K = batch_k(LOG2N, INV, LAY);
  using Blocks = int32_t[K][E];

  template <int P>
  __device__ __forceinline__ static void bfly(Blocks& v, int jl, int c, int d1, int d2,
                                              uint32_t half, int f) {
    const int im = ((jl >> P) << (P + 1)) | (jl & ((1 << P) - 1));
    const int in = im | (1 << P);
    const uint32_t e1 = (uint32_t)(INV ? d2 : d1);
    const uint32_t e2 = (uint32_t)(INV ? d1 : d2);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t ua = (uint32_t)v[k][im], ub = (uint32_t)v[k][in];
      const uint32_t kk = (uint32_t)c * (ua + ub) + half;
      v[k][im] = (int32_t)(kk + e1 * ub) >> f;
      v[k][in] = (int32_t)(kk + e2 * ua) >> f;
    }
  }

  // Register pass p: the lane's pairs are lane * E/2 + jl; `row` holds N/2
  // entries of 3 words.  The multipliers of 4 pairs (three 16-byte loads) are
  // fetched one group ahead of their use; the empty asm statements with a
  // memory clobber keep the compiler from hoisting loads further (which
  // would cost registers the K blocks need).
  template <int P>
  __device__ __forceinline__ static void reg_pass(Blocks& v, const int* row, int lane,
                                                  uint32_t half, int f) {
    constexpr int NP = E / 2;
    constexpr SetTableShape sh{LOG2N, LOG2E, 1, 0};
    const int* base = row + lane * sh.seg();
    if constexpr (NP % 4 == 0) {
      const int4* b4 = reinterpret_cast<const int4*>(base);
      int4 na = b4[0], nb = b4[1], nc = b4[2];
#pragma unroll
      for (int q = 0; q < NP / 4; ++q) {
        const int4 a = na, b = nb, c = nc;
        if (q + 1 < NP / 4) {
          na = b4[3 * (q + 1)];
          nb = b4[3 * (q + 1) + 1];
          nc = b4[3 * (q + 1) + 2];
        }
        asm volatile("" ::: "memory");
        bfly<P>(v, 4 * q + 0, a.x, a.y, a.z, half, f);
        bfly<P>(v, 4 * q + 1, a.w, b.x, b.y, half, f);
        bfly<P>(v, 4 * q + 2, b.z, b.w, c.x, half, f);
        bfly<P>(v, 4 * q + 3, c.y, c.z, c.w, half, f);
      }
    } else {
#pragma unroll
      for (int jl = 0; jl < NP; ++jl)
        bfly<P>(v, jl, base[3 * jl], base[3 * jl + 1], base[3 * jl + 2], half, f);
    }
  }

  // Lane pass p: partner lane = lane ^ 2^(p - LOG2E).  `row` holds (c, s)
  // for the m side and (c, -s) for the n side of each pair (layout in
  // SetTableShape); this lane's E elements use pairs jbase + i of its side.
  template <int P>
  __device__ __forceinline__ static void lane_pass(Blocks& v, const int* row, int lane,
                                                   uint32_t half, int f) {
    constexpr int Q = P - LOG2E;
    constexpr int D = 1 << Q;
    const int upper = (lane >> Q) & 1;  // this lane holds the n side
    const int jbase = ((lane >> (Q + 1)) << P) + ((lane & (D - 1)) << LOG2E);
    // forward: m side (c, s), n side (c, -s); inverse: the opposite
    const int side = upper ^ (INV ? 1 : 0);
    // chunk c = jbase + i + side (i even) is stored at c + 2 (c / E);
    // c / E = jbase / E for every i of this lane
    const int skew = 2 * (jbase >> LOG2E);
    const int4* base = reinterpret_cast<const int4*>(row) + jbase + side + skew;
#pragma unroll
    for (int i = 0; i < E; i += 2) {
      const int4 cs = base[i];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int32_t p0 = __shfl_xor_sync(kFullMask, v[k][i], D);
        const int32_t p1 = __shfl_xor_sync(kFullMask, v[k][i + 1], D);
        const uint32_t u0 =
            (uint32_t)cs.x * (uint32_t)v[k][i] + (uint32_t)cs.y * (uint32_t)p0 + half;
        const uint32_t u1 =
            (uint32_t)cs.z * (uint32_t)v[k][i + 1] + (uint32_t)cs.w * (uint32_t)p1 + half;
        v[k][i] = (int32_t)u0 >> f;
        v[k][i + 1] = (int32_t)u1 >> f;
      }
    }
  }

  template <int P>
  __device__ __forceinline__ static void pass(Blocks& v, const int* rtab, int lane,
                                              uint32_t half, int f) {
    constexpr SetTableShape sh{LOG2N, LOG2E, 1, 0};
    const int* row = rtab + sh.pass_offset(P);
    if constexpr (P < LOG2E)
      reg_pass<P>(v, row, lane, half, f);
    else
      lane_pass<P>(v, row, lane, half, f);
  }

  // Pass p of the transposed layout (all passes register passes; passes
  // p >= LOG2E act on bit p - LOG2E of the register index of the transposed
  // block): passes [P0, P1) in increasing order forward, decreasing inverse.
  template <int P0, int P1, int J = 0>
  __device__ __forceinline__ static void tpasses(Blocks& v, const int* rtab, int lane,
                                                 uint32_t half, int f) {
    if constexpr (J < P1 - P0) {
      constexpr int P = INV ? P1 - 1 - J : P0 + J;
      SetTableShape sh{LOG2N, LOG2E, 1, 0};
      sh.all_reg = true;
      reg_pass<(P < LOG2E ? P : P - LOG2E)>(v, rtab + sh.pass_offset(P), lane, half, f);
      tpasses<P0, P1, J + 1>(v, rtab, lane, half, f);
    }
  }

  // All passes of one round: increasing p forward, decreasing p inverse.
  template <int J>
  __device__ __forceinline__ static void round(Blocks& v, const int* rtab, int lane,
                                               uint32_t half, int f) {
    if constexpr (J < LOG2N) {
      pass<INV ? (LOG2N - 1 - J) : J>(v, rtab, lane, half, f);
      round<J + 1>(v, rtab, lane, half, f);
    }
  }
};

template <int LOG2N, int KIND, int LAY = 0>
__device__ __forceinline__ void batch_load(const BatchParams& p, long long b, int lane,
                                           int32_t (&v)[BatchMath<LOG2N, false, LAY>::E]) {
  constexpr int N = 1 << LOG2N;
  constexpr int E = BatchMath<LOG2N, false, LAY>::E;
  if constexpr (KIND == 0)
    load_i16<E>(static_cast<const int16_t*>(p.in) + b * N + lane * E, v);
  else
    load_i32<E>(static_cast<const int32_t*>(p.in) + b * N + lane * E, v);
}

template <int LOG2N, int KIND, int LAY = 0>
__device__ __forceinline__ void batch_store(const BatchParams& p, long long b, int lane,
                                            const int32_t (&v)[BatchMath<LOG2N, false, LAY>::E]) {
  constexpr int N = 1 << LOG2N;
  constexpr int E = BatchMath<LOG2N, false, LAY>::E;
  if constexpr (KIND == 0)
    store_i32<E>(static_cast<int32_t*>(p.out) + b * N + lane * E, v);
  else
    store_i16_sat<E>(static_cast<int16_t*>(p.out) + b * N + lane * E, v);
}

// A lane's permutation segment (see SetTableShape): 2E bytes in registers.
// OWN_ID (a block per lane, E >= 16): the own words are the identity, so
// only the E source bytes (the second half of the segment) are loaded.
template <int E, bool OWN_ID = false>
struct PermBytes {
  static constexpr int W = OWN_ID ? E / 4 : (2 * E + 3) / 4;
  uint32_t w[W < 4 ? W : (W + 3) / 4 * 4];
  __device__ __forceinline__ void load(const int* seg) {
    if constexpr (OWN_ID) seg += E / 4;
    if constexpr (W % 4 == 0) {
#pragma unroll
      for (int q = 0; q < W / 4; ++q) {
        const int4 t = reinterpret_cast<const int4*>(seg)[q];
        w[4 * q] = t.x; w[4 * q + 1] = t.y; w[4 * q + 2] = t.z; w[4 * q + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < W; ++q) w[q] = (uint32_t)seg[q];
    }
  }
  // word of this lane's element i in the region / of the element's gather source
  __device__ __forceinline__ int own(int i) const {
    if constexpr (OWN_ID) return i;
    return (w[i >> 2] >> (8 * (i & 3))) & 0xFF;
  }
  __device__ __forceinline__ int src(int i) const {
    constexpr int B = OWN_ID ? 0 : E;
    return (w[(B + i) >> 2] >> (8 * ((B + i) & 3))) & 0xFF;
  }
};

// Blocks of a lane group per pass through the permutation buffer: the
// buffer holds GROUPS x batch_perm_k block regions per warp, and a lane
// group's K blocks go through it in K / batch_perm_k passes.  Measured: one
// pass is fastest where the kernel's shared memory leaves enough L1 (fewer
// passes, more independent loads in flight); the 16x16 inverse runs one
// block per pass (a 16x16 region is 1 KB; measured 1-3% faster with two
// blocks per lane group), while two passes cost 4x4 blocks 8-10%.
__host__ __device__ constexpr int batch_perm_k(int log2n, int kind, int lay = 0) {
  return (log2n == 8 && kind == 1) ? 1 : batch_k(log2n, kind == 1, lay);
}
__host__ __device__ constexpr int perm_buf_words(int log2n, int kind, int lay = 0) {
  return (32 >> (log2n - batch_log2e(log2n, lay))) * batch_perm_k(log2n, kind, lay) *
         perm_region_words(log2n, lay);
}

// Whether a lane's permutation bytes skip the identity own words.
__host__ __device__ constexpr bool perm_own_id(int log2n, int lay) {
  return log2n == batch_log2e(log2n, lay) && (1 << log2n) >= 16;
}

// The permutation slot of one round for the K blocks of this lane group
// (regions of the warp's buffer `pbuf`): forward, the gather
// v'[e] = v[perm[e]]; inverse, its undoing v'[perm[e]] = v[e].
template <int LOG2N, int KIND, int LAY = 0>
__device__ __forceinline__ void perm_slot(
    int32_t (&v)[BatchMath<LOG2N, KIND == 1, LAY>::K][BatchMath<LOG2N, KIND == 1, LAY>::E],
    const PermBytes<BatchMath<LOG2N, KIND == 1, LAY>::E, perm_own_id(LOG2N, LAY)>& pb,
    int32_t* pbuf, int grp) {
  using M = BatchMath<LOG2N, KIND == 1, LAY>;
  constexpr int E = M::E;
  constexpr int K = M::K;
  constexpr int GROUPS = 32 / M::L;
  constexpr int RW = perm_region_words(LOG2N, LAY);
  constexpr int KP = batch_perm_k(LOG2N, KIND, LAY);
  static_assert(K % KP == 0, "permutation passes must cover the lane group's blocks");
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += KP) {
#pragma unroll
    for (int kk = 0; kk < KP; ++kk) {
      int32_t* region = pbuf + (kk * GROUPS + grp) * RW;
#pragma unroll
      for (int i = 0; i < E; ++i) region[KIND == 1 ? pb.src(i) : pb.own(i)] = v[k0 + kk][i];
    }
    __syncwarp();
#pragma unroll
    for (int kk = 0; kk < KP; ++kk) {
      const int32_t* region = pbuf + (kk * GROUPS + grp) * RW;
#pragma unroll
      for (int i = 0; i < E; ++i) v[k0 + kk][i] = region[KIND == 1 ? pb.own(i) : pb.src(i)];
    }
    __syncwarp();
  }
}

// Transposes of the K blocks of this lane group between the natural layout
// (lane l holds elements l E + i) and the transposed one (lane l holds
// elements i E + l; E = L), through the blocks' regions of the permutation
// buffer.  Word of element x = a E + 4 q + r (q: 16-byte chunk of lane a's
// row): a E + 4 (q ^ ((a E / 32) & (E / 4 - 1))) + r -- rows a and a + 32 / E
// start on the same bank, so the key a E / 32 gives them different chunk
// orders: a natural row is written or read as E / 4 16-byte chunks and a
// transposed column as E words, both without bank conflicts.
template <int LOG2N, int KIND, int LAY, bool TO_T>
__device__ __forceinline__ void tr_slot(
    int32_t (&v)[BatchMath<LOG2N, KIND == 1, LAY>::K][BatchMath<LOG2N, KIND == 1, LAY>::E],
    int32_t* pbuf, int grp, int lane) {
  using M = BatchMath<LOG2N, KIND == 1, LAY>;
  constexpr int E = M::E;
  constexpr int K = M::K;
  constexpr int GROUPS = 32 / M::L;
  constexpr int RW = perm_region_words(LOG2N, LAY);
  constexpr int KP = batch_perm_k(LOG2N, KIND, LAY);
  constexpr int QM = E / 4 - 1;
  static_assert(M::L == E && E % 4 == 0, "square blocks of whole chunks");
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += KP) {
#pragma unroll
    for (int kk = 0; kk < KP; ++kk) {
      int32_t* region = pbuf + (kk * GROUPS + grp) * RW;
      if constexpr (TO_T) {  // natural rows out
#pragma unroll
        for (int q = 0; q < E / 4; ++q)
          *reinterpret_cast<int4*>(region + lane * E + 4 * (q ^ ((lane * E / 32) & QM))) =
              make_int4(v[k0 + kk][4 * q], v[k0 + kk][4 * q + 1], v[k0 + kk][4 * q + 2],
                        v[k0 + kk][4 * q + 3]);
      } else {  // transposed columns out
#pragma unroll
        for (int i = 0; i < E; ++i)
          region[i * E + 4 * ((lane >> 2) ^ ((i * E / 32) & QM)) + (lane & 3)] = v[k0 + kk][i];
      }
    }
    __syncwarp();
#pragma unroll
    for (int kk = 0; kk < KP; ++kk) {
      const int32_t* region = pbuf + (kk * GROUPS + grp) * RW;
      if constexpr (TO_T) {  // transposed columns in
#pragma unroll
        for (int i = 0; i < E; ++i)
          v[k0 + kk][i] = region[i * E + 4 * ((lane >> 2) ^ ((i * E / 32) & QM)) + (lane & 3)];
      } else {  // natural rows in
#pragma unroll
        for (int q = 0; q < E / 4; ++q) {
          const int4 t =
              *reinterpret_cast<const int4*>(region + lane * E + 4 * (q ^ ((lane * E / 32) & QM)));
          v[k0 + kk][4 * q] = t.x;
          v[k0 + kk][4 * q + 1] = t.y;
          v[k0 + kk][4 * q + 2] = t.z;
          v[k0 + kk][4 * q + 3] = t.w;
        }
      }
    }
    __syncwarp();
  }
}

// Bucket of a slot: the largest k with starts[k] <= slot (empty buckets share
// their start with the next one, so the largest is non-empty).
__device__ __forceinline__ int bucket_of_slot(const int* starts, int num_sets, int slot) {
  int lo = 0, hi = num_sets + 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(starts + mid) <= slot) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- staging
// For N = 32 and 64 the kernels' input (int16 blocks forward, int32
// coefficients inverse) is copied into shared memory with cp.async one
// task ahead (and the block ids two tasks ahead), so the global-memory
// latency is off the critical path.  Stage layout, per warp: piece j (CH
// bytes) of lane l of lane group g in block k of the task at
// ((k J + j) 32 + g L + l) CH -- the reads of one (k, j) step are 32
// consecutive pieces (no bank conflicts) while the copies walk the task's
// blocks in global order (coalesced).
__host__ __device__ constexpr bool batch_staged(int log2n, int kind) {
  // measured: a gain where a block spans several lanes (N = 32, 64); larger
  // blocks leave no room for the stage next to the permutation buffer
  return (kind == 0 || kind == 1) && (log2n == 5 || log2n == 6);
}

template <int LOG2N, int KIND, int LAY = 0>
struct BatchStage {
  static constexpr int N = 1 << LOG2N;
  static constexpr int IB = KIND == 0 ? 2 : 4;  // input bytes per value
  static constexpr int E = 1 << batch_log2e(LOG2N, LAY);
  static constexpr int L = N / E;
  static constexpr int K = batch_k(LOG2N, KIND == 1, LAY);
  static constexpr int GROUPS = 32 / L;
  static constexpr int G = GROUPS * K;
  static constexpr int LANE_BYTES = E * IB;
  static constexpr int CH = LANE_BYTES < 16 ? LANE_BYTES : 16;  // bytes per copy
  static constexpr int J = LANE_BYTES / CH;                     // copies per lane and block
  static constexpr int CPB = L * J;                             // copies per block
  static constexpr int PER_LANE = K * J;                        // copies per lane and task
  static constexpr int BYTES = G * N * IB;
  static constexpr int IDS_BYTES = 2 * G * 4;                   // block ids of two tasks
  static_assert(G % 4 == 0 && BYTES % 16 == 0, "stage alignment");
};

// Shared memory of one warp: permutation buffer, then (staged kernels) the
// stage and the block ids, or (bulk-staged kernels) the stage and the
// warp's mbarrier.
template <int LOG2N, int KIND, bool STAGED = batch_staged(LOG2N, KIND), bool BULK = false,
          int LAY = 0>
__host__ __device__ constexpr int batch_warp_bytes() {
  return perm_buf_words(LOG2N, KIND, LAY) * 4 +
         (STAGED ? BatchStage<LOG2N, KIND, LAY>::BYTES + BatchStage<LOG2N, KIND, LAY>::IDS_BYTES : 0) +
         (BULK ? BatchStage<LOG2N, KIND, LAY>::BYTES + 16 : 0);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------- bulk stage
// Bulk-staged kernels: each warp task's blocks are copied into the warp's
// stage with one cp.async.bulk per block (issued by the lane that owns the
// slot; the copy engine moves the bytes), completing on the warp's
// mbarrier; a task is copied while the previous one computes.  Stage layout:
// slot s of the task at s * N * IB bytes.
__device__ __forceinline__ uint64_t batch_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of the mbarrier at shared address `bar`, at most
// about one second; false on timeout.
__device__ __forceinline__ bool batch_mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = batch_ns();
  for (uint32_t it = 0;; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && batch_ns() - t0 > 1000000000ull) return false;
  }
}

// Issue the copies of one task: slots l + 32 j of the task (j < GJ) with
// block ids ids[j] (-1: none).  Lane 0 announces the task's bytes on the
// barrier first.
template <int LOG2N, int KIND, int GJ, int LAY = 0>
__device__ __forceinline__ void bulk_issue(const BatchParams& p, const int (&ids)[GJ],
                                           char* stage, uint32_t bar, int lane32) {
  using St = BatchStage<LOG2N, KIND, LAY>;
  constexpr uint32_t BB = St::N * St::IB;
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < GJ; ++j)
    cnt += __popc(__ballot_sync(kFullMask, ids[j] >= 0 && (long long)ids[j] < p.nblocks));
  if (lane32 == 0)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((uint32_t)cnt * BB)
                 : "memory");
  // the stage was last read by this warp's generic loads (ordered by the
  // caller's __syncwarp); order them before the copy engine's writes
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
#pragma unroll
  for (int j = 0; j < GJ; ++j) {
    const int slot = lane32 + 32 * j;
    if (slot < St::G && ids[j] >= 0 && (long long)ids[j] < p.nblocks) {
      const char* src = static_cast<const char*>(p.in) + (long long)ids[j] * BB;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
          "[%3];" ::"r"(smem_u32(stage + slot * BB)),
          "l"(src), "r"(BB), "r"(bar)
          : "memory");
    }
  }
}

// This lane's E values of the block in stage slot `slot`.
template <int LOG2N, int KIND, int LAY = 0>
__device__ __forceinline__ void bulk_read(const char* stage, int slot, int lane,
                                          int32_t (&v)[BatchStage<LOG2N, KIND, LAY>::E]) {
  using St = BatchStage<LOG2N, KIND, LAY>;
  constexpr int LB = St::E * St::IB;  // bytes of one lane
  const char* src = stage + slot * (St::N * St::IB) + lane * LB;
#pragma unroll
  for (int q = 0; q < LB / 16; ++q) {
    const uint4 t = *reinterpret_cast<const uint4*>(src + 16 * q);
    const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      if constexpr (St::IB == 2) {
        v[q * 8 + 2 * x] = (int32_t)(int16_t)(w[x] & 0xffffu);
        v[q * 8 + 2 * x + 1] = (int32_t)w[x] >> 16;
      } else {
        v[q * 4 + x] = (int32_t)w[x];
      }
    }
  }
}

// Asynchronous global -> shared copy of BYTES (4, 8 or 16); zero-filled
// without reading when !valid.
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src, bool valid) {
  const int n = valid ? BYTES : 0;
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src),
                 "n"(BYTES), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Copy the G block ids of task t into `ids` (16-byte pieces).
template <int G>
__device__ __forceinline__ void stage_order(const BatchParams& p, long long t, int* ids,
                                            int lane32) {
  if (lane32 < G / 4)
    cp_async<16>(smem_u32(ids + 4 * lane32), p.order + t * G + 4 * lane32, true);
}

// Copy the input blocks listed in `ids` into the stage.
template <int LOG2N, int KIND, int LAY = 0>
__device__ __forceinline__ void stage_blocks(const BatchParams& p, const int* ids, char* stage,
                                             int lane32) {
  using St = BatchStage<LOG2N, KIND, LAY>;
  const char* in = static_cast<const char*>(p.in);
  const uint32_t sbase = smem_u32(stage);
#pragma unroll
  for (int u = 0; u < St::PER_LANE; ++u) {
    const int c = lane32 + 32 * u;
    const int s = c / St::CPB, q = c % St::CPB;
    const int b = ids[s];
    const bool valid = b >= 0 && (long long)b < p.nblocks;
    const int k = s / St::GROUPS, g = s % St::GROUPS;
    const int l = q / St::J, j = q % St::J;
    const uint32_t dst = sbase + (uint32_t)(((k * St::J + j) * 32 + g * St::L + l) * St::CH);
    const char* src = valid ? in + ((long long)b * St::N * St::IB + q * St::CH) : in;
    cp_async<St::CH>(dst, src, valid);
  }
}

// This lane's E values of block k of the staged task.
template <int LOG2N, int KIND, int LAY = 0>
__device__ __forceinline__ void stage_read(const char* stage, int k, int lane32,
                                           int32_t (&v)[BatchStage<LOG2N, KIND, LAY>::E]) {
  using St = BatchStage<LOG2N, KIND, LAY>;
  constexpr int VPC = St::CH / St::IB;  // values per copy
#pragma unroll
  for (int j = 0; j < St::J; ++j) {
    const char* src = stage + ((k * St::J + j) * 32 + lane32) * St::CH;
    uint32_t w[St::CH / 4];
    if constexpr (St::CH == 16) {
      const uint4 t = *reinterpret_cast<const uint4*>(src);
      w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
    } else if constexpr (St::CH == 8) {
      const uint2 t = *reinterpret_cast<const uint2*>(src);
      w[0] = t.x; w[1] = t.y;
    } else {
      w[0] = *reinterpret_cast<const uint32_t*>(src);
    }
#pragma unroll
    for (int x = 0; x < VPC; ++x) {
      if constexpr (St::IB == 2)
        v[j * VPC + x] = (x & 1) ? (int32_t)w[x / 2] >> 16 : (int32_t)(int16_t)(w[x / 2] & 0xffffu);
      else
        v[j * VPC + x] = (int32_t)w[x];
    }
  }
}

// ---------------------------------------------------------------- primary
// The integer DCT-II primary of the secondary-transform pipeline (Sec. VI)
// for 4x4 (N = 16) and 8x8 (N = 64) blocks, whose secondary HyGT covers every
// coefficient.  In the lane-group layout a lane holds RPL = E / M whole rows
// of its block (row l RPL + q in registers q M .. q M + M - 1); the row
// stage runs in registers, the column stage after a transpose through the
// block's region of the permutation buffer (word of (row r, column c):
// r S + c; S = 9 for 8x8 spreads a warp's accesses over the 32 banks), after
// which a lane holds RPL whole columns.
template <int LOG2N>
struct PrimaryShape {
  static constexpr int M = LOG2N == 4 ? 4 : 8;
  static constexpr int E = 1 << batch_log2e(LOG2N);
  static constexpr int RPL = E / M;
  static constexpr int S = M == 8 ? 9 : 4;
  static_assert(LOG2N == 4 || LOG2N == 6, "primary for 4x4 and 8x8 blocks");
  static_assert(S * (M - 1) + M <= perm_region_words(LOG2N), "region too small");
};

template <int LOG2N>
__device__ __forceinline__ void prim_rows_to_cols(const int32_t* src, int32_t* dst,
                                                  int32_t* region, int l) {
  using P = PrimaryShape<LOG2N>;
#pragma unroll
  for (int q = 0; q < P::RPL; ++q)
#pragma unroll
    for (int c = 0; c < P::M; ++c) region[(l * P::RPL + q) * P::S + c] = src[q * P::M + c];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < P::RPL; ++q)
#pragma unroll
    for (int r = 0; r < P::M; ++r) dst[q * P::M + r] = region[r * P::S + l * P::RPL + q];
  __syncwarp();
}

template <int LOG2N>
__device__ __forceinline__ void prim_cols_to_rows(const int32_t* src, int32_t* dst,
                                                  int32_t* region, int l) {
  using P = PrimaryShape<LOG2N>;
#pragma unroll
  for (int q = 0; q < P::RPL; ++q)
#pragma unroll
    for (int r = 0; r < P::M; ++r) region[r * P::S + l * P::RPL + q] = src[q * P::M + r];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < P::RPL; ++q)
#pragma unroll
    for (int c = 0; c < P::M; ++c) dst[q * P::M + c] = region[(l * P::RPL + q) * P::S + c];
  __syncwarp();
}

// Forward primary of the K blocks of a lane group: rows, then columns.
// Inverse: columns, then rows, with C transposed.  `pbuf` is the warp's
// permutation buffer (one region per block of the lane group).
template <int LOG2N, int KIND>
__device__ __forceinline__ void batch_primary(
    int32_t (&v)[BatchMath<LOG2N, KIND == 1>::K][BatchMath<LOG2N, KIND == 1>::E], int32_t* pbuf,
    int grp, int lane) {
  using P = PrimaryShape<LOG2N>;
  using Mth = BatchMath<LOG2N, KIND == 1>;
  constexpr int E = Mth::E, K = Mth::K, GROUPS = 32 / Mth::L;
  constexpr int RW = perm_region_words(LOG2N);
  constexpr bool INV = KIND == 1;
  static_assert(batch_perm_k(LOG2N, KIND) == K, "one buffer region per block");
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int32_t* region = pbuf + (k * GROUPS + grp) * RW;
    int32_t t[E], u[E];
    if (!INV) {
#pragma unroll
      for (int q = 0; q < P::RPL; ++q) dct_stage<P::M, false>(v[k] + q * P::M, t + q * P::M);
      prim_rows_to_cols<LOG2N>(t, u, region, lane);
#pragma unroll
      for (int q = 0; q < P::RPL; ++q) dct_stage<P::M, false>(u + q * P::M, t + q * P::M);
      prim_cols_to_rows<LOG2N>(t, v[k], region, lane);
    } else {
      prim_rows_to_cols<LOG2N>(v[k], u, region, lane);
#pragma unroll
      for (int q = 0; q < P::RPL; ++q) dct_stage<P::M, true>(u + q * P::M, t + q * P::M);
      prim_cols_to_rows<LOG2N>(t, u, region, lane);
#pragma unroll
      for (int q = 0; q < P::RPL; ++q) dct_stage<P::M, true>(u + q * P::M, v[k] + q * P::M);
    }
  }
}

// The tasks [t0, t1) of one warp.  `cache` holds the tables of sets
// [set_lo, set_lo + cached count) when CACHED, else tables are read from
// global memory.  `pbuf` is the warp's shared memory: G block regions of
// perm_region_words(LOG2N) words (the permutation buffer), then for staged
// kernels (STAGED: the input copied into shared memory one task ahead) the
// stage and the block ids (batch_warp_bytes in all).
template <int LOG2N, int KIND, bool CACHED, bool STAGED, bool PRIM = false, bool PF = false,
          bool BULK = false, int LAY = 0>
__device__ __forceinline__ void batch_tasks(const BatchParams& p, long long t0, long long t1,
                                            const int* cache, int set_lo, int32_t* pbuf) {
  using M = BatchMath<LOG2N, KIND == 1, LAY>;
  constexpr int E = M::E;
  constexpr int L = M::L;
  constexpr int K = M::K;
  constexpr int GROUPS = 32 / L;
  constexpr int G = GROUPS * K;
  constexpr int RW = perm_region_words(LOG2N, LAY);
  constexpr bool INV = (KIND == 1);
  static_assert(!(STAGED && BULK), "one staging scheme at a time");
  static_assert(!(BULK && LAY != 0), "the bulk stage reads a block with several lanes");
  static_assert(!(PRIM && LAY != 0), "the fused primary runs in the lane-group layout");
  static_assert(batch_group(LOG2N) % G == 0, "the schedule group must hold whole tasks");
  static_assert(!BULK || (LOG2N >= 4 && G == BatchStage<LOG2N, KIND, LAY>::G),
                "bulk copies of whole blocks need N * input bytes >= 16");
  const int lane32 = threadIdx.x & 31;
  const int lane = lane32 % L;
  const int grp = lane32 / L;
  const uint32_t half = 1u << (p.frac_bits - 1);
  const int f = p.frac_bits;
  const int R = p.rounds;
  const int S = p.num_sets;
  SetTableShape sh{LOG2N, M::LOG2E, R, p.perms};
  sh.all_reg = batch_layout_all_reg(LAY);
  const int rw = sh.round_words();

  char* stage = reinterpret_cast<char*>(pbuf + perm_buf_words(LOG2N, KIND, LAY));
  int* ids = reinterpret_cast<int*>(stage + BatchStage<LOG2N, KIND, LAY>::BYTES);  // [2][G]
  if constexpr (STAGED) {
    if (t0 >= t1) return;
    // prologue: ids of the first task, then its blocks and the next task's ids
    stage_order<G>(p, t0, ids + (t0 & 1) * G, lane32);
    cp_async_wait_all();
    __syncwarp();
    if (t0 + 1 < t1) stage_order<G>(p, t0 + 1, ids + ((t0 + 1) & 1) * G, lane32);
    stage_blocks<LOG2N, KIND, LAY>(p, ids + (t0 & 1) * G, stage, lane32);
    cp_async_commit();
  }

  // bulk stage: the task's block ids in registers (slot l + 32 j in lane l),
  // this task's and the next one's
  constexpr int GJ = (G + 31) / 32;
  char* bstage = reinterpret_cast<char*>(pbuf + perm_buf_words(LOG2N, KIND, LAY));
  const uint32_t bbar = smem_u32(bstage + BatchStage<LOG2N, KIND, LAY>::BYTES);
  uint32_t bphase = 0;
  int ids_cur[GJ], ids_next[GJ];
  if constexpr (BULK) {
    if (t0 >= t1) return;
    if (lane32 == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bbar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < GJ; ++j) {
      const int sl = lane32 + 32 * j;
      ids_cur[j] = sl < G ? __ldg(p.order + t0 * G + sl) : -1;
      ids_next[j] = (sl < G && t0 + 1 < t1) ? __ldg(p.order + (t0 + 1) * G + sl) : -1;
    }
    bulk_issue<LOG2N, KIND, GJ, LAY>(p, ids_cur, bstage, bbar, lane32);
  }

  int bucket = 0, bucket_end = 0;
  for (long long t = t0; t < t1; ++t) {
    const int slot = (int)(t * G);
    if (slot >= bucket_end) {  // warp-uniform
      bucket = bucket_of_slot(p.starts, S, slot);
      bucket_end = __ldg(p.starts + bucket + 1);
    }
    int b[K];
    bool active[K];
    int32_t v[K][E];
    if constexpr (BULK) {
      // every lane observes the phase (visibility of the copied bytes); the
      // decision to give up is warp-uniform
      if (!__all_sync(kFullMask, batch_mbar_wait(bbar, bphase))) {
        if (lane32 == 0 && p.status) atomicCAS(p.status, 0, 2);
        batch_mbar_wait(bbar, bphase);  // bounded wait for the copies in flight
        return;
      }
      bphase ^= 1u;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int sl = k * GROUPS + grp;  // sl / 32 == (k * GROUPS) / 32: GROUPS divides 32
        b[k] = __shfl_sync(kFullMask, ids_cur[(k * GROUPS) >> 5], sl & 31);
        active[k] = b[k] >= 0 && b[k] < p.nblocks;
        bulk_read<LOG2N, KIND, LAY>(bstage, sl, lane, v[k]);
      }
      __syncwarp();
      if (t + 1 < t1) {
#pragma unroll
        for (int j = 0; j < GJ; ++j) {
          ids_cur[j] = ids_next[j];
          const int sl = lane32 + 32 * j;
          ids_next[j] = (sl < G && t + 2 < t1) ? __ldg(p.order + (t + 2) * G + sl) : -1;
        }
        bulk_issue<LOG2N, KIND, GJ, LAY>(p, ids_cur, bstage, bbar, lane32);
      }
    } else if constexpr (STAGED) {
      cp_async_wait_all();
      __syncwarp();
#pragma unroll
      for (int k = 0; k < K; ++k) {
        b[k] = ids[(t & 1) * G + k * GROUPS + grp];
        active[k] = b[k] >= 0 && b[k] < p.nblocks;
        stage_read<LOG2N, KIND, LAY>(stage, k, lane32, v[k]);  // zero-filled when inactive
      }
      __syncwarp();
      if (t + 1 < t1) {  // next task's blocks, and the ids of the one after
        if (t + 2 < t1) stage_order<G>(p, t + 2, ids + (t & 1) * G, lane32);
        stage_blocks<LOG2N, KIND, LAY>(p, ids + ((t + 1) & 1) * G, stage, lane32);
      }
      cp_async_commit();
    } else {
      if constexpr (PF) {
        // pull the next task's blocks into L2 while this one computes: each
        // lane asks for the 128-byte lines of its own E values of each block
        if (t + 1 < t1) {
          constexpr int LB = E * (KIND == 0 ? 2 : 4);
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int nbk = __ldg(p.order + slot + G + k * GROUPS + grp);
            if (nbk >= 0 && nbk < p.nblocks) {
              const char* a = static_cast<const char*>(p.in) +
                              ((long long)nbk * (1 << LOG2N) + lane * E) * (KIND == 0 ? 2 : 4);
#pragma unroll
              for (int o = 0; o < LB; o += 128)
                asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a + o));
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        b[k] = __ldg(p.order + slot + k * GROUPS + grp);
        active[k] = b[k] >= 0 && b[k] < p.nblocks;
        if (active[k]) {
          batch_load<LOG2N, KIND, LAY>(p, b[k], lane, v[k]);
        } else {
#pragma unroll
          for (int i = 0; i < E; ++i) v[k][i] = 0;
        }
      }
    }
    if constexpr (PRIM && !INV) {  // primary first (also for the skip bucket)
      if (bucket != S + 1) batch_primary<LOG2N, KIND>(v, pbuf, grp, lane);
    }
    if (bucket < S) {
      const int* stab = CACHED ? cache + (size_t)(bucket - set_lo) * p.set_words
                               : p.ktab + (size_t)bucket * p.set_words;
      for (int rr = 0; rr < R; ++rr) {
        const int r = INV ? (R - 1 - rr) : rr;
        const bool has_perm = p.perms && ((p.perm_mask >> r) & 1u);
        PermBytes<E, perm_own_id(LOG2N, LAY)> pb;
        if (has_perm) pb.load(stab + sh.perm_offset(r) + lane * sh.perm_seg());
        if constexpr (batch_layout_all_reg(LAY)) {
          // passes 0 .. LOG2E-1 on the natural block, the rest on the
          // transposed one; the slot's gather reads the transposed block
          const int* rt = stab + r * rw;
          constexpr int LE = M::LOG2E;
          if (!INV) {
            M::template tpasses<0, LE>(v, rt, lane, half, f);
            tr_slot<LOG2N, KIND, LAY, true>(v, pbuf, grp, lane);
            M::template tpasses<LE, LOG2N>(v, rt, lane, half, f);
            if (has_perm)
              perm_slot<LOG2N, KIND, LAY>(v, pb, pbuf, grp);  // gather of slot r, transposing back
            else
              tr_slot<LOG2N, KIND, LAY, false>(v, pbuf, grp, lane);
          } else {
            if (has_perm)
              perm_slot<LOG2N, KIND, LAY>(v, pb, pbuf, grp);  // undo slot r's gather, transposing
            else
              tr_slot<LOG2N, KIND, LAY, true>(v, pbuf, grp, lane);
            M::template tpasses<LE, LOG2N>(v, rt, lane, half, f);
            tr_slot<LOG2N, KIND, LAY, false>(v, pbuf, grp, lane);
            M::template tpasses<0, LE>(v, rt, lane, half, f);
          }
        } else {
          if (INV && has_perm) perm_slot<LOG2N, KIND, LAY>(v, pb, pbuf, grp);  // undo slot r's gather
          M::template round<0>(v, stab + r * rw, lane, half, f);
          if (!INV && has_perm) perm_slot<LOG2N, KIND, LAY>(v, pb, pbuf, grp);  // gather of slot r
        }
      }
    } else if (bucket == S + 1) {  // bad set index: zeros, status
#pragma unroll
      for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int i = 0; i < E; ++i) v[k][i] = 0;
        if (active[k] && lane == 0 && p.status) atomicCAS(p.status, 0, 4);
      }
    }
    if constexpr (PRIM && INV) {  // inverse primary last
      if (bucket != S + 1) batch_primary<LOG2N, KIND>(v, pbuf, grp, lane);
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (active[k]) batch_store<LOG2N, KIND, LAY>(p, b[k], lane, v[k]);
  }
  if constexpr (STAGED) cp_async_wait_all();
}

// One CTA's share of a bucketed batch: CTA `cta` of `ncta` walks a contiguous
// range of warp tasks.  `smem` is the dynamic shared memory: the cached set
// tables (max_cached_sets x set_words) followed by batch_warp_bytes per warp.
// KIND 0: int16 -> int32 forward; KIND 1: int32 -> int16 inverse.
template <int LOG2N, int KIND, bool STAGED = batch_staged(LOG2N, KIND), bool PRIM = false,
          bool PF = false, bool BULK = false, int LAY = 0>
__device__ __forceinline__ void batch_cta(const BatchParams& p, long long cta, long long ncta,
                                          int32_t* smem) {
  constexpr int GS = batch_group(LOG2N);                      // schedule group
  constexpr int G = batch_task_group(LOG2N, KIND == 1, LAY);  // this kernel's task size

  // The schedule must have been built for this block count, set count and G.
  if (p.meta[1] != (int)p.nblocks || p.meta[2] != p.num_sets || p.meta[3] != GS) {
    if (threadIdx.x == 0 && cta == 0 && p.status) atomicCAS(p.status, 0, 1);
    return;
  }
  const long long ntasks = max(0LL, min((long long)p.meta[0], p.tmax)) * (GS / G);
  const int wpc = blockDim.x >> 5;
  const long long warps_total = ncta * wpc;
  const long long chunk = (ntasks + warps_total - 1) / warps_total;
  const int warp = threadIdx.x >> 5;
  const long long gw = cta * wpc + warp;
  const long long t0 = min(ntasks, gw * chunk);
  const long long t1 = min(ntasks, t0 + chunk);

  // Sets spanned by this CTA's tasks (consecutive in the sorted order).
  const long long c0 = min(ntasks, cta * wpc * chunk);
  const long long c1 = min(ntasks, c0 + (long long)wpc * chunk);
  int set_lo = 0, ncache = 0;
  if (c1 > c0) {
    const int bk_lo = bucket_of_slot(p.starts, p.num_sets, (int)(c0 * G));
    const int bk_hi = bucket_of_slot(p.starts, p.num_sets, (int)(c1 * G - 1));
    set_lo = min(bk_lo, p.num_sets);
    const int set_hi = min(bk_hi, p.num_sets - 1);
    ncache = set_hi >= set_lo ? set_hi - set_lo + 1 : 0;
  }
  const bool cached = ncache <= p.max_cached_sets;
  int32_t* cache = smem;
  int32_t* pbuf = smem + (size_t)p.max_cached_sets * p.set_words;
  if (cached && ncache > 0) {
    const int4* src = reinterpret_cast<const int4*>(p.ktab + (size_t)set_lo * p.set_words);
    int4* dst = reinterpret_cast<int4*>(cache);
    const int n4 = ncache * p.set_words / 4;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();

  int32_t* wbuf =
      pbuf + (size_t)warp * (batch_warp_bytes<LOG2N, KIND, STAGED, BULK, LAY>() / 4);
  if (cached)
    batch_tasks<LOG2N, KIND, true, STAGED, PRIM, PF, BULK, LAY>(p, t0, t1, cache, set_lo, wbuf);
  else
    batch_tasks<LOG2N, KIND, false, STAGED, PRIM, PF, BULK, LAY>(p, t0, t1, cache, set_lo, wbuf);
}

// Dynamic shared memory of batch_cta for block size 2^LOG2N without the set
// tables: batch_warp_bytes per warp.
template <int LOG2N, int KIND, bool STAGED = batch_staged(LOG2N, KIND), bool BULK = false,
          int LAY = 0>
__host__ __device__ inline size_t batch_pbuf_bytes(int threads) {
  return (size_t)(threads / 32) * batch_warp_bytes<LOG2N, KIND, STAGED, BULK, LAY>();
}

// The kernel may be launched with fewer threads than batch_threads (a
// multiple of 32): the launch tuning picks the warps per CTA.
template <int LOG2N, int KIND, bool STAGED, bool PRIM = false, bool PF = false,
          bool BULK = false, int LAY = 0>
__global__ void __launch_bounds__(batch_threads(LOG2N, KIND, LAY), 1)
    hygt_batch_kernel(BatchParams p) {
  extern __shared__ __align__(16) int32_t bsmem[];
  batch_cta<LOG2N, KIND, STAGED, PRIM, PF, BULK, LAY>(p, blockIdx.x, gridDim.x, bsmem);
}

// Launch tuning of the bucketed kernels (one per plan and direction): warps
// per CTA (0: batch_threads / 32), CTAs per SM (0: as many as fit), and
// how the next task's input is fetched ahead (-1: the measured default
// batch_staged; 0: not at all; 1: copied into shared memory one task ahead;
// 2: prefetched into L2 one task ahead; 3: copied into shared memory one
// task ahead by one bulk copy per block; 1, 2 and 3 for N >= 16), and the
// register layout (0: lane groups; 1: one lane per block, 4x4 and 8x8
// blocks, stages 0 to 2).
struct BatchTune {
  int warps = 0;
  int ctas_per_sm = 0;
  int stage = -1;
  int layout = 0;
};

// Set tables a CTA keeps in shared memory: as many as its share of the
// sorted order usually spans (a CTA that spans more reads the tables from
// global memory), and no more -- shared memory not taken stays L1 cache,
// which the kernels' global loads depend on.
__host__ inline int batch_cached_sets(size_t max_smem, size_t pbuf, size_t set_bytes,
                                      int num_sets, int ctas) {
  long long cap = 2 + (num_sets + ctas - 1) / (ctas > 0 ? ctas : 1);
  if (cap < 4) cap = 4;
  if (cap > 64) cap = 64;
  long long fit = max_smem > pbuf ? (long long)((max_smem - pbuf) / set_bytes) : 0;
  return (int)(fit < cap ? fit : cap);
}

// Launchers of one block size and direction (hygt_batch_launch.cuh,
// instantiated in batch_n*.cu).
template <int LOG2N, int KIND>
cudaError_t launch_batch_n(const BatchParams& p, cudaStream_t stream, const BatchTune& tune);
template <int LOG2N, int KIND>
cudaError_t launch_primary_n(const BatchParams& p, cudaStream_t stream, const BatchTune& tune);

// Host launchers (batch_int.cu, batch_fwd.cu, batch_inv.cu).
cudaError_t batch_build(const uint16_t* d_set, long long nblocks, int num_sets, int group,
                        void* d_work, cudaStream_t stream);
cudaError_t launch_batch_fwd(int log2n, const BatchParams& p, cudaStream_t stream,
                             const BatchTune& tune = BatchTune());
cudaError_t launch_batch_inv(int log2n, const BatchParams& p, cudaStream_t stream,
                             const BatchTune& tune = BatchTune());
// The same kernels with the DCT-II primary of the secondary-transform
// pipeline fused (log2n 4 or 6: 4x4 or 8x8 blocks).
cudaError_t launch_batch_primary(int log2n, int inverse, const BatchParams& p,
                                 cudaStream_t stream, const BatchTune& tune = BatchTune());
cudaError_t launch_batch_primary_fwd(int log2n, const BatchParams& p, cudaStream_t stream,
                                     const BatchTune& tune);
cudaError_t launch_batch_primary_inv(int log2n, const BatchParams& p, cudaStream_t stream,
                                     const BatchTune& tune);

}  // namespace hygt
