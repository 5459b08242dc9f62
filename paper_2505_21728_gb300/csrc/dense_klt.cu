// dense_klt.cu -- dense matrix transform y = K_set x per block (the matrix
// form of Eq. 3), the baseline the HyGT is compared with.
//
// Blocks are bucketed by set (the batch schedule, in tiles of 128 blocks),
// so every tile multiplies one 128 x N slice of blocks by one N x N matrix.
//
// BF16 tensor-core kernel (sm_103a tcgen05): a persistent, warp-specialised
// pipeline (producer warps gather and convert tiles into swizzled shared
// memory, one thread issues tcgen05.mma into tensor-memory accumulators,
// epilogue warps drain them with tcgen05.ld), described at the kernel.
//
// Integer CUDA-core kernel: y = floor((K_int x + 2^(f-1)) / 2^f) with
// K_int = round(2^f K), int32 arithmetic; a warp computes 32 blocks of one
// set, each lane one output row at a time.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "hygt_batch.cuh"
#include "hygt_dense.cuh"
#include "hygt_launch.cuh"

namespace hygt {

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);           // start address
  d |= (uint64_t)(16 >> 4) << 16;                   // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}

// Instruction descriptor, FP32 accumulator, both operands K-major:
// kind::f16 with BF16 A and B (format 1), or kind::f8f6f4 with E4M3 A and B
// (format 0).
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n, bool fp8) {
  return (1u << 4) | ((fp8 ? 0u : 1u) << 7) | ((fp8 ? 0u : 1u) << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

template <bool FP8>
__device__ __forceinline__ void mma_tc(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
  if constexpr (FP8)
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

// 16 consecutive FP32 columns of this thread's accumulator row.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
        "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
        "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}

// ---------------------------------------------------------------- BF16 kernel
// Warp-specialised persistent kernel, one tile of 128 blocks per pipeline
// step, three roles that hand tiles over through mbarriers:
//   warps 0-3  producer: warp w gathers blocks 32w .. 32w + 31 of the tile
//              (coalesced cp.async pieces), thread t converts block t
//              int16 -> BF16 into the 128-byte-swizzled K-major A stage
//              (STAGES stages), and keeps the set's matrix image (B) current;
//   warp 8     one thread issues N/16 tcgen05.mma (M = 128, K = 16) per tile
//              into one of ACC tensor-memory accumulators and commits them;
//   warps 4-7  epilogue: warp 4 + q reads accumulator lanes 32q.. with
//              tcgen05.ld and stores the FP32 outputs.
// So the gather of tile i + 1, the MMAs of tile i and the stores of tile
// i - 1 run at the same time.  Skip and bad-set tiles are handled by the
// producer alone (every role walks the same tile list and skips them).
// Every wait is bounded by a time limit; a role that gives up raises the
// CTA's abort flag, which the other roles' waits observe.
// Shared memory: A stages (BF16 or E4M3 tiles, swizzled), the B image, the
// raw ring (int16 tiles as gathered), the output row buffers (FP32 rows on
// their way to global memory), the FP8 row scales, barriers.  Raw and output rows are padded to an odd
// number of 16-byte units, so that thread t accessing row t hits distinct
// banks.
template <int N, bool FP8>
struct DenseTcShape {
  static constexpr int EB = FP8 ? 1 : 2;                  // operand bytes per element
  static constexpr int KP = FP8 && N < 128 ? 128 : N;     // K padded to whole 128-byte rows
  static constexpr int ROWB = KP * EB;                    // bytes of one operand row
  static constexpr int KB = ROWB / 128;                   // K blocks of 128 bytes
  static constexpr int KSTEPS = ROWB / 32;                // MMAs per tile (32 bytes of K each)
  static constexpr size_t A_BYTES = (size_t)128 * ROWB;
  static constexpr size_t B_BYTES = (size_t)N * ROWB;
  static constexpr int STAGES = N <= 64 ? 4 : 1;         // A stages
  static constexpr int ACC = N <= 64 ? 4 : 2;            // accumulators in tensor memory
  static constexpr int RAW = N <= 64 ? 4 : 0;            // raw tiles in flight (0: direct loads)
  static constexpr int ROW = N * 2 + 16;                 // raw row pitch (bytes)
  static constexpr size_t RAW_BYTES = (size_t)128 * ROW;
  static constexpr uint32_t TMEM_COLS = (uint32_t)(N * ACC);  // 256 or 512 (a power of 2)
  static constexpr int OUT = N <= 64 ? 2 : 0;            // output row buffers per thread (0: direct stores)
  static constexpr int OROW = N * 4 + 16;                // output row pitch (bytes)
  static constexpr size_t OUT_BYTES = (size_t)128 * OROW;
  // FP8: per-row scales of the last SR tiles (the producer runs at most
  // STAGES + ACC tiles ahead of the epilogue)
  static constexpr int SR = FP8 ? STAGES + ACC + 1 : 0;
  static constexpr size_t B_OFF = STAGES * A_BYTES;
  static constexpr size_t RAW_OFF = B_OFF + B_BYTES;
  static constexpr size_t OUT_OFF = RAW_OFF + RAW * RAW_BYTES;
  static constexpr size_t SC_OFF = OUT_OFF + OUT * OUT_BYTES;
  static constexpr size_t BAR_OFF = SC_OFF + (size_t)SR * 128 * 4;
  static constexpr size_t SMEM = BAR_OFF + 320;
  static constexpr int THREADS = 288;                   // 4 producer + 4 epilogue + 1 MMA warp
  static_assert(RAW_OFF % 16 == 0 && ROW % 16 == 0 && OUT_OFF % 16 == 0 && OROW % 16 == 0 &&
                    BAR_OFF % 16 == 0 && ROWB % 128 == 0,
                "alignment");
  static_assert((2 * STAGES + 2 * ACC + RAW + SR) * 8 + 8 <= 320, "barrier area");
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait for the completion of the mbarrier phase with parity `parity`, at
// most about one second, and not past the CTA's abort flag (if given).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort_flag) {
  const uint32_t a = smem_addr(bar);
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && ((abort_flag && *abort_flag) || global_ns() - t0 > 1000000000ull))
      return false;
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// 16 consecutive FP32 columns of this thread's accumulator row, without
// waiting (tcgen05.wait::ld before use).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* u) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
        "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
        "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
}

// Bulk copy shared -> global (16-byte aligned, size a multiple of 16), in
// this thread's current bulk group.
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until at most one of this thread's bulk groups still reads its source.
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completing on `bar`.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void dense_abort(volatile int* abort_flag, int* status) {
  *abort_flag = 1;
  if (status) atomicCAS(status, 0, 2);
}

// Bucket of consecutive tiles: a binary search over the bucket starts only
// when a tile leaves the current bucket.
struct BucketTracker {
  int bucket = 0, end = 0;
  __device__ __forceinline__ int at(const int* starts, int num_sets, int slot) {
    if (slot >= end) {
      bucket = bucket_of_slot(starts, num_sets, slot);
      end = __ldg(starts + bucket + 1);
    }
    return bucket;
  }
};

template <int N, bool FP8>
__global__ void __launch_bounds__(288, 1) dense_tc_kernel(DenseParams p) {
  using SH = DenseTcShape<N, FP8>;
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* b_img = dsm + SH::B_OFF;
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + SH::BAR_OFF);
  uint64_t* a_full = bars;                       // [STAGES], 128 producer arrivals
  uint64_t* a_free = bars + SH::STAGES;          // [STAGES], MMA commit
  uint64_t* acc_full = bars + 2 * SH::STAGES;    // [ACC], MMA commit
  uint64_t* acc_empty = acc_full + SH::ACC;      // [ACC], 128 epilogue arrivals
  uint64_t* raw_full = acc_empty + SH::ACC;      // [RAW], 128 producer arrivals + bytes
  uint64_t* sc_full = raw_full + SH::RAW;        // [SR], 128 producer arrivals (FP8)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sc_full + SH::SR);
  float* scale_ring = reinterpret_cast<float*>(dsm + SH::SC_OFF);  // [SR][128]
  unsigned char* raw = dsm + SH::RAW_OFF;
  unsigned char* out = dsm + SH::OUT_OFF;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int t = threadIdx.x;
  const int warp = t >> 5;

  if (p.meta[1] != (int)p.nblocks || p.meta[2] != p.num_sets || p.meta[3] != 128) {
    if (t == 0 && blockIdx.x == 0 && p.status) atomicCAS(p.status, 0, 1);
    return;
  }
  // the 128-byte swizzle needs 1024-byte aligned operand images
  if ((smem_addr(dsm) & 1023u) != 0) {
    if (t == 0 && p.status) atomicCAS(p.status, 0, 2);
    return;
  }
  if (warp == 8) tmem_alloc(tmem_slot, SH::TMEM_COLS);
  if (t == 0) {
    for (int i = 0; i < SH::STAGES; ++i) {
      mbar_init(a_full + i, 128);
      mbar_init(a_free + i, 1);
    }
    for (int i = 0; i < SH::ACC; ++i) {
      mbar_init(acc_full + i, 1);
      mbar_init(acc_empty + i, 128);
    }
    for (int i = 0; i < SH::RAW; ++i) mbar_init(raw_full + i, 128);
    for (int i = 0; i < SH::SR; ++i) mbar_init(sc_full + i, 128);
    *abort_flag = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const long long ntasks = max(0LL, min((long long)p.meta[0], p.tmax));
  const long long chunk = (ntasks + gridDim.x - 1) / gridDim.x;
  const long long t0 = min(ntasks, (long long)blockIdx.x * chunk);
  const long long t1 = min(ntasks, t0 + chunk);
  const int S = p.num_sets;

  if (warp < 4) {
    // ------------------------------------------------ producer
    // Thread t converts row t of every tile.  With a raw ring, the rows of the
    // next RAW tiles are in flight as cp.async pieces while this one is
    // converted (measured 17% faster than one bulk copy per row);
    // block ids are loaded one tile ahead of their use (idq holds the ids of
    // the tiles in flight, id_ahead the next one's).
    constexpr int IDQ = SH::RAW > 0 ? SH::RAW : 1;
    auto load_id = [&](long long task) {
      return task < t1 ? __ldg(p.order + task * 128 + t) : -1;
    };
    // The warp copies its 32 rows of the tile with 16-byte cp.async pieces
    // (a row's pieces in consecutive lanes: coalesced), each thread's
    // pieces completing with one arrival on the ring slot's barrier.
    auto issue_raw = [&](long long task, int b) {
      if constexpr (SH::RAW > 0) {
        const int rs = (int)((task - t0) % SH::RAW);
        constexpr int CPR = N * 2 / 16;  // pieces per row
        const int lane = t & 31;
        __syncwarp();  // the warp's rows in this slot have been read
        unsigned char* wrows = raw + (size_t)rs * SH::RAW_BYTES + (size_t)(t - lane) * SH::ROW;
#pragma unroll
        for (int j = 0; j < CPR; ++j) {
          const int c = j * 32 + lane, row = c / CPR, ch = c % CPR;
          const int rb = __shfl_sync(0xffffffffu, b, row);
          if (rb >= 0 && rb < p.nblocks)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                             smem_addr(wrows + (size_t)row * SH::ROW + ch * 16)),
                         "l"(p.x + (long long)rb * N + ch * 8)
                         : "memory");
        }
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                         smem_addr(raw_full + rs))
                     : "memory");
      }
    };
    int idq[IDQ];
#pragma unroll
    for (int d = 0; d < IDQ; ++d) idq[d] = load_id(t0 + d);
    if constexpr (SH::RAW > 0) {
#pragma unroll
      for (int d = 0; d < IDQ; ++d)
        if (t0 + d < t1) issue_raw(t0 + d, idq[d]);
    }
    int id_ahead = load_id(t0 + IDQ);
    int i = 0, cur_set = -1;
    bool aborted = false;
    BucketTracker bt;
    for (long long task = t0; task < t1; ++task) {
      const int slot = (int)(task * 128);
      const int bucket = bt.at(p.starts, S, slot);
      const int b = idq[0];
      const bool active = b >= 0 && b < p.nblocks;
      // this thread's row of the tile: from the raw ring, or straight from global memory
      const int4* xs;
      if constexpr (SH::RAW > 0) {
        const int rs = (int)((task - t0) % SH::RAW);
        if (!__all_sync(0xffffffffu,
                        mbar_wait_bounded(raw_full + rs, (uint32_t)((task - t0) / SH::RAW) & 1u,
                                          abort_flag))) {
          dense_abort(abort_flag, p.status);
          aborted = true;
          break;
        }
        xs = reinterpret_cast<const int4*>(raw + (size_t)rs * SH::RAW_BYTES + (size_t)t * SH::ROW);
      } else {
        xs = reinterpret_cast<const int4*>(p.x + (long long)(active ? b : 0) * N);
      }
      if (bucket >= S) {  // skip (identity) or bad set (zeros)
        if (active) {
          float* y = p.y + (long long)b * N;
          for (int c = 0; c < N / 8; ++c) {
            const int4 raw8 = SH::RAW > 0 ? xs[c] : __ldg(xs + c);
            const int16_t* h = reinterpret_cast<const int16_t*>(&raw8);
#pragma unroll
            for (int k = 0; k < 8; ++k) y[8 * c + k] = bucket == S ? (float)h[k] : 0.f;
          }
          if (bucket != S && p.status) atomicCAS(p.status, 0, 4);
        }
      } else {
        const int s = i % SH::STAGES;
        if (i >= SH::STAGES &&
            !__all_sync(0xffffffffu, mbar_wait_bounded(a_free + s,
                                                       (uint32_t)((i / SH::STAGES) - 1) & 1u,
                                                       abort_flag))) {
          dense_abort(abort_flag, p.status);
          aborted = true;
          break;
        }
        if (bucket != cur_set) {
          // every MMA issued so far must be done before the image is replaced
          if (i > 0) {
            const int j = i - 1;
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(a_free + j % SH::STAGES,
                                                           (uint32_t)(j / SH::STAGES) & 1u,
                                                           abort_flag))) {
              dense_abort(abort_flag, p.status);
              aborted = true;
              break;
            }
          }
          const int4* src = reinterpret_cast<const int4*>((FP8 ? p.kimg8 : p.kimg) +
                                                          (size_t)bucket * SH::B_BYTES);
          int4* dst = reinterpret_cast<int4*>(b_img);
          for (int k = t; k < (int)(SH::B_BYTES / 16); k += 128) dst[k] = __ldg(src + k);
          cur_set = bucket;
        }
        // A row t of stage s, 16-byte chunks at swizzled positions
        unsigned char* row = dsm + (size_t)s * SH::A_BYTES + (t >> 3) * 1024 + (t & 7) * 128;
        if constexpr (!FP8) {  // int16 -> bf16, 8 values per chunk
#pragma unroll 8
          for (int c = 0; c < N / 8; ++c) {
            int4 raw8 = !active ? make_int4(0, 0, 0, 0) : SH::RAW > 0 ? xs[c] : __ldg(xs + c);
            const int16_t* h = reinterpret_cast<const int16_t*>(&raw8);
            __nv_bfloat162 q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
              q[k] = __floats2bfloat162_rn((float)h[2 * k], (float)h[2 * k + 1]);
            const int kb = c >> 3, cc = c & 7;
            unsigned char* dst = row + kb * (128 * 128) + ((cc ^ (t & 7)) << 4);
            *reinterpret_cast<int4*>(dst) = *reinterpret_cast<int4*>(q);
          }
        } else {  // int16 -> e4m3 with a per-row scale, 16 values per chunk
          int amax = 0;
          if (active) {
#pragma unroll 8
            for (int c = 0; c < N / 8; ++c) {
              const int4 raw8 = SH::RAW > 0 ? xs[c] : __ldg(xs + c);
              const int16_t* h = reinterpret_cast<const int16_t*>(&raw8);
#pragma unroll
              for (int k = 0; k < 8; ++k) amax = max(amax, abs((int)h[k]));
            }
          }
          const float inv = amax > 0 ? 448.f / (float)amax : 1.f;
          scale_ring[(i % SH::SR) * 128 + t] = amax > 0 ? (float)amax / 448.f : 1.f;
#pragma unroll 4
          for (int c = 0; c < SH::KP / 16; ++c) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (active && c < N / 16) {
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const int4 raw8 = SH::RAW > 0 ? xs[2 * c + hh] : __ldg(xs + 2 * c + hh);
                const int16_t* h = reinterpret_cast<const int16_t*>(&raw8);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                  const __nv_fp8x2_storage_t q2 = __nv_cvt_float2_to_fp8x2(
                      make_float2((float)h[2 * k] * inv, (float)h[2 * k + 1] * inv),
                      __NV_SATFINITE, __NV_E4M3);
                  w[2 * hh + (k >> 1)] |= (uint32_t)q2 << (16 * (k & 1));
                }
              }
            }
            const int kb = c >> 3, cc = c & 7;
            unsigned char* dst = row + kb * (128 * 128) + ((cc ^ (t & 7)) << 4);
            *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(a_full + s);
        if constexpr (FP8) mbar_arrive(sc_full + i % SH::SR);
        ++i;
      }
      // advance the id queue; this thread's raw row is read, so its slot takes
      // the tile RAW ahead (generic reads ordered before the asynchronous write)
#pragma unroll
      for (int d = 0; d + 1 < IDQ; ++d) idq[d] = idq[d + 1];
      idq[IDQ - 1] = id_ahead;
      if constexpr (SH::RAW > 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (task + SH::RAW < t1) issue_raw(task + SH::RAW, id_ahead);
      }
      id_ahead = load_id(task + IDQ + 1);
    }
    if constexpr (SH::RAW > 0) {
      // let copies still in flight land before the CTA exits
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    (void)aborted;
  } else if (warp < 8) {
    // ------------------------------------------------ epilogue
    const int r = t - 128;  // accumulator lane = tile row
    const uint32_t lane_base = tmem + ((uint32_t)((warp - 4) * 32) << 16);
    int i = 0;
    BucketTracker bt;
    int b_next = t0 < t1 ? __ldg(p.order + t0 * 128 + r) : -1;
    for (long long task = t0; task < t1; ++task) {
      const int slot = (int)(task * 128);
      const int bucket = bt.at(p.starts, S, slot);
      const int b = b_next;  // ids one tile ahead
      b_next = task + 1 < t1 ? __ldg(p.order + (task + 1) * 128 + r) : -1;
      if (bucket >= S) continue;
      const int a = i % SH::ACC;
      const bool active = b >= 0 && b < p.nblocks;
      if (!mbar_wait_bounded(acc_full + a, (uint32_t)(i / SH::ACC) & 1u, abort_flag)) {
        dense_abort(abort_flag, p.status);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* y = p.y + (long long)(active ? b : 0) * N;
      float osc = 1.f;  // FP8: row scale x set scale
      if constexpr (FP8) {
        if (!mbar_wait_bounded(sc_full + i % SH::SR, (uint32_t)(i / SH::SR) & 1u, abort_flag)) {
          dense_abort(abort_flag, p.status);
          break;
        }
        osc = scale_ring[(i % SH::SR) * 128 + r] * __ldg(p.kscale + bucket);
      }
      if constexpr (SH::OUT > 0) {
        // whole row into registers, accumulator released, row staged in
        // shared memory and written by one bulk copy
        uint32_t u[N];
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) tmem_ld16_async(lane_base + (uint32_t)(a * N + c0), u + c0);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(acc_empty + a);
        unsigned char* orow = out + (size_t)(i & 1) * SH::OUT_BYTES + (size_t)r * SH::OROW;
        bulk_wait_read1();  // the copy that last read this buffer is done with it
        if (active) {
#pragma unroll
          for (int c = 0; c < N; c += 4) {
            if constexpr (FP8) {
              *reinterpret_cast<float4*>(orow + 4 * c) =
                  make_float4(__uint_as_float(u[c]) * osc, __uint_as_float(u[c + 1]) * osc,
                              __uint_as_float(u[c + 2]) * osc, __uint_as_float(u[c + 3]) * osc);
            } else {
              *reinterpret_cast<uint4*>(orow + 4 * c) = make_uint4(u[c], u[c + 1], u[c + 2], u[c + 3]);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bulk_store(y, orow, N * 4);
        }
        bulk_commit();  // one group per tile, so groups alternate between the two buffers
      } else {
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
          float v[16];
          tmem_ld16(lane_base + (uint32_t)(a * N + c0), v);
          if (active) {
#pragma unroll
            for (int k = 0; k < 16; k += 4)
              *reinterpret_cast<float4*>(y + c0 + k) =
                  make_float4(v[k] * osc, v[k + 1] * osc, v[k + 2] * osc, v[k + 3] * osc);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(acc_empty + a);
      }
      ++i;
    }
    if constexpr (SH::OUT > 0) bulk_wait_all();
  } else if (t == 256) {
    // ------------------------------------------------ MMA issuer
    constexpr uint32_t kIdesc = tc_idesc(128, N, FP8);
    const uint32_t b0 = smem_addr(b_img);
    int i = 0;
    BucketTracker bt;
    for (long long task = t0; task < t1; ++task) {
      const int slot = (int)(task * 128);
      const int bucket = bt.at(p.starts, S, slot);
      if (bucket >= S) continue;
      const int s = i % SH::STAGES, a = i % SH::ACC;
      if (!mbar_wait_bounded(a_full + s, (uint32_t)(i / SH::STAGES) & 1u, abort_flag) ||
          (i >= SH::ACC &&
           !mbar_wait_bounded(acc_empty + a, (uint32_t)((i / SH::ACC) - 1) & 1u, abort_flag))) {
        dense_abort(abort_flag, p.status);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_addr(dsm + (size_t)s * SH::A_BYTES);
#pragma unroll
      for (int k = 0; k < SH::KSTEPS; ++k) {
        const uint32_t ka = (uint32_t)((k >> 2) * (128 * 128) + (k & 3) * 32);
        const uint32_t kb = (uint32_t)((k >> 2) * (N * 128) + (k & 3) * 32);
        mma_tc<FP8>(tmem + (uint32_t)(a * N), sw128_desc(a0 + ka), sw128_desc(b0 + kb), kIdesc,
                    k > 0 ? 1u : 0u);
      }
      mma_commit(a_free + s);
      mma_commit(acc_full + a);
      ++i;
    }
    // the tensor memory is released below: wait for the last MMAs issued,
    // also after an abort
    if (i > 0) {
      const int j = i - 1;
      if (!mbar_wait_bounded(a_free + j % SH::STAGES, (uint32_t)(j / SH::STAGES) & 1u, nullptr))
        dense_abort(abort_flag, p.status);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 8) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem_dealloc(tmem, SH::TMEM_COLS);
  }
}

// ---------------------------------------------------------------- int32 kernel
// One lane per block: the lane holds its block's N values in registers; the
// warp's 32 blocks share the set, so every multiplier K_int[i][k] is read by
// all lanes at once (a broadcast from the CTA's shared copy of the matrix).
// Four outputs are formed at a time and stored as one 16-byte vector.
template <int N>
__global__ void __launch_bounds__(256) dense_int_kernel(DenseParams p) {
  __shared__ __align__(16) int32_t km[N * N];
  if (p.meta[1] != (int)p.nblocks || p.meta[2] != p.num_sets || p.meta[3] != 128) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && p.status) atomicCAS(p.status, 0, 1);
    return;
  }
  // CTA tasks are 128-block tiles (one bucket each); warp w takes rows 32w..
  const long long ntasks = max(0LL, min((long long)p.meta[0], p.tmax));
  const long long chunk = (ntasks + gridDim.x - 1) / gridDim.x;
  const long long t0 = min(ntasks, (long long)blockIdx.x * chunk);
  const long long t1 = min(ntasks, t0 + chunk);
  const int half = 1 << (p.frac_bits - 1);
  int cached = -1;  // the bucket is CTA-uniform, so every thread tracks the same value
  BucketTracker bt;
  for (long long task = t0; task < t1; ++task) {
    const int slot = (int)(task * 128);
    const int bucket = bt.at(p.starts, p.num_sets, slot);
    if (bucket < p.num_sets && bucket != cached) {
      __syncthreads();
      const int16_t* K = p.kint + (size_t)bucket * N * N;
      for (int i = threadIdx.x; i < N * N; i += blockDim.x) km[i] = (int32_t)__ldg(K + i);
      __syncthreads();
      cached = bucket;
    }
    for (int row = threadIdx.x; row < 128; row += blockDim.x) {
      const int b = __ldg(p.order + slot + row);
      const bool active = b >= 0 && b < p.nblocks;
      int32_t x[N];
      {
        uint32_t w[N / 2];
        if (active) load_words<N / 2>(p.x + (long long)b * N, w);
        else
          for (int k = 0; k < N / 2; ++k) w[k] = 0;
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
          x[2 * k] = (int32_t)(int16_t)(w[k] & 0xffffu);
          x[2 * k + 1] = (int32_t)w[k] >> 16;
        }
      }
      int32_t* y = p.yint + (long long)(active ? b : 0) * N;
      if (bucket < p.num_sets) {
#pragma unroll 1
        for (int i = 0; i < N; i += 4) {
          int32_t acc[4] = {half, half, half, half};
#pragma unroll
          for (int k = 0; k < N; k += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int4 kv = *reinterpret_cast<const int4*>(&km[(i + q) * N + k]);
              acc[q] += kv.x * x[k] + kv.y * x[k + 1] + kv.z * x[k + 2] + kv.w * x[k + 3];
            }
          }
          if (active)
            *reinterpret_cast<int4*>(y + i) =
                make_int4(acc[0] >> p.frac_bits, acc[1] >> p.frac_bits, acc[2] >> p.frac_bits,
                          acc[3] >> p.frac_bits);
        }
      } else if (active) {
        for (int k = 0; k < N; ++k) y[k] = bucket == p.num_sets ? x[k] : 0;
        if (bucket != p.num_sets && p.status) atomicCAS(p.status, 0, 4);
      }
    }
  }
}

// ---------------------------------------------------------------- launchers
template <int N, bool FP8>
static cudaError_t launch_tc(const DenseParams& p, cudaStream_t stream) {
  using SH = DenseTcShape<N, FP8>;
  auto kern = dense_tc_kernel<N, FP8>;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  // Shared memory per CTA is padded so that the CTAs resident on an SM never
  // ask for more than the 512 tensor-memory columns of the SM: allocation
  // then never has to wait.
  const int max_ctas = 512 / (int)SH::TMEM_COLS;
  size_t smem = SH::SMEM;
  const size_t sm_total = 228 * 1024;
  if (smem * (size_t)(max_ctas + 1) <= sm_total) smem = sm_total / (size_t)(max_ctas + 1) + 1024;
  if (smem > (size_t)info.max_smem_optin) return cudaErrorInvalidConfiguration;
  err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SH::THREADS, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  if (occ > max_ctas) return cudaErrorInvalidConfiguration;
  long long grid = (long long)occ * info.sms;
  const long long tiles = (p.nblocks + 127) / 128 + p.num_sets + 2;
  if (grid > tiles) grid = tiles;
  kern<<<(unsigned)grid, SH::THREADS, smem, stream>>>(p);
  return cudaGetLastError();
}

template <int N>
static cudaError_t launch_int(const DenseParams& p, cudaStream_t stream) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  const DeviceInfo info = device_info(dev);
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dense_int_kernel<N>, 128, 0);
  if (err != cudaSuccess) return err;
  if (occ < 1) occ = 1;
  long long grid = (long long)occ * info.sms;
  const long long tiles = (p.nblocks + 127) / 128 + p.num_sets + 2;
  if (grid > tiles) grid = tiles;
  dense_int_kernel<N><<<(unsigned)grid, 128, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_dense(int log2n, int kind, const DenseParams& p, cudaStream_t stream) {
  if (kind == 0 || kind == 2) {
    const bool fp8 = kind == 2;
    switch (log2n) {
      case 6: return fp8 ? launch_tc<64, true>(p, stream) : launch_tc<64, false>(p, stream);
      case 8: return fp8 ? launch_tc<256, true>(p, stream) : launch_tc<256, false>(p, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (log2n) {
    case 4: return launch_int<16>(p, stream);
    case 6: return launch_int<64>(p, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hygt
