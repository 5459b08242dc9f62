// pmpt.cu -- the general Parametric Multi-pass Transform with explicit index
// vectors (sm_103a).
//
// A pass is a parallel-Givens matrix over an arbitrary cover of 0..N-1 by
// N/2 disjoint pairs (m_j, n_j) (Sec. IV, Eq. 7-8), each pair with its own
// angle; the transform is the product of the passes, the first applied first
// (Sec. III, Eq. 5), and the inverse runs them in reverse with the angles
// negated (Eq. 9).  Unlike the HyGT, whose pairs follow from the hypercube,
// every pair costs its two indices in memory (Sec. IV), and the pairs of a
// pass can join any two elements, so a block is not split over lanes by a
// fixed pattern.
//
// Mapping.  A warp task is G = max(1, 256 / N) consecutive blocks: the warp
// copies them (coalesced) into a shared-memory region per block of N + 1
// words, and every pass spreads its G N/2 <= 128 rotations over the 32
// lanes (item w: block w / (N/2), pair w mod (N/2); at most four per lane,
// fixed for the task); each item reads its pair's packed indices and
// multipliers (one 8-byte load, L1-cached), gathers the two values from the
// block's region, rotates them and writes them back; __syncwarp()
// separates the passes.  Integer rotations round half up,
// floor((c a + s b + 2^(f-1)) / 2^f) (Sec. IV, Fig. 5 conversion), with
// int32 intermediates; the inverse output saturates to int16.  Set index
// 0xFFFF is the identity; any other index >= num_sets zeroes the block and
// records HYGT_ERR_SET_INDEX.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hygt.h"
#include "hygt_launch.cuh"

struct hygt_pmpt_s {
  int n = 0, passes = 0, num_sets = 0;
  int angle_bits = 0, frac_bits = 0;
  int is_float = 0;
  int device = 0;
  uint2* d_mncs = nullptr;    // (m | n << 16, int16 c | int16 s << 16) per pair, [S][P][N/2]
  float2* d_csf = nullptr;    // (cos, sin) per pair
  uint32_t* d_mn = nullptr;   // m | n << 16 per pair (FP32 calls)
};

namespace hygt {

constexpr int kPmptThreads = 256;

struct PmptParams {
  const void* in;
  void* out;
  const uint16_t* set;
  long long nblocks;
  int n, passes, num_sets, frac_bits;
  int group;  // blocks per warp task
  const uint2* mncs;
  const uint32_t* mn;
  const float2* csf;
  int* status;
};

// Items of a lane in a task: item it = lane + 32 u (u < kPmptItems) is
// rotation j = it mod (N/2) of block it / (N/2); a task holds at most 128
// rotations per pass (G N/2 <= 128), so 4 items per lane cover it.
constexpr int kPmptItems = 4;

// KIND: 0 integer forward, 1 integer inverse, 2 FP32 forward, 3 FP32 inverse.
template <int KIND>
__global__ void __launch_bounds__(kPmptThreads) hygt_pmpt_kernel(PmptParams p) {
  constexpr bool INV = (KIND & 1) != 0;
  constexpr bool F32 = KIND >= 2;
  extern __shared__ __align__(16) int32_t psm[];
  const int N = p.n, half = p.n / 2, G = p.group, RS = p.n + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  int32_t* reg = psm + (size_t)warp * (G * RS + G);  // G regions, then G set indices
  int* bset = reg + G * RS;
  float* regf = reinterpret_cast<float*>(reg);
  const long long ntasks = (p.nblocks + G - 1) / G;
  const uint32_t rnd = 1u << (p.frac_bits - 1);
  const int f = p.frac_bits;
  const size_t pass_stride = (size_t)half;

  for (long long t = (long long)blockIdx.x * wpc + warp; t < ntasks;
       t += (long long)gridDim.x * wpc) {
    const long long b0 = t * G;
    const int nb = (int)min((long long)G, p.nblocks - b0);
    // blocks in (coalesced): element e = lane + 32 x of the task, block and
    // index advanced without division
    {
      int blk = lane / N, i = lane - blk * N;
      const int step_blk = 32 / N, step_i = 32 - step_blk * N;
      for (int e = lane; e < nb * N; e += 32) {
        const long long g = b0 * N + e;
        if constexpr (F32)
          regf[blk * RS + i] = __ldcs(static_cast<const float*>(p.in) + g);
        else if constexpr (INV)
          reg[blk * RS + i] = __ldcs(static_cast<const int32_t*>(p.in) + g);
        else
          reg[blk * RS + i] = __ldcs(static_cast<const int16_t*>(p.in) + g);
        blk += step_blk;
        i += step_i;
        if (i >= N) { i -= N; ++blk; }
      }
    }
    for (int k = lane; k < nb; k += 32) {  // a task may hold more than 32 blocks
      const int s = p.set ? (int)__ldg(p.set + b0 + k) : 0;
      bset[k] = s;
      if (s != 0xFFFF && s >= p.num_sets && p.status) atomicCAS(p.status, 0, HYGT_ERR_SET_INDEX);
    }
    __syncwarp();
    // this lane's rotations: region offset and table offset of pass 0
    int rbase[kPmptItems];
    long long tbase[kPmptItems];
#pragma unroll
    for (int u = 0; u < kPmptItems; ++u) {
      const int it = lane + 32 * u;
      const int blk = it / half, j = it - blk * half;
      rbase[u] = blk * RS;
      tbase[u] = -1;
      if (it < nb * half) {
        const int s = bset[blk];
        if (s < p.num_sets) tbase[u] = (long long)s * p.passes * half + j;
      }
    }
    for (int kk = 0; kk < p.passes; ++kk) {
      const int k = INV ? p.passes - 1 - kk : kk;
      uint2 ent[kPmptItems];
      float2 entf[kPmptItems];
      uint32_t mnf[kPmptItems];
#pragma unroll
      for (int u = 0; u < kPmptItems; ++u) {  // the loads first: independent
        if (tbase[u] < 0) continue;
        const size_t e = (size_t)tbase[u] + (size_t)k * pass_stride;
        if constexpr (F32) {
          entf[u] = __ldg(p.csf + e);
          mnf[u] = __ldg(p.mn + e);
        } else {
          ent[u] = __ldg(p.mncs + e);
        }
      }
#pragma unroll
      for (int u = 0; u < kPmptItems; ++u) {
        if (tbase[u] < 0) continue;
        if constexpr (F32) {
          const int m = (int)(mnf[u] & 0xFFFFu), q = (int)(mnf[u] >> 16);
          const float c = entf[u].x, sn = INV ? -entf[u].y : entf[u].y;
          const float a = regf[rbase[u] + m], bb = regf[rbase[u] + q];
          regf[rbase[u] + m] = fmaf(c, a, sn * bb);
          regf[rbase[u] + q] = fmaf(c, bb, -sn * a);
        } else {
          const int m = (int)(ent[u].x & 0xFFFFu), q = (int)(ent[u].x >> 16);
          const int32_t c = (int32_t)(int16_t)(ent[u].y & 0xFFFFu);
          const int32_t s0 = (int32_t)ent[u].y >> 16;
          const int32_t sn = INV ? -s0 : s0;
          const uint32_t a = (uint32_t)reg[rbase[u] + m], bb = (uint32_t)reg[rbase[u] + q];
          reg[rbase[u] + m] = (int32_t)((uint32_t)c * a + (uint32_t)sn * bb + rnd) >> f;
          reg[rbase[u] + q] = (int32_t)((uint32_t)c * bb - (uint32_t)sn * a + rnd) >> f;
        }
      }
      __syncwarp();
    }
    // blocks out (coalesced); bad set index: zeros
    {
      int blk = lane / N, i = lane - blk * N;
      const int step_blk = 32 / N, step_i = 32 - step_blk * N;
      for (int e = lane; e < nb * N; e += 32) {
        const long long g = b0 * N + e;
        const int s = bset[blk];
        const bool bad = s != 0xFFFF && s >= p.num_sets;
        if constexpr (F32) {
          __stcs(static_cast<float*>(p.out) + g, bad ? 0.f : regf[blk * RS + i]);
        } else if constexpr (INV) {
          const int32_t v = bad ? 0 : reg[blk * RS + i];
          __stcs(static_cast<int16_t*>(p.out) + g, (int16_t)max(-32768, min(32767, v)));
        } else {
          __stcs(static_cast<int32_t*>(p.out) + g, bad ? 0 : reg[blk * RS + i]);
        }
        blk += step_blk;
        i += step_i;
        if (i >= N) { i -= N; ++blk; }
      }
    }
    __syncwarp();
  }
}

static cudaError_t launch_pmpt(int kind, const PmptParams& p, cudaStream_t stream) {
  int dev = 0;
  cudaGetDevice(&dev);
  const DeviceInfo info = device_info(dev);
  const int wpc = kPmptThreads / 32;
  const size_t smem = (size_t)wpc * (p.group * (p.n + 1) + p.group) * 4;
  const long long ntasks = (p.nblocks + p.group - 1) / p.group;
  long long grid = (long long)info.sms * 4;
  if ((ntasks + wpc - 1) / wpc < grid) grid = (ntasks + wpc - 1) / wpc;
  if (grid < 1) grid = 1;
  switch (kind) {
    case 0: hygt_pmpt_kernel<0><<<(int)grid, kPmptThreads, smem, stream>>>(p); break;
    case 1: hygt_pmpt_kernel<1><<<(int)grid, kPmptThreads, smem, stream>>>(p); break;
    case 2: hygt_pmpt_kernel<2><<<(int)grid, kPmptThreads, smem, stream>>>(p); break;
    default: hygt_pmpt_kernel<3><<<(int)grid, kPmptThreads, smem, stream>>>(p); break;
  }
  return cudaGetLastError();
}

}  // namespace hygt

namespace {

void free_pmpt(hygt_pmpt p) {
  if (!p) return;
  if (p->d_mn) cudaFree(p->d_mn);
  if (p->d_mncs) cudaFree(p->d_mncs);
  if (p->d_csf) cudaFree(p->d_csf);
  delete p;
}

template <typename T>
hygt_status upload_vec(T** dst, const std::vector<T>& v) {
  if (cudaMalloc(reinterpret_cast<void**>(dst), v.size() * sizeof(T)) != cudaSuccess) {
    *dst = nullptr;
    cudaGetLastError();
    return HYGT_ERR_OOM;
  }
  if (cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return HYGT_ERR_CUDA;
  return HYGT_OK;
}

hygt_status pmpt_status(cudaError_t e) {
  if (e == cudaSuccess) return HYGT_OK;
  if (e == cudaErrorMemoryAllocation) return HYGT_ERR_OOM;
  return HYGT_ERR_CUDA;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

hygt_status pmpt_run(int kind, hygt_pmpt pm, const void* in, void* out, const uint16_t* d_set,
                     int64_t nblocks, hygt_stream stream, int* d_status) {
  if (!pm || nblocks < 0 || nblocks > ((int64_t)1 << 40)) return HYGT_ERR_ARG;
  if (kind < 2 && pm->is_float) return HYGT_ERR_UNSUPPORTED;
  if (nblocks == 0) return HYGT_OK;
  if (!in || !out || !aligned(in, 4) || !aligned(out, 4)) return HYGT_ERR_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HYGT_ERR_CUDA;
  if (dev != pm->device) return HYGT_ERR_ARG;
  hygt::PmptParams p{};
  p.in = in;
  p.out = out;
  p.set = d_set;
  p.nblocks = nblocks;
  p.n = pm->n;
  p.passes = pm->passes;
  p.num_sets = pm->num_sets;
  p.frac_bits = pm->frac_bits > 0 ? pm->frac_bits : 8;
  p.group = pm->n >= 256 ? 1 : 256 / pm->n;
  p.mncs = pm->d_mncs;
  p.mn = pm->d_mn;
  p.csf = pm->d_csf;
  p.status = d_status;
  return pmpt_status(hygt::launch_pmpt(kind, p, (cudaStream_t)stream));
}

}  // namespace

extern "C" {

hygt_status hygt_pmpt_create(hygt_pmpt* out, int n, int passes, int num_sets,
                             const uint8_t* angle_idx, const float* theta, const uint16_t* m_idx,
                             const uint16_t* n_idx, int angle_bits, int frac_bits) {
  if (!out) return HYGT_ERR_ARG;
  *out = nullptr;
  if (n < 2 || n > 256 || (n & 1) || passes < 1 || passes > 4096 || num_sets < 1 ||
      num_sets > 65535 || !m_idx || !n_idx || (!angle_idx == !theta))
    return HYGT_ERR_ARG;
  if (angle_idx && (angle_bits < 1 || angle_bits > 8 || frac_bits < 1 || frac_bits > 14))
    return HYGT_ERR_ARG;
  const int half = n / 2;
  const size_t pairs = (size_t)num_sets * passes * half;
  // the index vectors of every pass must cover 0..N-1 exactly once (Eq. 7)
  std::vector<uint32_t> mn(pairs);
  std::vector<int> seen(n);
  for (size_t sp = 0; sp < (size_t)num_sets * passes; ++sp) {
    std::fill(seen.begin(), seen.end(), 0);
    for (int j = 0; j < half; ++j) {
      const int m = m_idx[sp * half + j], k = n_idx[sp * half + j];
      if (m >= n || k >= n || m == k || seen[m] || seen[k]) return HYGT_ERR_ARG;
      seen[m] = seen[k] = 1;
      mn[sp * half + j] = (uint32_t)m | ((uint32_t)k << 16);
    }
  }
  hygt_pmpt p = new (std::nothrow) hygt_pmpt_s();
  if (!p) return HYGT_ERR_OOM;
  p->n = n;
  p->passes = passes;
  p->num_sets = num_sets;
  p->angle_bits = angle_idx ? angle_bits : 0;
  p->frac_bits = angle_idx ? frac_bits : 0;
  p->is_float = angle_idx ? 0 : 1;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    free_pmpt(p);
    return HYGT_ERR_CUDA;
  }
  std::vector<float2> csf(pairs);
  std::vector<uint32_t> cs;
  const double two_pi = 6.283185307179586476925286766559;
  if (angle_idx) {
    // on-the-fly conversion of Sec. IV (Fig. 5): q -> round(2^f cos), round(2^f sin)
    cs.resize(pairs);
    const double scale = std::ldexp(1.0, frac_bits);
    for (size_t e = 0; e < pairs; ++e) {
      const double th = two_pi * (double)angle_idx[e] / (double)(1 << angle_bits);
      const long c = std::lround(scale * std::cos(th)), s = std::lround(scale * std::sin(th));
      cs[e] = ((uint32_t)(uint16_t)(int16_t)c) | ((uint32_t)(uint16_t)(int16_t)s << 16);
      csf[e] = make_float2((float)std::cos(th), (float)std::sin(th));
    }
  } else {
    for (size_t e = 0; e < pairs; ++e) {
      const double th = (double)theta[e];
      csf[e] = make_float2((float)std::cos(th), (float)std::sin(th));
    }
  }
  hygt_status s = upload_vec(&p->d_mn, mn);
  if (s == HYGT_OK) s = upload_vec(&p->d_csf, csf);
  if (s == HYGT_OK && !cs.empty()) {
    std::vector<uint2> mncs(pairs);
    for (size_t e = 0; e < pairs; ++e) mncs[e] = make_uint2(mn[e], cs[e]);
    s = upload_vec(&p->d_mncs, mncs);
  }
  if (s != HYGT_OK) {
    free_pmpt(p);
    return s;
  }
  *out = p;
  return HYGT_OK;
}

void hygt_pmpt_destroy(hygt_pmpt pm) { free_pmpt(pm); }

size_t hygt_pmpt_param_bytes(int n, int passes, int num_sets) {
  if (n < 2 || n > 256 || (n & 1) || passes < 1 || num_sets < 1) return 0;
  // one byte per angle and one byte per index (N <= 256): three per pair
  return (size_t)num_sets * (size_t)passes * (size_t)(n / 2) * 3;
}

hygt_status hygt_pmpt_forward(hygt_pmpt pm, const int16_t* d_x, int32_t* d_y,
                              const uint16_t* d_set, int64_t nblocks, hygt_stream stream,
                              int* d_status) {
  return pmpt_run(0, pm, d_x, d_y, d_set, nblocks, stream, d_status);
}

hygt_status hygt_pmpt_inverse(hygt_pmpt pm, const int32_t* d_y, int16_t* d_x,
                              const uint16_t* d_set, int64_t nblocks, hygt_stream stream,
                              int* d_status) {
  return pmpt_run(1, pm, d_y, d_x, d_set, nblocks, stream, d_status);
}

hygt_status hygt_pmpt_forward_f32(hygt_pmpt pm, const float* d_x, float* d_y,
                                  const uint16_t* d_set, int64_t nblocks, hygt_stream stream,
                                  int* d_status) {
  return pmpt_run(2, pm, d_x, d_y, d_set, nblocks, stream, d_status);
}

hygt_status hygt_pmpt_inverse_f32(hygt_pmpt pm, const float* d_y, float* d_x,
                                  const uint16_t* d_set, int64_t nblocks, hygt_stream stream,
                                  int* d_status) {
  return pmpt_run(3, pm, d_y, d_x, d_set, nblocks, stream, d_status);
}

}  // extern "C"
