// secondary.cu -- kernel and launcher of the secondary-transform pipeline
// (see hygt_secondary.cuh).
#include "hygt_launch.cuh"
#include "hygt_secondary.cuh"

namespace hygt {

// One separable primary stage over the task's blocks: src -> dst.  dim 0:
// along rows (item = block, row, k); dim 1: along columns (item = block,
// k, column).  TR: use C^T (inverse).
template <bool TR>
__device__ __forceinline__ void sec_stage(const int32_t* src, int32_t* dst, const int32_t* C,
                                          int M, int log2m, int nb, int RS, int dim, int lane) {
  const int M2 = M * M;
  for (int w = lane; w < nb * M2; w += 32) {
    const int blk = w >> (2 * log2m);
    const int r = (w >> log2m) & (M - 1), k = w & (M - 1);
    const int32_t* s = src + blk * RS;
    uint32_t acc = 128u;
    if (dim == 0) {  // output (row r, k) from row r
#pragma unroll 8
      for (int i = 0; i < M; ++i)
        acc += (uint32_t)(TR ? C[i * M + k] : C[k * M + i]) * (uint32_t)s[r * M + i];
      dst[blk * RS + r * M + k] = (int32_t)acc >> 8;
    } else {         // output (k, column r) from column r
#pragma unroll 8
      for (int i = 0; i < M; ++i)
        acc += (uint32_t)(TR ? C[i * M + k] : C[k * M + i]) * (uint32_t)s[i * M + r];
      dst[blk * RS + k * M + r] = (int32_t)acc >> 8;
    }
  }
  __syncwarp();
}

template <int INV>
__global__ void __launch_bounds__(kSecThreads) hygt_secondary_kernel(const SecondaryParams p) {
  extern __shared__ __align__(16) int32_t ssm[];
  const int log2m = p.log2m, M = 1 << log2m, M2 = M * M;
  const int s = 1 << (p.log2n >> 1), log2s = p.log2n >> 1;
  const int N = 1 << p.log2n, half = N >> 1;
  const int G = p.group, RS = M2 + 1;
  int32_t* C = ssm;
  for (int i = threadIdx.x; i < M2; i += blockDim.x) C[i] = p.C[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpc = blockDim.x >> 5;
  int32_t* A = ssm + M2 + (size_t)warp * (2 * G * RS + G);
  int32_t* B = A + G * RS;
  int* bset = B + G * RS;
  const long long ntasks = (p.nblocks + G - 1) / G;
  const uint32_t rnd = 1u << (p.frac_bits - 1);
  const int f = p.frac_bits;
  const int R = p.rounds;

  for (long long t = (long long)blockIdx.x * wpc + warp; t < ntasks;
       t += (long long)gridDim.x * wpc) {
    const long long b0 = t * G;
    const int nb = (int)min((long long)G, p.nblocks - b0);
    for (int e = lane; e < nb * M2; e += 32) {
      const int blk = e >> (2 * log2m), i = e & (M2 - 1);
      const long long g = b0 * M2 + e;
      A[blk * RS + i] = INV ? __ldcs(static_cast<const int32_t*>(p.in) + g)
                            : (int32_t)__ldcs(static_cast<const int16_t*>(p.in) + g);
    }
    for (int k = lane; k < nb; k += 32) {
      const int st = p.set ? (int)__ldg(p.set + b0 + k) : 0;
      bset[k] = st;
      if (st != 0xFFFF && st >= p.num_sets && p.status) atomicCAS(p.status, 0, 4);
    }
    __syncwarp();
    if (!INV) {
      sec_stage<false>(A, B, C, M, log2m, nb, RS, 0, lane);  // rows
      sec_stage<false>(B, A, C, M, log2m, nb, RS, 1, lane);  // columns
    }
    // the HyGT on the top-left s x s coefficients (element e at row e / s,
    // column e mod s of the block)
    for (int rr = 0; rr < R; ++rr) {
      const int r = INV ? R - 1 - rr : rr;
      const bool has_perm = p.perm && ((p.perm_mask >> r) & 1u);
      if (INV && has_perm) {  // undo slot r's gather: v_prev[perm[i]] = v[i]
        for (int w = lane; w < nb * N; w += 32) {
          const int blk = w >> p.log2n, i = w & (N - 1);
          const int st = bset[blk];
          if (st >= p.num_sets) continue;
          const int d = __ldg(p.perm + ((size_t)st * R + r) * N + i);
          B[blk * RS + d] = A[blk * RS + (i >> log2s) * M + (i & (s - 1))];
        }
        __syncwarp();
        for (int w = lane; w < nb * N; w += 32) {
          const int blk = w >> p.log2n, i = w & (N - 1);
          if (bset[blk] >= p.num_sets) continue;
          A[blk * RS + (i >> log2s) * M + (i & (s - 1))] = B[blk * RS + i];
        }
        __syncwarp();
      }
      for (int pp = 0; pp < p.log2n; ++pp) {
        const int ps = INV ? p.log2n - 1 - pp : pp;
        for (int w = lane; w < nb * half; w += 32) {
          const int blk = w >> (p.log2n - 1), j = w & (half - 1);
          const int st = bset[blk];
          if (st >= p.num_sets) continue;  // skip sentinel or bad index
          const int m = ((j >> ps) << (ps + 1)) | (j & ((1 << ps) - 1));
          const int n = m + (1 << ps);
          const uint32_t cs = __ldg(p.tab + (((size_t)st * R + r) * p.log2n + ps) * half + j);
          const int32_t c = (int32_t)(int16_t)(cs & 0xFFFFu);
          const int32_t s0 = (int32_t)cs >> 16;
          const int32_t sn = INV ? -s0 : s0;
          int32_t* pm = A + blk * RS + (m >> log2s) * M + (m & (s - 1));
          int32_t* pn = A + blk * RS + (n >> log2s) * M + (n & (s - 1));
          const uint32_t a = (uint32_t)*pm, b = (uint32_t)*pn;
          *pm = (int32_t)((uint32_t)c * a + (uint32_t)sn * b + rnd) >> f;
          *pn = (int32_t)((uint32_t)c * b - (uint32_t)sn * a + rnd) >> f;
        }
        __syncwarp();
      }
      if (!INV && has_perm) {  // gather of slot r: v'[i] = v[perm[i]]
        for (int w = lane; w < nb * N; w += 32) {
          const int blk = w >> p.log2n, i = w & (N - 1);
          const int st = bset[blk];
          if (st >= p.num_sets) continue;
          const int src = __ldg(p.perm + ((size_t)st * R + r) * N + i);
          B[blk * RS + i] = A[blk * RS + (src >> log2s) * M + (src & (s - 1))];
        }
        __syncwarp();
        for (int w = lane; w < nb * N; w += 32) {
          const int blk = w >> p.log2n, i = w & (N - 1);
          if (bset[blk] >= p.num_sets) continue;
          A[blk * RS + (i >> log2s) * M + (i & (s - 1))] = B[blk * RS + i];
        }
        __syncwarp();
      }
    }
    if (INV) {
      sec_stage<true>(A, B, C, M, log2m, nb, RS, 1, lane);  // columns
      sec_stage<true>(B, A, C, M, log2m, nb, RS, 0, lane);  // rows
    }
    for (int e = lane; e < nb * M2; e += 32) {
      const int blk = e >> (2 * log2m), i = e & (M2 - 1);
      const long long g = b0 * M2 + e;
      const int st = bset[blk];
      const bool bad = st != 0xFFFF && st >= p.num_sets;
      const int32_t v = bad ? 0 : A[blk * RS + i];
      if (INV)
        __stcs(static_cast<int16_t*>(p.out) + g, (int16_t)max(-32768, min(32767, v)));
      else
        __stcs(static_cast<int32_t*>(p.out) + g, v);
    }
    __syncwarp();
  }
}

cudaError_t launch_secondary(int inverse, const SecondaryParams& p, cudaStream_t stream) {
  int dev = 0;
  cudaGetDevice(&dev);
  const DeviceInfo info = device_info(dev);
  const size_t smem = secondary_smem(p.log2m, p.group);
  const int wpc = kSecThreads / 32;
  const long long ntasks = (p.nblocks + p.group - 1) / p.group;
  const int per_sm = (int)(info.max_smem_optin / (smem + 1024));
  long long grid = (long long)info.sms * (per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm));
  if ((ntasks + wpc - 1) / wpc < grid) grid = (ntasks + wpc - 1) / wpc;
  if (grid < 1) grid = 1;
  auto kern = inverse ? hygt_secondary_kernel<1> : hygt_secondary_kernel<0>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<(int)grid, kSecThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace hygt
