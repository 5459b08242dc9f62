// hygt_secondary.cuh -- the secondary-transform pipeline of Sec. VI in one
// kernel (sm_103a): integer 2-D DCT-II primary of an M x M residual block,
// then the integer HyGT on the top-left s x s coefficients (s = 4 for 4 x 4
// blocks, 8 for 8 x 8 and larger), the other coefficients passed through;
// the inverse runs the inverse HyGT on the sub-block, then the inverse
// DCT-II, and saturates to int16.
//
// Primary (the paper does not fix it; read as the orthonormal DCT-II with
// the HyGT's 8-bit precision): C = round(256 D), D[k][i] =
// a_k cos(pi (2i + 1) k / (2M)); each 1-D stage rounds half up,
// y_k = floor((sum_i C[k][i] x_i + 128) / 256); forward rows then columns,
// inverse columns then rows with C^T.  The sub-block is the HyGT's vector in
// raster order.  Every sum stays within int32 for int16 residuals
// (|C| <= 256 sqrt(2/M)).
//
// Mapping.  A warp task is G = max(1, 512 / M^2) consecutive blocks in two
// shared-memory regions per block (A and B, M^2 + 1 words each): the warp
// copies the blocks in (coalesced), computes the row stage A -> B and the
// column stage B -> A with one output per lane-item (M multiply-adds each,
// C cached in shared memory), applies the HyGT passes to the sub-block in A
// (one rotation per lane-item, multipliers from the plan's packed table,
// the permutation slots through B), and copies the blocks out.  The HyGT's
// rounding and int32 arithmetic are those of the other integer kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hygt {

constexpr int kSecThreads = 256;
constexpr int kSecMaxM = 32;

struct SecondaryParams {
  const void* in;
  void* out;
  const uint16_t* set;
  long long nblocks;
  int log2m;            // primary block side M = 2^log2m (2..5)
  int log2n;            // HyGT size N = s^2 (4 or 6)
  int rounds, num_sets, frac_bits;
  unsigned perm_mask;
  const uint32_t* tab;  // (c | s << 16) per pair, [S][R][log2n][N/2]
  const uint8_t* perm;  // [S][R][N] or nullptr
  int group;            // blocks per warp task
  int* status;
  int16_t C[kSecMaxM * kSecMaxM];  // primary matrix, row k = basis k
};

// Shared memory of one launch (bytes).
__host__ __device__ inline size_t secondary_smem(int log2m, int group) {
  const int M2 = 1 << (2 * log2m);
  return (size_t)(1 << (2 * log2m)) * 4 +                                  // C
         (size_t)(kSecThreads / 32) * ((size_t)2 * group * (M2 + 1) + group) * 4;
}

cudaError_t launch_secondary(int inverse, const SecondaryParams& p, cudaStream_t stream);

}  // namespace hygt
