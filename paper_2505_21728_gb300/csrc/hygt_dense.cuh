// hygt_dense.cuh -- parameters of the dense matrix-transform kernels.
#pragma once

#include <stdint.h>

#include <cuda_runtime.h>

namespace hygt {

struct DenseParams {
  const int16_t* x;             // [B][N]
  float* y;                     // [B][N] (BF16 kernel)
  int32_t* yint;                // [B][N] (integer kernel)
  const int* order;             // schedule (tiles of 128 blocks)
  const int* starts;
  const int* meta;
  long long nblocks;
  long long tmax;
  const unsigned char* kimg;    // BF16 swizzled images, [S][N * N * 2 bytes]
  const unsigned char* kimg8;   // E4M3 swizzled images (K padded to 128), [S][N * max(N, 128) bytes]
  const float* kscale;          // E4M3 scale of each set's matrix, [S]
  const int16_t* kint;          // integer matrices round(2^f K), [S][N][N]
  int num_sets;
  int frac_bits;
  int* status;
};

// kind 0: BF16 tensor cores (N = 64, 256); kind 1: int32 CUDA cores (N = 16, 64);
// kind 2: FP8 (E4M3, per-block and per-set scales) tensor cores (N = 64, 256).
cudaError_t launch_dense(int log2n, int kind, const DenseParams& p, cudaStream_t stream);

}  // namespace hygt
