// hygt_primary.cuh -- the integer DCT-II primary of the secondary-transform
// pipeline (Sec. VI) inside the set-bucketed HyGT kernels, for 4x4 and 8x8
// blocks, whose secondary HyGT covers every coefficient (N = M^2).
//
// The matrix C = round(256 D), D[k][i] = a_k cos(pi (2i + 1) k / (2M)),
// a_0 = sqrt(1/M), a_k = sqrt(2/M) (orthonormal DCT-II; rounded half away
// from zero), is evaluated at compile time from its definition (cosine by
// range reduction and a Taylor series, square root by Newton's method), so
// the multiply-adds take it as immediates.  No entry of 256 D lies within
// 1e-6 of a rounding tie, far above the error of these evaluations.
//
// Each 1-D stage rounds half up, y_k = floor((sum_i C[k][i] x_i + 128) / 256),
// in int32 (exact for int16 residuals: |sum| < 2^25).  Forward: rows, then
// columns; inverse: columns, then rows, with C transposed.
#pragma once

#include <stdint.h>

#include <utility>

namespace hygt {

namespace primary_detail {
constexpr double kPi = 3.14159265358979323846264338327950288;
__host__ __device__ constexpr double cos_taylor(double x) {  // |x| <= pi
  double term = 1.0, sum = 1.0;
  for (int n = 1; n < 30; ++n) {
    term *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double cos_cx(double x) {
  // reduce to [-pi, pi]
  const double two_pi = 2.0 * kPi;
  while (x > kPi) x -= two_pi;
  while (x < -kPi) x += two_pi;
  return cos_taylor(x);
}
__host__ __device__ constexpr double sqrt_cx(double v) {
  double r = v > 1.0 ? v : 1.0;
  for (int it = 0; it < 100; ++it) r = 0.5 * (r + v / r);
  return r;
}
__host__ __device__ constexpr int round_half_away(double v) {
  return v >= 0.0 ? (int)(v + 0.5) : -(int)(-v + 0.5);
}
}  // namespace primary_detail

// C[k][i] of the M-point integer DCT-II.
template <int M>
__host__ __device__ constexpr int dct_coef(int k, int i) {
  using namespace primary_detail;
  const double a = k == 0 ? sqrt_cx(1.0 / M) : sqrt_cx(2.0 / M);
  return round_half_away(256.0 * a * cos_cx(kPi * (2.0 * i + 1.0) * k / (2.0 * M)));
}

// The coefficient as a compile-time constant.
template <int M, int K, int I>
struct DctCoef {
  static constexpr int value = dct_coef<M>(K, I);
};

// out[K] = floor((sum_i C'[K][i] in[i] + 128) / 256), C' = C or C^T (TR),
// the coefficients as immediates.
template <int M, bool TR, int K, int... I>
__device__ __forceinline__ int32_t dct_dot(const int32_t* in, std::integer_sequence<int, I...>) {
  uint32_t acc = 128u;
  ((acc += (uint32_t)DctCoef<M, TR ? I : K, TR ? K : I>::value * (uint32_t)in[I]), ...);
  return (int32_t)acc >> 8;
}

template <int M, bool TR, int... K>
__device__ __forceinline__ void dct_stage_seq(const int32_t* in, int32_t* out,
                                              std::integer_sequence<int, K...>) {
  ((out[K] = dct_dot<M, TR, K>(in, std::make_integer_sequence<int, M>())), ...);
}

// One 1-D stage on M values in registers.
template <int M, bool TR>
__device__ __forceinline__ void dct_stage(const int32_t* in, int32_t* out) {
  dct_stage_seq<M, TR>(in, out, std::make_integer_sequence<int, M>());
}

}  // namespace hygt
