// oz_split.h -- the exponent-aligned BF16 slicing of the tensor-core form
// (Ozaki scheme): one double-FP32 value, scaled so that |H + L| <= 2^BETA,
// as five slices of BETA = 7 bits.  Compiles as CUDA device code and as host
// C++ (FP32 additions with round-to-nearest on both), so the CPU tests check
// the bounds below on this very code (tests/test_oz_split.py).
//
// Slice s is the running residual rounded to a multiple of 2^(-BETA s)
// (round to nearest, by adding and removing 1.5 2^(23 - BETA s)), so each
// slice carries its own weight.  The first three slices come from H alone,
// with exact residuals; the residual is then at most 2^-15 and takes the low
// part L in one FP32 addition whose rounding is below 2^-37; the last two
// slices come from that sum.  Slices s >= 1 are integer multiples of
// 2^(-BETA s) of magnitude <= 64, except the fourth: <= 64.5 + |L| 2^21 (it
// rounds the residual plus L), which stays below 256 for |L| <= 2^-14 -- so
// every slice is exact in BF16 and the levels 0 and 1 never see L.  |H + L - sum of slices| <= 2^-29 + 2^-37
// (2^-36 of the scale 2^7).
#pragma once

#ifdef __CUDACC__
#define OZS_HD __host__ __device__ __forceinline__
#else
#define OZS_HD inline
#endif

namespace modal {
namespace ozs {

constexpr int BETA = 7;    // bits per slice
constexpr int SLICES = 5;  // slices per value
constexpr int FOLD = 3;    // slice before which L joins the residual

#ifdef __CUDACC__
__host__ __device__
#endif
constexpr float pow2c(int k) {
  return k >= 0 ? (float)(1ull << k) : 1.0f / (float)(1ull << -k);
}

OZS_HD float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
OZS_HD float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

OZS_HD void split_hl(float H, float L, float (&q)[SLICES]) {
  float r = H;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int s = 0; s < SLICES; ++s) {
    const float m = 1.5f * pow2c(23 - BETA * s);
    if (s == FOLD) r = add_rn(r, L);
    q[s] = sub_rn(add_rn(r, m), m);
    if (s + 1 < SLICES) r = sub_rn(r, q[s]);  // exact
  }
}

}  // namespace ozs
}  // namespace modal
