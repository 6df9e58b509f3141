// fp_bits.h -- double-FP32 values (hi + lo) of the tensor-core form: their
// running sum, and conversions between FP64 and double-FP32 by integer
// operations on the bits, for the prologue and the epilogues (this part's
// FP64 pipe runs at 1/64 of the FP32 rate, and these conversions touch every
// value of M and every running sum of a tile).  Each conversion equals its
// plain-FP64 counterpart bit for bit (the same rounding), with the FP64 route
// kept for the rare inputs outside the fast path.  The file compiles as CUDA
// device code and as host C++, so the CPU tests check it with g++
// (tests/test_fp_bits.py).
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define FPB_HD __host__ __device__ __forceinline__
#define FPB_HD_NOINLINE __host__ __device__ __noinline__
#else
#define FPB_HD inline
#define FPB_HD_NOINLINE inline
#endif

namespace modal {
namespace fpb {

FPB_HD uint32_t f_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
#endif
}
FPB_HD float f_from(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, 4);
  return x;
#endif
}
FPB_HD uint64_t d_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, 8);
  return u;
#endif
}
FPB_HD double d_from(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, 8);
  return x;
#endif
}
// int -> float, rounded to nearest (ties to even)
FPB_HD float int_to_f_rn(int i) {
#ifdef __CUDA_ARCH__
  return __int2float_rn(i);
#else
  return (float)i;
#endif
}

// out of line: inlined in every unrolled epilogue it cost the GEMM 3.5 %
FPB_HD_NOINLINE double f32_scaled_f64_slow(float x, int e) { return ldexp((double)x, e); }

// x 2^e as a double (= ldexp((double)x, e)), assembled from the bits of x.
// Exact; a zero keeps its sign; a subnormal x, or a result outside the
// normal double range, goes through ldexp.  A double-FP32 value (hi, lo)
// scaled by 2^e is then f32_scaled_f64(hi, e) + f32_scaled_f64(lo, e), one
// exact FP64 addition.
FPB_HD double f32_scaled_f64(float x, int e) {
  const uint32_t u = f_bits(x);
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  if ((u & 0x7fffffffu) == 0u) return d_from(sign);
  const uint32_t ex = (u >> 23) & 0xffu;
  const int E = (int)ex + (1023 - 127) + e;
  if (ex == 0u || ex == 0xffu || E <= 0 || E >= 2047) return f32_scaled_f64_slow(x, e);
  return d_from(sign | ((uint64_t)E << 52) | ((uint64_t)(u & 0x7fffffu) << 29));
}

struct f2 {
  float h, l;
};

// x as hi + lo: hi = x rounded to FP32, lo = (x - hi) rounded to FP32
FPB_HD f2 df_from_d(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

// out of line, so that the rare inputs' FP64 route is a branch taken only by
// them rather than work every caller does
FPB_HD_NOINLINE f2 df_from_d_slow(double x) { return df_from_d(x); }

// The same split with integer operations: hi is x rounded to 24 significant
// bits (to nearest, ties to even), and x - hi, an integer of at most 29 bits
// times 2^(e - 52), goes to FP32 through the rounding integer-to-float
// conversion and an exponent shift.  Zeros, and exponents where hi or lo
// could leave the normal FP32 range (|x| < 2^-73 or >= 2^127), take
// df_from_d.
FPB_HD f2 df_from_d_fast(double x) {
  const uint64_t u = d_bits(x);
  const int ex = (int)((u >> 52) & 0x7ffu);
  if (ex < 950 || ex > 1149) return df_from_d_slow(x);
  const uint32_t sign = (uint32_t)(u >> 63) << 31;
  const uint64_t mant = (u & 0xfffffffffffffull) | (1ull << 52);
  uint32_t m24 = (uint32_t)(mant >> 29);
  int rem = (int)(mant & 0x1fffffffu);  // units of 2^(e - 52)
  if (rem > (1 << 28) || (rem == (1 << 28) && (m24 & 1u))) {
    ++m24;
    rem -= 1 << 29;
  }
  int eh = ex - 1023 + 127;
  if (m24 == (1u << 24)) {  // rounded up to the next power of two
    m24 >>= 1;
    ++eh;
  }
  const float h = f_from(sign | ((uint32_t)eh << 23) | (m24 & 0x7fffffu));
  if (rem == 0) return {h, 0.f};
  const int r = (int)f_bits(int_to_f_rn(rem)) + ((ex - 1075) * (1 << 23));
  return {h, f_from((uint32_t)r ^ sign)};
}

// (hi, lo) += (bh, bl): the running double-FP32 sums of the GEMM drains
// (compensated summation of the chunk sums across the slices).  The high
// parts meet in an error-free two-sum (Knuth); the low parts and that error
// are added in FP32 and the pair is renormalised -- ~2^-48 of the sum per
// step, FP32 operations only.
FPB_HD void df_add(float &hi, float &lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  float e = (hi - (s - bb)) + (bh - bb);
  e += lo + bl;
  hi = s + e;
  lo = e - (hi - s);
}

}  // namespace fpb
}  // namespace modal
