// Scalar fixed-point arithmetic of the FP64-accurate split products
// (oz_gemm.cu; Ozaki, Ogita, Oishi & Rump 2012), host and device: the
// kernels call it, and CPU tests compile it for the host and check it
// against the definitions in exact arithmetic.
//   oz_digits       one FP64 value x below a given exponent ex (|x| < 2^ex)
//                   as OZ_S = 8 balanced signed 8-bit digits, each returned
//                   as the bf16 bit pattern of the integer (|q| <= 128,
//                   exact in bf16);
//   oz_fixed_value  the exact int64 sums of a product back to FP64,
//                   correctly rounded.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#endif

namespace mpl {

OZ_HD unsigned long long oz_bits_of_double(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

OZ_HD float oz_float_of_bits(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof f);
  return f;
#endif
}

OZ_HD double oz_double_of_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

OZ_HD uint32_t oz_bits_of_float(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  std::memcpy(&b, &f, sizeof b);
  return b;
#endif
}

// Signed field of len bits of x starting at bit pos.
OZ_HD int oz_sext_field(uint32_t x, int pos, int len) {
  return ((int)(x << (32 - pos - len))) >> (32 - len);
}

// bf16 bit pattern of an integer |q| <= 256 (at most 8 significant bits, so
// exact): 1.5 2^23 + q is exact in FP32, removing 1.5 2^23 leaves q, and
// the upper half of q's FP32 pattern is its bf16 pattern.  Two full-rate
// operations instead of an integer-to-float conversion.
OZ_HD uint16_t oz_bf16_of_small_int(int q) {
  const float fq = oz_float_of_bits(0x4B400000u + (uint32_t)q) - 12582912.0f;
  return (uint16_t)(oz_bits_of_float(fq) >> 16);
}

// x is taken from its bit pattern to the 64-bit fixed point
// U = round(x 2^(63 - ex)) (half away from zero), |U| < 2^63, and
// U = sum_i q_i 2^(56 - 8i) exactly, each q_i the nearest integer (half up)
// of what remains above 2^(56 - 8i) after the digits before it.  Same value
// as x 2^(7 - ex) = sum_i q_i 2^(-8i) up to 2^(ex - 64).
//
// What remains above 2^(56 - 8i) is the low 64 - 8i bits of U read as a
// two's-complement number (each half-up digit leaves a remainder in
// [-2^(s-1), 2^(s-1)), s = 64 - 8i), so q_i = floor(t_i / 2 + 1/2) with t_i
// the signed 9-bit field of U at bits 63 - 8i .. 55 - 8i, and the last digit
// is the signed low byte: eight 32-bit field extractions on the integer
// pipes (GB300 runs FP64 at 1/64 of the FP32 rate), no 64-bit shifts or
// subtractions.
OZ_HD void oz_digits(double x, int ex, uint16_t out[8]) {
  const unsigned long long bits = oz_bits_of_double(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  const long long frac = (long long)(bits & 0xFFFFFFFFFFFFFULL);
  const long long M = E ? (frac | (1LL << 52)) : frac;  // |x| = M 2^(max(E, 1) - 1075)
  const int sft = (E ? E : 1) - 1075 + 63 - ex;          // U = M 2^sft
  long long U;
  if (M == 0 || sft <= -64) U = 0;
  else if (sft >= 0) U = M << sft;                       // below 2^63 because |x| < 2^ex
  else U = (M >> (-sft)) + ((M >> (-sft - 1)) & 1);      // nearest, half up
  if (bits >> 63) U = -U;
  const uint32_t lo = (uint32_t)(unsigned long long)U, hi = (uint32_t)((unsigned long long)U >> 32);
  const uint32_t mid = (hi << 1) | (lo >> 31);           // bits 62 .. 31 of U
  out[0] = oz_bf16_of_small_int((oz_sext_field(hi, 23, 9) + 1) >> 1);
  out[1] = oz_bf16_of_small_int((oz_sext_field(hi, 15, 9) + 1) >> 1);
  out[2] = oz_bf16_of_small_int((oz_sext_field(hi, 7, 9) + 1) >> 1);
  out[3] = oz_bf16_of_small_int((oz_sext_field(mid, 0, 9) + 1) >> 1);
  out[4] = oz_bf16_of_small_int((oz_sext_field(lo, 23, 9) + 1) >> 1);
  out[5] = oz_bf16_of_small_int((oz_sext_field(lo, 15, 9) + 1) >> 1);
  out[6] = oz_bf16_of_small_int((oz_sext_field(lo, 7, 9) + 1) >> 1);
  out[7] = oz_bf16_of_small_int(oz_sext_field(lo, 0, 8));
}

// x 2^k: a multiplication by the power of two when 2^k is a normal double
// (exact unless the result is subnormal), ldexp otherwise -- the value of
// ldexp(x, k) without its FP64 instruction sequence on the device.
OZ_HD double oz_scale2(double x, int k) {
  if (k >= -1022 && k <= 1023) return x * oz_double_of_bits((unsigned long long)(k + 1023) << 52);
  return ldexp(x, k);
}

// The FP64 value of one accumulator pair of a product, 2^ex (hi 2^-24 +
// lo 2^-56) = 2^(ex - 56) (top 2^32 + low) with top = hi + floor(lo / 2^32)
// and low = lo mod 2^32 (|hi| < 2^59, |lo| < 2^62, so |top| < 2^60), rounded
// once to nearest-even (while the result is normal):
//   -2^53 <= top < 2^53: top and low are exact doubles, so the one addition
//     is the only rounding;
//   otherwise the exact value top + low 2^-32 has magnitude >= 2^53, its unit
//     in the last place is >= 2 units of top, the rounding midpoints are
//     integers, and low only decides on which side of a midpoint at top the
//     value lies: 2 top + [low != 0] (a sticky bit below top, < 2^61) rounded
//     once and halved gives the same double.
OZ_HD double oz_fixed_value(long long hi, long long lo, int ex) {
  const long long top = hi + (lo >> 32);
  const long long low = lo & 0xFFFFFFFFLL;
  if (top >= -(1LL << 53) && top < (1LL << 53))
    return oz_scale2((double)top, ex - 24) + oz_scale2((double)low, ex - 56);
  return oz_scale2((double)(2 * top + (low != 0 ? 1 : 0)), ex - 25);
}

}  // namespace mpl
