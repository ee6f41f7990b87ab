#pragma once

#include <cstdint>

namespace ite {

// Format conversions by integer operations on the bit patterns.  GB300 runs
// FP64 instructions, conversions from and to FP64 among them, at 1/64 of the
// fp32 rate, and these kernels convert every element they move.
//
// double -> binary format with `mb` mantissa bits and an 8-bit exponent (bf16:
// mb = 7, fp32: mb = 23), rounded to nearest even; magnitudes below the
// format's normal range become signed zero, above it infinity.  Returns the
// bit pattern in the low 1 + 8 + mb bits.
template <int MB>
__device__ __forceinline__ uint32_t dbl_to_e8(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << (8 + MB);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return sign | (0xFFu << MB) | (m ? (1u << (MB - 1)) : 0u);
  int ex = e - 1023 + 127;
  if (ex <= 0) return sign;
  constexpr int SH = 52 - MB;
  unsigned long long mant = m >> SH;
  const unsigned long long rem = m & ((1ull << SH) - 1), half = 1ull << (SH - 1);
  if (rem > half || (rem == half && (mant & 1))) {
    if (++mant == (1ull << MB)) {
      mant = 0;
      ++ex;
    }
  }
  if (ex >= 255) return sign | (0xFFu << MB);
  return sign | ((uint32_t)ex << MB) | (uint32_t)mant;
}

// fp32 -> double, exact (subnormal inputs included)
__device__ __forceinline__ double f32_to_dbl(float f) {
  const uint32_t u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  int e = (int)((u >> 23) & 0xFF);
  uint32_t m = u & 0x7FFFFFu;
  if (e == 0xFF) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | ((unsigned long long)m << 29)));
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)sign);
    const int lz = __clz(m) - 8;                       // shift the leading 1 to bit 23
    m = (m << lz) & 0x7FFFFFu;
    e = 1 - lz;
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) |
                                          ((unsigned long long)m << 29)));
}

__device__ __forceinline__ float dbl_to_f32(double x) { return __uint_as_float(dbl_to_e8<23>(x)); }

}  // namespace ite
