// FP64 <-> FP32 conversions in integer arithmetic.
//
// On GB300 the hardware conversion instructions between FP64 and FP32 issue
// to the FP64 pipe, whose throughput is about 1/60 of the FP32 pipe; the
// integer pipe is not the bottleneck of these kernels.  Both functions work
// directly on the IEEE-754 binary64 / binary32 bit layouts:
//   binary64: sign (1) | exponent (11, bias 1023) | fraction (52)
//   binary32: sign (1) | exponent (8, bias 127)   | fraction (23)
// Values outside the binary32 normal range are handled as follows: magnitudes
// below 2^-126 become signed zero (no subnormals), magnitudes of 2^128 or more
// and NaN become signed infinity, so the kernels' non-finite check still fires.
#pragma once

#include <cstdint>

namespace dg {

// binary64 -> binary32, rounding to nearest (ties away from zero).
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned sign = static_cast<unsigned>(bits >> 32) & 0x80000000u;
  const unsigned long long mag = bits & 0x7fffffffffffffffull;
  // Add half a binary32 ulp at fraction bit 28, then keep exponent and the top
  // 23 fraction bits: (mag >> 29) holds the 11-bit exponent in bits 33..23 of
  // a 64-bit value; its low 32 bits hold exponent bits 8..0 in bits 31..23.
  // The rebias by -896 (= 1023 - 127) is, modulo 2^9 on that 9-bit field, an
  // addition of 128 << 23.
  const unsigned long long r = mag + (1ull << 28);
  unsigned f = static_cast<unsigned>(r >> 29) + 0x40000000u;
  const unsigned hi = static_cast<unsigned>(mag >> 32);
  f = hi < 0x38100000u ? 0u : f;              // below 2^-126: zero
  f = hi >= 0x47f00000u ? 0x7f800000u : f;     // 2^128 and above, inf, NaN
  return __uint_as_float(f | sign);
}

// binary32 -> binary64, exact for normal numbers.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned sign = b & 0x80000000u;
  const unsigned mag = b & 0x7fffffffu;
  // exponent rebias +896 at bit 20 of the high word; fraction split 20 + 3 bits
  unsigned hi = (mag >> 3) + 0x38000000u;
  unsigned lo = b << 29;
  hi = mag < 0x00800000u ? 0u : hi;            // zero and subnormals: zero
  lo = mag < 0x00800000u ? 0u : lo;
  hi = mag >= 0x7f800000u ? 0x7ff00000u : hi;  // inf, NaN: infinity
  lo = mag >= 0x7f800000u ? 0u : lo;
  return __hiloint2double(static_cast<int>(hi | sign), static_cast<int>(lo));
}

// binary32 -> binary64 for finite inputs (exact for normal numbers; zero and
// subnormals give zero).  Infinity and NaN are not preserved -- callers that
// use it detect non-finite inputs themselves.
__device__ __forceinline__ double f32_to_f64_finite(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned mag = b & 0x7fffffffu;
  const bool tiny = mag < 0x00800000u;
  const unsigned hi = tiny ? 0u : ((mag >> 3) + 0x38000000u) | (b & 0x80000000u);
  const unsigned lo = tiny ? 0u : b << 29;
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

template <typename TO, typename TI>
__device__ __forceinline__ TO cvt(TI x) {
  if constexpr (sizeof(TO) == sizeof(TI)) {
    return x;
  } else if constexpr (sizeof(TO) == 4) {
    return f64_to_f32(x);
  } else {
    return f32_to_f64(x);
  }
}

}  // namespace dg
