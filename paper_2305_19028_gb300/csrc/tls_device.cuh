// Device helpers shared by several translation units.
#pragma once
#include <cstdint>

namespace tls {

// FP64 -> FP32 conversion with round-to-nearest-even, done with integer instructions only
// (the FP64 pipe, which the hardware conversion uses, is far too narrow on this GPU to convert
// every entry of A). Handles zeros, FP32 subnormals, overflow to infinity and NaN.
static __device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(bits >> 63) << 31;
  const int exp = (int)((bits >> 52) & 0x7FF);
  const unsigned long long mant = bits & 0xFFFFFFFFFFFFFull;
  if (exp == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (mant ? 0x400000u : 0u));
  int e32 = exp - 1023 + 127;
  if (e32 >= 255) return __uint_as_float(sign | 0x7F800000u);
  // significand with the implicit bit, 53 bits; keep 24 (normal) or fewer (subnormal)
  unsigned long long sig = (exp == 0) ? mant : (mant | (1ull << 52));
  int shift = 29;                       // 53 - 24
  if (e32 <= 0) {                        // FP32 subnormal (or underflow to zero)
    shift += 1 - e32;
    e32 = 0;
    if (shift > 63) return __uint_as_float(sign);
  }
  const unsigned long long q = sig >> shift;
  const unsigned long long rem = sig & ((1ull << shift) - 1);
  const unsigned long long half = 1ull << (shift - 1);
  unsigned long long r = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
  // r holds the 24-bit significand (with the implicit bit for normals); a carry bumps the exponent
  unsigned int out;
  if (e32 == 0) {
    out = (unsigned int)r;               // subnormal (a carry into bit 23 gives the smallest normal)
  } else {
    if (r == (1ull << 24)) { r >>= 1; ++e32; }
    if (e32 >= 255) return __uint_as_float(sign | 0x7F800000u);
    out = ((unsigned int)e32 << 23) | ((unsigned int)r & 0x7FFFFFu);
  }
  return __uint_as_float(sign | out);
}


}  // namespace tls
