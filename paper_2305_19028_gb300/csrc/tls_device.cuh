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


// a = hi + lo + e with hi = fl32(a) (round to nearest even, as f64_to_f32_rn) and
// lo = fl32(a - hi), so |e| <= 2^-48 |a|: the FP64 value as an unevaluated pair of FP32 numbers.
// Integer arithmetic only (no FP64 instruction): with a = sig 2^E (sig the 53-bit significand),
// hi keeps the top 24 bits of sig rounded, and a - hi = D 2^E exactly with D = sig - 2^29 round(
// sig / 2^29), |D| <= 2^28. lo = 0 where hi is not a normal FP32 number (|a| < 2^-126, overflow,
// Inf, NaN): there the pair's error is below 2^-149 or the value is not finite in FP32 anyway.
static __device__ __forceinline__ void f64_split_f32(double a, float& hi, float& lo) {
  hi = f64_to_f32_rn(a);
  lo = 0.f;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  const int exp = (int)((bits >> 52) & 0x7FF);
  const int e32 = exp - 1023 + 127;
  if (exp == 0x7FF || e32 <= 0 || e32 >= 255) return;
  const unsigned long long sig = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long q = sig >> 29;
  const unsigned long long rem = sig & ((1ull << 29) - 1);
  const unsigned long long half = 1ull << 28;
  const bool up = rem > half || (rem == half && (q & 1));
  const int D = up ? (int)rem - (1 << 29) : (int)rem;           // |D| <= 2^28
  if (D == 0) return;
  // lo = D 2^E, E = exp - 1075 in [-178, 75]: one exact power-of-two product, or two when 2^E
  // is below the normal range
  const int E = exp - 1075;
  float v = __int2float_rn(D);
  if (E >= -126) {
    v *= __uint_as_float((unsigned int)(E + 127) << 23);
  } else {
    v *= __uint_as_float((unsigned int)(E + 64 + 127) << 23);
    v *= __uint_as_float((unsigned int)(127 - 64) << 23);
  }
  lo = (bits >> 63) ? -v : v;
}


// ---- double-FP32 arithmetic (error-free transforms on FP32 pairs), shared by the dense and
// batched residual passes
// (the _rn intrinsics keep the compiler from contracting a product into a later add, which
// would break the error-free transforms)
static __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += (ah + al) (xh + xl): ah xh exactly (FMA), the cross terms ah xl and al xh in
// FP32, al xl (2^-48 of the product) dropped
static __device__ __forceinline__ void df_fma(float ah, float al, float xh, float xl, float& hi,
                                       float& lo) {
  const float p = __fmul_rn(ah, xh);
  float e = __fmaf_rn(ah, xh, -p);
  e = __fmaf_rn(ah, xl, e);
  e = __fmaf_rn(al, xh, e);
  float s, t;
  two_sum(hi, p, s, t);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, e));
}


// (hi, lo) += (bh, bl): the pair sum (TwoSum of the leading parts, the low parts added)
static __device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  hi = s;
  lo = __fadd_rn(__fadd_rn(lo, bl), e);
}

}  // namespace tls
