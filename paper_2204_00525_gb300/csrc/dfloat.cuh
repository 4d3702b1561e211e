// Double-float arithmetic on the FP32 pipe: a value is an unevaluated sum hi + lo of two
// floats (about 47 significant bits).  Used by the mixed-precision head/tail scans, which
// must keep their prefix sums accurate without paying for FP64 instructions (GB300 runs
// FP64 at 1/64 of the FP32 rate).
//
// Building blocks (published error-free transformations):
//   two_sum   Knuth's TwoSum: s + e == a + b exactly (6 additions).
//   fast_two  Dekker's Fast2Sum for |a| >= |b|: s + e == a + b exactly (3 additions).
//   two_prod  FMA-based product: p + e == a * b exactly (Ogita, Rump, Oishi 2005).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fig {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  dfl r;
  fast_two(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.hi, -a.lo}; }

// a * b for a double-float a and a float b.
__device__ __forceinline__ dfl df_mul_f(dfl a, float b) {
  const float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);          // two_prod error
  e = fmaf(a.lo, b, e);
  dfl r;
  fast_two(p, e, r.hi, r.lo);
  return r;
}

// Integer -> float without conversion instructions (64-bit conversions run on the FP64
// pipe of this part): a float of exponent 2^23 holds an integer below 2^23 in its
// mantissa, so or-ing the integer in and subtracting 2^23 is exact.
__device__ __forceinline__ float small_u23_to_float(uint32_t v) {     // v < 2^23
  return __uint_as_float(0x4B000000u | v) - 8388608.0f;
}

// Exact split of a non-negative integer below 2^31 into hi + lo floats: the high 15 bits
// scaled by 2^16 plus the low 16 bits, renormalised by Fast2Sum (both exact in float).
__device__ __forceinline__ dfl df_from_count(int32_t p) {
  const uint32_t u = (uint32_t)p;
  const float h = small_u23_to_float(u >> 16) * 65536.0f;
  const float l = small_u23_to_float(u & 0xFFFFu);
  dfl r;
  fast_two(h, l, r.hi, r.lo);
  return r;
}

// Split a double x into hi + lo with |x - hi - lo| <= 2^-47 |x| without FP64 or
// conversion instructions: hi takes the sign, the exponent and the leading 23 bits of
// the mantissa (truncated); lo is the remaining 29-bit integer u, rounded to a multiple of
// 64 (|error| <= 32), times 2^(e - 1075).  The rounding uses a float of exponent 2^29,
// whose mantissa steps are 64: adding (u + 32) / 64 to its bit pattern gives 2^29 + 64 k
// (a carry into the exponent gives 2^30 = 2^29 + 64 * 2^23), and subtracting 2^29 is
// exact (Sterbenz).  Outside |x| in [2^-74, 2^127] (zero, tiny or huge values) the FP64
// conversion is used instead.
// Out-of-line on purpose: inlined, the compiler if-converts this rare path and issues its
// FP64 conversions for every element.
static __device__ __noinline__ dfl df_from_double_wide(double x) {
  if (x == 0.0) return dfl{0.0f, 0.0f};
  const float h = (float)x;
  return dfl{h, (float)(x - (double)h)};
}

__device__ __forceinline__ dfl df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FFull);
  if (e < 949 || e > 1150) return df_from_double_wide(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const float h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
  const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);   // 2^(e - 1075)
  const uint32_t u = (uint32_t)(m & 0x1FFFFFFFull);
  const float k64 = __uint_as_float((156u << 23) + ((u + 32u) >> 6)) - 536870912.0f;
  float l = k64 * scale;
  if (sign) l = -l;
  return dfl{h, l};
}

__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// hi + lo as a double with integer instructions only (the conversions above issue at the
// FP64 rate).  hi's 24-bit significand is placed at bits 39-62 of a signed 64-bit integer S
// and lo's is added at its own exponent (bits below bit 0 dropped), S is renormalised by at
// most one left shift (hi a power of two, lo negative) and rounded to 53 bits (half up):
// exact whenever the sum fits in 53 bits, which a normalised pair (|lo| <= ulp(hi) / 2, as
// Fast2Sum leaves it) with lo at most 29 binades below hi's last bit does, and within one
// unit in the last place otherwise.  Zero, subnormal, infinite or NaN parts and
// unnormalised pairs take the conversions, out of line.
static __device__ __noinline__ double df_to_double_wide(float hi, float lo) { return (double)hi + (double)lo; }

__device__ __forceinline__ double df_to_double_int(float hi, float lo) {
  const uint32_t hb = __float_as_uint(hi), lb = __float_as_uint(lo);
  const int eh = (int)((hb >> 23) & 0xFFu), el = (int)((lb >> 23) & 0xFFu);
  const bool lo_zero = (lb & 0x7FFFFFFFu) == 0u;
  const int d = eh - (el == 0 ? 1 : el);          // binades between the two exponents
  if (eh == 0 || eh == 255 || (!lo_zero && (el == 255 || d < 24))) return df_to_double_wide(hi, lo);
  long long S = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 39;
  if (hb >> 31) S = -S;
  if (!lo_zero) {
    const long long L = (long long)((lb & 0x7FFFFFu) | (el ? 0x800000u : 0u));
    const int sh = 39 - d;
    const long long Lv = sh >= 0 ? (L << sh) : (sh > -24 ? (L >> -sh) : 0ll);
    S += (lb >> 31) ? -Lv : Lv;
  }
  const unsigned long long sign = S < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long M = (unsigned long long)(S < 0 ? -S : S);
  int e = eh - 127 + 1023;
  if (M < (1ull << 62)) {                        // one step below hi's binade
    M <<= 1;
    e -= 1;
  }
  M += 1ull << 9;                                // round bits 9..0 (half up)
  if (M >= (1ull << 63)) {
    M >>= 1;
    e += 1;
  }
  M >>= 10;
  return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | (M & ((1ull << 52) - 1))));
}

}  // namespace fig
