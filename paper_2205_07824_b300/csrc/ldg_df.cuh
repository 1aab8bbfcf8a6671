// Double-float arithmetic on the FP32 pipes: a value is the unevaluated sum h + l of two
// floats (Dekker's double-length numbers, Numer. Math. 18, 1971), carrying a 48-bit
// significand. Sums use Knuth's error-free TwoSum (TAOCP vol. 2, 4.2.2), products the
// exact FMA form of Dekker's TwoProduct (p = a*b rounded, e = fma(a, b, -p)).
//
// Every rounding step is written with the _rn intrinsics, which the compiler neither
// contracts into FMAs nor reassociates: the error-free transformations rely on each
// operation being rounded exactly once.
//
// Accuracy. Converting an FP64 value keeps its leading 24 significant bits in h and the
// next 29 rounded to 24 in l (relative error < 2^-47); a sum or product adds a relative
// error of a few units of 2^-48 of its operands (the l*l term of a product is dropped).
// A length-n dot product therefore carries about n 2^-48 times the sum of |terms|, as an
// FP64 one carries n 2^-53 times it. Range: a pair keeps its 48 bits while l is a normal
// float, for magnitudes from about 2^-102 (2e-31) to 2^128 (3e38); below, l goes
// subnormal and the precision falls off; FP64 values below 2^-126 convert to zero and
// above the float range to infinity.
#pragma once
#include <cuda_runtime.h>

namespace ldg {

struct __align__(8) df {
  float h, l;
  df() = default;
  __host__ __device__ constexpr df(float hi, float lo) : h(hi), l(lo) {}
  __device__ __forceinline__ explicit df(double x);
  __device__ __forceinline__ explicit df(int x) : h((float)x), l(0.f) {}
  __device__ __forceinline__ explicit operator double() const;
};

// product a*b before normalisation: p = fl(a.h b.h) and everything else in e
struct dfp {
  float p, e;
  __device__ __forceinline__ operator df() const;
};

// dot-product accumulator: s is the running float sum, c collects every rounding error
// (and the low parts) in plain float; normalised once, when converted to df
struct dfa {
  float s, c;
  dfa() = default;
  __device__ __forceinline__ explicit dfa(int) : s(0.f), c(0.f) {}
  __device__ __forceinline__ dfa(df x) : s(x.h), c(x.l) {}
  __device__ __forceinline__ dfa(dfp x) : s(x.p), c(x.e) {}
  __device__ __forceinline__ operator df() const;
};

// s + e exactly, when |a| >= |b| or a == 0 (Dekker's Fast2Sum)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// a + b = s + err exactly, for any a, b (Knuth's TwoSum)
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Split of an FP64 value by its bits: h = x truncated to 24 significant bits (exactly a
// float), l = the remaining 29 bits rounded to a float. Integer work only, plus one
// integer-to-float conversion, so the FP64 unit is not involved.
__device__ __forceinline__ df::df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int ex = (int)((hw >> 20) & 0x7ffu);  // biased FP64 exponent
  const unsigned sign = hw & 0x80000000u;
  // float with the same sign, exponent ex - 1023 + 127 and FP64 mantissa bits 51..29
  const unsigned fb = sign | ((unsigned)(ex - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
  // the rest, (lw mod 2^29) * 2^(ex - 1075), with the sign of x; the power of two is
  // applied in one factor, or as 2^(ex - 975) * 2^-100 where 2^(ex - 1075) is no
  // normal float (ex < 949)
  const bool one = ex >= 949;
  const float s1 = __uint_as_float((unsigned)(one ? ex - 948 : ex - 848) << 23);
  const float s2 = one ? 1.f : 0x1p-100f;
  const float rest = __fmul_rn(__fmul_rn(__uint2float_rn(lw & 0x1fffffffu), s1), s2);
  const bool normal = ex >= 897 && ex <= 1150;
  // above the float range: infinity, or a quiet NaN for a NaN
  const unsigned big = sign | 0x7f800000u | ((ex == 2047 && ((hw & 0xfffffu) | lw)) ? 0x400000u : 0u);
  h = normal ? __uint_as_float(fb) : (ex > 1150 ? __uint_as_float(big) : 0.f);
  l = normal ? __uint_as_float(__float_as_uint(rest) | sign) : 0.f;
}

// h + l in FP64: both floats widened exactly by their bits, one FP64 add
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((unsigned long long)u << 32));  // +-0
  if (e == 0u || e == 0xffu) return (double)f;  // subnormal, inf, nan: rare path
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(e + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ df::operator double() const { return widen(h) + widen(l); }

__device__ __forceinline__ dfp::operator df() const { return fast_two_sum(p, e); }
__device__ __forceinline__ dfa::operator df() const { return fast_two_sum(s, c); }

__device__ __forceinline__ dfp operator*(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dfp{p, e};
}
__device__ __forceinline__ dfp operator-(dfp a) { return dfp{-a.p, -a.e}; }
__device__ __forceinline__ df operator-(df a) { return df(-a.h, -a.l); }

__device__ __forceinline__ dfa& operator+=(dfa& a, dfp b) {
  float err;
  a.s = two_sum(a.s, b.p, err);
  a.c = __fadd_rn(a.c, __fadd_rn(err, b.e));
  return a;
}
__device__ __forceinline__ dfa& operator-=(dfa& a, dfp b) { return a += -b; }
__device__ __forceinline__ dfa& operator+=(dfa& a, df b) { return a += dfp{b.h, b.l}; }
__device__ __forceinline__ dfa& operator-=(dfa& a, df b) { return a += dfp{-b.h, -b.l}; }

__device__ __forceinline__ df operator+(df a, df b) {
  float err;
  const float s = two_sum(a.h, b.h, err);
  return fast_two_sum(s, __fadd_rn(err, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator+(dfp a, df b) { return df(a) + b; }
__device__ __forceinline__ df operator+(df a, dfp b) { return a + df(b); }
__device__ __forceinline__ df operator+(dfp a, dfp b) {
  dfa s(a);
  s += b;
  return df(s);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }
__device__ __forceinline__ df& operator+=(df& a, dfp b) {
  dfa s(a);
  s += b;
  return a = df(s);
}
__device__ __forceinline__ df& operator-=(df& a, dfp b) { return a += -b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = df(a * b); }

__device__ __forceinline__ bool operator>=(df a, df b) { return a.h > b.h || (a.h == b.h && a.l >= b.l); }

// Accumulator type of a dot product in arithmetic R (R itself, except for double-float)
template <class R> struct AccOf { typedef R type; };
template <> struct AccOf<df> { typedef dfa type; };

}  // namespace ldg
