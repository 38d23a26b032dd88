// dfloat.cuh -- double-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about
// 48 significant bits.  GB300 executes FP64 at a small fraction of its FP32 rate, so the
// kernels of the FP64 iterative refinement evaluate their sums of products in this
// representation instead: the data stay FP64 in memory and only the arithmetic moves.
//
// Building blocks (error-free transformations):
//  * two_sum: Knuth's TwoSum (The Art of Computer Programming, vol. 2, 4.2.2), s + e = a + b
//    exactly for any a, b, in six additions;
//  * fast_two_sum: Dekker's Fast2Sum (Dekker 1971), the same for |a| >= |b| in three;
//  * two_prod: p + e = a * b exactly with one fused multiply-add (the FMA-based form of
//    Dekker's product);
//  * dot2: the compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot
//    product", SIAM J. Sci. Comput. 26, 2005), extended to double-float operands: the hi
//    products are summed error-free with two_sum, every rounding error and the lo cross
//    terms go into a float compensation, and the result is the double-float s + c.
// The additions and products use the explicitly rounded intrinsics so that the compiler
// cannot contract them into fused operations that would break the transformations.
//
// Conversions: d2df splits a double into hi (its 24 leading significand bits) and lo
// (the next 24, rounded toward zero) by integer operations on its bit pattern, so that
// loading FP64 data costs no FP64 instruction; df2d widens both floats the same way and
// joins them with one FP64 addition.
#pragma once
#include <cstdint>

namespace hp {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  const float e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
  return {s, e};
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// Accumulator of a compensated sum of double-float products and terms.
struct Dot2 {
  float s = 0.f, c = 0.f;
  // += x (double-float)
  __device__ __forceinline__ void add(dfl x) {
    const dfl t = two_sum(s, x.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, x.lo));
  }
  // += a * x (double-float operands); the lo * lo term is below the format's precision
  __device__ __forceinline__ void fma(dfl a, dfl x) {
    const dfl p = two_prod(a.hi, x.hi);
    const float cross = __fmaf_rn(a.hi, x.lo, __fmul_rn(a.lo, x.hi));
    const dfl t = two_sum(s, p.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, __fadd_rn(p.lo, cross)));
  }
  // -= a * x
  __device__ __forceinline__ void fms(dfl a, dfl x) { fma(dfl{-a.hi, -a.lo}, x); }
  // s + c as a normalised pair (two_sum: c may exceed s after cancellation)
  __device__ __forceinline__ dfl result() const { return two_sum(s, c); }
};

// double -> double-float by bit manipulation (no FP64 instruction).  hi holds the 24
// leading significand bits (truncated), lo the next 24 (truncated): the pair is within
// 2^-47 of x, relatively.  Doubles whose hi or lo would leave the normal float range
// (zero, subnormal or tiny, huge, infinite, NaN) go through the FP64 conversion.
__device__ __forceinline__ dfl d2df(double x) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned sgn = static_cast<unsigned>(u >> 32) & 0x80000000u;
  const int e = static_cast<int>((u >> 52) & 0x7ffu);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  const int eh = e - 1023 + 127;  // float biased exponent of hi
  if ((u << 1) == 0ull) return {__uint_as_float(sgn), 0.f};  // +-0
  if (eh <= 53 || eh >= 255) {
    const float h = __double2float_rn(x);
    return {h, isfinite(h) ? __double2float_rn(x - (double)h) : 0.f};
  }
  const float hi = __uint_as_float(sgn | (static_cast<unsigned>(eh) << 23) | static_cast<unsigned>(m >> 29));
  const unsigned ml = static_cast<unsigned>(m & 0x1FFFFFFFull);  // the 29 bits below hi
  float lo = 0.f;
  if (ml) {
    const int k = 31 - __clz(ml);  // leading one of ml: bit k (0..28); lo = ml 2^(eh - 127 - 52)
    const unsigned mant = k >= 23 ? (ml >> (k - 23)) : (ml << (23 - k));
    lo = __uint_as_float(sgn | (static_cast<unsigned>(eh + k - 52) << 23) | (mant & 0x7FFFFFu));
  }
  return {hi, lo};
}

// float -> double, exact, by bit manipulation (zero and normal floats; anything else
// through the FP64 conversion)
__device__ __forceinline__ double f2d(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (u << 1) == 0u ? __hiloint2double((int)(u & 0x80000000u), 0) : (double)x;
  const unsigned m = u & 0x7FFFFFu;
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// double-float -> double: hi and lo widened exactly by bit manipulation, then one FP64
// addition (the correctly rounded hi + lo)
__device__ __forceinline__ double df2d(dfl v) { return f2d(v.hi) + f2d(v.lo); }

}  // namespace hp
