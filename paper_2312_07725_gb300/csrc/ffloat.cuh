// Unevaluated sums of two floats ("float-float", about 48 significant bits)
// on the FP32 pipe, which runs ~74x faster than FP64 on this part.
// Algorithms: Knuth's TwoSum (error-free addition), Dekker's FastTwoSum
// (|a| >= |b|), and the FMA form of the error-free product (TwoProduct).
#pragma once

struct ff {
  float hi, lo;
};

// FP64 <-> FP32 conversions with integer operations.  The hardware
// conversions execute on the FP64 pipe, which bounds every residual kernel on
// this part; these use the integer pipe.  IEEE-754 binary64 -> binary32 drops
// 29 fraction bits, rounding to nearest (ties away from zero): the carry of the
// rounding add runs into the exponent field by itself.  Results below the
// binary32 normal range become signed zero, above it signed infinity; NaN
// stays NaN.  binary32 -> binary64 is exact for normal numbers and zero
// (subnormal floats, which the kernels never hold, flush to zero).
__device__ __forceinline__ float d2f_i(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long r = b + (1ull << 28);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const unsigned int ahi = (unsigned int)(r >> 32) & 0x7fffffffu;
  // exponent (mod 2^9) and 23 fraction bits; subtracting 896 << 23 rebases the
  // exponent from bias 1023 to 127 (mod 2^32 this adds 0x40000000)
  unsigned int f = (unsigned int)(r >> 29) + 0x40000000u;
  f = ahi < (897u << 20) ? 0u : f;
  f = ahi >= (1151u << 20) ? 0x7f800000u : f;
  // NaN, tested on the two 32-bit words (the compiler turns the same test on the
  // 64-bit pattern into an FP64 instruction)
  const unsigned int bh = (unsigned int)(b >> 32) & 0x7fffffffu, bl = (unsigned int)b;
  f = (bh > 0x7ff00000u) | ((bh == 0x7ff00000u) & (bl != 0u)) ? 0x7fc00000u : f;
  return __uint_as_float(f | sign);
}

__device__ __forceinline__ double f2d_i(float x) {
  const unsigned int u = __float_as_uint(x), a = u & 0x7fffffffu, sign = u & 0x80000000u;
  unsigned int hi = sign | ((a >> 3) + (896u << 20)), lo = a << 29;
  if (a < 0x00800000u) {  // zero (subnormals flushed)
    hi = sign;
    lo = 0u;
  } else if (a >= 0x7f800000u) {  // infinity, NaN
    hi = sign | 0x7ff00000u | (a > 0x7f800000u ? 0x00080000u : 0u);
    lo = 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// split of a double into hi + lo, hi the nearest float: x - hi is exact, so
// hi + lo carries about 48 bits of x
__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = d2f_i(x);
  return ff{h, d2f_i(x - f2d_i(h))};
}

__device__ __forceinline__ double ff_to_double(ff a) { return f2d_i(a.hi) + f2d_i(a.lo); }

// -x, and x with its sign flipped when neg, on the integer pipe (an FP64
// negation that no FMA absorbs costs an FP64 addition)
__device__ __forceinline__ double neg_i(double x) {
  return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}
__device__ __forceinline__ double neg_if(double x, bool neg) {
  return __hiloint2double(__double2hiint(x) ^ (neg ? (int)0x80000000 : 0), __double2loint(x));
}
// x > 0 (false for zero, negative and NaN), decided on the bit pattern
__device__ __forceinline__ bool pos_i(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000LL;
}

// x as hi + lo on the integer pipe (ff_from_double without its FP64
// subtraction): hi the nearest float (d2f_i, ties away from zero), lo the
// leading 24 bits of the remainder x - hi (truncated: x - hi - lo is below
// 2^-48 |x|).  For normal x with 2^-100 < |x| < 2^100, where hi and lo are
// normal floats (lo below the FP32 range becomes 0).
__device__ __forceinline__ ff ff_split_i(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const float h = d2f_i(x);
  // remainder of the 53-bit significand after rounding it to 24 bits
  const unsigned int low = (unsigned int)b & 0x1fffffffu;
  const int R = (int)low - ((low & 0x10000000u) ? 0x20000000 : 0);
  if (R == 0) return ff{h, 0.0f};
  const unsigned int a = R < 0 ? (unsigned int)(-R) : (unsigned int)R;
  const int p = 31 - __clz((int)a);  // leading bit of |R| (<= 28)
  const unsigned int sig = p >= 23 ? (a >> (p - 23)) : (a << (23 - p));
  // |lo| = a 2^(E - 1075), E the binary64 exponent field: FP32 exponent field p + E - 948
  const int fe = p + (int)((b >> 52) & 0x7ffu) - 948;
  if (fe <= 0) return ff{h, 0.0f};
  const unsigned int sign = ((unsigned int)(b >> 32) & 0x80000000u) ^ (R < 0 ? 0x80000000u : 0u);
  return ff{h, __uint_as_float(sign | ((unsigned int)fe << 23) | (sig & 0x7fffffu))};
}

// an int as a double on the integer pipe (exact)
__device__ __forceinline__ double i2d_i(int n) {
  if (n == 0) return 0.0;
  const unsigned int a = n < 0 ? 0u - (unsigned int)n : (unsigned int)n;
  const int p = 31 - __clz((int)a);
  const unsigned long long bits = ((unsigned long long)(n < 0 ? 1u : 0u) << 63) |
                                  ((unsigned long long)(1023 + p) << 52) |
                                  (((unsigned long long)a << (52 - p)) & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

// hi + lo as a double on the integer pipe (ff_to_double without its FP64
// addition): the two 24-bit significands are added as integers at their
// offset, the sum is renormalised by at most one position and its top 53 bits
// kept (truncated: an error below 2^-52 of the value; exact when lo lies
// within 29 bits below hi's last bit).  Requires |lo| < |hi| / 2 or hi == 0;
// subnormal floats count as zero, and hi must not be Inf or NaN.
__device__ __forceinline__ double ff_join_i(ff a) {
  const unsigned int bh = __float_as_uint(a.hi), bl = __float_as_uint(a.lo);
  const unsigned int eh = (bh >> 23) & 0xffu, el = (bl >> 23) & 0xffu;
  if (eh == 0u) return f2d_i(a.lo);
  if (el == 0u) return f2d_i(a.hi);
  const unsigned int sh = eh - el;  // >= 1 when |lo| < |hi| / 2
  // significands with their leading bits at bit 62 (hi) and 62 - sh (lo)
  const unsigned long long H = (unsigned long long)((bh & 0x7fffffu) | 0x800000u) << 39;
  const unsigned long long L =
      sh < 63u ? ((unsigned long long)((bl & 0x7fffffu) | 0x800000u) << 39) >> sh : 0ull;
  unsigned long long S = ((bh ^ bl) & 0x80000000u) ? H - L : H + L;
  unsigned int e = eh + 896u;  // binary64 biased exponent of bit 62
  if (S >> 63) {
    S >>= 1;
    ++e;
  } else if (!(S >> 62)) {
    S <<= 1;
    --e;
  }
  const unsigned long long bits = ((unsigned long long)(bh & 0x80000000u) << 32) |
                                  ((unsigned long long)e << 52) | ((S >> 10) & 0xfffffffffffffull);
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// a + b without the final renormalisation (7 instead of 10 additions): hi + lo
// carries the same sum, but |lo| may exceed half an ulp of hi by a little.  For
// operands of further float-float products, reciprocals and differences only,
// not for accumulators.
__device__ __forceinline__ ff ff_add_nn(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return ff{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  ff r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// acc + c * x
__device__ __forceinline__ ff ff_fma(ff c, ff x, ff acc) { return ff_add(acc, ff_mul(c, x)); }

// a b without the final renormalisation (operands of further products only)
__device__ __forceinline__ ff ff_mul_nn(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff{p, e};
}

// c + x for a float-float c and a float |x| << |c| (x + c.lo rounded once)
__device__ __forceinline__ ff ff_add_small(ff c, float x) {
  ff r;
  fast_two_sum(c.hi, __fadd_rn(x, c.lo), r.hi, r.lo);
  return r;
}
