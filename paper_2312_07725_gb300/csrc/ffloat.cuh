// Unevaluated sums of two floats ("float-float", about 48 significant bits)
// on the FP32 pipe, which runs ~74x faster than FP64 on this part.
// Algorithms: Knuth's TwoSum (error-free addition), Dekker's FastTwoSum
// (|a| >= |b|), and the FMA form of the error-free product (TwoProduct).
#pragma once

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float h) { return ff{h, 0.0f}; }

// exact split of a double into hi + lo (hi the nearest float)
__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return ff{h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

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
