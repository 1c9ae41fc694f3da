// FP64 natural logarithm and exponential for the residual kernels, by P. T. P.
// Tang's table-driven method (ACM TOMS 15, 1989, for exp; ACM TOMS 16, 1990,
// for log), in 4 FP64-pipe operations each: the FP64 pipe bounds every kernel
// on this part, so only the reduced argument and the additions that carry the
// result's leading bits are FP64, and the small correction terms (below 2^-13
// of the result) are float-float on the FP32 pipe, joined to a double on the
// integer pipe.  Tables: mathfn_tables.h (gen_mathfn_tables.py).
//
// nsfr_log: x = 2^k m, m in [1, 2); with c_j ~ 1/(1 + (j + 1/2)/128), j the
//   top 7 fraction bits of m, r = m c_j - 1 is formed by one FMA (|r| <= 2^-8)
//   and ln x = k ln 2 - ln c_j + log1p(r), log1p(r) = r + r^2 q(r) by its
//   Taylor polynomial to r^7 (truncation below 2^-58): ln x = t1 + (r + c),
//   t1 = k ln2_hi - ln c_j (hi) in FP64, c = r^2 q(r) + k ln2_lo - ln c_j (lo)
//   (|c| < 2^-16) in float-float.  The error is about one ulp of
//   max(|ln x|, ln 2): absolute accuracy near x = 1, which is what the entropy
//   variables and the logarithmic means need.
// nsfr_exp: x = (32 k + j) ln2/32 + r, |r| <= ln2/64 (n = 32 k + j rounded in
//   FP32: off by one at most, near a tie, which leaves |r| below 1.01 ln2/64),
//   with the reduction in Cody and Waite's two-constant form;
//   e^x = 2^k 2^(j/32) (1 + expm1(r)), expm1(r) = r + r^2 q(r) by its Taylor
//   polynomial to r^6 (truncation below 2^-58): with s = 2^(j/32) (hi, lo),
//   e^x = 2^k (s_hi + (s_hi r + c)), c = s_hi r^2 q(r) + s_lo (|c| < 2^-13) in
//   float-float, 2^k added to the exponent field.  About one ulp.
// Arguments outside the reduced ranges (x <= 0, subnormal, infinite or NaN
// for nsfr_log; |x| >= 700 or NaN for nsfr_exp) go to the CUDA library
// functions; the kernels never produce them for physical states.
#pragma once

#include "ffloat.cuh"
#include "mathfn_tables.h"

// where the tables are read from: the global arrays, or a copy a kernel has
// staged in shared memory (nsfr_stage_tables)
struct MathTables {
  const double* c;    // [128] c_j
  const double* lhi;  // [128] -ln c_j, leading part
  const double* llo;  // [128] -ln c_j, trailing part
  const double* shi;  // [32] 2^(j/32), leading part
  const double* slo;  // [32] 2^(j/32), trailing part
};
#define NSFR_MATH_TABLE_DOUBLES (3 * 128 + 2 * 32)

__device__ __forceinline__ MathTables nsfr_global_tables() {
  return MathTables{NSFR_LOG_C, NSFR_LOG_LHI, NSFR_LOG_LLO, NSFR_EXP_SHI, NSFR_EXP_SLO};
}

// copy the tables into sm[0 .. NSFR_MATH_TABLE_DOUBLES) (all threads of the
// block take part; a __syncthreads must follow before use)
__device__ __forceinline__ MathTables nsfr_stage_tables(double* sm) {
  for (int i = threadIdx.x; i < NSFR_MATH_TABLE_DOUBLES; i += blockDim.x) {
    double v;
    if (i < 128) v = NSFR_LOG_C[i];
    else if (i < 256) v = NSFR_LOG_LHI[i - 128];
    else if (i < 384) v = NSFR_LOG_LLO[i - 256];
    else if (i < 416) v = NSFR_EXP_SHI[i - 384];
    else v = NSFR_EXP_SLO[i - 416];
    sm[i] = v;
  }
  return MathTables{sm, sm + 128, sm + 256, sm + 384, sm + 416};
}

// the out-of-range arguments' path, a call rather than inlined code (inlined,
// the compiler evaluates parts of it on every call and selects)
static __device__ __noinline__ double nsfr_log_slow(double x) { return log(x); }
static __device__ __noinline__ double nsfr_exp_slow(double x) { return exp(x); }

__device__ __forceinline__ double nsfr_log(double x, const MathTables& T) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  if (hi - 0x00100000u >= 0x7fe00000u) return nsfr_log_slow(x);
  const int k = (int)(hi >> 20) - 1023;
  const int j = (int)((hi >> 13) & 127u);
  const double m = __hiloint2double((int)((hi & 0x000fffffu) | 0x3ff00000u), (int)lo);
  const double r = fma(m, T.c[j], -1.0);
  // q = -1/2 + r w, w = 1/3 + r q2, q2 = -1/4 + r/5 - r^2/6 + r^3/7: w and q in
  // float-float (r/3 and r w need more than FP32's 24 bits), q2 in FP32
  const ff rf = ff_split_i(r);
  const float q2 = fmaf(fmaf(fmaf(1.0f / 7.0f, rf.hi, -1.0f / 6.0f), rf.hi, 0.2f), rf.hi, -0.25f);
  const ff w = ff_add_small(ff{0x1.555556p-2f, -0x1.555556p-27f}, __fmul_rn(rf.hi, q2));
  const ff q = ff_add_nn(ff{-0.5f, 0.0f}, ff_mul_nn(rf, w));
  // c = r^2 q + (k ln2_lo + llo_j), renormalised for the join
  const ff t2 = ff_add_nn(ff_mul_nn(ff{(float)k, 0.0f}, ff{0x1.ef357ap-45f, -0x1.87131ap-70f}),
                          ff{d2f_i(T.llo[j]), 0.0f});
  const ff c = ff_add(ff_mul_nn(ff_mul_nn(rf, rf), q), t2);
  const double t1 = fma(i2d_i(k), NSFR_LN2_HI, T.lhi[j]);
  return t1 + (r + ff_join_i(c));
}

__device__ __forceinline__ double nsfr_exp(double x, const MathTables& T) {
  const unsigned int ahi = (unsigned int)__double2hiint(x) & 0x7fffffffu;
  if (ahi >= 0x4085e000u) return nsfr_exp_slow(x);  // |x| >= 700, infinity, NaN
  // n = round(32 x / ln 2) in FP32: 1.5 2^23 fixes the binade, so n is the
  // difference of the bit patterns
  const float tn = __fmaf_rn(d2f_i(x), 0x1.715476p+5f, 12582912.0f);
  const int n = (int)__float_as_uint(tn) - 0x4b400000;
  const double ndn = i2d_i(-n);  // -n as a double, so that no FP64 negation is needed
  const double r = fma(ndn, NSFR_EXP_L2, fma(ndn, NSFR_EXP_L1, x));
  const int j = n & 31, k = n >> 5;
  // q = 1/2 + r w, w = 1/6 + r z, z = 1/24 + r (1/120 + r/720): z, w and q in
  // float-float (their leading terms need more than FP32's 24 bits)
  const ff rf = ff_split_i(r);
  const ff z = ff_add_small(ff{0x1.555556p-5f, -0x1.555556p-30f},
                            __fmul_rn(rf.hi, fmaf(1.0f / 720.0f, rf.hi, 1.0f / 120.0f)));
  const ff w = ff_add_nn(ff{0x1.555556p-3f, -0x1.555556p-28f}, ff_mul_nn(rf, z));
  const ff q = ff_add_nn(ff{0.5f, 0.0f}, ff_mul_nn(rf, w));
  const double sh = T.shi[j];
  // c = s_hi r^2 q + s_lo, renormalised for the join
  const ff c = ff_add(ff_mul_nn(ff_split_i(sh), ff_mul_nn(ff_mul_nn(rf, rf), q)), ff{d2f_i(T.slo[j]), 0.0f});
  const double y = sh + fma(sh, r, ff_join_i(c));
  return __hiloint2double(__double2hiint(y) + (int)((unsigned int)k << 20), __double2loint(y));
}

__device__ __forceinline__ double nsfr_log(double x) { return nsfr_log(x, nsfr_global_tables()); }
__device__ __forceinline__ double nsfr_exp(double x) { return nsfr_exp(x, nsfr_global_tables()); }
