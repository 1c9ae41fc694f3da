// FP64 natural logarithm and exponential for the residual kernels, by P. T. P.
// Tang's table-driven method (ACM TOMS 15, 1989, for exp; ACM TOMS 16, 1990,
// for log), in about 10 (log) and 11 (exp) FP64-pipe operations; the FP64
// pipe bounds every kernel on this part.  Tables: mathfn_tables.h
// (gen_mathfn_tables.py).
//
// nsfr_log: x = 2^k m, m in [1, 2); with c_j ~ 1/(1 + (j + 1/2)/128), j the
//   top 7 fraction bits of m, r = m c_j - 1 is formed by one FMA (|r| <= 2^-8)
//   and ln x = k ln 2 - ln c_j + log1p(r), log1p(r) by its Taylor polynomial
//   to r^7 (truncation below 2^-58), the terms from r^4 on in FP32.  The error
//   is about one ulp of max(|ln x|, ln 2): absolute accuracy near x = 1, which
//   is what the entropy variables and the logarithmic means need.
// nsfr_exp: x = (32 k + j) ln2/32 + r, |r| <= ln2/64, with the reduction in
//   Cody and Waite's two-constant form; e^x = 2^k 2^(j/32) (1 + expm1(r)),
//   expm1(r) by its Taylor polynomial to r^6 (truncation below 2^-58), the
//   terms from r^5 on in FP32, 2^k added to the exponent field.  About one ulp.
// Arguments outside the reduced ranges (x <= 0, subnormal, infinite or NaN
// for nsfr_log; |x| >= 700 or NaN for nsfr_exp) go to the CUDA library
// functions; the kernels never produce them for physical states.
#pragma once

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

// FP32 tails of the polynomials: the log's r^4 q2(r) and the exp's r^5 q3(r)
// carry factors |r|^4 <= 2^-32 and |r|^5 <= 2^-32, so FP32's relative rounding
// (below 2^-22 after three operations, plus the truncation of r) contributes
// less than 2^-56 absolute, while every leading term stays FP64.  The
// conversions are integer bit operations (the FP64 pipe is the bound).
__device__ __forceinline__ float tail_arg_f(double r) {
  // r truncated to float; |r| < 2^-126 (zero included) gives 0
  const unsigned int hi = (unsigned int)__double2hiint(r), lo = (unsigned int)__double2loint(r);
  const unsigned int a = hi & 0x7fffffffu;
  const unsigned int f = a < (897u << 20) ? 0u : (((a - (896u << 20)) << 3) | (lo >> 29));
  return __uint_as_float(f | (hi & 0x80000000u));
}
__device__ __forceinline__ double tail_val_d(float t) {
  // a normal float to double (exactly)
  const unsigned int u = __float_as_uint(t), a = u & 0x7fffffffu;
  return __hiloint2double((int)((u & 0x80000000u) | ((a >> 3) + (896u << 20))), (int)(a << 29));
}

__device__ __forceinline__ double nsfr_log(double x, const MathTables& T) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  if (hi - 0x00100000u >= 0x7fe00000u) return log(x);
  const int k = (int)(hi >> 20) - 1023;
  const int j = (int)((hi >> 13) & 127u);
  const double m = __hiloint2double((int)((hi & 0x000fffffu) | 0x3ff00000u), (int)lo);
  const double r = fma(m, T.c[j], -1.0);
  // log1p(r) = r + r^2 q(r),  q = -1/2 + r (1/3 + r q2),  q2 = -1/4 + r/5 - r^2/6 + r^3/7 in FP32
  const float rf = tail_arg_f(r);
  const float q2 = fmaf(fmaf(fmaf(1.0f / 7.0f, rf, -1.0f / 6.0f), rf, 0.2f), rf, -0.25f);
  const double q = fma(fma(tail_val_d(q2), r, 1.0 / 3.0), r, -0.5);
  // k as a double: 2^52 + 2^31 + k read from its bit pattern, minus 2^52 + 2^31
  const double kd = __hiloint2double(0x43300000, (int)((unsigned int)k + 0x80000000u)) - 4503601774854144.0;
  const double t1 = fma(kd, NSFR_LN2_HI, T.lhi[j]);
  const double t2 = fma(kd, NSFR_LN2_LO, T.llo[j]);
  return t1 + (fma(r * r, q, r) + t2);
}

__device__ __forceinline__ double nsfr_exp(double x, const MathTables& T) {
  const unsigned int ahi = (unsigned int)__double2hiint(x) & 0x7fffffffu;
  if (ahi >= 0x4085e000u) return exp(x);  // |x| >= 700, infinity, NaN
  // n = round(32 x / ln 2) in the low word of t (1.5 2^52 fixes the exponent)
  const double t = fma(x, NSFR_EXP_INV_L, 6755399441055744.0);
  const int n = __double2loint(t);
  const double nd = t - 6755399441055744.0;
  const double r = fma(-nd, NSFR_EXP_L2, fma(-nd, NSFR_EXP_L1, x));
  const int j = n & 31, k = n >> 5;
  // expm1(r) = r + r^2 (1/2 + r/6 + r^2/24 + r^3 q3),  q3 = 1/120 + r/720 in FP32
  const float q3 = fmaf(1.0f / 720.0f, tail_arg_f(r), 1.0f / 120.0f);
  const double q = fma(fma(fma(tail_val_d(q3), r, 1.0 / 24.0), r, 1.0 / 6.0), r, 0.5);
  const double p = fma(r * r, q, r);
  const double sh = T.shi[j];
  const double y = sh + fma(sh, p, T.slo[j]);
  return __hiloint2double(__double2hiint(y) + (int)((unsigned int)k << 20), __double2loint(y));
}

__device__ __forceinline__ double nsfr_log(double x) { return nsfr_log(x, nsfr_global_tables()); }
__device__ __forceinline__ double nsfr_exp(double x) { return nsfr_exp(x, nsfr_global_tables()); }
