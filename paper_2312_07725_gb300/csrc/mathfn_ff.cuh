// Natural logarithm and exponential in float-float arithmetic (pairs of
// floats, ~48 significant bits) for the FP32-bulk kernels, which must not wait
// on the FP64 pipe.  The same table-driven method as mathfn.cuh (P. T. P.
// Tang, ACM TOMS 15, 1989 and 16, 1990), with float tables
// (mathfn_tables.h, gen_mathfn_tables.py):
//
// ff_log: x = 2^k m, m in [1, 2) from x.hi (x.lo scaled by the same power of
//   two); with cf_j ~ 1/(1 + (j + 1/2)/128), j the top 7 fraction bits of m,
//   r = m cf_j - 1 as a float-float (m_hi cf_j by an FMA TwoProduct, its
//   leading part minus 1 exact since it lies within 2^-8 of 1, the two small
//   remainders summed in float), and ln x = k ln 2 - ln cf_j + log1p(r) with
//   log1p(r) = r - r^2/2 + r^3 q(r), r and r^2/2 in float-float and r^3 q in
//   float (|r| < 2^-8: q to r^4, truncation below 2^-66).  Error about 2^-46
//   of max(|ln x|, 0.7) (measured below 2^-44).
// ff_exp: n = round(64 x / ln 2), r = x - n ln2/64 with ln2/64 = L1 + L2 + L3
//   (n L1 and x.hi - n L1 exact, n L2 and x.lo joined by TwoProduct and
//   TwoSum), e^x = 2^(n>>6) 2^((n&63)/64) (1 + expm1(r)), expm1(r) = r +
//   r^2/2 + r^3 q(r), |r| <= ln2/128 (q to r^3, truncation below 2^-64).
//   Relative error about 2^-46 (measured below 2^-44).
// Arguments: ff_log wants x.hi positive and normal; ff_exp wants |x.hi| < 87
// (a normal float result).  The kernels check the states that reach them.
#pragma once

#include "ffloat.cuh"
#include "mathfn_tables.h"

struct MathTablesF {
  const float* c;    // [128] cf_j
  const float* lhi;  // [128] -ln cf_j, leading float
  const float* llo;  // [128] -ln cf_j, trailing float
  const float* shi;  // [64] 2^(j/64), leading float
  const float* slo;  // [64] 2^(j/64), trailing float
};
#define NSFR_MATH_TABLE_FLOATS (3 * 128 + 2 * 64)

__device__ __forceinline__ MathTablesF nsfr_global_tables_f() {
  return MathTablesF{NSFR_FLOG_C, NSFR_FLOG_LHI, NSFR_FLOG_LLO, NSFR_FEXP_SHI, NSFR_FEXP_SLO};
}

// copy the tables into sm[0 .. NSFR_MATH_TABLE_FLOATS) (all threads of the
// block take part; a __syncthreads must follow before use)
__device__ __forceinline__ MathTablesF nsfr_stage_tables_f(float* sm) {
  for (int i = threadIdx.x; i < NSFR_MATH_TABLE_FLOATS; i += blockDim.x) {
    float v;
    if (i < 128) v = NSFR_FLOG_C[i];
    else if (i < 256) v = NSFR_FLOG_LHI[i - 128];
    else if (i < 384) v = NSFR_FLOG_LLO[i - 256];
    else if (i < 448) v = NSFR_FEXP_SHI[i - 384];
    else v = NSFR_FEXP_SLO[i - 448];
    sm[i] = v;
  }
  return MathTablesF{sm, sm + 128, sm + 256, sm + 384, sm + 448};
}

// 2^e for an integer e with a normal float result
__device__ __forceinline__ float ff_pow2(int e) { return __uint_as_float((unsigned int)(e + 127) << 23); }

__device__ __forceinline__ ff ff_log(ff x, const MathTablesF& T) {
  const unsigned int b = __float_as_uint(x.hi);
  const int k = (int)(b >> 23) - 127;
  const int j = (int)((b >> 16) & 127u);
  const float mh = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
  const float ml = x.lo * ff_pow2(-k);
  const float c = T.c[j];
  // m cf_j - 1 = (p - 1) + (e + m_lo cf_j), p + e = m_hi cf_j exactly
  const float p = __fmul_rn(mh, c);
  const float e = __fmaf_rn(mh, c, -p);
  ff r;
  two_sum(__fsub_rn(p, 1.0f), __fmaf_rn(ml, c, e), r.hi, r.lo);
  // log1p(r) = r - r^2/2 + r^3 q(r),  q = 1/3 - r/4 + r^2/5 - r^3/6 + r^4/7
  const float s2 = __fmul_rn(r.hi, r.hi);
  const float s2e = __fmaf_rn(2.0f * r.hi, r.lo, __fmaf_rn(r.hi, r.hi, -s2));
  const float q = __fmaf_rn(
      __fmaf_rn(__fmaf_rn(__fmaf_rn(1.0f / 7.0f, r.hi, -1.0f / 6.0f), r.hi, 0.2f), r.hi, -0.25f), r.hi,
      1.0f / 3.0f);
  const float t3 = __fmul_rn(__fmul_rn(s2, r.hi), q);
  const ff l1p = ff_add(r, ff{-0.5f * s2, __fmaf_rn(-0.5f, s2e, t3)});
  // k ln 2 - ln cf_j: k A and k B exact (|k| < 2^9), k C in float
  const float kf = (float)k;
  ff kl;
  fast_two_sum(kf * NSFR_FLN2_A, kf * NSFR_FLN2_B, kl.hi, kl.lo);
  kl.lo = __fmaf_rn(kf, NSFR_FLN2_C, kl.lo);
  return ff_add(ff_add(kl, ff{T.lhi[j], T.llo[j]}), l1p);
}

__device__ __forceinline__ ff ff_exp(ff x, const MathTablesF& T) {
  const float nf = rintf(__fmul_rn(x.hi, NSFR_FEXP_INV_L));
  const int n = (int)nf;
  // r = x - n (L1 + L2 + L3): x.hi - n L1 is exact, n L2 = p2 + e2 exactly, and
  // x.lo (up to 2^-24 |x|) joins by a TwoSum too, so that its rounding does not
  // grow with |x|
  const float r1 = __fmaf_rn(-nf, NSFR_FEXP_L1, x.hi);
  const float p2 = __fmul_rn(nf, NSFR_FEXP_L2);
  const float e2 = __fmaf_rn(nf, NSFR_FEXP_L2, -p2);
  float a, b, c, d;
  two_sum(r1, -p2, a, b);
  two_sum(a, x.lo, c, d);
  ff r;
  fast_two_sum(c, __fadd_rn(__fadd_rn(b, d), __fmaf_rn(-nf, NSFR_FEXP_L3, -e2)), r.hi, r.lo);
  const int j = n & 63, k = n >> 6;
  // expm1(r) = r + r^2/2 + r^3 q(r),  q = 1/6 + r/24 + r^2/120 + r^3/720
  const float s2 = __fmul_rn(r.hi, r.hi);
  const float s2e = __fmaf_rn(2.0f * r.hi, r.lo, __fmaf_rn(r.hi, r.hi, -s2));
  const float q =
      __fmaf_rn(__fmaf_rn(__fmaf_rn(1.0f / 720.0f, r.hi, 1.0f / 120.0f), r.hi, 1.0f / 24.0f), r.hi, 1.0f / 6.0f);
  const float t3 = __fmul_rn(__fmul_rn(s2, r.hi), q);
  const ff em1 = ff_add(r, ff{0.5f * s2, __fmaf_rn(0.5f, s2e, t3)});
  const ff S{T.shi[j], T.slo[j]};
  const ff y = ff_add(S, ff_mul(S, em1));
  const float sc = ff_pow2(k);
  return ff{y.hi * sc, y.lo * sc};
}
