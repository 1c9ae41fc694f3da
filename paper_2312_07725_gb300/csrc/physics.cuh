// Device physics for the Euler equations (Sec. "Systems of Equations").
//
// Entropy U = -rho s/(gamma-1), s = ln p - gamma ln rho; entropy variables
// v = [(gamma-s)/(gamma-1) - beta|u|^2, 2 beta u, -2 beta], beta = rho/(2p);
// entropy potential psi = rho u.  Two-point flux: Chandrashekar's entropy
// conserving, kinetic-energy preserving flux (the solution of the Tadmor
// shuffle condition, Eq. tadmor shuffle, in the variables rho, u, beta),
// whose logarithmic means use Ismail and Roe's series for nearly equal
// arguments.  Face dissipation: Roe's linearisation (Sec. "Nonlinear
// Stability").
//
// FP64 work is the cost of every kernel on this part (FP32 runs ~74x
// faster), so the per-node record (Rec) stores what makes each pair cheap:
// rho, 2 beta, u/2, |u|^2/4, ln rho, ln beta.  Arithmetic means are then plain
// sums, and reciprocals are FP64 refinements of an FP32 seed.
#pragma once

#include "ffloat.cuh"
#include "nsfr_internal.h"

// Below this value of f^2 = ((a-b)/(a+b))^2 the log mean uses its series; the
// truncation of the series is then below the FP64 rounding level.
#define NSFR_LM_EPS 1.0e-4

struct Rec {
  double r, b2, u0, u1, u2, qq, lr, lb;  // rho, 2 beta, u/2, |u|^2/4, ln rho, ln beta
};

__device__ __forceinline__ Rec load_rec(const double* P, int stride) {
  Rec a;
  a.r = P[P_RHO * stride];
  a.b2 = P[P_B2 * stride];
  a.u0 = P[P_UH * stride];
  a.u1 = P[(P_UH + 1) * stride];
  a.u2 = P[(P_UH + 2) * stride];
  a.qq = P[P_QQ * stride];
  a.lr = P[P_LRHO * stride];
  a.lb = P[P_LBETA * stride];
  return a;
}

// the six fields without the logs (records staged without them)
__device__ __forceinline__ Rec load_rec6(const double* P, int stride) {
  Rec a;
  a.r = P[P_RHO * stride];
  a.b2 = P[P_B2 * stride];
  a.u0 = P[P_UH * stride];
  a.u1 = P[(P_UH + 1) * stride];
  a.u2 = P[(P_UH + 2) * stride];
  a.qq = P[P_QQ * stride];
  a.lr = 0.0;
  a.lb = 0.0;
  return a;
}

__device__ __forceinline__ void store_rec(double* P, int stride, const Rec& a) {
  P[P_RHO * stride] = a.r;
  P[P_B2 * stride] = a.b2;
  P[P_UH * stride] = a.u0;
  P[(P_UH + 1) * stride] = a.u1;
  P[(P_UH + 2) * stride] = a.u2;
  P[P_QQ * stride] = a.qq;
  P[P_LRHO * stride] = a.lr;
  P[P_LBETA * stride] = a.lb;
}

// Reciprocals.  The seed comes from the FP32 unit: the mantissa m in [1, 2)
// of |x|, truncated to 23 bits, goes through rcp.approx.ftz.f32 (<= 1 ulp),
// and the exponent of 1/x = 2^(1023-e) (1/m) is rebuilt with integer
// operations, so that the seed (relative error <= 2^-22) costs no FP64-pipe
// slot; the FP64 reciprocal approximation, which it replaces, occupies that
// pipe for about 2.5 FMA slots.  Valid for normal |x| in [2^-1021, 2^1021].
// Refinement, with e = 1 - x r:
//   Newton            r <- r + r e            (error e^2 <= 2^-44),
//   third order       r <- r + r (e + e^2)    (error e^3 <= 2^-66: the FP64 result).
__device__ __forceinline__ double rcp_seed(double x) {
  const unsigned int hi = (unsigned int)__double2hiint(x), lo = (unsigned int)__double2loint(x);
  // m = 1.f, f the top 23 fraction bits of x
  const unsigned int mb = 0x3f800000u | (__funnelshift_l(lo, hi, 3) & 0x007fffffu);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(mb)));
  const unsigned int rb = __float_as_uint(rf);  // 1/m in (1/2, 1]: FP32 exponent 126 or 127
  // FP64 exponent field of the seed: (rb's FP32 exponent - 127) + (1023 - e) + 1023
  const unsigned int shi = ((rb >> 3) + (1919u << 20) - (hi & 0x7ff00000u)) | (hi & 0x80000000u);
  return __hiloint2double((int)shi, (int)(rb << 29));
}
__device__ __forceinline__ double rcp_newton1(double x) {
  const double r = rcp_seed(x);
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ double rcp_full(double x) {
  const double r = rcp_seed(x);
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// x 2^k (k small) by moving the exponent field: exact, and off the FP64 pipe.
// Zero stays zero; a subnormal x (never a state quantity) takes the multiply.
// (The rare path is a call, not inlined: inlined, the compiler evaluates its
// multiply on every call and selects, which costs the FP64 operation this
// avoids.)
static __device__ __noinline__ double mul_pow2_slow(double x, double scale) { return x * scale; }
template <int K>
__device__ __forceinline__ double mul_pow2(double x) {
  const int hi = __double2hiint(x);
  if ((hi & 0x7ff00000) == 0) {
    if ((hi & 0x7fffffff) == 0 && __double2loint(x) == 0) return x;  // +-0
    return mul_pow2_slow(x, K >= 0 ? (double)(1LL << K) : 1.0 / (double)(1LL << -K));
  }
  return __hiloint2double(hi + K * (1 << 20), __double2loint(x));
}

// u < NSFR_LM_EPS for u = f^2 >= 0, decided on the integer bit pattern
__device__ __forceinline__ bool lm_small(double u) {
  return __double_as_longlong(u) < __double_as_longlong(NSFR_LM_EPS);
}

__device__ __forceinline__ double horner4(const double* c, double u) {
  return fma(fma(fma(c[3], u, c[2]), u, c[1]), u, c[0]);
}

// Float-float rho and 2 beta of a record, split once per node, for the series
// branch of the log means below.
struct RecF {
  ff r, b2;
};
__device__ __forceinline__ RecF recf_of(const Rec& a) { return RecF{ff_split_i(a.r), ff_split_i(a.b2)}; }

__device__ __forceinline__ float rcp32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// a / b, b > 0, in float-float from r, the FP32 reciprocal of b.hi, and one
// correction (about 2^-44 relative; the result is not renormalised)
__device__ __forceinline__ ff ff_div_nn(ff a, ff b, float r) {
  const float q1 = __fmul_rn(a.hi, r);
  const float p = __fmul_rn(q1, b.hi);
  const float pe = __fmaf_rn(q1, b.hi, -p);
  // a - q1 b: a.hi - p is exact (the two are within a few ulps of each other)
  const float rem = __fmaf_rn(-q1, b.lo, __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo));
  return ff{q1, __fmul_rn(rem, r)};
}

// 1/x for an FP64 x > 0 from a float-float approximation xf of it and r, the
// FP32 reciprocal of xf.hi: the float-float seed r + r (1 - xf r) (~2^-45),
// joined on the integer pipe, and one FP64 Newton step -- two FP64
// operations, to the accuracy of rcp_full's three.
static __device__ __noinline__ double rcp_full_slow(double x) { return rcp_full(x); }
__device__ __forceinline__ double rcp_from_ff(double x, ff xf, float r) {
  if (!(xf.hi > 1.0e-37f && xf.hi < 1.0e37f)) return rcp_full_slow(x);  // outside the FP32 seed's range (a call)
  const float e = __fmaf_rn(-xf.lo, r, __fmaf_rn(-xf.hi, r, 1.0f));
  const double r0 = ff_join_i(ff{r, __fmul_rn(r, e)});
  return fma(r0, fma(-x, r0, 1.0), r0);
}

// 1/x for an FP64 x > 0 in two FP64 operations: rcp_from_ff of x's
// integer-pipe split (rcp_full outside the FP32 range).
__device__ __forceinline__ double rcp_ff(double x) {
  const ff xf = ff_split_i(x);
  return rcp_from_ff(x, xf, rcp32(xf.hi));
}

// The series branch of a logarithmic mean on the FP32 pipe.  With
// f = d / s = (a - b)/(a + b) and u = f^2 formed in float-float from the
// float-float difference and sum of a, b (rs the FP32 reciprocal of s.hi),
// lm_u_ff returns false when u >= NSFR_LM_EPS (the caller takes the log
// branch in FP64); otherwise lm_tail_ff(u, c) gives the series' part beyond
// its constant term, eps = u (c1 + u (c2 + u c3)), c = {c1 hi, c1 lo, c2 hi,
// c2 lo, c3}, as a double.  |eps| <= 1e-4 |c1|, and eps is good to about
// 2^-40 of itself, so c0 + eps in FP64 matches the FP64 Horner form to its
// rounding: the series costs no FP64 operation (eps's two floats are joined
// on the integer pipe) instead of the FP64 ratio, square and Horner chain.
// f, u and the tail keep ~44 bits: the float-float inputs (2^-48) and the sum
// and difference (2^-47 of the larger operand) put ~2^-49 into f, i.e. below
// 2^-55 into c0 + eps when u < 1e-4.  A sum outside the FP32 range (and a
// NaN) takes the log branch.
__device__ __forceinline__ bool lm_uf_ff(ff d, ff s, float rs, ff& f, ff& u) {
  if (!(s.hi > 1.0e-37f && s.hi < 1.0e37f)) return false;
  f = ff_div_nn(d, s, rs);
  const float uh = __fmul_rn(f.hi, f.hi);
  u = ff{uh, __fmaf_rn(__fmul_rn(2.0f, f.hi), f.lo, __fmaf_rn(f.hi, f.hi, -uh))};
  return uh < (float)NSFR_LM_EPS;
}
__device__ __forceinline__ bool lm_u_ff(ff d, ff s, float rs, ff& u) {
  ff f;
  return lm_uf_ff(d, s, rs, f, u);
}

// c1 + u (c2 + u c3) in float-float (not renormalised), the tail u (c1 + ...)
// as float-float, and the tail joined to a double
__device__ __forceinline__ ff lm_poly_ffv(ff u, const float* c) {
  float ts, te;
  two_sum(c[2], __fmul_rn(u.hi, c[4]), ts, te);
  const ff t{ts, __fadd_rn(te, c[3])};                   // c2 + u c3
  return ff_add_nn(ff{c[0], c[1]}, ff_mul_nn(u, t));     // c1 + u (c2 + u c3)
}
__device__ __forceinline__ ff lm_tail_ffv(ff u, const float* c) { return ff_mul_nn(u, lm_poly_ffv(u, c)); }
__device__ __forceinline__ double lm_tail_ff(ff u, const float* c) { return ff_join_i(lm_tail_ffv(u, c)); }

__device__ __forceinline__ bool lm_series_ff(ff d, ff s, float rs, const float* c, double& eps) {
  ff u;
  if (!lm_u_ff(d, s, rs, u)) return false;
  eps = lm_tail_ff(u, c);
  return true;
}

// the same from float-float a, b
__device__ __forceinline__ bool lm_series_ff(ff a, ff b, const float* c, double& eps) {
  const ff s = ff_add_nn(a, b);
  return lm_series_ff(ff_add_nn(a, ff_neg(b)), s, rcp32(s.hi), c, eps);
}

// Record of a conserved state; flags rho <= 0, p <= 0 or NaN.  ln rho and
// ln beta come from the face-state pass, which already formed them.
__device__ __forceinline__ Rec rec_from_conserved(double r, double m0, double m1, double m2, double E, double lr,
                                                  double lb, double gm1, int* flag) {
  Rec a;
  const double ir = rcp_full(r);
  const double u0 = m0 * ir, u1 = m1 * ir, u2 = m2 * ir;
  const double q2 = fma(u0, u0, fma(u1, u1, u2 * u2));
  const double p = gm1 * fma(-0.5 * r, q2, E);
  if (!(r > 0.0) || !(p > 0.0)) atomicOr(flag, 1);
  a.r = r;
  a.b2 = r * rcp_full(p);
  a.u0 = 0.5 * u0;
  a.u1 = 0.5 * u1;
  a.u2 = 0.5 * u2;
  a.qq = 0.25 * q2;
  a.lr = lr;
  a.lb = lb;
  return a;
}

// ln rho and ln beta of a state for the log-mean branch.  RecLogs takes them
// from a record; PtrLogs reads them from memory only when a log mean needs
// them, so that the common series path neither stages nor holds the logs.
struct RecLogs {
  const Rec& a;
  __device__ __forceinline__ double lr() const { return a.lr; }
  __device__ __forceinline__ double lb() const { return a.lb; }
  __device__ __forceinline__ double r() const { return a.r; }
  __device__ __forceinline__ double b2() const { return a.b2; }
};
struct PtrLogs {
  const double* p;  // ln rho at p[0], ln beta at p[off]: fields of a record with field stride off
  int off;
  __device__ __forceinline__ double lr() const { return p[0]; }
  __device__ __forceinline__ double lb() const { return p[off]; }
  // the record's FP64 rho and 2 beta (for kernels that stage them in float-float only)
  __device__ __forceinline__ double r() const { return p[(P_RHO - P_LRHO) * off]; }
  __device__ __forceinline__ double b2() const { return p[(P_B2 - P_LRHO) * off]; }
};

// Chandrashekar's flux, F = f_s(A, B) . n, n the averaged metric row (n0, n1, n2):
//   rho_ln = (rho_a + rho_b) Gh(u_r),   1/(2(gamma-1) beta_ln) = F4g(u_b) / (2 beta_a + 2 beta_b),
//   p_hat  = (rho_a + rho_b) / (2 beta_a + 2 beta_b),
//   F_rho = rho_ln u.n,  F_m = F_rho u + p_hat n,  F_E = F_rho (1/(2(gamma-1) beta_ln) - |u|^2_bar/2) + u.F_m,
// with the log means' series branch on the FP32 pipe (lm_series_ff, from the
// float-float rho and 2 beta of the two nodes).  ec_flux_over_sr_ff returns
// the flux divided by s = rho_a + rho_b, and s: every component carries that
// factor (rho_ln = s G(u_r), p_hat = s / (2 beta_a + 2 beta_b), and F_E is
// linear in both), so a caller that accumulates w F folds s into the weight
// and saves the two products by s.  On the series branch
//   F_rho / s = Gh(u_r) u.n = (u.n / 2) (1 + eps_r),
//   h = F4g(u_b) / s2 - qs = (F4g(0) + eps_b) / s2 - qs,
// and the FP64 work left is the sums, 1/s2, the FMAs that add the eps and the
// flux; off it rho_ln / s = (rho_a - rho_b) / ((ln rho_a - ln rho_b) s), and
// the differences rho_a - rho_b and 2 beta_a - 2 beta_b are formed in FP64 on
// that branch only.
template <class LA, class LB>
__device__ __forceinline__ double ec_flux_over_sr_ff(const Rec& A, const Rec& B, const RecF& Af, const RecF& Bf,
                                                     double n0, double n1, double n2, const OpsGL& K, const LA& la,
                                                     const LB& lb, double F[5]) {
  const double sr = A.r + B.r, s2 = A.b2 + B.b2;
  const ff s2f = ff_add_nn(Af.b2, Bf.b2);
  const float rs2 = rcp32(s2f.hi);
  const double rb2 = rcp_from_ff(s2, s2f, rs2);
  const double qs = A.qq + B.qq;
  const double v0 = A.u0 + B.u0, v1 = A.u1 + B.u1, v2 = A.u2 + B.u2;  // u_bar
  const double un = fma(v0, n0, fma(v1, n1, v2 * n2));
  double er, eb, Fr, h;
  if (lm_series_ff(Af.r, Bf.r, K.lmg_ff, er)) {
    const double uh = mul_pow2<-1>(un);
    Fr = fma(uh, er, uh);
  } else {
    Fr = (A.r - B.r) / ((la.lr() - lb.lr()) * sr) * un;
  }
  if (lm_series_ff(ff_add_nn(Af.b2, ff_neg(Bf.b2)), s2f, rs2, K.lmb_ff, eb))
    h = fma(eb, rb2, fma(K.f4g[0], rb2, -qs));
  else
    h = K.inv_gm1 * (la.lb() - lb.lb()) / (A.b2 - B.b2) - qs;
  F[0] = Fr;
  F[1] = fma(Fr, v0, rb2 * n0);
  F[2] = fma(Fr, v1, rb2 * n1);
  F[3] = fma(Fr, v2, rb2 * n2);
  F[4] = fma(v2, F[3], fma(v1, F[2], fma(v0, F[1], Fr * h)));
  return sr;
}

// The same flux itself, not divided by s: rho_ln = (s/2)(1 + eps_r).
template <class LA, class LB>
__device__ __forceinline__ void ec_flux_ff(const Rec& A, const Rec& B, const RecF& Af, const RecF& Bf, double n0,
                                           double n1, double n2, const OpsGL& K, const LA& la, const LB& lb,
                                           double F[5]) {
  const double sr = A.r + B.r, s2 = A.b2 + B.b2;
  const ff s2f = ff_add_nn(Af.b2, Bf.b2);
  const float rs2 = rcp32(s2f.hi);
  const double rb2 = rcp_from_ff(s2, s2f, rs2);
  const double qs = A.qq + B.qq;
  double er, eb, rln, h;
  if (lm_series_ff(Af.r, Bf.r, K.lmg_ff, er)) {
    const double sh = mul_pow2<-1>(sr);
    rln = fma(sh, er, sh);
  } else {
    rln = (A.r - B.r) / (la.lr() - lb.lr());
  }
  if (lm_series_ff(ff_add_nn(Af.b2, ff_neg(Bf.b2)), s2f, rs2, K.lmb_ff, eb))
    h = fma(eb, rb2, fma(K.f4g[0], rb2, -qs));
  else
    h = K.inv_gm1 * (la.lb() - lb.lb()) / (A.b2 - B.b2) - qs;
  const double ph = sr * rb2;
  const double v0 = A.u0 + B.u0, v1 = A.u1 + B.u1, v2 = A.u2 + B.u2;  // u_bar
  const double un = fma(v0, n0, fma(v1, n1, v2 * n2));
  const double Fr = rln * un;
  F[0] = Fr;
  F[1] = fma(Fr, v0, ph * n0);
  F[2] = fma(Fr, v1, ph * n1);
  F[3] = fma(Fr, v2, ph * n2);
  F[4] = fma(v2, F[3], fma(v1, F[2], fma(v0, F[1], Fr * h)));
}

__device__ __forceinline__ RecF recf_split(const Rec& a) { return RecF{ff_split_i(a.r), ff_split_i(a.b2)}; }

// Chandrashekar's flux with Ranocha's pressure terms (Sec. "Results": the EC
// runs use Chandrashekar's flux with Ranocha's pressure fix), F = f_s(A, B) . n:
// the same mass flux and internal-energy term, the arithmetic pressure mean in
// the momentum flux and the cross product mean as the pressure work,
//   F_m = F_rho u_bar + (p_a + p_b)/2 n,
//   F_E = F_rho (1/(2(gamma-1) beta_ln) + u_a . u_b / 2) + (p_a u_b.n + p_b u_a.n)/2.
// pa, pb are the two pressures (rho / (2 beta)); with the half velocities h of
// the records u_a . u_b / 2 = 2 h_a . h_b and u_b . n / 2 = u_bar . n - h_a . n.
// The log means' series branch runs on the FP32 pipe, as in ec_flux_over_sr_ff:
// rho_ln = (s/2)(1 + eps_r), 1/(2(gamma-1) beta_ln) = (F4g(0) + eps_b) / s2.
template <class LA, class LB>
__device__ __forceinline__ void ranocha_flux_ff(const Rec& A, const Rec& B, const RecF& Af, const RecF& Bf,
                                                double pa, double pb, double n0, double n1, double n2,
                                                const OpsGL& K, const LA& la, const LB& lb, double F[5]) {
  double er, eb, rln, ibg;
  if (lm_series_ff(Af.r, Bf.r, K.lmg_ff, er)) {
    const double sh = mul_pow2<-1>(A.r + B.r);
    rln = fma(sh, er, sh);
  } else {
    rln = (A.r - B.r) / (la.lr() - lb.lr());
  }
  const ff s2f = ff_add_nn(Af.b2, Bf.b2);
  const float rs2 = rcp32(s2f.hi);
  if (lm_series_ff(ff_add_nn(Af.b2, ff_neg(Bf.b2)), s2f, rs2, K.lmb_ff, eb)) {
    const double rb2 = rcp_from_ff(A.b2 + B.b2, s2f, rs2);
    ibg = fma(eb, rb2, K.f4g[0] * rb2);
  } else {
    ibg = K.inv_gm1 * (la.lb() - lb.lb()) / (A.b2 - B.b2);
  }
  const double v0 = A.u0 + B.u0, v1 = A.u1 + B.u1, v2 = A.u2 + B.u2;  // u_bar
  const double un = fma(v0, n0, fma(v1, n1, v2 * n2));
  const double an = fma(A.u0, n0, fma(A.u1, n1, A.u2 * n2));     // u_a . n / 2
  const double hab = fma(A.u0, B.u0, fma(A.u1, B.u1, A.u2 * B.u2));  // u_a . u_b / 4
  const double Fr = rln * un;
  const double pm = mul_pow2<-1>(pa + pb);
  F[0] = Fr;
  F[1] = fma(Fr, v0, pm * n0);
  F[2] = fma(Fr, v1, pm * n1);
  F[3] = fma(Fr, v2, pm * n2);
  F[4] = fma(Fr, fma(2.0, hab, ibg), fma(pa, un - an, pb * an));
}

__device__ __forceinline__ double pressure_of(const Rec& a) { return a.r * rcp_full(a.b2); }

// D = |A_n| (u_R - u_L): Roe-averaged flux Jacobian along n (non-unit),
// applied through its eigen-decomposition (acoustic waves q -+ a, entropy
// and shear waves q), scaled by |n|.
__device__ __forceinline__ void roe_dissipation(const Rec& L, const Rec& R, double n0, double n1, double n2,
                                                double gamma, double D[5]) {
  const double nn = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
  const double in = 1.0 / nn;
  const double h0 = n0 * in, h1 = n1 * in, h2 = n2 * in;
  const double pL = L.r / L.b2, pR = R.r / R.b2;
  const double gg = gamma / (gamma - 1.0);
  const double HL = gg * pL / L.r + 2.0 * L.qq, HR = gg * pR / R.r + 2.0 * R.qq;
  const double sL = sqrt(L.r), sR = sqrt(R.r);
  const double wl = sL / (sL + sR), wr = 1.0 - wl;
  const double uh0 = 2.0 * (wl * L.u0 + wr * R.u0), uh1 = 2.0 * (wl * L.u1 + wr * R.u1),
               uh2 = 2.0 * (wl * L.u2 + wr * R.u2);
  const double Hh = wl * HL + wr * HR;
  const double q2h = uh0 * uh0 + uh1 * uh1 + uh2 * uh2;
  const double a2 = (gamma - 1.0) * (Hh - 0.5 * q2h);
  const double ah = sqrt(a2);
  const double rh = sL * sR;
  const double qh = uh0 * h0 + uh1 * h1 + uh2 * h2;
  const double dr = R.r - L.r, dp = pR - pL;
  const double du0 = 2.0 * (R.u0 - L.u0), du1 = 2.0 * (R.u1 - L.u1), du2 = 2.0 * (R.u2 - L.u2);
  const double dq = du0 * h0 + du1 * h1 + du2 * h2;
  const double al1 = (dp - rh * ah * dq) / (2.0 * a2);
  const double al5 = (dp + rh * ah * dq) / (2.0 * a2);
  const double al2 = dr - dp / a2;
  const double t0 = du0 - dq * h0, t1 = du1 - dq * h1, t2 = du2 - dq * h2;  // shear jump
  const double l1 = fabs(qh - ah), l2 = fabs(qh), l5 = fabs(qh + ah);
  const double c1 = l1 * al1, c5 = l5 * al5, c2 = l2 * al2, cs = l2 * rh;
  D[0] = nn * (c1 + c5 + c2);
  D[1] = nn * (c1 * (uh0 - ah * h0) + c5 * (uh0 + ah * h0) + c2 * uh0 + cs * t0);
  D[2] = nn * (c1 * (uh1 - ah * h1) + c5 * (uh1 + ah * h1) + c2 * uh1 + cs * t1);
  D[3] = nn * (c1 * (uh2 - ah * h2) + c5 * (uh2 + ah * h2) + c2 * uh2 + cs * t2);
  D[4] = nn * (c1 * (Hh - qh * ah) + c5 * (Hh + qh * ah) + c2 * 0.5 * q2h + cs * (uh0 * t0 + uh1 * t1 + uh2 * t2));
}

// D = R |Lambda| T R^T [[v]]: entropy-variable matrix dissipation along n,
// scaled by |n|.  [[v]] = v(R) - v(L) from the records (s = (1-gamma) ln rho
// - ln 2 beta, v = ((gamma - s)/(gamma-1) - beta |u|^2, 2 beta u, -2 beta));
// R, Lambda: eigenvectors and speeds of the flux Jacobian (acoustic q -+ a,
// entropy and shear waves q, q = u . n^), T Barth's scaling (rho/(2 gamma),
// rho (gamma-1)/gamma, p, p, rho/(2 gamma)) so that R T R^T = du/dv, all at
// the state (rho_ln, u_bar, p_hat) of the EC flux.  The shear waves act
// through the projection I - n^ n^T.
__device__ __forceinline__ void es_dissipation(const Rec& L, const Rec& R, double n0, double n1, double n2,
                                               const OpsGL& K, double D[5]) {
  const double g = K.gamma, ln2 = 0.69314718055994530942;
  const double sL = (1.0 - g) * L.lr - (L.lb + ln2), sR = (1.0 - g) * R.lr - (R.lb + ln2);
  const double dv0 = (sL - sR) * K.inv_gm1 - 2.0 * (R.b2 * R.qq - L.b2 * L.qq);
  const double dm0 = 2.0 * (R.b2 * R.u0 - L.b2 * L.u0), dm1 = 2.0 * (R.b2 * R.u1 - L.b2 * L.u1),
               dm2 = 2.0 * (R.b2 * R.u2 - L.b2 * L.u2);
  const double dv4 = L.b2 - R.b2;
  // averaged state
  const double sr = L.r + R.r, dr = L.r - R.r;
  const double fr = dr / sr, ur = fr * fr;
  const double rho = lm_small(ur) ? sr * horner4(K.gh, ur) : dr / (L.lr - R.lr);
  const double u0 = L.u0 + R.u0, u1 = L.u1 + R.u1, u2 = L.u2 + R.u2;
  const double p = sr / (L.b2 + R.b2);
  const double nn = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
  const double h0 = n0 / nn, h1 = n1 / nn, h2 = n2 / nn;
  const double a = sqrt(g * p / rho);
  const double qn = u0 * h0 + u1 * h1 + u2 * h2;
  const double q2 = u0 * u0 + u1 * u1 + u2 * u2;
  const double H = a * a * K.inv_gm1 + 0.5 * q2;
  const double t_ac = rho / (2.0 * g), t_en = rho * (g - 1.0) / g;
  // r . [[v]] for r = (1, u -+ a n^, H -+ a q) and the entropy wave (1, u, q2/2)
  const double wm = dv0 + (u0 - a * h0) * dm0 + (u1 - a * h1) * dm1 + (u2 - a * h2) * dm2 + (H - a * qn) * dv4;
  const double wp = dv0 + (u0 + a * h0) * dm0 + (u1 + a * h1) * dm1 + (u2 + a * h2) * dm2 + (H + a * qn) * dv4;
  const double we = dv0 + u0 * dm0 + u1 * dm1 + u2 * dm2 + 0.5 * q2 * dv4;
  const double c1 = fabs(qn - a) * t_ac * wm, c5 = fabs(qn + a) * t_ac * wp, c2 = fabs(qn) * t_en * we;
  const double z0 = dm0 + u0 * dv4, z1 = dm1 + u1 * dv4, z2 = dm2 + u2 * dv4;
  const double zn = h0 * z0 + h1 * z1 + h2 * z2;
  const double P0 = z0 - h0 * zn, P1 = z1 - h1 * zn, P2 = z2 - h2 * zn;
  const double cs = fabs(qn) * p;
  D[0] = nn * (c1 + c2 + c5);
  D[1] = nn * (c1 * (u0 - a * h0) + c2 * u0 + c5 * (u0 + a * h0) + cs * P0);
  D[2] = nn * (c1 * (u1 - a * h1) + c2 * u1 + c5 * (u1 + a * h1) + cs * P1);
  D[3] = nn * (c1 * (u2 - a * h2) + c2 * u2 + c5 * (u2 + a * h2) + cs * P2);
  D[4] = nn * (c1 * (H - a * qn) + c2 * 0.5 * q2 + c5 * (H + a * qn) + cs * (u0 * P0 + u1 * P1 + u2 * P2));
}

// f*(u~_L, u~_R; n): the EC flux (Chandrashekar's or, vf = NSFR_FLUX_RANOCHA,
// with Ranocha's pressure terms), minus (1/2)|A_n|(u_R - u_L) (Roe) or minus
// (1/2) R |Lambda| T R^T [[v]] (entropy-variable matrix dissipation).
__device__ __forceinline__ void face_flux(const Rec& L, const Rec& R, double n0, double n1, double n2,
                                          const OpsGL& K, int kind, int vf, double F[5]) {
  const RecF Lf = recf_split(L), Rf = recf_split(R);
  if (vf == NSFR_FLUX_RANOCHA)
    ranocha_flux_ff(L, R, Lf, Rf, pressure_of(L), pressure_of(R), n0, n1, n2, K, RecLogs{L}, RecLogs{R}, F);
  else
    ec_flux_ff(L, R, Lf, Rf, n0, n1, n2, K, RecLogs{L}, RecLogs{R}, F);
  if (kind == NSFR_FACE_EC_ROE || kind == NSFR_FACE_EC_ES) {
    double D[5];
    if (kind == NSFR_FACE_EC_ROE) roe_dissipation(L, R, n0, n1, n2, K.gamma, D);
    else es_dissipation(L, R, n0, n1, n2, K, D);
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k] -= 0.5 * D[k];
  }
}
