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
#pragma once

#include "nsfr_internal.h"

// Below this value of f^2 = ((a-b)/(a+b))^2 the log mean uses the series; the
// truncation of the series is then below the FP64 rounding level.
#define NSFR_LM_EPS 1.0e-4

struct Prim {
  double r, u0, u1, u2, b, lr, lb, q2;  // rho, velocity, beta, ln rho, ln beta, |u|^2
};

__device__ __forceinline__ Prim load_prim(const double* P, int stride) {
  Prim a;
  a.r = P[P_RHO * stride];
  a.u0 = P[P_U * stride];
  a.u1 = P[P_V * stride];
  a.u2 = P[P_W * stride];
  a.b = P[P_BETA * stride];
  a.lr = P[P_LRHO * stride];
  a.lb = P[P_LBETA * stride];
  a.q2 = P[P_Q2 * stride];
  return a;
}

__device__ __forceinline__ void store_prim(double* P, int stride, const Prim& a) {
  P[P_RHO * stride] = a.r;
  P[P_U * stride] = a.u0;
  P[P_V * stride] = a.u1;
  P[P_W * stride] = a.u2;
  P[P_BETA * stride] = a.b;
  P[P_LRHO * stride] = a.lr;
  P[P_LBETA * stride] = a.lb;
  P[P_Q2 * stride] = a.q2;
}

// Primitive record of a conserved state; flags rho <= 0, p <= 0, NaN.
__device__ __forceinline__ Prim prim_from_conserved(double r, double m0, double m1, double m2, double E,
                                                    double gamma, int* flag) {
  Prim a;
  const double ir = 1.0 / r;
  a.r = r;
  a.u0 = m0 * ir;
  a.u1 = m1 * ir;
  a.u2 = m2 * ir;
  a.q2 = a.u0 * a.u0 + a.u1 * a.u1 + a.u2 * a.u2;
  const double p = (gamma - 1.0) * (E - 0.5 * r * a.q2);
  if (!(r > 0.0) || !(p > 0.0)) atomicOr(flag, 1);
  a.b = 0.5 * r / p;
  a.lr = log(r);
  a.lb = log(a.b);
  return a;
}

// sum_k u^k/(2k+1), k <= 3: atanh(f)/f with u = f^2
__device__ __forceinline__ double lm_series_F(double u) {
  return 1.0 + u * (1.0 / 3.0 + u * (1.0 / 5.0 + u * (1.0 / 7.0)));
}
// its reciprocal f/atanh(f) = 1 - u/3 - 4u^2/45 - 44u^3/945 - ...
__device__ __forceinline__ double lm_series_G(double u) {
  return 1.0 + u * (-1.0 / 3.0 + u * (-4.0 / 45.0 + u * (-44.0 / 945.0)));
}

// rho_ln, 1/beta_ln and p_hat = rho_bar/(2 beta_bar) of a pair.
__device__ __forceinline__ void ec_means(const Prim& A, const Prim& B, double& rln, double& ibln, double& ph) {
  const double sr = A.r + B.r, dr = A.r - B.r;
  const double sb = A.b + B.b, db = A.b - B.b;
  const double rsr = 1.0 / sr, rsb = 1.0 / sb;
  const double fr = dr * rsr, fb = db * rsb;
  const double ur = fr * fr, ub = fb * fb;
  if (ur < NSFR_LM_EPS) {
    rln = 0.5 * sr * lm_series_G(ur);
  } else {
    rln = dr / (A.lr - B.lr);
  }
  if (ub < NSFR_LM_EPS) {
    ibln = 2.0 * rsb * lm_series_F(ub);
  } else {
    ibln = (A.lb - B.lb) / db;
  }
  ph = 0.5 * sr * rsb;
}

// F = f_s(A, B) . n with n the (already averaged) metric row.
__device__ __forceinline__ void ec_flux(const Prim& A, const Prim& B, double n0, double n1, double n2,
                                        double inv2gm1, double F[5]) {
  double rln, ibln, ph;
  ec_means(A, B, rln, ibln, ph);
  const double u0 = 0.5 * (A.u0 + B.u0), u1 = 0.5 * (A.u1 + B.u1), u2 = 0.5 * (A.u2 + B.u2);
  const double un = u0 * n0 + u1 * n1 + u2 * n2;
  const double Fr = rln * un;
  F[0] = Fr;
  F[1] = Fr * u0 + ph * n0;
  F[2] = Fr * u1 + ph * n1;
  F[3] = Fr * u2 + ph * n2;
  const double q2 = 0.5 * (A.q2 + B.q2);
  F[4] = Fr * (ibln * inv2gm1 - 0.5 * q2) + u0 * F[1] + u1 * F[2] + u2 * F[3];
}

// D = |A_n| (u_R - u_L): Roe-averaged flux Jacobian along n (non-unit),
// applied through its eigen-decomposition (acoustic waves q -+ a, entropy
// and shear waves q), scaled by |n|.
__device__ __forceinline__ void roe_dissipation(const Prim& L, const Prim& R, double n0, double n1, double n2,
                                                double gamma, double D[5]) {
  const double nn = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
  const double in = 1.0 / nn;
  const double h0 = n0 * in, h1 = n1 * in, h2 = n2 * in;
  const double pL = 0.5 * L.r / L.b, pR = 0.5 * R.r / R.b;
  const double gg = gamma / (gamma - 1.0);
  const double HL = gg * pL / L.r + 0.5 * L.q2, HR = gg * pR / R.r + 0.5 * R.q2;
  const double sL = sqrt(L.r), sR = sqrt(R.r);
  const double wl = sL / (sL + sR), wr = 1.0 - wl;
  const double uh0 = wl * L.u0 + wr * R.u0, uh1 = wl * L.u1 + wr * R.u1, uh2 = wl * L.u2 + wr * R.u2;
  const double Hh = wl * HL + wr * HR;
  const double q2h = uh0 * uh0 + uh1 * uh1 + uh2 * uh2;
  const double a2 = (gamma - 1.0) * (Hh - 0.5 * q2h);
  const double ah = sqrt(a2);
  const double rh = sL * sR;
  const double qh = uh0 * h0 + uh1 * h1 + uh2 * h2;
  const double dr = R.r - L.r, dp = pR - pL;
  const double du0 = R.u0 - L.u0, du1 = R.u1 - L.u1, du2 = R.u2 - L.u2;
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

// f*(u~_L, u~_R; n): EC flux, minus (1/2)|A_n|(u_R - u_L) with Roe dissipation.
__device__ __forceinline__ void face_flux(const Prim& L, const Prim& R, double n0, double n1, double n2,
                                          double gamma, double inv2gm1, int kind, double F[5]) {
  ec_flux(L, R, n0, n1, n2, inv2gm1, F);
  if (kind == NSFR_FACE_EC_ROE) {
    double D[5];
    roe_dissipation(L, R, n0, n1, n2, gamma, D);
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k] -= 0.5 * D[k];
  }
}
