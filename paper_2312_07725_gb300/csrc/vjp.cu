// Reverse-mode (VJP) kernels of du/dt(u; x), written by hand.
//
// du/dt = -A R(u; C) with A = Pi~ (W J)^{-1} Pi~^T (Eq. weight-adj ESFR mass)
// symmetric, so for a cotangent rbar:
//   Rbar = -A rbar,  Jbar_i = -(sum_k zbar_ki y_ki) / (w_i J_i^2),  zbar = -Pi~^T rbar, y = Pi~^T R.
// R (Eq. NSFR, sum-factorised) is reversed term by term:
//   volume pair  R_a += c F, R_b -= c F           -> Fbar = c (Rbar_a - Rbar_b)
//   hybrid       R_a += s w t_a (phi_a + f* - sum_b t_b phi_b)
//                -> f*bar = sum_a s w t_a Rbar_a =: rho,  phi_a bar = s w t_a Rbar_a - t_a rho
// and each two-point flux F(A, B; n) is reversed to cotangents of the primitive
// records (rho, u, beta) of both states and of n.  Face states are entropy
// projections u~_f = u(t_s . v(u)) (Sec. "Nonlinearly Stable Flux
// Reconstruction"); their cotangents are gathered per face (own element and
// neighbour in separate slots, no atomics) and mapped back through u(v), the
// extrapolation and v(u) by vjp_face_kernel.  The metric cotangents (volume
// rows, the shared face rows, J) are mapped to the control points by
// vjp_metric_kernel, the reverse of the conservative-curl construction
// (Sec. "Computational Space", Eq. GCL).  FP64 throughout; EC face flux.
#include "kernel_common.cuh"
#include "mathfn.cuh"
#include "physics.cuh"

namespace {
using namespace nsfr_k;

struct PR {
  double r, u0, u1, u2, b;  // rho, velocity, beta = rho / (2p)
};

// Node splits for the reverse fluxes: rho and beta as float-float.
struct PRF {
  ff r, b;
};

// log mean L(a, b) and its partial derivatives.  Series branch, as the
// forward kernels form the log means: L = s G(u)/2 with s = a + b,
// f = (a - b)/s, u = f^2 < NSFR_LM_EPS and G = f/atanh f = 1 - u/3 - 4u^2/45
// - 44u^3/945 (next term below 1e-16), so that dL/da = G/2 + 2 G'(u) f b/s and
// dL/db = G/2 - 2 G'(u) f a/s:
//   L = (s/2)(1 + eps_G),  dL/da = 1/2 + (eps_G/2 + 2 G'(u) f b/s),
//   dL/db = 1/2 + (eps_G/2 - 2 G'(u) f a/s),
// eps_G = G - 1, with f, u and the parenthesised corrections (below 7e-3)
// in float-float from float-float a, b (sf their sum, rs the FP32 reciprocal
// of sf.hi), joined on the integer pipe: 4 FP64 operations instead of about
// 17.  Returns whether the series branch was taken (u set); otherwise
// L = (a - b)/(ln a - ln b) and its derivatives in FP64 (reciprocals by an
// FP32 seed and a third-order step, rcp_full: a division costs several times
// as many FP64-pipe operations).
__device__ __forceinline__ bool logmean_grad_ff(double a, double b, ff af, ff bf, ff sf, float rs, const OpsGL& K,
                                                double& L, double& La, double& Lb, ff& u) {
  ff f;
  if (lm_uf_ff(ff_add_nn(af, ff_neg(bf)), sf, rs, f, u)) {
    const ff eg = lm_tail_ffv(u, K.lmg_ff);
    // 2 G'(u) f / s, 1/s from rs and one float-float correction
    const float e = __fmaf_rn(-sf.lo, rs, __fmaf_rn(-sf.hi, rs, 1.0f));
    const ff t = ff_mul_nn(ff_mul_nn(lm_poly_ffv(u, K.lmgd_ff), f), ff{rs, __fmul_rn(rs, e)});
    const ff t2{2.0f * t.hi, 2.0f * t.lo};
    const ff eh{0.5f * eg.hi, 0.5f * eg.lo};
    const double sh = mul_pow2<-1>(a + b);
    L = fma(sh, ff_join_i(eg), sh);
    La = 0.5 + ff_join_i(ff_add(eh, ff_mul_nn(t2, bf)));
    Lb = 0.5 + ff_join_i(ff_add(eh, ff_neg(ff_mul_nn(t2, af))));
    return true;
  }
  const double iD = rcp_full(nsfr_log(a) - nsfr_log(b));
  L = (a - b) * iD;
  La = (1.0 - L * rcp_full(a)) * iD;
  Lb = (L * rcp_full(b) - 1.0) * iD;
  return false;
}

// reverse of F = f_s(A, B) . n (Chandrashekar): accumulates into Ab, Bb, nb.
// The forward flux, with u_bar = (u_A + u_B)/2, s_b = beta_A + beta_B and
// h = 1/(2 (gamma-1) beta_ln):
//   F_rho = rho_ln (u_bar . n),   F_m = F_rho u_bar + p_hat n,   p_hat = (rho_A + rho_B)/(2 s_b),
//   F_E = F_rho (h - |u|^2_bar/2) + u_bar . F_m = F_rho (h + u_A . u_B/2) + p_hat (u_bar . n)
// (|u_bar|^2 - |u|^2_bar/2 = u_A . u_B/2), reversed term by term.  F is
// linear in n, so a caller may pass a multiple of n with Fb divided by it.
// Af, Bf: the float-float rho and beta of A and B (the log means' series
// branch, logmean_grad_ff); 1/s_b from a float-float seed and one Newton step,
// and on the series branch 1/beta_ln = (1/s_b)(2 atanh(f)/f) = (1/s_b)(2 + eps_a).
__device__ __forceinline__ void ec_flux_vjp(const PR& A, const PR& B, const PRF& Af, const PRF& Bf, double n0,
                                            double n1, double n2, const OpsGL& K, const double Fb[5], PR& Ab,
                                            PR& Bb, double nb[3]) {
  double rl, rla, rlb, bl, bla, blb;
  ff ur, ub;
  const ff sr = ff_add_nn(Af.r, Bf.r), sb = ff_add_nn(Af.b, Bf.b);
  const float rsb = rcp32(sb.hi);
  logmean_grad_ff(A.r, B.r, Af.r, Bf.r, sr, rcp32(sr.hi), K, rl, rla, rlb, ur);
  const double isb = rcp_from_ff(A.b + B.b, sb, rsb);
  double ibl;
  if (logmean_grad_ff(A.b, B.b, Af.b, Bf.b, sb, rsb, K, bl, bla, blb, ub))
    ibl = fma(isb, ff_join_i(lm_tail_ffv(ub, K.lma_ff)), mul_pow2<1>(isb));
  else
    ibl = rcp_full(bl);
  const double v0 = mul_pow2<-1>(A.u0 + B.u0), v1 = mul_pow2<-1>(A.u1 + B.u1), v2 = mul_pow2<-1>(A.u2 + B.u2);
  const double un = fma(v0, n0, fma(v1, n1, v2 * n2));
  const double F0 = rl * un;
  const double hs = mul_pow2<-1>(isb);  // dp_hat/drho_A = dp_hat/drho_B
  const double ph = (A.r + B.r) * hs;
  const double h = mul_pow2<-1>(K.inv_gm1 * ibl);
  const double uab = fma(A.u0, B.u0, fma(A.u1, B.u1, A.u2 * B.u2));
  // reverse
  const double t4 = Fb[4];
  const double F0b = fma(t4, fma(0.5, uab, h), fma(Fb[1], v0, fma(Fb[2], v1, fma(Fb[3], v2, Fb[0]))));
  const double phb = fma(t4, un, fma(Fb[1], n0, fma(Fb[2], n1, Fb[3] * n2)));
  const double hb = t4 * F0;
  const double uabb = mul_pow2<-1>(hb);
  const double unb = fma(F0b, rl, t4 * ph);  // u_bar . n: through F_rho and F_E
  // u_bar cotangent (F_rho Fb_m + unb n) shared by both sides, halved, plus the u_A . u_B term
  const double F0h = mul_pow2<-1>(F0), unbh = mul_pow2<-1>(unb);
  const double g0 = fma(unbh, n0, F0h * Fb[1]), g1 = fma(unbh, n1, F0h * Fb[2]), g2 = fma(unbh, n2, F0h * Fb[3]);
  Ab.u0 += fma(uabb, B.u0, g0);
  Ab.u1 += fma(uabb, B.u1, g1);
  Ab.u2 += fma(uabb, B.u2, g2);
  Bb.u0 += fma(uabb, A.u0, g0);
  Bb.u1 += fma(uabb, A.u1, g1);
  Bb.u2 += fma(uabb, A.u2, g2);
  nb[0] += fma(ph, Fb[1], unb * v0);
  nb[1] += fma(ph, Fb[2], unb * v1);
  nb[2] += fma(ph, Fb[3], unb * v2);
  const double rlb_ = F0b * un;
  const double blb_ = -hb * h * ibl;
  const double rq = phb * hs;         // p_hat's share of the rho cotangents
  const double bq = -phb * ph * isb;  // and of the beta cotangents (dp_hat/dbeta = -p_hat/s_b)
  Ab.r += fma(rlb_, rla, rq);
  Bb.r += fma(rlb_, rlb, rq);
  Ab.b += fma(blb_, bla, bq);
  Bb.b += fma(blb_, blb, bq);
}

__device__ __forceinline__ PR pr_from_conserved(const double* U, int stride, double gamma) {
  PR a;
  a.r = U[0];
  const double ir = rcp_ff(a.r);
  a.u0 = U[stride] * ir;
  a.u1 = U[2 * stride] * ir;
  a.u2 = U[3 * stride] * ir;
  const double q2 = a.u0 * a.u0 + a.u1 * a.u1 + a.u2 * a.u2;
  const double p = (gamma - 1.0) * (U[4 * stride] - mul_pow2<-1>(a.r) * q2);
  a.b = mul_pow2<-1>(a.r) * rcp_ff(p);
  return a;
}

// (rho, u, beta) cotangent plus a direct pressure cotangent -> conserved cotangent
__device__ __forceinline__ void conserved_bar(const PR& a, double gamma, const PR& pb, double pbar_direct,
                                              double Ub[5]) {
  // p = rho / (2 beta): 1/(2p) = beta/rho, beta/p = 2 beta^2/rho
  const double q2 = a.u0 * a.u0 + a.u1 * a.u1 + a.u2 * a.u2;
  const double ir = rcp_ff(a.r);
  double rb = pb.r + pb.b * a.b * ir;
  const double pbar = pbar_direct - 2.0 * pb.b * a.b * a.b * ir;
  // p = (gamma-1)(E - |m|^2/(2 rho))
  const double g1 = gamma - 1.0;
  const double Eb = g1 * pbar;
  double mb0 = -g1 * pbar * a.u0, mb1 = -g1 * pbar * a.u1, mb2 = -g1 * pbar * a.u2;
  rb += g1 * pbar * 0.5 * q2;
  // u = m / rho
  mb0 += pb.u0 * ir;
  mb1 += pb.u1 * ir;
  mb2 += pb.u2 * ir;
  rb -= (pb.u0 * a.u0 + pb.u1 * a.u1 + pb.u2 * a.u2) * ir;
  Ub[0] = rb;
  Ub[1] = mb0;
  Ub[2] = mb1;
  Ub[3] = mb2;
  Ub[4] = Eb;
}

// (igm1 = 1/(gamma-1); the exact doublings and halvings are exponent adds)
__device__ __forceinline__ void entropy_vars(const PR& a, double gamma, double igm1, double v[5]) {
  const double q2 = a.u0 * a.u0 + a.u1 * a.u1 + a.u2 * a.u2;
  const double p = mul_pow2<-1>(a.r) * rcp_ff(a.b);
  const double s = nsfr_log(p) - gamma * nsfr_log(a.r);
  const double b2 = mul_pow2<1>(a.b);
  v[0] = (gamma - s) * igm1 - a.b * q2;
  v[1] = b2 * a.u0;
  v[2] = b2 * a.u1;
  v[3] = b2 * a.u2;
  v[4] = neg_i(b2);
}

// face state from entropy variables (forward) as a primitive record
__device__ __forceinline__ PR pr_from_entropy(const double v[5], double gamma, double igm1) {
  PR a;
  const double v5 = v[4], iv5 = rcp_full(v5);
  a.b = neg_i(mul_pow2<-1>(v5));
  a.u0 = -v[1] * iv5;
  a.u1 = -v[2] * iv5;
  a.u2 = -v[3] * iv5;
  const double vm2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  const double lr = -gamma * igm1 + v[0] - 0.5 * vm2 * iv5 - nsfr_log(-v5) * igm1;
  a.r = nsfr_exp(lr);
  return a;
}

// reverse of pr_from_entropy: (rho, u, beta) cotangent -> v cotangent
__device__ __forceinline__ void entropy_bar_from_pr(const double v[5], const PR& a, double gamma, double igm1,
                                                    const PR& pb, double vb[5]) {
  const double v5 = v[4], iv5 = rcp_full(v5), iv52 = iv5 * iv5;
  const double vm2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  vb[0] = 0.0;
  vb[1] = vb[2] = vb[3] = 0.0;
  vb[4] = -0.5 * pb.b;
  const double ub[3] = {pb.u0, pb.u1, pb.u2};
  for (int c = 0; c < 3; ++c) {
    vb[1 + c] += -ub[c] * iv5;
    vb[4] += ub[c] * v[1 + c] * iv52;
  }
  const double lb = pb.r * a.r;
  vb[0] += lb;
  for (int c = 0; c < 3; ++c) vb[1 + c] += -lb * v[1 + c] * iv5;
  vb[4] += lb * (0.5 * vm2 * iv52 - igm1 * iv5);
}

// reverse of entropy_vars: v cotangent -> (rho, u, beta) cotangent and direct p cotangent
__device__ __forceinline__ void pr_bar_from_entropy_bar(const PR& a, double gamma, double igm1, const double vb[5],
                                                        PR& pb, double& pbar) {
  const double q2 = a.u0 * a.u0 + a.u1 * a.u1 + a.u2 * a.u2;
  const double ir = rcp_ff(a.r);  // 1/p = 2 beta / rho
  const double u[3] = {a.u0, a.u1, a.u2};
  double bb = -2.0 * vb[4] - vb[0] * q2;
  double ubv[3];
  for (int c = 0; c < 3; ++c) {
    bb += 2.0 * vb[1 + c] * u[c];
    ubv[c] = 2.0 * a.b * vb[1 + c] - 2.0 * a.b * u[c] * vb[0];
  }
  const double sb = -vb[0] * igm1;
  pbar = 2.0 * sb * a.b * ir;
  pb.r = -gamma * sb * ir;
  pb.u0 = ubv[0];
  pb.u1 = ubv[1];
  pb.u2 = ubv[2];
  pb.b = bb;
}

__device__ __forceinline__ PR pr_load(const double* P, int stride) {
  PR a;
  a.r = P[0];
  a.u0 = P[stride];
  a.u1 = P[2 * stride];
  a.u2 = P[3 * stride];
  a.b = P[4 * stride];
  return a;
}

// face record (K1 layout) -> primitive record
__device__ __forceinline__ PR pr_from_face(const double* f, int nfp) {
  const Rec R = load_rec(f, nfp);
  PR a;
  a.r = R.r;
  a.u0 = mul_pow2<1>(R.u0);
  a.u1 = mul_pow2<1>(R.u1);
  a.u2 = mul_pow2<1>(R.u2);
  a.b = mul_pow2<-1>(R.b2);
  return a;
}

// --------------------------------------------------------------------------
// volume reverse: one thread per line, like volume_kernel
// --------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(threads_for(N), 2)
    vjp_volume_kernel(const double* __restrict__ u, const double* __restrict__ rbar, const double* __restrict__ Rfwd,
                      const double* __restrict__ metric, const double* __restrict__ nf_plus,
                      const double* __restrict__ face, const double* __restrict__ wj, OpsGL ops, int nx, int ny,
                      int nz, int ne, double* __restrict__ ubar, double* __restrict__ fbar_own,
                      double* __restrict__ fbar_nbr, double* __restrict__ nfbar, double* __restrict__ mbar,
                      double* __restrict__ Jbar, const double* __restrict__ nrec, double* __restrict__ pbq) {
  constexpr int NV = N * N * N, NFP = N * N, NL = 3 * NFP;
  extern __shared__ double sm[];
  const int epb = blockDim.x / NL;
  const int e0 = blockIdx.x * epb;
  double* P = sm;                          // [epb][5][NV] primitive records
  double* Rb = P + (size_t)epb * 5 * NV;   // [epb][5][NV] Rbar
  double* Pb = Rb + (size_t)epb * 5 * NV;  // [epb][5][NV] record cotangents
  double* Y = Pb + (size_t)epb * 5 * NV;   // [epb][5][NV] Pi~^T R (for Jbar)
  PRF* Pf = reinterpret_cast<PRF*>(Y + (size_t)epb * 5 * NV);  // [epb][NV] rho, beta as float-float
  const double g = ops.gamma;
  const int nel = min(epb, ne - e0);
  const int total = nel * 5 * NV;

  if (ops.uncol) {
    // The uncollocated scheme: the line phase runs on the N GL points with the
    // projected state's records (the forward projection pass's node records),
    // and du^/dt = -Pt (W J)^{-1} A R_q (A = (chi Pi~1)^T, Pt = Pi~1, dense 1D
    // sweeps), so Rbar_q = A^T (W J)^{-1} Pt^T (-rbar), rbar at the ns^3
    // solution nodes.
    __shared__ double AT[NSFR_MAXN * NSFR_MAXN], PtT[NSFR_MAXN * NSFR_MAXN];
    const int ns = ops.ns, nsv = ns * ns * ns;
    for (int t = threadIdx.x; t < N * N; t += blockDim.x) AT[(t % N) * N + t / N] = ops.A[t];
    for (int t = threadIdx.x; t < ns * N; t += blockDim.x) PtT[(t % N) * ns + t / N] = ops.Pt[t];  // Pt: ns x N
    for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
      const int le = t / NV, node = t % NV;
      const double* rec = nrec + (size_t)(e0 + le) * NSFR_NFIELD * NV + node;
      double* p = P + (size_t)le * 5 * NV + node;
      p[0] = rec[P_RHO * NV];
      p[NV] = mul_pow2<1>(rec[P_UH * NV]);
      p[2 * NV] = mul_pow2<1>(rec[(P_UH + 1) * NV]);
      p[3 * NV] = mul_pow2<1>(rec[(P_UH + 2) * NV]);
      p[4 * NV] = mul_pow2<-1>(rec[P_B2 * NV]);
    }
    for (int t = threadIdx.x; t < nel * 5 * nsv; t += blockDim.x)
      Y[(size_t)(t / nsv) * NV + t % nsv] = -rbar[(size_t)e0 * 5 * nsv + t];
    __syncthreads();
    psweep(PtT, ns, N, Y, Pb, 5 * nel, NV, 0, ns, ns, ns);
    psweep(PtT, ns, N, Pb, Rb, 5 * nel, NV, 1, N, ns, ns);
    psweep(PtT, ns, N, Rb, Y, 5 * nel, NV, 2, N, N, ns);
    for (int t = threadIdx.x; t < total; t += blockDim.x) Y[t] /= wj[(size_t)(e0 + t / (5 * NV)) * NV + t % NV];
    __syncthreads();
    psweep(AT, N, N, Y, Pb, 5 * nel, NV, 0, N, N, N);
    psweep(AT, N, N, Pb, Y, 5 * nel, NV, 1, N, N, N);
    psweep(AT, N, N, Y, Rb, 5 * nel, NV, 2, N, N, N);
  } else {
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV;
    const PR a = pr_from_conserved(u + (size_t)(e0 + le) * 5 * NV + node, NV, g);
    double* p = P + (size_t)le * 5 * NV + node;
    p[0] = a.r;
    p[NV] = a.u0;
    p[2 * NV] = a.u1;
    p[3 * NV] = a.u2;
    p[4 * NV] = a.b;
  }
  // zbar = -Pi~^T rbar ; (y = Pi~^T R) ; Rbar = Pi~ D zbar with D = 1/(wJ)
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    Rb[t] = -rbar[(size_t)e0 * 5 * NV + t];
    if (Rfwd) Y[t] = Rfwd[(size_t)e0 * 5 * NV + t];
  }
  __syncthreads();
  auto sweep = [&](double* X, int d, bool transpose) {
    const int st = (d == 0) ? 1 : (d == 1 ? N : N * N);
    for (int t = threadIdx.x; t < nel * 5 * NFP; t += blockDim.x) {
      const int line = t % NFP, lk = t / NFP;
      int base, stride;
      line_geometry<N>(d, line % N, line / N, base, stride);
      double* x = X + (size_t)lk * NV + base;
      double dot = 0.0;
      for (int a = 0; a < N; ++a) dot = fma(transpose ? ops.hv[a] : ops.gv[a], x[a * st], dot);
      for (int a = 0; a < N; ++a) x[a * st] = fma(-(transpose ? ops.gv[a] : ops.hv[a]), dot, x[a * st]);
    }
  };
  if (ops.has_K) {
    for (int dd = 0; dd < 3; ++dd) {
      sweep(Rb, dd, true);
      if (Rfwd) sweep(Y, dd, true);
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV;
    const double wJ = wj[(size_t)(e0 + le) * NV + node];
    double db = 0.0;
    for (int k = 0; k < 5; ++k) {
      const size_t i = (size_t)(le * 5 + k) * NV + node;
      db += Rb[i] * Y[i];
      Rb[i] /= wJ;
    }
    // D = 1/(w J) -> Jbar = Dbar * dD/dJ = -Dbar / (w J^2)
    if (Rfwd) {
      const int i = node % N, j = (node / N) % N, k = node / (N * N);
      const double w3 = ops.w[i] * ops.w[j] * ops.w[k];
      const double J = wJ / w3;
      Jbar[(size_t)(e0 + le) * NV + node] += -db / (wJ * J);
    }
  }
  __syncthreads();
  if (ops.has_K) {
    for (int dd = 0; dd < 3; ++dd) {
      sweep(Rb, dd, false);
      __syncthreads();
    }
  }
  }  // collocated
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV;
    const double* p = P + (size_t)le * 5 * NV + node;
    Pf[t] = PRF{ff_split_i(p[0]), ff_split_i(p[4 * NV])};
  }
  __syncthreads();

  // line phase
  const int le = threadIdx.x / NL, l = threadIdx.x % NL, e = e0 + le;
  const bool valid = le < nel;
  const int d = l / NFP, line = l % NFP, l0 = line % N, l1 = line / N;
  int base, stride;
  line_geometry<N>(d, l0, l1, base, stride);
  PR ab[N];
  double mb[N][3];
  for (int a = 0; a < N; ++a) {
    ab[a] = PR{0, 0, 0, 0, 0};
    mb[a][0] = mb[a][1] = mb[a][2] = 0.0;
  }
  if (valid) {
    const double* Pe = P + (size_t)le * 5 * NV + base;
    const PRF* Pfe = Pf + (size_t)le * NV + base;
    const double* Re = Rb + (size_t)le * 5 * NV + base;
    const double* Me = metric + ((size_t)e * 9 + 3 * d) * NV + base;
    const double wperp = ops.w[l0] * ops.w[l1];
    // the fluxes take the sums of the two metric rows with halved cotangents (F
    // is linear in n), so that the row cotangent is nb itself
    const double hw = 0.5 * wperp;
    for (int a = 0; a < N; ++a) {
      const PR A = pr_load(Pe + a * stride, NV);
      for (int b = a + 1; b < N; ++b) {
        const PR B = pr_load(Pe + b * stride, NV);
        const double c = hw * ops.S1[a * N + b];
        double Fb[5];
        for (int k = 0; k < 5; ++k) Fb[k] = c * (Re[k * NV + a * stride] - Re[k * NV + b * stride]);
        double nb[3] = {0.0, 0.0, 0.0};
        ec_flux_vjp(A, B, Pfe[a * stride], Pfe[b * stride], Me[a * stride] + Me[b * stride],
                    Me[NV + a * stride] + Me[NV + b * stride], Me[2 * NV + a * stride] + Me[2 * NV + b * stride], ops,
                    Fb, ab[a], ab[b], nb);
        for (int c2 = 0; c2 < 3; ++c2) {
          mb[a][c2] += nb[c2];
          mb[b][c2] += nb[c2];
        }
      }
    }
    for (int s = 0; s < 2; ++s) {
      const int f = 2 * d + s;
      const int enb = nbr_index(e, d, s, nx, ny, nz);
      const PR Fo = pr_from_face(face + (((size_t)e * 6 + f) * NSFR_NFIELD) * NFP + line, NFP);
      const PR Fn = pr_from_face(face + (((size_t)enb * 6 + 2 * d + 1 - s) * NSFR_NFIELD) * NFP + line, NFP);
      const PRF Fof{ff_split_i(Fo.r), ff_split_i(Fo.b)}, Fnf{ff_split_i(Fn.r), ff_split_i(Fn.b)};
      const double* nf = nf_plus + (((size_t)(s ? e : enb) * 3 + d) * 3) * NFP + line;
      const double f0 = nf[0], f1 = nf[NFP], f2 = nf[2 * NFP];
      const double* t = s ? ops.tp : ops.tm;
      const double sw = (s ? 1.0 : -1.0) * wperp;
      double rho[5] = {0, 0, 0, 0, 0};
      for (int a = 0; a < N; ++a) {
        const double st = sw * t[a];
        for (int k = 0; k < 5; ++k) rho[k] = fma(st, Re[k * NV + a * stride], rho[k]);
      }
      PR fob{0, 0, 0, 0, 0}, fnb{0, 0, 0, 0, 0};
      double nfb[3] = {0.0, 0.0, 0.0};
      // face flux f* = F(L, R; n_f)
      if (s) ec_flux_vjp(Fo, Fn, Fof, Fnf, f0, f1, f2, ops, rho, fob, fnb, nfb);
      else ec_flux_vjp(Fn, Fo, Fnf, Fof, f0, f1, f2, ops, rho, fnb, fob, nfb);
      // hybrid terms (metric-row sums with halved cotangents, as above)
      for (int a = 0; a < N; ++a) {
        const PR A = pr_load(Pe + a * stride, NV);
        const double th = 0.5 * t[a];
        double Fb[5];
        for (int k = 0; k < 5; ++k) Fb[k] = th * fma(sw, Re[k * NV + a * stride], -rho[k]);
        double nb[3] = {0.0, 0.0, 0.0};
        ec_flux_vjp(A, Fo, Pfe[a * stride], Fof, Me[a * stride] + f0, Me[NV + a * stride] + f1,
                    Me[2 * NV + a * stride] + f2, ops, Fb, ab[a], fob, nb);
        for (int c2 = 0; c2 < 3; ++c2) {
          mb[a][c2] += nb[c2];
          nfb[c2] += nb[c2];
        }
      }
      double* fo = fbar_own + (((size_t)e * 6 + f) * 5) * NFP + line;
      double* fn = fbar_nbr + (((size_t)e * 6 + f) * 5) * NFP + line;
      fo[0] = fob.r;
      fo[NFP] = fob.u0;
      fo[2 * NFP] = fob.u1;
      fo[3 * NFP] = fob.u2;
      fo[4 * NFP] = fob.b;
      fn[0] = fnb.r;
      fn[NFP] = fnb.u0;
      fn[2 * NFP] = fnb.u1;
      fn[3 * NFP] = fnb.u2;
      fn[4 * NFP] = fnb.b;
      if (mbar) {
        double* nfo = nfbar + (((size_t)e * 6 + f) * 3) * NFP + line;
        for (int c2 = 0; c2 < 3; ++c2) nfo[c2 * NFP] = nfb[c2];
      }
    }
    if (mbar)
      for (int a = 0; a < N; ++a)
        for (int c2 = 0; c2 < 3; ++c2) mbar[((size_t)e * 9 + 3 * d + c2) * NV + base + a * stride] += mb[a][c2];
  }
  // record cotangents meet in shared memory (d = 0, 1, 2)
  for (int dd = 0; dd < 3; ++dd) {
    if (valid && d == dd) {
      double* pb = Pb + (size_t)le * 5 * NV + base;
      for (int a = 0; a < N; ++a) {
        const double x[5] = {ab[a].r, ab[a].u0, ab[a].u1, ab[a].u2, ab[a].b};
        for (int k = 0; k < 5; ++k) {
          if (dd == 0) pb[k * NV + a * stride] = x[k];
          else pb[k * NV + a * stride] += x[k];
        }
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int lq = t / NV, node = t % NV;
    const PR pb = pr_load(Pb + (size_t)lq * 5 * NV + node, NV);
    if (ops.uncol) {  // record cotangents at the GL points, for the projection's reverse
      double* q = pbq + (size_t)(e0 + lq) * 5 * NV + node;
      q[0] = pb.r;
      q[NV] = pb.u0;
      q[2 * NV] = pb.u1;
      q[3 * NV] = pb.u2;
      q[4 * NV] = pb.b;
      continue;
    }
    const PR a = pr_load(P + (size_t)lq * 5 * NV + node, NV);
    double Ub[5];
    conserved_bar(a, g, pb, 0.0, Ub);
    double* ub = ubar + (size_t)(e0 + lq) * 5 * NV + node;
    for (int k = 0; k < 5; ++k) ub[k * NV] += Ub[k];
  }
}

// --------------------------------------------------------------------------
// face reverse: face-state cotangents -> volume state cotangents
// --------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(threads_for(N), 2)
    vjp_face_kernel(const double* __restrict__ u, const double* __restrict__ fbar_own,
                    const double* __restrict__ fbar_nbr, OpsGL ops, int nx, int ny, int nz, int ne,
                    double* __restrict__ ubar) {
  constexpr int NV = N * N * N, NFP = N * N, NL = 3 * NFP;
  extern __shared__ double sm[];
  const int epb = blockDim.x / NL;
  const int e0 = blockIdx.x * epb;
  double* V = sm;                         // [epb][5][NV] entropy variables
  double* Vb = V + (size_t)epb * 5 * NV;  // [epb][5][NV] their cotangents
  const double g = ops.gamma;
  const int nel = min(epb, ne - e0);
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV;
    const PR a = pr_from_conserved(u + (size_t)(e0 + le) * 5 * NV + node, NV, g);
    double v[5];
    entropy_vars(a, g, ops.inv_gm1, v);
    for (int k = 0; k < 5; ++k) V[(size_t)(le * 5 + k) * NV + node] = v[k];
  }
  __syncthreads();
  const int le = threadIdx.x / NL, l = threadIdx.x % NL, e = e0 + le;
  const bool valid = le < nel;
  const int d = l / NFP, line = l % NFP;
  int base, stride;
  line_geometry<N>(d, line % N, line / N, base, stride);
  double vbl[N][5];
  for (int a = 0; a < N; ++a)
    for (int k = 0; k < 5; ++k) vbl[a][k] = 0.0;
  if (valid) {
    const double* Ve = V + (size_t)le * 5 * NV + base;
    for (int s = 0; s < 2; ++s) {
      const int f = 2 * d + s;
      const int enb = nbr_index(e, d, s, nx, ny, nz);
      const double* t = s ? ops.tp : ops.tm;
      double vf[5];
      for (int k = 0; k < 5; ++k) {
        double x = 0.0;
        for (int a = 0; a < N; ++a) x += t[a] * Ve[k * NV + a * stride];
        vf[k] = x;
      }
      const PR fa = pr_from_entropy(vf, g, ops.inv_gm1);
      const double* o = fbar_own + (((size_t)e * 6 + f) * 5) * NFP + line;
      const double* q = fbar_nbr + (((size_t)enb * 6 + 2 * d + 1 - s) * 5) * NFP + line;
      const PR pb{o[0] + q[0], o[NFP] + q[NFP], o[2 * NFP] + q[2 * NFP], o[3 * NFP] + q[3 * NFP],
                  o[4 * NFP] + q[4 * NFP]};
      double vfb[5];
      entropy_bar_from_pr(vf, fa, g, ops.inv_gm1, pb, vfb);
      for (int a = 0; a < N; ++a)
        for (int k = 0; k < 5; ++k) vbl[a][k] += t[a] * vfb[k];
    }
  }
  for (int dd = 0; dd < 3; ++dd) {
    if (valid && d == dd) {
      double* vb = Vb + (size_t)le * 5 * NV + base;
      for (int a = 0; a < N; ++a)
        for (int k = 0; k < 5; ++k) {
          if (dd == 0) vb[k * NV + a * stride] = vbl[a][k];
          else vb[k * NV + a * stride] += vbl[a][k];
        }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int lq = t / NV, node = t % NV;
    const PR a = pr_from_conserved(u + (size_t)(e0 + lq) * 5 * NV + node, NV, g);
    double vb[5];
    for (int k = 0; k < 5; ++k) vb[k] = Vb[(size_t)(lq * 5 + k) * NV + node];
    PR pb;
    double pbar;
    pr_bar_from_entropy_bar(a, g, ops.inv_gm1, vb, pb, pbar);
    double Ub[5];
    conserved_bar(a, g, pb, pbar, Ub);
    double* ub = ubar + (size_t)(e0 + lq) * 5 * NV + node;
    for (int k = 0; k < 5; ++k) ub[k * NV] += Ub[k];
  }
}

// --------------------------------------------------------------------------
// projection reverse (uncollocated scheme): record cotangents at the GL points
// and at the face points -> cotangent of the solution coefficients u^
// --------------------------------------------------------------------------
// The forward projection (projection.cu), with ns Lobatto solution nodes and N
// GL points per direction:
//   u_q = chi u^,  v_q = v(u_q),  v~^ = Pi v_q,
//   w_q = chi v~^  -> the volume records u(w_q),
//   w_f = (l_s along d) (chi, chi across) v~^  -> the face records u(w_f).
// Reversed: wbar from the record cotangents through u(w) (entropy_bar_from_pr),
// v~^bar = chi^T wbar_q + sum_faces (l_s, chi, chi)^T wbar_f, v_q bar = Pi^T v~^bar,
// u_q bar through v(u) (pr_bar_from_entropy_bar, conserved_bar), u^bar = chi^T u_q bar.
// One element per CTA (grid-stride); all sweeps on shared memory.
template <int N>
__global__ void __launch_bounds__(256) vjp_projection_kernel(const double* __restrict__ u,
                                                             const double* __restrict__ pbq,
                                                             const double* __restrict__ fbar_own,
                                                             const double* __restrict__ fbar_nbr, OpsGL ops, int nx,
                                                             int ny, int nz, int ne, double* __restrict__ ubar) {
  constexpr int NV = N * N * N, NFP = N * N, SL = 5 * NV;
  extern __shared__ double sm[];
  double* B0 = sm;  // six [5][NV] buffers
  double* B1 = B0 + SL;
  double* B2 = B1 + SL;
  double* B3 = B2 + SL;
  double* B4 = B3 + SL;
  double* B5 = B4 + SL;
  __shared__ double chiT[NSFR_MAXN * NSFR_MAXN], PiT[NSFR_MAXN * NSFR_MAXN];
  __shared__ double lay[5 * NSFR_MAXN * NSFR_MAXN], mid[5 * NSFR_MAXN * NSFR_MAXN];
  const int ns = ops.ns, nsv = ns * ns * ns;
  const double g = ops.gamma;
  for (int t = threadIdx.x; t < N * ns; t += blockDim.x) {
    chiT[(t % ns) * N + t / ns] = ops.chi[t];  // chi: N x ns
    PiT[(t % N) * ns + t / N] = ops.Pi[t];     // Pi: ns x N
  }
  for (int e = blockIdx.x; e < ne; e += gridDim.x) {
    for (int t = threadIdx.x; t < 5 * nsv; t += blockDim.x) B0[(t / nsv) * NV + t % nsv] = u[(size_t)e * 5 * nsv + t];
    __syncthreads();
    // forward: u_q (B1), v_q (B2), v~^ (B3), w_q (B4)
    psweep(ops.chi, ns, N, B0, B2, 5, NV, 0, ns, ns, ns);
    psweep(ops.chi, ns, N, B2, B3, 5, NV, 1, N, ns, ns);
    psweep(ops.chi, ns, N, B3, B1, 5, NV, 2, N, N, ns);
    for (int t = threadIdx.x; t < NV; t += blockDim.x) {
      const PR a = pr_from_conserved(B1 + t, NV, g);
      double v[5];
      entropy_vars(a, g, ops.inv_gm1, v);
      for (int k = 0; k < 5; ++k) B2[k * NV + t] = v[k];
    }
    __syncthreads();
    psweep(ops.Pi, N, ns, B2, B4, 5, NV, 0, N, N, N);
    psweep(ops.Pi, N, ns, B4, B5, 5, NV, 1, ns, N, N);
    psweep(ops.Pi, N, ns, B5, B3, 5, NV, 2, ns, ns, N);
    psweep(ops.chi, ns, N, B3, B5, 5, NV, 0, ns, ns, ns);
    psweep(ops.chi, ns, N, B5, B0, 5, NV, 1, N, ns, ns);
    psweep(ops.chi, ns, N, B0, B4, 5, NV, 2, N, N, ns);
    // wbar_q (B5) from the volume record cotangents
    for (int t = threadIdx.x; t < NV; t += blockDim.x) {
      double w[5], wb[5];
      for (int k = 0; k < 5; ++k) w[k] = B4[k * NV + t];
      const PR a = pr_from_entropy(w, g, ops.inv_gm1);
      const double* q = pbq + (size_t)e * 5 * NV + t;
      const PR pb{q[0], q[NV], q[2 * NV], q[3 * NV], q[4 * NV]};
      entropy_bar_from_pr(w, a, g, ops.inv_gm1, pb, wb);
      for (int k = 0; k < 5; ++k) B5[k * NV + t] = wb[k];
    }
    __syncthreads();
    // v~^bar = chi^T wbar_q -> B0 (ns^3)
    psweep(chiT, N, ns, B5, B4, 5, NV, 0, N, N, N);
    psweep(chiT, N, ns, B4, B2, 5, NV, 1, ns, N, N);
    psweep(chiT, N, ns, B2, B0, 5, NV, 2, ns, ns, N);
    // faces, one at a time: the layer l_s . v~^ along d (lay, ns^2), across the
    // first transverse direction (mid, N x ns), across the second (the face
    // points, N^2); reversed the same way into B0
    for (int f = 0; f < 6; ++f) {
      const int d = f / 2, side = f % 2;
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;  // transverse directions, lower first
      const double* ls = side ? ops.ls_p : ops.ls_m;
      auto vidx = [&](int a, int b, int c) {  // node of v~^ with index a along d, b along t1, c along t2
        int x[3];
        x[d] = a;
        x[t1] = b;
        x[t2] = c;
        return x[0] + ns * (x[1] + ns * x[2]);
      };
      for (int t = threadIdx.x; t < 5 * ns * ns; t += blockDim.x) {
        const int k = t / (ns * ns), b = (t / ns) % ns, c = t % ns;
        double acc = 0.0;
        for (int a = 0; a < ns; ++a) acc = fma(ls[a], B3[k * NV + vidx(a, b, c)], acc);
        lay[(k * ns + b) * ns + c] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 5 * N * ns; t += blockDim.x) {
        const int k = t / (N * ns), i = (t / ns) % N, c = t % ns;
        double acc = 0.0;
        for (int b = 0; b < ns; ++b) acc = fma(ops.chi[i * ns + b], lay[(k * ns + b) * ns + c], acc);
        mid[(k * N + i) * ns + c] = acc;
      }
      __syncthreads();
      // w_f at the face points and its cotangent (own + neighbour's slot), into B2 (5 x N^2)
      const int enb = nbr_index(e, d, side, nx, ny, nz);
      for (int t = threadIdx.x; t < NFP; t += blockDim.x) {
        const int i = t % N, j = t / N;  // face point t = i + N j (i along t1, j along t2)
        double w[5], wb[5];
        for (int k = 0; k < 5; ++k) {
          double acc = 0.0;
          for (int c = 0; c < ns; ++c) acc = fma(ops.chi[j * ns + c], mid[(k * N + i) * ns + c], acc);
          w[k] = acc;
        }
        const PR a = pr_from_entropy(w, g, ops.inv_gm1);
        const double* o = fbar_own + (((size_t)e * 6 + f) * 5) * NFP + t;
        const double* q = fbar_nbr + (((size_t)enb * 6 + 2 * d + 1 - side) * 5) * NFP + t;
        const PR pb{o[0] + q[0], o[NFP] + q[NFP], o[2 * NFP] + q[2 * NFP], o[3 * NFP] + q[3 * NFP],
                    o[4 * NFP] + q[4 * NFP]};
        entropy_bar_from_pr(w, a, g, ops.inv_gm1, pb, wb);
        for (int k = 0; k < 5; ++k) B2[k * NFP + t] = wb[k];
      }
      __syncthreads();
      // reverse across t2 (mid bar), across t1 (layer bar), along d into B0
      for (int t = threadIdx.x; t < 5 * N * ns; t += blockDim.x) {
        const int k = t / (N * ns), i = (t / ns) % N, c = t % ns;
        double acc = 0.0;
        for (int j = 0; j < N; ++j) acc = fma(ops.chi[j * ns + c], B2[k * NFP + i + N * j], acc);
        mid[(k * N + i) * ns + c] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 5 * ns * ns; t += blockDim.x) {
        const int k = t / (ns * ns), b = (t / ns) % ns, c = t % ns;
        double acc = 0.0;
        for (int i = 0; i < N; ++i) acc = fma(ops.chi[i * ns + b], mid[(k * N + i) * ns + c], acc);
        lay[(k * ns + b) * ns + c] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 5 * nsv; t += blockDim.x) {
        const int k = t / nsv, node = t % nsv;
        const int x[3] = {node % ns, (node / ns) % ns, node / (ns * ns)};
        B0[k * NV + node] = fma(ls[x[d]], lay[(k * ns + x[t1]) * ns + x[t2]], B0[k * NV + node]);
      }
      __syncthreads();
    }
    // v_q bar = Pi^T v~^bar -> B2 (N^3)
    psweep(PiT, ns, N, B0, B4, 5, NV, 0, ns, ns, ns);
    psweep(PiT, ns, N, B4, B5, 5, NV, 1, N, ns, ns);
    psweep(PiT, ns, N, B5, B2, 5, NV, 2, N, N, ns);
    // u_q bar through v(u) -> B4
    for (int t = threadIdx.x; t < NV; t += blockDim.x) {
      const PR a = pr_from_conserved(B1 + t, NV, g);
      double vb[5], Ub[5];
      for (int k = 0; k < 5; ++k) vb[k] = B2[k * NV + t];
      PR pb;
      double pbar;
      pr_bar_from_entropy_bar(a, g, ops.inv_gm1, vb, pb, pbar);
      conserved_bar(a, g, pb, pbar, Ub);
      for (int k = 0; k < 5; ++k) B4[k * NV + t] = Ub[k];
    }
    __syncthreads();
    // u^bar += chi^T u_q bar
    psweep(chiT, N, ns, B4, B5, 5, NV, 0, N, N, N);
    psweep(chiT, N, ns, B5, B2, 5, NV, 1, ns, N, N);
    psweep(chiT, N, ns, B2, B0, 5, NV, 2, ns, ns, N);
    for (int t = threadIdx.x; t < 5 * nsv; t += blockDim.x)
      ubar[(size_t)e * 5 * nsv + t] += B0[(t / nsv) * NV + t % nsv];
    __syncthreads();
  }
}

// --------------------------------------------------------------------------
// metric reverse: (C bar, shared face-row bar, J bar) -> control-point bar
// --------------------------------------------------------------------------
__device__ void msweep(const double* A, bool transpose, int rows, int k, int m, const double* in, double* out, int d,
                       int ex, int ey, int ez) {
  // forward: out(ext with m along d) = A (m x k) applied along d; transpose: A^T (k x m)
  int ox = ex, oy = ey, oz = ez;
  if (d == 0) ox = m;
  if (d == 1) oy = m;
  if (d == 2) oz = m;
  const int total = ox * oy * oz;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int x = t % ox, y = (t / ox) % oy, z = t / (ox * oy);
    double s = 0.0;
    for (int b = 0; b < k; ++b) {
      int xi = x, yi = y, zi = z, r;
      if (d == 0) { r = x; xi = b; }
      else if (d == 1) { r = y; yi = b; }
      else { r = z; zi = b; }
      const double a = transpose ? A[b * rows + r] : A[r * rows + b];
      s += a * in[xi + ex * (yi + ey * zi)];
    }
    out[t] = s;
  }
  __syncthreads();
}

// field slots of the metric reverse (see vjp_metric_kernel)
#define NSFR_VJP_METRIC_SLOTS 40

// out = A (N x N, or A^T) applied along direction D of an N x N x L block
// (x fastest; L = N for a cube, 1 for a face layer), A in shared memory
template <int N, int L, int D, bool TR>
__device__ __forceinline__ void nsweep(const double* A, const double* in, double* out) {
  constexpr int NT = N * N * L, ST = D == 0 ? 1 : (D == 1 ? N : N * N);
  for (int t = threadIdx.x; t < NT; t += blockDim.x) {
    const int r = (t / ST) % N;
    const double* src = in + (t - r * ST);
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < N; ++b) s = fma(TR ? A[b * N + r] : A[r * N + b], src[b * ST], s);
    out[t] = s;
  }
  __syncthreads();
}
template <int N, bool TR>
__device__ __forceinline__ void nsweep_d(const double* A, const double* in, double* out, int d) {
  if (d == 0) nsweep<N, N, 0, TR>(A, in, out);
  else if (d == 1) nsweep<N, N, 1, TR>(A, in, out);
  else nsweep<N, N, 2, TR>(A, in, out);
}
// along all three directions
template <int N, bool TR>
__device__ __forceinline__ void nsweep3(const double* A, const double* in, double* out, double* t1, double* t2) {
  nsweep<N, N, 0, TR>(A, in, t1);
  nsweep<N, N, 1, TR>(A, t1, t2);
  nsweep<N, N, 2, TR>(A, t2, out);
}

// S: doubles per field slot, at least max(n^3, q^3) (NSFR_VJP_METRIC_SLOTS
// slots), then the operators E (n x q), D (n x n), I (n x n) and the element's
// first control point.  Slots whose lifetimes do not overlap are shared: the
// control points become V once the Lobatto coordinates exist, and the Jacobian
// a = I3(dX) of the determinant part, which runs first, gives way to the metric
// cotangent Clb; the accumulation order is that of the plain sequence.
template <int N>
__global__ void vjp_metric_kernel(const double* __restrict__ ctrl, OpsGeo g, const double* __restrict__ mbar,
                                  const double* __restrict__ nfbar, const double* __restrict__ Jbar, int nx, int ny,
                                  int nz, int S, double* __restrict__ xbar) {
  extern __shared__ double sm[];
  constexpr int n = N, nv = N * N * N, nfp = N * N;
  const int q = g.q, q3 = q * q * q;
  double* Xe = sm;           // 3: control points; V (3) once X exists
  double* V = Xe;
  double* X = Xe + 3 * S;    // 3 (LGL)
  double* dX = X + 3 * S;    // 9
  double* A = dX + 9 * S;    // 9: a = d x / d xi at GL nodes, then its cotangent; then Clb
  double* Clb = A;           //    (the cotangent of the LGL metric)
  double* dXb = A + 9 * S;   // 9
  double* Xb = dXb + 9 * S;  // 3
  double* T1 = Xb + 3 * S;
  double* T2 = T1 + S;
  double* T3 = T2 + S;
  double* T4 = T3 + S;
  double* Es = T4 + S;       // n x q
  double* Dl = Es + N * NSFR_MAXN;
  double* Ig = Dl + N * N;
  double* X0 = Ig + N * N;   // the first control point
  const int e = blockIdx.x;
  for (int t = threadIdx.x; t < N * q; t += blockDim.x) Es[t] = g.E[t];
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    Dl[t] = g.Dl[t];
    Ig[t] = g.I[t];
  }
  for (int t = threadIdx.x; t < 3 * q3; t += blockDim.x) Xe[(t % 3) * S + t / 3] = ctrl[(size_t)e * q3 * 3 + t];
  if (threadIdx.x < 3) X0[threadIdx.x] = ctrl[(size_t)e * q3 * 3 + threadIdx.x];
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    msweep(Es, false, q, q, n, Xe + c * S, T1, 0, q, q, q);
    msweep(Es, false, q, q, n, T1, T2, 1, n, q, q);
    msweep(Es, false, q, q, n, T2, X + c * S, 2, n, n, q);
  }
  for (int k = 0; k < 3; ++k)
    for (int m = 0; m < 3; ++m) nsweep_d<N, false>(Dl, X + m * S, dX + (k * 3 + m) * S, k);
  for (int t = threadIdx.x; t < 9 * S; t += blockDim.x) dXb[t] = 0.0;
  for (int t = threadIdx.x; t < 3 * S; t += blockDim.x) Xb[t] = 0.0;
  __syncthreads();
  // J = det(a), a = I3(dX) at GL nodes: abar = Jbar cof(a) (in place), dXb += I3^T(abar)
  for (int r = 0; r < 9; ++r) nsweep3<N, false>(Ig, dX + r * S, A + r * S, T1, T2);
  for (int t = threadIdx.x; t < nv; t += blockDim.x) {
    const double a00 = A[0 * S + t], a01 = A[1 * S + t], a02 = A[2 * S + t];
    const double a10 = A[3 * S + t], a11 = A[4 * S + t], a12 = A[5 * S + t];
    const double a20 = A[6 * S + t], a21 = A[7 * S + t], a22 = A[8 * S + t];
    const double jb = Jbar[(size_t)e * nv + t];
    A[0 * S + t] = jb * (a11 * a22 - a12 * a21);
    A[1 * S + t] = jb * (a12 * a20 - a10 * a22);
    A[2 * S + t] = jb * (a10 * a21 - a11 * a20);
    A[3 * S + t] = jb * (a02 * a21 - a01 * a22);
    A[4 * S + t] = jb * (a00 * a22 - a02 * a20);
    A[5 * S + t] = jb * (a01 * a20 - a00 * a21);
    A[6 * S + t] = jb * (a01 * a12 - a02 * a11);
    A[7 * S + t] = jb * (a02 * a10 - a00 * a12);
    A[8 * S + t] = jb * (a00 * a11 - a01 * a10);
  }
  __syncthreads();
  for (int r = 0; r < 9; ++r) {
    nsweep3<N, true>(Ig, A + r * S, T3, T1, T2);
    for (int t = threadIdx.x; t < nv; t += blockDim.x) dXb[r * S + t] += T3[t];
    __syncthreads();
  }
  // metric = I3 (C_lgl)  ->  Clb = I3^T (mbar), in the slots a no longer needs
  for (int r = 0; r < 9; ++r) {
    for (int t = threadIdx.x; t < nv; t += blockDim.x) T3[t] = mbar[((size_t)e * 9 + r) * nv + t];
    __syncthreads();
    nsweep3<N, true>(Ig, T3, Clb + r * S, T1, T2);
  }
  // shared face rows: own +face (slot 2d+1) and the +neighbour's -face (slot 2d)
  for (int d = 0; d < 3; ++d) {
    int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
    if (d == 0) ex = (ex + 1) % nx;
    else if (d == 1) ey = (ey + 1) % ny;
    else ez = (ez + 1) % nz;
    const int ep = ex + nx * (ey + ny * ez);
    for (int c = 0; c < 3; ++c) {
      for (int t = threadIdx.x; t < nfp; t += blockDim.x)
        T3[t] = nfbar[(((size_t)e * 6 + 2 * d + 1) * 3 + c) * nfp + t] +
                nfbar[(((size_t)ep * 6 + 2 * d) * 3 + c) * nfp + t];
      __syncthreads();
      // forward: face = I (x) I applied to the layer: reverse with I^T along both
      nsweep<N, 1, 1, true>(Ig, T3, T4);
      nsweep<N, 1, 0, true>(Ig, T4, T3);
      double* dst = Clb + (d * 3 + c) * S;
      for (int t = threadIdx.x; t < nfp; t += blockDim.x) {
        const int f0 = t % n, f1 = t / n;
        int x, y, z;
        if (d == 0) { x = n - 1; y = f0; z = f1; }
        else if (d == 1) { x = f0; y = n - 1; z = f1; }
        else { x = f0; y = f1; z = n - 1; }
        dst[x + n * (y + n * z)] += T3[t];
      }
      __syncthreads();
    }
  }
  // C_lgl[i][c] = -curl_i(V^(c)), V^(c)_k = (X_l - X_l,0) dX[k][m], (c, m, l) cyclic
  for (int c = 0; c < 3; ++c) {
    const int m = (c + 1) % 3, l = (c + 2) % 3;
    // Vbar_k from Clb[.][c]: i=0: -(D1 V2 - D2 V1); i=1: -(D2 V0 - D0 V2); i=2: -(D0 V1 - D1 V0)
    for (int t = threadIdx.x; t < 3 * S; t += blockDim.x) V[t] = 0.0;
    __syncthreads();
    const int da[3] = {1, 2, 0}, va[3] = {2, 0, 1};
    const int db[3] = {2, 0, 1}, vb[3] = {1, 2, 0};
    for (int i = 0; i < 3; ++i) {
      nsweep_d<N, true>(Dl, Clb + (i * 3 + c) * S, T1, da[i]);
      nsweep_d<N, true>(Dl, Clb + (i * 3 + c) * S, T2, db[i]);
      for (int t = threadIdx.x; t < nv; t += blockDim.x) {
        V[va[i] * S + t] -= T1[t];
        V[vb[i] * S + t] += T2[t];
      }
      __syncthreads();
    }
    const double x0 = X0[l];
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
      const double xl = X[l * S + t] - x0;
      for (int k = 0; k < 3; ++k) {
        Xb[l * S + t] += V[k * S + t] * dX[(k * 3 + m) * S + t];
        dXb[(k * 3 + m) * S + t] += V[k * S + t] * xl;
      }
    }
    __syncthreads();
  }
  // dX[k][m] = D_k X_m
  for (int k = 0; k < 3; ++k)
    for (int m = 0; m < 3; ++m) {
      nsweep_d<N, true>(Dl, dXb + (k * 3 + m) * S, T1, k);
      for (int t = threadIdx.x; t < nv; t += blockDim.x) Xb[m * S + t] += T1[t];
      __syncthreads();
    }
  // X = E3(Xe) -> xbar += E3^T(Xb)
  for (int c = 0; c < 3; ++c) {
    msweep(Es, true, q, n, q, Xb + c * S, T1, 0, n, n, n);
    msweep(Es, true, q, n, q, T1, T2, 1, q, n, n);
    msweep(Es, true, q, n, q, T2, T3, 2, q, q, n);
    for (int t = threadIdx.x; t < q3; t += blockDim.x) xbar[((size_t)e * q3 + t) * 3 + c] += T3[t];
    __syncthreads();
  }
}

template <int N>
cudaError_t launch_vjp_n(nsfr_ctx* ctx, const double* u, const double* dbar, double* ubar, double* xbar,
                         const double* Rfwd, cudaStream_t s) {
  constexpr int NV = N * N * N;
  constexpr int epb = epb_for(N);
  const int grid = (ctx->ne + epb - 1) / epb;
  // per element: P, Rbar, record cotangents, Y (5 NV doubles each), then the node splits (NV PRF)
  size_t smem = (size_t)epb * NV * (20 * sizeof(double) + sizeof(PRF));
  cudaError_t err =
      cudaFuncSetAttribute(vjp_volume_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  nsfr_prof_begin(ctx, 6, s);
  vjp_volume_kernel<N><<<grid, threads_for(N), smem, s>>>(
      u, dbar, xbar ? Rfwd : nullptr, ctx->metric, ctx->nfp_plus, ctx->face, ctx->wj, ctx->ops, ctx->nx, ctx->ny,
      ctx->nz, ctx->ne, ubar, ctx->vjp_fown, ctx->vjp_fnbr, ctx->vjp_nfbar, xbar ? ctx->vjp_mbar : nullptr,
      ctx->vjp_jbar, ctx->nrec, ctx->vjp_pbq);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (ctx->uncol) {
    smem = (size_t)6 * 5 * NV * sizeof(double);
    if ((err = cudaFuncSetAttribute(vjp_projection_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem)) != cudaSuccess)
      return err;
    nsfr_prof_begin(ctx, 5, s);
    vjp_projection_kernel<N><<<ctx->ne < 152 * 16 ? ctx->ne : 152 * 16, 256, smem, s>>>(
        u, ctx->vjp_pbq, ctx->vjp_fown, ctx->vjp_fnbr, ctx->ops, ctx->nx, ctx->ny, ctx->nz, ctx->ne, ubar);
    nsfr_prof_end(ctx, s);
    ctx->launches++;
    return cudaGetLastError();
  }
  smem = (size_t)epb * 10 * NV * sizeof(double);
  if ((err = cudaFuncSetAttribute(vjp_face_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return err;
  nsfr_prof_begin(ctx, 5, s);
  vjp_face_kernel<N><<<grid, threads_for(N), smem, s>>>(u, ctx->vjp_fown, ctx->vjp_fnbr, ctx->ops, ctx->nx, ctx->ny,
                                                        ctx->nz, ctx->ne, ubar);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace

// field slot of the metric reverse: max(n^3, q^3) doubles rounded up to 32; the
// block has as many threads (at most 256), so that a pass over a field is one sweep
static int vjp_metric_slot(const nsfr_ctx* ctx) {
  const int nv = ctx->gops.n * ctx->gops.n * ctx->gops.n, q3 = ctx->gops.q * ctx->gops.q * ctx->gops.q;
  const int m = nv > q3 ? nv : q3;
  return (m + 31) / 32 * 32;
}
// the field slots, the operators E (n x NSFR_MAXN), D and I (n x n) and the first
// control point (4 doubles)
size_t nsfr_vjp_metric_smem(const nsfr_ctx* ctx) {
  const int n = ctx->gops.n;
  return ((size_t)NSFR_VJP_METRIC_SLOTS * vjp_metric_slot(ctx) + (size_t)n * NSFR_MAXN + 2 * (size_t)n * n + 4) *
         sizeof(double);
}

cudaError_t nsfr_launch_vjp(nsfr_ctx* ctx, const double* u, const double* dbar, double* ubar, double* xbar,
                            cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  const double* Rfwd = ctx->rtmp;
  switch (ctx->n) {
    case 2: err = launch_vjp_n<2>(ctx, u, dbar, ubar, xbar, Rfwd, s); break;
    case 3: err = launch_vjp_n<3>(ctx, u, dbar, ubar, xbar, Rfwd, s); break;
    case 4: err = launch_vjp_n<4>(ctx, u, dbar, ubar, xbar, Rfwd, s); break;
    case 5: err = launch_vjp_n<5>(ctx, u, dbar, ubar, xbar, Rfwd, s); break;
    case 6: err = launch_vjp_n<6>(ctx, u, dbar, ubar, xbar, Rfwd, s); break;
    case 7: err = launch_vjp_n<7>(ctx, u, dbar, ubar, xbar, Rfwd, s); break;
    case 8: err = launch_vjp_n<8>(ctx, u, dbar, ubar, xbar, Rfwd, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (err != cudaSuccess || !xbar) return err;
  const int S = vjp_metric_slot(ctx);
  const size_t smem = nsfr_vjp_metric_smem(ctx);
  void (*vjp_metric_kernel_p)(const double*, OpsGeo, const double*, const double*, const double*, int, int, int, int,
                              double*) = nullptr;
  switch (ctx->gops.n) {
    case 2: vjp_metric_kernel_p = vjp_metric_kernel<2>; break;
    case 3: vjp_metric_kernel_p = vjp_metric_kernel<3>; break;
    case 4: vjp_metric_kernel_p = vjp_metric_kernel<4>; break;
    case 5: vjp_metric_kernel_p = vjp_metric_kernel<5>; break;
    case 6: vjp_metric_kernel_p = vjp_metric_kernel<6>; break;
    case 7: vjp_metric_kernel_p = vjp_metric_kernel<7>; break;
    case 8: vjp_metric_kernel_p = vjp_metric_kernel<8>; break;
    default: return cudaErrorInvalidValue;
  }
  if ((err = cudaFuncSetAttribute(vjp_metric_kernel_p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
      cudaSuccess)
    return err;
  nsfr_prof_begin(ctx, 7, s);
  vjp_metric_kernel_p<<<ctx->ne, S < 256 ? S : 256, smem, s>>>(ctx->ctrl, ctx->gops, ctx->vjp_mbar, ctx->vjp_nfbar,
                                                                ctx->vjp_jbar, ctx->nx, ctx->ny, ctx->nz, S, xbar);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}
