// NSFR-EC volume/hybrid/surface kernel, FP32-bulk form.
//
// Same discretisation as volume_kernel (Eq. NSFR with sum-factorised
// Hadamard products, Eq. weight-adj ESFR mass, fused RK stage), with the work
// split by precision:
//   FP64  the entropy projection (the shared face-state kernel), the state,
//         and the logarithmic means of pairs whose values differ by more than
//         about 3% (the log branch, with the face-state pass's logs);
//   float-float (FP32 pairs, ~48 bits)  the scalars made from the log means
//         -- rho_ln, p_hat = rho_bar / (2 beta_bar) and the energy coefficient
//         H = 1/(2(gamma-1) beta_ln) + p_hat/rho_ln -- on the series branch,
//         where each is a constant plus an O(f^2) correction that FP32 carries
//         to ~1e-7 of itself, and the mass flux rho_ln u.n with its
//         accumulation;
//   FP32  the momentum and energy flux arithmetic and their accumulation, and
//         the mass-inverse contractions.
// The fluxes are formed as deviations from the state of the element's first
// node (rho_ref, u_ref, p_ref): subtracting p_ref n from the momentum flux
// leaves R unchanged (the scheme is free-stream preserving, Sec. "Free-stream
// Preservation"), and because R is linear in the flux values,
//   F_m = F_rho u_bar + p_hat n      -> F_m' = F_rho (u_bar - u_ref) + (p_hat - p_ref) n,
//                                        R_m = R(F_m') + u_ref R_rho,
//   F_E = F_rho (H - |u|^2_bar/2 + |u_bar|^2), H = 1/(2(gamma-1) beta_ln) + p_hat/rho_ln
//                                     -> F_E' = F_E - E_ref F_rho, E_ref = H_ref + |u_ref|^2/2,
//                                        R_E = R(F_E') + E_ref R_rho,
// exactly.  Only O(deviation) quantities then meet FP32 rounding; the mass
// residual, which u_ref and E_ref (~250 for the Taylor-Green vortex) multiply,
// is kept to ~48 bits.
#include <type_traits>

#include "ffloat.cuh"
#include "kernel_common.cuh"
#include "mathfn_ff.cuh"
#include "physics.cuh"

namespace {
using namespace nsfr_k;

// a node of the bulk kernels: rho, 2 beta, u/2 as float-float (split from the
// FP64 records in the FP32-bulk form, the float-float records in its variant);
// the FP64 values and the logs are read from the records when a log mean
// leaves its series branch
template <bool FF>
struct BNode {
  ff r, b2;
  ff u0, u1, u2;  // u/2
  float qq;       // |u|^2/4
};

template <bool FF>
__device__ __forceinline__ BNode<FF> bnode_from_rec(const Rec& a) {
  BNode<FF> b;
  b.r = ff_split_i(a.r);
  b.b2 = ff_split_i(a.b2);
  b.u0 = ff_split_i(a.u0);
  b.u1 = ff_split_i(a.u1);
  b.u2 = ff_split_i(a.u2);
  b.qq = d2f_i(a.qq);
  return b;
}

struct BRef {
  double p, H;       // p_ref, H_ref = gamma p_ref / ((gamma - 1) rho_ref)
  ff pf, Hf;         // the same as float-float
  ff u0, u1, u2;     // u_ref
  float kin;         // |u_ref|^2 / 2
};

// 1/x as float-float for x > 0 (normal): the FP32 seed r0 (rcp32(x.hi)) and
// one correction r0 (1 - x r0), with 1 - x r0 formed by FMAs (error ~2^-46
// relative)
__device__ __forceinline__ ff ff_rcp(ff x, float r0) {
  const float e = __fmaf_rn(-x.lo, r0, __fmaf_rn(-x.hi, r0, 1.0f));
  ff r;
  fast_two_sum(r0, __fmul_rn(r0, e), r.hi, r.lo);
  return r;
}
__device__ __forceinline__ ff ff_rcp(ff x) { return ff_rcp(x, rcp32(x.hi)); }

// a - b for close float-float values (|a - b| << |a|): the hi difference is exact
__device__ __forceinline__ float ff_diff(ff a, ff b) { return (a.hi - b.hi) + (a.lo - b.lo); }


// series branch of the log means in float-float: u = f^2 below this
#define NSFR_LM_EPS32 1.0e-3f

// deviation flux of a pair: Fr (mass, float-float), Fm = F_m - u_ref F_rho - p_ref n,
// FE = F_E - (H_ref + |u_ref|^2/2) F_rho; (n0, n1, n2) the averaged metric row.
// With f = (a - b)/(a + b), u = f^2 for rho and for 2 beta:
//   rho_ln = (rho_bar) G(u_r),  G = f/atanh(f) = 1 - u/3 - 4u^2/45 - 44u^3/945 - ...
//   H s2 = p_hat s2 / rho_ln + s2 / (2 (gamma-1) beta_ln) = 2 atanh(f_r)/f_r + F4g(u_b)
//        = (2 + 2/(gamma-1)) + u_r P_a(u_r) + u_b P_b(u_b)
// (s2 = 2 beta_a + 2 beta_b), truncated where the next term is below 1e-13 (u < 1e-3).
// The FP32-bulk form: the log means to FP64 accuracy as the FP64 path forms
// them -- the series branch (u < 1e-4) from the nodes' float-float rho and
// 2 beta with float-float tails good to ~2^-40 of themselves (lm_u_ff,
// lm_tail_ffv), the FP64 records and logs off it -- and the scalars made from
// them in float-float: rho_ln = (s/2)(1 + eps_G(u_r)), H s2 = (2 + F4g(0)) +
// eps_a(u_r) + eps_b(u_b), eps_a the series of 2 atanh(f_r)/f_r - 2.
template <class LA, class LB>
__device__ __forceinline__ void bulk_flux(const BNode<false>& A, const BNode<false>& B, ff n0, ff n1, ff n2,
                                          const BRef& ref, const OpsGL& K, const LA& la, const LB& lb, ff& Fr,
                                          float Fm[3], float& FE) {
  const ff sr = ff_add_nn(A.r, B.r), s2 = ff_add_nn(A.b2, B.b2);
  const float rs2 = rcp32(s2.hi);
  const ff rb2 = ff_rcp(s2, rs2);
  ff ur, ub, rln, cx;  // cx = H s2 - (2 + 2/(gamma-1))
  if (lm_u_ff(ff_add_nn(A.r, ff_neg(B.r)), sr, rcp32(sr.hi), ur)) {
    const ff sh{0.5f * sr.hi, 0.5f * sr.lo};
    rln = ff_add(sh, ff_mul_nn(sh, lm_tail_ffv(ur, K.lmg_ff)));
    cx = lm_tail_ffv(ur, K.lma_ff);
  } else {  // FP64 from the records and the logs of the face-state pass
    const double dr = la.r() - lb.r(), dl = la.lr() - lb.lr();
    rln = ff_split_i(dr / dl);
    cx = ff_split_i(fma(la.r() + lb.r(), dl / dr, -K.fr2[0]));
  }
  if (lm_u_ff(ff_add_nn(A.b2, ff_neg(B.b2)), s2, rs2, ub)) {
    cx = ff_add(cx, lm_tail_ffv(ub, K.lmb_ff));
  } else {
    const double sb = la.b2() + lb.b2(), db = la.b2() - lb.b2();
    cx = ff_add(cx, ff_split_i(fma(K.inv_gm1 * (la.lb() - lb.lb()), sb / db, -K.f4g[0])));
  }
  const ff H = ff_mul(ff_add(ff{K.cab_hi, K.cab_lo}, cx), rb2);
  const float dp = ff_diff(ff_mul(sr, rb2), ref.pf);
  const float dH = ff_diff(H, ref.Hf);
  const ff v0 = ff_add_nn(A.u0, B.u0), v1 = ff_add_nn(A.u1, B.u1), v2 = ff_add_nn(A.u2, B.u2);
  const ff un = ff_add_nn(ff_add_nn(ff_mul(v0, n0), ff_mul(v1, n1)), ff_mul(v2, n2));
  Fr = ff_mul(rln, un);
  const float f = Fr.hi;
  const float w0 = ff_diff(v0, ref.u0), w1 = ff_diff(v1, ref.u1), w2 = ff_diff(v2, ref.u2);
  Fm[0] = fmaf(f, w0, dp * n0.hi);
  Fm[1] = fmaf(f, w1, dp * n1.hi);
  Fm[2] = fmaf(f, w2, dp * n2.hi);
  const float du2 = fmaf(w0, v0.hi + ref.u0.hi, fmaf(w1, v1.hi + ref.u1.hi, w2 * (v2.hi + ref.u2.hi)));
  FE = f * (dH + du2 + ref.kin - (A.qq + B.qq));
}

// The float-float variant: the same scalars in float-float on the series branch.
template <class LA, class LB>
__device__ __forceinline__ void bulk_flux(const BNode<true>& A, const BNode<true>& B, ff n0, ff n1, ff n2,
                                          const BRef& ref, const OpsGL& K, const LA& la, const LB& lb, ff& Fr,
                                          float Fm[3], float& FE) {
  const ff sr = ff_add_nn(A.r, B.r), s2 = ff_add_nn(A.b2, B.b2);
  const float dr = ff_diff(A.r, B.r), d2 = ff_diff(A.b2, B.b2);
  const ff rb2 = ff_rcp(s2);
  float rsr;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rsr) : "f"(sr.hi));
  const float fr = dr * rsr, fb = d2 * rb2.hi;
  const float ur = fr * fr, ub = fb * fb;
  ff rln;
  float cx;  // H s2 - (2 + 2/(gamma-1))
  if (ur < NSFR_LM_EPS32) {
    const float g = ur * fmaf(fmaf(K.lmg[2], ur, K.lmg[1]), ur, K.lmg[0]);
    rln = ff_add_small(ff{0.5f * sr.hi, 0.5f * sr.lo}, 0.5f * sr.hi * g);
    cx = ur * fmaf(fmaf(K.lma[2], ur, K.lma[1]), ur, K.lma[0]);
  } else {  // FP64 with the logs of the face-state pass
    const double srd = ff_to_double(sr), drd = ff_to_double(A.r) - ff_to_double(B.r);
    const double dl = la.lr() - lb.lr();
    rln = ff_from_double(drd / dl);
    cx = d2f_i(fma(srd, dl / drd, -2.0));
  }
  if (ub < NSFR_LM_EPS32) {
    cx += ub * fmaf(fmaf(K.lmb[2], ub, K.lmb[1]), ub, K.lmb[0]);
  } else {
    const double s2d = ff_to_double(s2), d2d = ff_to_double(A.b2) - ff_to_double(B.b2);
    cx += d2f_i(fma(K.inv_gm1 * (la.lb() - lb.lb()), s2d / d2d, -2.0 * K.inv_gm1));
  }
  const ff H = ff_mul(ff_add_small(ff{K.cab_hi, K.cab_lo}, cx), rb2);
  const float dp = ff_diff(ff_mul(sr, rb2), ref.pf);
  const float dH = ff_diff(H, ref.Hf);
  const ff v0 = ff_add_nn(A.u0, B.u0), v1 = ff_add_nn(A.u1, B.u1), v2 = ff_add_nn(A.u2, B.u2);
  const ff un = ff_add_nn(ff_add_nn(ff_mul(v0, n0), ff_mul(v1, n1)), ff_mul(v2, n2));
  Fr = ff_mul(rln, un);
  const float f = Fr.hi;
  // velocity deviations to float accuracy (the hi difference rounded once, the lo
  // difference added)
  const float w0 = ff_diff(v0, ref.u0), w1 = ff_diff(v1, ref.u1), w2 = ff_diff(v2, ref.u2);
  Fm[0] = fmaf(f, w0, dp * n0.hi);
  Fm[1] = fmaf(f, w1, dp * n1.hi);
  Fm[2] = fmaf(f, w2, dp * n2.hi);
  // |u_bar|^2 - |u_ref|^2/2 - |u|^2_bar/2, with |u_bar|^2 - |u_ref|^2 = (u_bar - u_ref).(u_bar + u_ref)
  const float du2 = fmaf(w0, v0.hi + ref.u0.hi, fmaf(w1, v1.hi + ref.u1.hi, w2 * (v2.hi + ref.u2.hi)));
  FE = f * (dH + du2 + ref.kin - (A.qq + B.qq));
}

// a x for a power of two a (exact)
__device__ __forceinline__ ff ff_scale(ff x, float a) { return ff{x.hi * a, x.lo * a}; }

__device__ __forceinline__ float2 ff_pack(ff x) { return make_float2(x.hi, x.lo); }

// K1 for FP32-bulk contexts: the entropy projection of face_state_kernel --
// v(u) at the nodes, t_s . v along every line to both faces, u(v~) at the face
// nodes -- in float-float arithmetic with the float-float log and exp, so that
// it does not wait on the FP64 pipe (about 1e-14 relative in every output).
// Node records: rho, 2 beta, u/2, |u|^2/4 as float-float pairs packed in the
// 8-byte slots (read by volume_bulk_kernel only), ln rho and ln beta in FP64;
// face records in FP64, as the face-flux kernel reads them.
template <int N>
__global__ void __launch_bounds__(threads_for(N)) face_state_bulk_kernel(const double* __restrict__ u, OpsGL ops,
                                                                         double* __restrict__ face,
                                                                         double* __restrict__ nrec, int ne,
                                                                         int* flag) {
  constexpr int NV = N * N * N, NFP = N * N, NL = 3 * NFP;
  extern __shared__ double sm[];
  const int epb = blockDim.x / NL;
  const int e0 = blockIdx.x * epb;
  ff* V = reinterpret_cast<ff*>(sm);  // [epb][5][NV] entropy variables
  const MathTablesF T = nsfr_stage_tables_f(reinterpret_cast<float*>(V + (size_t)epb * 5 * NV));
  const ff G = ff_from_double(ops.gamma), GM1 = ff_from_double(ops.gamma - 1.0);
  const ff IGM1 = ff_from_double(ops.inv_gm1), LN2 = ff_from_double(0.69314718055994530942);
  __syncthreads();
  for (int t = threadIdx.x; t < epb * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV, e = e0 + le;
    if (e >= ne) continue;
    const double* ue = u + (size_t)e * 5 * NV + node;
    const ff r = ff_from_double(ue[0]), m0 = ff_from_double(ue[NV]), m1 = ff_from_double(ue[2 * NV]),
             m2 = ff_from_double(ue[3 * NV]), E = ff_from_double(ue[4 * NV]);
    const ff ir = ff_rcp(r);
    const ff u0 = ff_mul(m0, ir), u1 = ff_mul(m1, ir), u2 = ff_mul(m2, ir);
    const ff q2 = ff_add(ff_add(ff_mul(u0, u0), ff_mul(u1, u1)), ff_mul(u2, u2));
    const ff p = ff_mul(ff_add(E, ff_neg(ff_mul(ff_scale(r, 0.5f), q2))), GM1);
    if (!(r.hi > 0.0f) || !(p.hi > 0.0f)) atomicOr(flag, 1);
    const ff b2 = ff_mul(r, ff_rcp(p));  // 2 beta = rho / p
    const ff lr = ff_log(r, T), lp = ff_log(p, T);
    // v0 = (gamma - s)/(gamma - 1) - beta |u|^2,  s = ln p - gamma ln rho
    const ff gs = ff_add(ff_add(G, ff_neg(lp)), ff_mul(G, lr));
    ff* v = V + (size_t)le * 5 * NV + node;
    v[0] = ff_add(ff_mul(gs, IGM1), ff_neg(ff_mul(ff_scale(b2, 0.5f), q2)));
    v[NV] = ff_mul(b2, u0);
    v[2 * NV] = ff_mul(b2, u1);
    v[3 * NV] = ff_mul(b2, u2);
    v[4 * NV] = ff_neg(b2);
    float2* rec = reinterpret_cast<float2*>(nrec + (size_t)e * NSFR_NFIELD * NV) + node;
    rec[P_RHO * NV] = ff_pack(r);
    rec[P_B2 * NV] = ff_pack(b2);
    rec[P_UH * NV] = ff_pack(ff_scale(u0, 0.5f));
    rec[(P_UH + 1) * NV] = ff_pack(ff_scale(u1, 0.5f));
    rec[(P_UH + 2) * NV] = ff_pack(ff_scale(u2, 0.5f));
    rec[P_QQ * NV] = ff_pack(ff_scale(q2, 0.25f));
    double* recd = nrec + (size_t)e * NSFR_NFIELD * NV + node;
    recd[P_LRHO * NV] = ff_to_double(lr);
    recd[P_LBETA * NV] = ff_to_double(ff_add(ff_add(lr, ff_neg(lp)), ff_neg(LN2)));  // ln rho - ln 2p
  }
  __syncthreads();
  const int le = threadIdx.x / NL, l = threadIdx.x % NL, e = e0 + le;
  if (le >= epb || e >= ne) return;
  const int d = l / NFP, line = l % NFP;
  int base, stride;
  line_geometry<N>(d, line % N, line / N, base, stride);
  const ff* v = V + (size_t)le * 5 * NV + base;
  ff vm[5], vp[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    ff am{0.0f, 0.0f}, ap{0.0f, 0.0f};
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const ff x = v[k * NV + a * stride];
      am = ff_fma(ff{ops.tmf[a], ops.tmlo[a]}, x, am);
      ap = ff_fma(ff{ops.tpf[a], ops.tplo[a]}, x, ap);
    }
    vm[k] = am;
    vp[k] = ap;
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const ff* w = s ? vp : vm;
    if (!(w[4].hi < 0.0f)) atomicOr(flag, 1);
    const ff b2 = ff_neg(w[4]);  // 2 beta
    const ff ib2 = ff_rcp(b2);
    const ff u0 = ff_mul(w[1], ib2), u1 = ff_mul(w[2], ib2), u2 = ff_mul(w[3], ib2);
    const ff q2 = ff_add(ff_add(ff_mul(u0, u0), ff_mul(u1, u1)), ff_mul(u2, u2));
    // s = gamma - (gamma - 1)(v0 + beta |u|^2), ln rho = -(s + ln 2 beta)/(gamma - 1)
    const ff sent = ff_add(G, ff_neg(ff_mul(GM1, ff_add(ff_mul(ff_scale(b2, 0.5f), q2), w[0]))));
    const ff L5 = ff_log(b2, T);
    const ff lr = ff_neg(ff_mul(ff_add(sent, L5), IGM1));
    Rec P;
    P.r = ff_to_double(ff_exp(lr, T));
    P.b2 = ff_to_double(b2);
    P.u0 = ff_to_double(ff_scale(u0, 0.5f));
    P.u1 = ff_to_double(ff_scale(u1, 0.5f));
    P.u2 = ff_to_double(ff_scale(u2, 0.5f));
    P.qq = ff_to_double(ff_scale(q2, 0.25f));
    P.lr = ff_to_double(lr);
    P.lb = ff_to_double(ff_add(L5, ff_neg(LN2)));
    store_rec(face + (((size_t)e * 6 + 2 * d + s) * NSFR_NFIELD) * NFP + line, NFP, P);
  }
}

// reference state of an element: its node 0 (u_ref from the same float-float
// split of u/2 that the node records hold, doubled exactly)
// from an FP64 node record (FP32-bulk form)
__device__ __forceinline__ BRef make_ref(const Rec& a, const OpsGL& ops) {
  BRef r;
  const double ib2 = rcp_full(a.b2);
  r.p = a.r * ib2;
  r.H = ops.gamma * ops.inv_gm1 * ib2;
  r.pf = ff_from_double(r.p);
  r.Hf = ff_from_double(r.H);
  const ff h0 = ff_from_double(a.u0), h1 = ff_from_double(a.u1), h2 = ff_from_double(a.u2);
  r.u0 = ff{2.0f * h0.hi, 2.0f * h0.lo};
  r.u1 = ff{2.0f * h1.hi, 2.0f * h1.lo};
  r.u2 = ff{2.0f * h2.hi, 2.0f * h2.lo};
  const float x = r.u0.hi, y = r.u1.hi, z = r.u2.hi;
  r.kin = 0.5f * fmaf(x, x, fmaf(y, y, z * z));
  return r;
}

// from the float-float fields of its node record: rho, 2 beta, u/2 (float-float variant)
__device__ __forceinline__ BRef make_ref(ff rho, ff b2, ff h0, ff h1, ff h2, const OpsGL& ops) {
  BRef r;
  const double ib2 = rcp_full(ff_to_double(b2));
  r.p = ff_to_double(rho) * ib2;
  r.H = ops.gamma * ops.inv_gm1 * ib2;
  r.pf = ff_from_double(r.p);
  r.Hf = ff_from_double(r.H);
  r.u0 = ff{2.0f * h0.hi, 2.0f * h0.lo};
  r.u1 = ff{2.0f * h1.hi, 2.0f * h1.lo};
  r.u2 = ff{2.0f * h2.hi, 2.0f * h2.lo};
  const float x = r.u0.hi, y = r.u1.hi, z = r.u2.hi;
  r.kin = 0.5f * fmaf(x, x, fmaf(y, y, z * z));
  return r;
}

template <int N>
__device__ __forceinline__ void rank_one_sweep_f(float* X, int nel, int d, bool transpose, const OpsGL& ops) {
  constexpr int NV = N * N * N, NFP = N * N;
  const int st = (d == 0) ? 1 : (d == 1 ? N : N * N);
  const int nlines = nel * 5 * NFP;
  for (int t = threadIdx.x; t < nlines; t += blockDim.x) {
    const int line = t % NFP, lk = t / NFP;
    int base, stride;
    line_geometry<N>(d, line % N, line / N, base, stride);
    float* x = X + (size_t)lk * NV + base;
    float dot = 0.0f;
#pragma unroll
    for (int a = 0; a < N; ++a) dot = fmaf(transpose ? ops.hvf[a] : ops.gvf[a], x[a * st], dot);
#pragma unroll
    for (int a = 0; a < N; ++a) x[a * st] = fmaf(-(transpose ? ops.gvf[a] : ops.hvf[a]), dot, x[a * st]);
  }
}

// Y = A along direction d of X (FP32), nslab slabs of stride st, extents (ex, ey,
// ez) in and m along d out; A is m x k row-major, or with trans the transpose of
// a k x m row-major matrix.  Ends with a barrier.
__device__ void fsweep(const float* __restrict__ A, bool trans, int k, int m, const float* X, float* Y, int nslab,
                       int st, int d, int ex, int ey, int ez) {
  int ox = ex, oy = ey, oz = ez;
  if (d == 0) ox = m;
  if (d == 1) oy = m;
  if (d == 2) oz = m;
  const int per = ox * oy * oz;
  for (int t = threadIdx.x; t < nslab * per; t += blockDim.x) {
    const int sl = t / per, q = t % per;
    const int x = q % ox, y = (q / ox) % oy, z = q / (ox * oy);
    const float* in = X + (size_t)sl * st;
    float acc = 0.0f;
    for (int b = 0; b < k; ++b) {
      int xi = x, yi = y, zi = z, r;
      if (d == 0) { r = x; xi = b; }
      else if (d == 1) { r = y; yi = b; }
      else { r = z; zi = b; }
      const float a = trans ? A[b * m + r] : A[r * k + b];
      acc = fmaf(a, in[xi + ex * (yi + ey * zi)], acc);
    }
    Y[(size_t)sl * st + q] = acc;
  }
  __syncthreads();
}

// The FP32-bulk epilogue of the uncollocated scheme (solution on the ns Lobatto
// nodes, the N GL points of the line phase), the FP32 form of the FP64 kernel's:
// R_q (FP64, [nel][5][NV]) in FP32, then R^ = chi^T R_q (raw residual) or
// du^/dt = -Pi~ (W J)^{-1} (chi Pi~1)^T R_q by dense 1D sweeps, and the store or
// the RK stage update on the ns^3 solution nodes.  X and Y: [nel][5][NV] floats.
template <int N>
__device__ void uncol_epilogue_f(const double* Rd, float* X, float* Y, int nel, int e0, const OpsGL& ops,
                                 const float* __restrict__ invwj32, int epi, const RkArgs& rk, double* out) {
  constexpr int NV = N * N * N;
  const int ns = ops.ns, nsv = ns * ns * ns, nsl = nel * 5;
  for (int t = threadIdx.x; t < nsl * NV; t += blockDim.x) X[t] = d2f_i(Rd[t]);
  __syncthreads();
  const float* res;
  if (epi == EPI_RAW) {
    fsweep(ops.chif, true, N, ns, X, Y, nsl, NV, 0, N, N, N);
    fsweep(ops.chif, true, N, ns, Y, X, nsl, NV, 1, ns, N, N);
    fsweep(ops.chif, true, N, ns, X, Y, nsl, NV, 2, ns, ns, N);
    res = Y;
  } else {
    fsweep(ops.Af, false, N, N, X, Y, nsl, NV, 0, N, N, N);
    fsweep(ops.Af, false, N, N, Y, X, nsl, NV, 1, N, N, N);
    fsweep(ops.Af, false, N, N, X, Y, nsl, NV, 2, N, N, N);
    for (int t = threadIdx.x; t < nsl * NV; t += blockDim.x) Y[t] *= invwj32[(size_t)(e0 + t / (5 * NV)) * NV + t % NV];
    __syncthreads();
    fsweep(ops.Ptf, false, N, ns, Y, X, nsl, NV, 0, N, N, N);
    fsweep(ops.Ptf, false, N, ns, X, Y, nsl, NV, 1, ns, N, N);
    fsweep(ops.Ptf, false, N, ns, Y, X, nsl, NV, 2, ns, ns, N);
    res = X;
  }
  const size_t off = (size_t)e0 * 5 * nsv;
  const double bdt = rk.b * rk.dt, adt = rk.a_next * rk.dt;
  for (int t = threadIdx.x; t < nsl * nsv; t += blockDim.x) {
    const double r = f2d_i(res[(size_t)(t / nsv) * NV + t % nsv]);
    if (epi == EPI_RAW) {
      out[off + t] = r;
    } else if (epi == EPI_DUDT) {
      out[off + t] = neg_i(r);
    } else {
      const double k = neg_i(r);
      if (rk.last) {
        rk.unext[off + t] = fma(bdt, k, rk.acc[off + t]);
      } else {
        const double u0 = rk.u0[off + t];
        rk.acc[off + t] = fma(bdt, k, rk.first ? u0 : rk.acc[off + t]);
        rk.unext[off + t] = fma(adt, k, u0);
      }
    }
  }
}

// shared-memory layout per element (SoA over the NV nodes)
//   floats : r, 2 beta as float-float                          4 NV
//   doubles: R (combined), epilogue                            5 NV
//   floats : u/2 hi(3) lo(3), |u|^2/4, metric hi(9) lo(9)     25 NV
//   floats : line sums R_rho hi, lo, R_m(3), R_E', one slab
//            per direction                                     18 NV
// preceded by the elements' reference states (BRef, 64 bytes each).
// The float-float metric rows (w_perp / 2 C), face rows (w_perp C_f) and
// 1/(w J) come from bulk_tables_kernel, once per geometry.
template <int N, bool FF>
__global__ void __launch_bounds__(bulk_threads(N, FF), bulk_ctas(N, FF))
    volume_bulk_kernel(const double* __restrict__ nrec, const float* __restrict__ metric32,
                       const double* __restrict__ nf_s, const float* __restrict__ nf32,
                       const double* __restrict__ face, const double* __restrict__ fstar,
                       const float* __restrict__ invwj32, const double* __restrict__ src, OpsGL ops, int nx,
                       int ny, int nz, int e_beg, int ne, int epi, RkArgs rk, double* out, int* flag) {
  // elements e_beg .. ne-1 (the whole mesh's neighbours stay reachable)
  constexpr int NV = N * N * N, NFP = N * N, NL = 3 * NFP;
  extern __shared__ double sm[];
  const int epb = blockDim.x / NL;
  const int e0 = e_beg + blockIdx.x * epb;
  BRef* Refs = (BRef*)sm;                          // [epb]
  float* Pdf = (float*)(Refs + epb);               // [epb][4][NV] rho, 2 beta as float-float
  double* Rd = (double*)(Pdf + (size_t)epb * 4 * NV);  // [epb][5][NV]
  float* Pf = (float*)(Rd + (size_t)epb * 5 * NV); // [epb][25][NV]
  float* Ra = Pf + (size_t)epb * 25 * NV;          // [epb][3][6][NV]
  float* Xf = Pf;                                  // epilogue (aliases Pf)

  for (int t = threadIdx.x; t < epb * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV, e = e0 + le;
    if (e >= ne) continue;
    ff u0, u1, u2;
    float qq;
    if constexpr (FF) {
      // the float-float fields of the node record (face_state_bulk_kernel)
      const float2* rec = reinterpret_cast<const float2*>(nrec + (size_t)e * NSFR_NFIELD * NV) + node;
      const float2 fr2 = rec[P_RHO * NV], fb2 = rec[P_B2 * NV], f0 = rec[P_UH * NV], f1 = rec[(P_UH + 1) * NV],
                   f2 = rec[(P_UH + 2) * NV], fq = rec[P_QQ * NV];
      u0 = ff{f0.x, f0.y};
      u1 = ff{f1.x, f1.y};
      u2 = ff{f2.x, f2.y};
      qq = fq.x;
      if (node == 0) Refs[le] = make_ref(ff{fr2.x, fr2.y}, ff{fb2.x, fb2.y}, u0, u1, u2, ops);
      float* pd = Pdf + (size_t)le * 4 * NV + node;
      pd[0] = fr2.x;
      pd[NV] = fr2.y;
      pd[2 * NV] = fb2.x;
      pd[3 * NV] = fb2.y;
    } else {
      // the FP64 node record (face_state_kernel)
      const Rec a = load_rec6(nrec + (size_t)e * NSFR_NFIELD * NV + node, NV);
      if (node == 0) Refs[le] = make_ref(a, ops);
      const ff r = ff_split_i(a.r), b2 = ff_split_i(a.b2);
      float* pd = Pdf + (size_t)le * 4 * NV + node;
      pd[0] = r.hi;
      pd[NV] = r.lo;
      pd[2 * NV] = b2.hi;
      pd[3 * NV] = b2.lo;
      u0 = ff_split_i(a.u0);
      u1 = ff_split_i(a.u1);
      u2 = ff_split_i(a.u2);
      qq = d2f_i(a.qq);
    }
    float* pf = Pf + (size_t)le * 25 * NV + node;
    pf[0] = u0.hi;
    pf[NV] = u1.hi;
    pf[2 * NV] = u2.hi;
    pf[3 * NV] = u0.lo;
    pf[4 * NV] = u1.lo;
    pf[5 * NV] = u2.lo;
    pf[6 * NV] = qq;
    const float* m32 = metric32 + (size_t)e * 18 * NV + node;
#pragma unroll
    for (int r = 0; r < 18; ++r) pf[(7 + r) * NV] = m32[r * NV];
  }
  __syncthreads();

  for (int t = threadIdx.x; t < epb * 18 * NV; t += blockDim.x) Ra[t] = 0.0f;
  __syncthreads();

  // line phase: one thread per line, the line's sums in the direction's slab
  // of Ra (node a's in registers while a is the outer pair index), added in
  // the order of a plain per-line accumulation
  const int le = threadIdx.x / NL, l = threadIdx.x % NL, e = e0 + le;
  const int d = l / NFP, line = l % NFP, l0 = line % N, l1 = line / N;
  int base, stride;
  line_geometry<N>(d, l0, l1, base, stride);
  if (le < epb && e < ne) {
    const float* pdf = Pdf + (size_t)le * 4 * NV + base;
    const float* pf = Pf + (size_t)le * 25 * NV + base;
    const double* Le = nrec + ((size_t)e * NSFR_NFIELD + P_LRHO) * NV + base;  // ln rho, ln beta (read only off the series path)
    float* Rl = Ra + ((size_t)le * 18 + 6 * d) * NV + base;
    const BRef ref = Refs[le];
    auto node_at = [&](int a) {
      BNode<FF> b;
      b.r = ff{pdf[a * stride], pdf[NV + a * stride]};
      b.b2 = ff{pdf[2 * NV + a * stride], pdf[3 * NV + a * stride]};
      b.u0 = ff{pf[a * stride], pf[3 * NV + a * stride]};
      b.u1 = ff{pf[NV + a * stride], pf[4 * NV + a * stride]};
      b.u2 = ff{pf[2 * NV + a * stride], pf[5 * NV + a * stride]};
      b.qq = pf[6 * NV + a * stride];
      return b;
    };
    auto metric_at = [&](int a, int c) {
      return ff{pf[(7 + 3 * d + c) * NV + a * stride], pf[(16 + 3 * d + c) * NV + a * stride]};
    };
    // accumulate a pair's (or hybrid) flux, scaled by c, into node a's sums
    auto add_to = [&](int a, ff c, const ff& Fr, const float Fm[3], float FE) {
      float* r = Rl + a * stride;
      const ff s_ = ff_fma(c, Fr, ff{r[0], r[NV]});
      r[0] = s_.hi;
      r[NV] = s_.lo;
#pragma unroll
      for (int k = 0; k < 3; ++k) r[(2 + k) * NV] = fmaf(c.hi, Fm[k], r[(2 + k) * NV]);
      r[5 * NV] = fmaf(c.hi, FE, r[5 * NV]);
    };
#pragma unroll 1
    for (int a = 0; a < N - 1; ++a) {
      const BNode<FF> A = node_at(a);
      const ff na0 = metric_at(a, 0), na1 = metric_at(a, 1), na2 = metric_at(a, 2);
      float* ra = Rl + a * stride;
      ff Rr = ff{ra[0], ra[NV]};
      float Rm0 = ra[2 * NV], Rm1 = ra[3 * NV], Rm2 = ra[4 * NV], Re = ra[5 * NV];
#pragma unroll 1
      for (int b = a + 1; b < N; ++b) {
        const BNode<FF> B = node_at(b);
        ff Fr;
        float Fm[3], FE;
        bulk_flux(A, B, ff_add_nn(na0, metric_at(b, 0)), ff_add_nn(na1, metric_at(b, 1)),
                  ff_add_nn(na2, metric_at(b, 2)),
                  ref, ops, PtrLogs{Le + a * stride, NV}, PtrLogs{Le + b * stride, NV}, Fr, Fm, FE);
        const ff c{ops.S1f[a * N + b], ops.S1lo[a * N + b]};
        Rr = ff_fma(c, Fr, Rr);
        Rm0 = fmaf(c.hi, Fm[0], Rm0);
        Rm1 = fmaf(c.hi, Fm[1], Rm1);
        Rm2 = fmaf(c.hi, Fm[2], Rm2);
        Re = fmaf(c.hi, FE, Re);
        add_to(b, ff_neg(c), Fr, Fm, FE);
      }
      ra[0] = Rr.hi;
      ra[NV] = Rr.lo;
      ra[2 * NV] = Rm0;
      ra[3 * NV] = Rm1;
      ra[4 * NV] = Rm2;
      ra[5 * NV] = Re;
    }
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      const int enb = nbr_index(e, d, s, nx, ny, nz);
      const double* fo = face + (((size_t)e * 6 + 2 * d + s) * NSFR_NFIELD) * NFP + line;
      const size_t fe = (size_t)(s ? e : enb) * 3 + d;  // the element whose + face this is
      const double* nf = nf_s + fe * 3 * NFP + line;  // w_perp C_f
      const double* fsp = fstar + fe * 5 * NFP + line;
      const float* g32 = nf32 + fe * 6 * NFP + line;  // the same as float-float: hi(3), lo(3)
      // the FP64 face flux in the element's deviation form:
      //   F_m' = F_m - u_ref F_rho - p_ref n,  F_E' = F_E - E_ref F_rho
      // (formed where it is used, so that it is not live across the hybrid loop)
      auto face_flux_dev = [&](ff& sr_, float sm_[3], float& se_) {
        const double F0 = fsp[0];
        sr_ = ff_from_double(F0);
        sm_[0] = d2f_i(fma(-ref.p, nf[0], fma(-ff_to_double(ref.u0), F0, fsp[NFP])));
        sm_[1] = d2f_i(fma(-ref.p, nf[NFP], fma(-ff_to_double(ref.u1), F0, fsp[2 * NFP])));
        sm_[2] = d2f_i(fma(-ref.p, nf[2 * NFP], fma(-ff_to_double(ref.u2), F0, fsp[3 * NFP])));
        se_ = d2f_i(fma(-(ref.H + f2d_i(ref.kin)), F0, fsp[4 * NFP]));
      };
      ff sr_;
      float sm_[3], se_;
      if (ops.lgl) {
        // LGL: t_s is the unit vector of the end node, so the hybrid terms reduce
        // to f* at that node
        face_flux_dev(sr_, sm_, se_);
        add_to(s ? N - 1 : 0, ff{s ? 1.0f : -1.0f, 0.0f}, sr_, sm_, se_);
        continue;
      }
      const BNode<FF> Fo = bnode_from_rec<FF>(load_rec6(fo, NFP));
      const ff h0{0.5f * g32[0], 0.5f * g32[3 * NFP]}, h1{0.5f * g32[NFP], 0.5f * g32[4 * NFP]},
          h2{0.5f * g32[2 * NFP], 0.5f * g32[5 * NFP]};
      const float* tf = s ? ops.tpf : ops.tmf;
      const float* tl = s ? ops.tplo : ops.tmlo;
      const float sg = s ? 1.0f : -1.0f;
      ff tr = ff{0.0f, 0.0f};
      float tm[3] = {0.0f, 0.0f, 0.0f}, te = 0.0f;
#pragma unroll 1
      for (int a = 0; a < N; ++a) {
        const BNode<FF> A = node_at(a);
        ff Fr;
        float Fm[3], FE;
        bulk_flux(A, Fo, ff_add_nn(metric_at(a, 0), h0), ff_add_nn(metric_at(a, 1), h1),
                  ff_add_nn(metric_at(a, 2), h2),
                  ref, ops, PtrLogs{Le + a * stride, NV}, PtrLogs{fo + P_LRHO * NFP, NFP}, Fr, Fm, FE);
        const ff ta{tf[a], tl[a]};
        tr = ff_fma(ta, Fr, tr);
#pragma unroll
        for (int k = 0; k < 3; ++k) tm[k] = fmaf(ta.hi, Fm[k], tm[k]);
        te = fmaf(ta.hi, FE, te);
        add_to(a, ff{sg * tf[a], sg * tl[a]}, Fr, Fm, FE);
      }
      face_flux_dev(sr_, sm_, se_);
      const ff dr_ = ff_add(sr_, ff_neg(tr));
      float dm[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) dm[k] = sm_[k] - tm[k];
      const float de = se_ - te;
#pragma unroll 1
      for (int a = 0; a < N; ++a) add_to(a, ff{sg * tf[a], sg * tl[a]}, dr_, dm, de);
    }
  }
  __syncthreads();
  // the directions meet in a fixed order (d = 0, 1, 2), into slab 0
  for (int t = threadIdx.x; t < min(epb, ne - e0) * NV; t += blockDim.x) {
    const int lq = t / NV, node = t % NV;
    float* ra = Ra + (size_t)lq * 18 * NV + node;
    ff r = ff_add(ff_add(ff{ra[0], ra[NV]}, ff{ra[6 * NV], ra[7 * NV]}), ff{ra[12 * NV], ra[13 * NV]});
    ra[0] = r.hi;
    ra[NV] = r.lo;
#pragma unroll
    for (int k = 2; k < 6; ++k) ra[k * NV] = (ra[k * NV] + ra[(6 + k) * NV]) + ra[(12 + k) * NV];
  }
  __syncthreads();
  const int nel = min(epb, ne - e0);
  // R in FP64: R_m = R(F_m') + u_ref R_rho, R_E = R(F_E') + E_ref R_rho
  // (the momentum's p_ref part needs no term back: its residual vanishes)
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int lq = t / NV, node = t % NV;
    const float* ra = Ra + (size_t)lq * 18 * NV + node;
    const BRef rf = Refs[lq];
    const double Rrho = f2d_i(ra[0]) + f2d_i(ra[NV]);
    double* rd = Rd + (size_t)lq * 5 * NV + node;
    rd[0] = Rrho;
    rd[NV] = fma(ff_to_double(rf.u0), Rrho, f2d_i(ra[2 * NV]));
    rd[2 * NV] = fma(ff_to_double(rf.u1), Rrho, f2d_i(ra[3 * NV]));
    rd[3 * NV] = fma(ff_to_double(rf.u2), Rrho, f2d_i(ra[4 * NV]));
    rd[4 * NV] = fma(rf.H + f2d_i(rf.kin), Rrho, f2d_i(ra[5 * NV]));
    if (src) {  // a volume source: R - W J q
      const double* q = src + ((size_t)(e0 + lq) * 5) * NV + node;
#pragma unroll
      for (int k = 0; k < 5; ++k) rd[k * NV] -= q[k * NV];
    }
  }
  __syncthreads();
  if (ops.uncol) {  // solution on the Lobatto nodes: back from the GL points (Pf is free again)
    uncol_epilogue_f<N>(Rd, Xf, Xf + (size_t)epb * 5 * NV, nel, e0, ops, invwj32, epi, rk, out);
    return;
  }
  const int total = nel * 5 * NV;
  const size_t off = (size_t)e0 * 5 * NV;
  if (epi == EPI_RAW) {
    for (int t = threadIdx.x; t < total; t += blockDim.x) out[off + t] = Rd[t];
    return;
  }
  // weight-adjusted inverse in FP32
  for (int t = threadIdx.x; t < total; t += blockDim.x) Xf[t] = d2f_i(Rd[t]);
  __syncthreads();
  if (ops.has_K) {
    for (int dd = 0; dd < 3; ++dd) {
      rank_one_sweep_f<N>(Xf, nel, dd, true, ops);
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int lq = t / (5 * NV), node = t % NV;
    Xf[t] *= invwj32[(size_t)(e0 + lq) * NV + node];
  }
  __syncthreads();
  if (ops.has_K) {
    for (int dd = 0; dd < 3; ++dd) {
      rank_one_sweep_f<N>(Xf, nel, dd, false, ops);
      __syncthreads();
    }
  }
  if (epi == EPI_DUDT) {
    for (int t = threadIdx.x; t < total; t += blockDim.x) out[off + t] = neg_i(f2d_i(Xf[t]));
  } else {
    const double bdt = rk.b * rk.dt, adt = rk.a_next * rk.dt;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const double k = neg_i(f2d_i(Xf[t]));
      if (rk.last) {
        rk.unext[off + t] = fma(bdt, k, rk.acc[off + t]);
      } else {
        const double u0 = rk.u0[off + t];
        rk.acc[off + t] = fma(bdt, k, rk.first ? u0 : rk.acc[off + t]);
        rk.unext[off + t] = fma(adt, k, u0);
      }
    }
  }
}

template <int N, bool FF>
cudaError_t launch_bulk_n(nsfr_ctx* ctx, const double* u, double* out, int epi, const RkArgs* rk, cudaStream_t s) {
  constexpr int NV = N * N * N;
  constexpr int epb = bulk_epb(N, FF);
  const int eb = ctx->vol_b, ee = ctx->vol_e < 0 ? ctx->ne : ctx->vol_e;
  const int grid = (ee - eb + epb - 1) / epb;
  if (grid <= 0) return cudaSuccess;
  const size_t smem = (size_t)epb * (sizeof(BRef) + NV * (7 * sizeof(double) + 43 * sizeof(float)));
  cudaError_t err =
      cudaFuncSetAttribute(volume_bulk_kernel<N, FF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  RkArgs r = rk ? *rk : RkArgs{};
  nsfr_prof_begin(ctx, 2, s);
  volume_bulk_kernel<N, FF><<<grid, bulk_threads(N, FF), smem, s>>>(ctx->nrec, ctx->metric32, ctx->nf_s,
                                                           ctx->nfp_plus32, ctx->face, ctx->fstar, ctx->invwj32,
                                                           epi == EPI_RAW ? nullptr : ctx->src_on, ctx->ops, ctx->nx,
                                                           ctx->ny, ctx->nz, eb, ee, epi, r, out, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace

namespace {
// float-float tables of one geometry for the bulk kernel, from the scaled
// FP64 rows: metric rows w_perp/2 C -> metric32[e][18][nv] (9 hi rows, then 9
// lo rows), face rows w_perp C_f -> nf32[e][3][6][nfp] (hi xyz, lo xyz),
// 1/(w J) -> invwj32[e][nv]
__global__ void bulk_tables_kernel(const double* __restrict__ metric_s, const double* __restrict__ nf_s,
                                   const double* __restrict__ invwj, OpsGL ops, int ne, float* __restrict__ metric32,
                                   float* __restrict__ nf32, float* __restrict__ invwj32) {
  const int n = ops.n, nv = n * n * n, nfp = n * n;
  const size_t nm = (size_t)ne * 9 * nv, nf = (size_t)ne * 9 * nfp, nj = (size_t)ne * nv;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nm + nf + nj; t += (size_t)gridDim.x * blockDim.x) {
    if (t < nm) {
      const size_t e = t / (9 * nv);
      const int r = (int)(t / nv % 9), node = (int)(t % nv);
      const ff m = ff_from_double(metric_s[t]);
      metric32[(e * 18 + r) * nv + node] = m.hi;
      metric32[(e * 18 + 9 + r) * nv + node] = m.lo;
    } else if (t < nm + nf) {
      const size_t q = t - nm, ed = q / (3 * nfp);  // e * 3 + d
      const int c = (int)(q / nfp % 3), line = (int)(q % nfp);
      const ff g = ff_from_double(nf_s[q]);
      nf32[(ed * 6 + c) * nfp + line] = g.hi;
      nf32[(ed * 6 + 3 + c) * nfp + line] = g.lo;
    } else {
      const size_t q = t - nm - nf;
      invwj32[q] = d2f_i(invwj[q]);
    }
  }
}
}  // namespace

cudaError_t nsfr_launch_bulk_tables(nsfr_ctx* ctx, cudaStream_t s) {
  bulk_tables_kernel<<<152 * 8, 256, 0, s>>>(ctx->metric_s, ctx->nf_s, ctx->invwj, ctx->ops, ctx->ne,
                                             ctx->metric32, ctx->nfp_plus32, ctx->invwj32);
  ctx->launches++;
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_face_bulk_n(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  constexpr int NV = N * N * N, NFP = N * N;
  constexpr int epb = epb_for(N);
  const int eb = ctx->fs_b, ee = ctx->fs_e < 0 ? ctx->ne : ctx->fs_e;  // as launch_face_n
  const int grid = (ee - eb + epb - 1) / epb;
  if (grid <= 0) return cudaSuccess;
  const size_t smem = (size_t)epb * 5 * NV * sizeof(ff) + NSFR_MATH_TABLE_FLOATS * sizeof(float);
  cudaError_t err =
      cudaFuncSetAttribute(face_state_bulk_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  nsfr_prof_begin(ctx, 1, s);
  face_state_bulk_kernel<N><<<grid, threads_for(N), smem, s>>>(
      u + (size_t)eb * 5 * NV, ctx->ops, ctx->face + (size_t)eb * 6 * NSFR_NFIELD * NFP,
      ctx->nrec + (size_t)eb * NSFR_NFIELD * NV, ee - eb, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t nsfr_launch_face_states_bulk(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  switch (ctx->n) {
    case 2: return launch_face_bulk_n<2>(ctx, u, s);
    case 3: return launch_face_bulk_n<3>(ctx, u, s);
    case 4: return launch_face_bulk_n<4>(ctx, u, s);
    case 5: return launch_face_bulk_n<5>(ctx, u, s);
    case 6: return launch_face_bulk_n<6>(ctx, u, s);
    case 7: return launch_face_bulk_n<7>(ctx, u, s);
    case 8: return launch_face_bulk_n<8>(ctx, u, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t nsfr_launch_volume_bulk(nsfr_ctx* ctx, const double* u, double* out, int epi, const RkArgs* rk,
                                    cudaStream_t s) {
  const bool ff = ctx->precision == NSFR_FP32_BULK_FF;
  switch (ctx->n) {
    case 2: return ff ? launch_bulk_n<2, true>(ctx, u, out, epi, rk, s) : launch_bulk_n<2, false>(ctx, u, out, epi, rk, s);
    case 3: return ff ? launch_bulk_n<3, true>(ctx, u, out, epi, rk, s) : launch_bulk_n<3, false>(ctx, u, out, epi, rk, s);
    case 4: return ff ? launch_bulk_n<4, true>(ctx, u, out, epi, rk, s) : launch_bulk_n<4, false>(ctx, u, out, epi, rk, s);
    case 5: return ff ? launch_bulk_n<5, true>(ctx, u, out, epi, rk, s) : launch_bulk_n<5, false>(ctx, u, out, epi, rk, s);
    case 6: return ff ? launch_bulk_n<6, true>(ctx, u, out, epi, rk, s) : launch_bulk_n<6, false>(ctx, u, out, epi, rk, s);
    case 7: return ff ? launch_bulk_n<7, true>(ctx, u, out, epi, rk, s) : launch_bulk_n<7, false>(ctx, u, out, epi, rk, s);
    case 8: return ff ? launch_bulk_n<8, true>(ctx, u, out, epi, rk, s) : launch_bulk_n<8, false>(ctx, u, out, epi, rk, s);
  }
  return cudaErrorInvalidValue;
}
