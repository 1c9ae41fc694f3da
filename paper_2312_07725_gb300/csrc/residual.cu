// NSFR-EC residual kernels (FP64 path).
//
// K1  face_state_kernel: entropy projection to the faces (Sec. "Nonlinearly
//     Stable Flux Reconstruction", entropy projected variables).  With the
//     collocated GL basis v^ = v(u) nodal, and each face state is
//     u~_f = u(t_s . v) along the line that ends on the face node.  The
//     kernel stores the primitive record of u~_f (rho, u, beta, ln rho,
//     ln beta, |u|^2), which is all the face fluxes need.
// K1b face_flux_kernel: the numerical flux f*(u~_L, u~_R; w_perp C_f) of every
//     face node, once per face (C_f the shared face row), for both elements
//     that share the face.
// K2  volume_kernel: Eq. NSFR with the sum-factorised Hadamard products
//     (Sec. "Scalable Evaluations"), one thread per line of an element:
//       volume:  R_a += sum_{b} w_perp S1[a,b] f_s(u_a, u_b) . (C_a + C_b)/2
//                (each unordered pair evaluated once: S1 is skew),
//       hybrid:  R_a += s w_perp t_s[a] (phi_a + f* - sum_b t_s[b] phi_b),
//                phi_a = f_s(u_a, u~_f) . (C_a + C_f)/2,
//       surface: f* read from K1b;
//     the three directions' line sums meet in shared memory, then the
//     epilogue applies the weight-adjusted inverse (Eq. weight-adj ESFR mass,
//     Pi~^T, 1/(w J), Pi~, each a 1D contraction per direction) and either
//     stores du/dt or performs the RK stage update in place.
#include "async_copy.cuh"
#include "kernel_common.cuh"
#include "mathfn.cuh"
#include "physics.cuh"

// stage the volume kernel's node records with bulk asynchronous copies (1) or a
// plain load loop (0)
#ifndef NSFR_VOL_STAGE_TMA
#define NSFR_VOL_STAGE_TMA 1
#endif

namespace {
using namespace nsfr_k;

template <int N>
__global__ void __launch_bounds__(threads_for(N)) face_state_kernel(const double* __restrict__ u, OpsGL ops,
                                                                    double* __restrict__ face,
                                                                    double* __restrict__ nrec, int ne, int* flag) {
  constexpr int NV = N * N * N, NFP = N * N, NL = 3 * NFP;
  extern __shared__ double sm[];
  const int epb = blockDim.x / NL;
  const int e0 = blockIdx.x * epb;
  const double g = ops.gamma, gm1 = g - 1.0, igm1 = ops.inv_gm1;
  const double ln2 = 0.69314718055994530942;
  // constants of v_1 and of ln rho~ (below): (gamma + ln 2)/(gamma-1), -gamma/(gamma-1), -1/(gamma-1)
  const double cv0 = (g + ln2) * igm1, ngig = -g * igm1, nigm1 = -igm1;
  const MathTables T = nsfr_stage_tables(sm + (size_t)epb * 5 * NV);
  __syncthreads();
  // v(u) at every node of the block's elements; the node records (rho, 2 beta,
  // u/2, |u|^2/4, ln rho, ln beta) are kept for the volume kernels
  for (int t = threadIdx.x; t < epb * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV, e = e0 + le;
    if (e >= ne) continue;
    const double* ue = u + (size_t)e * 5 * NV + node;
    const double r = ue[0], m0 = ue[NV], m1 = ue[2 * NV], m2 = ue[3 * NV], E = ue[4 * NV];
    // (negations by neg_i and the sign tests by pos_i run on the integer pipe)
    const double ir = rcp_ff(r);
    const double u0 = m0 * ir, u1 = m1 * ir, u2 = m2 * ir;
    const double q2 = fma(u0, u0, fma(u1, u1, u2 * u2));
    const double p = gm1 * fma(neg_i(mul_pow2<-1>(r)), q2, E);
    if (!pos_i(r) || !pos_i(p)) atomicOr(flag, 1);
    const double b2 = r * rcp_ff(p);  // 2 beta = rho / p
    const double lr = nsfr_log(r, T), l2p = nsfr_log(mul_pow2<1>(p), T);
    // v_1 = (gamma - s)/(gamma-1) - beta |u|^2 with s = ln p - gamma ln rho = ln 2p - ln 2 - gamma ln rho
    double* v = sm + (size_t)le * 5 * NV + node;
    v[0] = fma(neg_i(mul_pow2<-1>(b2)), q2, fma(igm1, fma(g, lr, neg_i(l2p)), cv0));
    v[NV] = b2 * u0;
    v[2 * NV] = b2 * u1;
    v[3 * NV] = b2 * u2;
    v[4 * NV] = neg_i(b2);
    Rec a;
    a.r = r;
    a.b2 = b2;
    a.u0 = mul_pow2<-1>(u0);
    a.u1 = mul_pow2<-1>(u1);
    a.u2 = mul_pow2<-1>(u2);
    a.qq = mul_pow2<-2>(q2);
    a.lr = lr;
    a.lb = lr - l2p;  // ln beta = ln rho - ln 2p
    store_rec(nrec + (size_t)e * NSFR_NFIELD * NV + node, NV, a);
  }
  __syncthreads();
  const int le = threadIdx.x / NL, l = threadIdx.x % NL, e = e0 + le;
  if (le >= epb || e >= ne) return;
  const int d = l / NFP, line = l % NFP;
  int base, stride;
  line_geometry<N>(d, line % N, line / N, base, stride);
  const double* v = sm + (size_t)le * 5 * NV + base;
  double vm[5], vp[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    double am = 0.0, ap = 0.0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const double x = v[k * NV + a * stride];
      am = fma(ops.tm[a], x, am);
      ap = fma(ops.tp[a], x, ap);
    }
    vm[k] = am;
    vp[k] = ap;
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const double* w = s ? vp : vm;
    const double b2 = neg_i(w[4]);            // 2 beta = -v_5
    if (!pos_i(b2)) atomicOr(flag, 1);
    const double iv = rcp_ff(b2);
    const double u0 = w[1] * iv, u1 = w[2] * iv, u2 = w[3] * iv;  // u = -v_{2..4} / v_5
    const double q2 = fma(u0, u0, fma(u1, u1, u2 * u2));
    const double L5 = nsfr_log(b2, T);        // ln(2 beta)
    // s = gamma - (gamma-1)(v_1 + beta |u|^2) = (1-gamma) ln rho - ln(2 beta), so
    // ln rho = (v_1 + beta |u|^2) - (gamma + ln(2 beta))/(gamma-1)
    const double lr = fma(nigm1, L5, fma(mul_pow2<-1>(b2), q2, w[0] + ngig));
    Rec P;
    P.r = nsfr_exp(lr, T);
    P.b2 = b2;
    P.u0 = mul_pow2<-1>(u0);
    P.u1 = mul_pow2<-1>(u1);
    P.u2 = mul_pow2<-1>(u2);
    P.qq = mul_pow2<-2>(q2);
    P.lr = lr;
    P.lb = L5 - ln2;
    store_rec(face + (((size_t)e * 6 + 2 * d + s) * NSFR_NFIELD) * NFP + line, NFP, P);
  }
}

// f* of the + face of element e in direction d, for every face node, on the
// face row scaled by the node's w_perp (f* is linear in the face row, its Roe
// part positively homogeneous): fstar[e][d][5][n^2].  L is the element's own + face state, R
// the neighbour's - face state; both carry the same face-node index.
// Elements [e_beg, e_end).
template <int N>
__global__ void __launch_bounds__(256) face_flux_kernel(const double* __restrict__ face,
                                                        const double* __restrict__ nf_s, OpsGL ops, int nx, int ny,
                                                        int nz, int e_beg, int e_end, int face_kind, int vf,
                                                        double* __restrict__ fstar) {
  constexpr int NFP = N * N;
  const int t = e_beg * 3 * NFP + blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= e_end * 3 * NFP) return;
  const int node = t % NFP, ed = t / NFP, d = ed % 3, e = ed / 3;
  const int enb = nbr_index(e, d, 1, nx, ny, nz);
  const Rec L = load_rec(face + (((size_t)e * 6 + 2 * d + 1) * NSFR_NFIELD) * NFP + node, NFP);
  const Rec R = load_rec(face + (((size_t)enb * 6 + 2 * d) * NSFR_NFIELD) * NFP + node, NFP);
  const double* nf = nf_s + (size_t)ed * 3 * NFP + node;
  double F[5];
  face_flux(L, R, nf[0], nf[NFP], nf[2 * NFP], ops, face_kind, vf, F);
  double* o = fstar + (size_t)ed * 5 * NFP + node;
#pragma unroll
  for (int k = 0; k < 5; ++k) o[k * NFP] = F[k];
}

// The first RK4 stage's update from a stored k = du/dt, as the volume kernel's
// fused epilogue performs it: acc = u0 + b dt k and, in place, k <- u0 + a dt k.
__global__ void __launch_bounds__(256) rk_first_update_kernel(const double* __restrict__ u0, double* __restrict__ k,
                                                              double* __restrict__ acc, double bdt, double adt,
                                                              long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double kk = k[i], u = u0[i];
    acc[i] = fma(bdt, kk, u);
    k[i] = fma(adt, kk, u);
  }
}

// Pi~1^T (transpose) or Pi~1 along direction d for every line of X[nel][5][NV],
// in place: Pi~1 x = x - hv (g . x), Pi~1^T x = x - g (hv . x).
template <int N>
__device__ __forceinline__ void rank_one_sweep(double* X, int nel, int d, bool transpose, const OpsGL& ops) {
  constexpr int NV = N * N * N, NFP = N * N;
  const int st = (d == 0) ? 1 : (d == 1 ? N : N * N);
  const int nlines = nel * 5 * NFP;
  for (int t = threadIdx.x; t < nlines; t += blockDim.x) {
    const int line = t % NFP, lk = t / NFP;  // lk = element*5 + var
    int base, stride;
    line_geometry<N>(d, line % N, line / N, base, stride);
    double* x = X + (size_t)lk * NV + base;
    double dot = 0.0;
#pragma unroll
    for (int a = 0; a < N; ++a) dot = fma(transpose ? ops.hv[a] : ops.gv[a], x[a * st], dot);
#pragma unroll
    for (int a = 0; a < N; ++a) x[a * st] = fma(-(transpose ? ops.gv[a] : ops.hv[a]), dot, x[a * st]);
  }
}

// Two-point flux of the line phase, up to a factor it returns (the caller folds
// it into its accumulation weights): Chandrashekar's (VF =
// NSFR_FLUX_CHANDRASHEKAR) divided by rho_a + rho_b, or Ranocha's pressure
// terms with factor 1, its node pressures riding in the records' |u|^2/4 slot
// (that flux has no use for |u|^2).
template <int VF, class LA, class LB>
__device__ __forceinline__ double vol_flux(const Rec& A, const Rec& B, const RecF& Af, const RecF& Bf, double n0,
                                           double n1, double n2, const OpsGL& K, const LA& la, const LB& lb,
                                           double F[5]) {
  if (VF == NSFR_FLUX_RANOCHA) {
    ranocha_flux_ff(A, B, Af, Bf, A.qq, B.qq, n0, n1, n2, K, la, lb, F);
    return 1.0;
  }
  return ec_flux_over_sr_ff(A, B, Af, Bf, n0, n1, n2, K, la, lb, F);
}

// Rows of the pair table pm of one element and direction: the n(n-1)/2 volume
// pairs a < b in the line phase's loop order, then the hybrid rows s n + a of
// node a and side s.  pm is [ne][3 d][NPP][3 comps][n^2 lines].
__host__ __device__ constexpr int pair_rows(int n) { return n * (n - 1) / 2 + 2 * n; }

// The stage state itself is not read: its node records come from the
// face-state pass (nrec), so the epilogue may write the next stage state over
// the buffer the stage started from.
template <int N, int VF>
__global__ void __launch_bounds__(vol_threads(N), vol_ctas(N)) volume_kernel(const double* __restrict__ nrec,
                                                                const double* __restrict__ pm,
                                                                const double* __restrict__ face,
                                                                const double* __restrict__ fstar,
                                                                const double* __restrict__ invwj,
                                                                const double* __restrict__ src, OpsGL ops, int nx,
                                                                int ny, int nz, int e_beg, int ne, int epi,
                                                                RkArgs rk, double* out, int* flag) {
  // elements e_beg .. ne-1 (the whole mesh's neighbours stay reachable)
  constexpr int NV = N * N * N, NFP = N * N, NL = 3 * NFP, NPP = pair_rows(N);
  extern __shared__ __align__(128) double sm[];
  const int epb = blockDim.x / NL;
  const int e0 = e_beg + blockIdx.x * epb;
  const int nel = min(epb, ne - e0);
  double* P = sm;                          // [epb][6][NV] node records (the logs stay in nrec)
  double* Ra = P + (size_t)epb * 6 * NV;   // [epb][3][5][NV] line sums, one slab per direction
  double* Rs = P;                          // [epb][5][NV] residual (after the line phase)
  ff* Pf = (ff*)(Ra + (size_t)epb * 15 * NV);  // [epb][2][NV] rho, 2 beta as float-float

  // prologue: node records (fields rho .. |u|^2/4) of the block's elements
#if NSFR_VOL_STAGE_TMA
  // one bulk copy per element: the six fields are contiguous in nrec (48 NV
  // bytes at a 64 NV-byte element stride, both multiples of 16)
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    nsfr_async::mbar_init(&bar, 1);
    nsfr_async::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    constexpr uint32_t bytes = 6 * NV * sizeof(double);
    nsfr_async::mbar_arrive_expect_tx(&bar, bytes * nel);
    for (int le = 0; le < nel; ++le)
      nsfr_async::bulk_g2s(P + (size_t)le * 6 * NV, nrec + (size_t)(e0 + le) * NSFR_NFIELD * NV, bytes, &bar);
  }
  for (int t = threadIdx.x; t < epb * 15 * NV; t += blockDim.x) Ra[t] = 0.0;
  const bool arrived = nsfr_async::mbar_wait_bounded(&bar, 0);
  if (__syncthreads_or(!arrived)) {
    // the copies did not complete in time: report it, give them one more
    // bounded wait and leave without using the buffer
    if (threadIdx.x == 0) atomicOr(flag, NSFR_FLAG_WAIT_TIMEOUT);
    nsfr_async::mbar_wait_bounded(&bar, 0);
    return;
  }
#else
  for (int t = threadIdx.x; t < epb * 6 * NV; t += blockDim.x) {
    const int le = t / (6 * NV);
    if (le >= nel) continue;
    P[t] = nrec[((size_t)(e0 + le) * NSFR_NFIELD) * NV + t % (6 * NV)];
  }
  for (int t = threadIdx.x; t < epb * 15 * NV; t += blockDim.x) Ra[t] = 0.0;
#endif
  __syncthreads();
  // float-float rho and 2 beta of every node (the log means' series branch);
  // Ranocha's flux takes the pressure rho / (2 beta) in place of |u|^2/4
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV;
    double* pe = P + (size_t)le * 6 * NV + node;
    const double r = pe[P_RHO * NV], b2 = pe[P_B2 * NV];
    Pf[(size_t)le * 2 * NV + node] = ff_split_i(r);
    Pf[((size_t)le * 2 + 1) * NV + node] = ff_split_i(b2);
    if (VF == NSFR_FLUX_RANOCHA) pe[P_QQ * NV] = r * rcp_full(b2);
  }
  __syncthreads();

  // line phase: one thread per line; the line's sums live in the direction's
  // slab of Ra (only this thread touches them), node a's in registers while
  // a is the outer pair index -- the additions keep the order of a plain
  // per-line accumulation.  The averaged metric row of each pair comes from
  // the pair table, scaled by w_perp / 2 (constant along a line) and, for
  // Chandrashekar's flux, by the pair's weight S1_ab (t_s,a for a hybrid row):
  // the fluxes are linear in the metric row, so only that flux's own factor
  // s = rho_a + rho_b remains; Ranocha's takes S1_ab and t_s,a here.  The next
  // row is loaded while the current flux is evaluated.
  const int le = threadIdx.x / NL, l = threadIdx.x % NL, e = e0 + le;
  const int d = l / NFP, line = l % NFP, l0 = line % N, l1 = line / N;
  int base, stride;
  line_geometry<N>(d, l0, l1, base, stride);
  if (le < nel) {
    const double* Pe = P + (size_t)le * 6 * NV + base;
    const ff* Pfe = Pf + (size_t)le * 2 * NV + base;
    auto recf_at = [&](int a) { return RecF{Pfe[a * stride], Pfe[NV + a * stride]}; };
    const double* Le = nrec + ((size_t)e * NSFR_NFIELD + P_LRHO) * NV + base;  // ln rho, ln beta (read only off the series path)
    const double* Pm = pm + ((size_t)e * 3 + d) * NPP * 3 * NFP + line;      // row q, component c at Pm[(3 q + c) NFP]
    double* Rl = Ra + ((size_t)le * 15 + 5 * d) * NV + base;
    // volume-volume pairs along the line: each unordered pair once (S1 is skew)
    double m0 = Pm[0], m1 = Pm[NFP], m2 = Pm[2 * NFP];
    int q = 0;
#pragma unroll 1
    for (int a = 0; a < N - 1; ++a) {
      const Rec A = load_rec6(Pe + a * stride, NV);
      const RecF Af = recf_at(a);
      double Racc[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) Racc[k] = Rl[k * NV + a * stride];
#pragma unroll 1
      for (int b = a + 1; b < N; ++b) {
        const double n0 = m0, n1 = m1, n2 = m2;
        ++q;  // the rows run on into the hybrid rows, so row q exists
        m0 = Pm[3 * q * NFP];
        m1 = Pm[(3 * q + 1) * NFP];
        m2 = Pm[(3 * q + 2) * NFP];
        const Rec B = load_rec6(Pe + b * stride, NV);
        double F[5];
        const double fs = vol_flux<VF>(A, B, Af, recf_at(b), n0, n1, n2, ops, PtrLogs{Le + a * stride, NV},
                                       PtrLogs{Le + b * stride, NV}, F);
        const double c = VF == NSFR_FLUX_RANOCHA ? ops.S1[a * N + b] : fs;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          Racc[k] = fma(c, F[k], Racc[k]);
          Rl[k * NV + b * stride] = fma(-c, F[k], Rl[k * NV + b * stride]);
        }
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) Rl[k * NV + a * stride] = Racc[k];
    }
    // hybrid volume-face terms and face fluxes, both ends of the line
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      const int enb = nbr_index(e, d, s, nx, ny, nz);
      const double* fo = face + (((size_t)e * 6 + 2 * d + s) * NSFR_NFIELD) * NFP + line;
      const size_t fe = (size_t)(s ? e : enb) * 3 + d;  // the element whose + face this is
      const double* fsp = fstar + fe * 5 * NFP + line;
      const double sw = s ? 1.0 : -1.0;
      if (ops.lgl) {
        // LGL: t_s is the unit vector of the end node, so the hybrid terms
        // t_a (phi_a + f* - sum_b t_b phi_b) reduce to f* at that node
        double* Re = Rl + (s ? N - 1 : 0) * stride;
#pragma unroll
        for (int k = 0; k < 5; ++k) Re[k * NV] = fma(sw, fsp[k * NFP], Re[k * NV]);
        continue;
      }
      Rec Fo = load_rec6(fo, NFP);
      if (VF == NSFR_FLUX_RANOCHA) Fo.qq = pressure_of(Fo);
      const RecF Fof = recf_of(Fo);
      const double* t = s ? ops.tp : ops.tm;
      const double* Ph = Pm + 3 * (N * (N - 1) / 2 + s * N) * NFP;  // hybrid rows: (C_a + C_f) w_perp / 2
      double tphi[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll 1
      for (int a = 0; a < N; ++a) {
        const Rec A = load_rec6(Pe + a * stride, NV);
        double F[5];
        const double fs = vol_flux<VF>(A, Fo, recf_at(a), Fof, Ph[3 * a * NFP], Ph[(3 * a + 1) * NFP],
                                       Ph[(3 * a + 2) * NFP], ops,
                                       PtrLogs{Le + a * stride, NV}, PtrLogs{fo + P_LRHO * NFP, NFP}, F);
        const double ta = VF == NSFR_FLUX_RANOCHA ? t[a] : fs;
        const double swt = neg_if(ta, !s);  // s t_a, the sign flipped on the integer pipe
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          tphi[k] = fma(ta, F[k], tphi[k]);
          Rl[k * NV + a * stride] = fma(swt, F[k], Rl[k * NV + a * stride]);
        }
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) tphi[k] = fsp[k * NFP] - tphi[k];
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const double swt = neg_if(t[a], !s);
#pragma unroll
        for (int k = 0; k < 5; ++k) Rl[k * NV + a * stride] = fma(swt, tphi[k], Rl[k * NV + a * stride]);
      }
    }
  }
  __syncthreads();
  // the three directions meet in a fixed order (d = 0, 1, 2); the records are
  // no longer needed, so the sum goes over them
  for (int t = threadIdx.x; t < nel * 5 * NV; t += blockDim.x) {
    const int lq = t / (5 * NV), r = t % (5 * NV);
    const double* ra = Ra + (size_t)lq * 15 * NV + r;
    double rv = (ra[0] + ra[5 * NV]) + ra[10 * NV];
    if (src) rv -= src[(size_t)e0 * 5 * NV + t];  // a volume source: R - W J q
    Rs[t] = rv;
  }
  __syncthreads();

  const int total = nel * 5 * NV;
  if (ops.uncol) {  // solution on the Lobatto nodes: back from the GL points (Ra is free again)
    uncol_epilogue<N>(Rs, Ra, nel, e0, ops, invwj, epi, rk, out);
    return;
  }
  if (epi != EPI_RAW) {
    // weight-adjusted inverse: Pi~^T along xi, eta, zeta; 1/(w J); Pi~ along xi, eta, zeta
    if (ops.has_K) {
      for (int dd = 0; dd < 3; ++dd) {
        rank_one_sweep<N>(Rs, nel, dd, true, ops);
        __syncthreads();
      }
    }
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int lq = t / (5 * NV), node = t % NV;
      Rs[t] *= invwj[(size_t)(e0 + lq) * NV + node];
    }
    __syncthreads();
    if (ops.has_K) {
      for (int dd = 0; dd < 3; ++dd) {
        rank_one_sweep<N>(Rs, nel, dd, false, ops);
        __syncthreads();
      }
    }
  }
  // store
  const size_t off = (size_t)e0 * 5 * NV;
  if (epi == EPI_RAW) {
    for (int t = threadIdx.x; t < total; t += blockDim.x) out[off + t] = Rs[t];
  } else if (epi == EPI_DUDT) {
    for (int t = threadIdx.x; t < total; t += blockDim.x) out[off + t] = neg_i(Rs[t]);
  } else {
    const double bdt = rk.b * rk.dt, adt = rk.a_next * rk.dt;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const double k = neg_i(Rs[t]);  // (the negations on the integer pipe)
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

template <int N>
cudaError_t launch_face_n(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  constexpr int NV = N * N * N, NFP = N * N;
  constexpr int epb = epb_for(N);
  // elements [fs_b, fs_e): the kernel touches only its own elements' data, so a
  // range is the same launch on offset pointers
  const int eb = ctx->fs_b, ee = ctx->fs_e < 0 ? ctx->ne : ctx->fs_e;
  const int grid = (ee - eb + epb - 1) / epb;
  if (grid <= 0) return cudaSuccess;
  const size_t smem = ((size_t)epb * 5 * NV + NSFR_MATH_TABLE_DOUBLES) * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(face_state_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  nsfr_prof_begin(ctx, 1, s);
  face_state_kernel<N><<<grid, threads_for(N), smem, s>>>(
      u + (size_t)eb * 5 * NV, ctx->ops, ctx->face + (size_t)eb * 6 * NSFR_NFIELD * NFP,
      ctx->nrec + (size_t)eb * NSFR_NFIELD * NV, ee - eb, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_face_flux_n(nsfr_ctx* ctx, cudaStream_t s) {
  // elements [ff_b, ff_e): each writes only its own + faces' fluxes
  const int eb = ctx->ff_b, ee = ctx->ff_e < 0 ? ctx->ne : ctx->ff_e;
  if ((long long)ctx->ne * 3 * N * N > 0x7fffffffLL) return cudaErrorInvalidValue;
  const long long total = (long long)(ee - eb) * 3 * N * N;
  if (total <= 0) return cudaSuccess;
  const int grid = (int)((total + 255) / 256);
  nsfr_prof_begin(ctx, 8, s);
  face_flux_kernel<N><<<grid, 256, 0, s>>>(ctx->face, ctx->nf_s, ctx->ops, ctx->nx, ctx->ny, ctx->nz, eb, ee,
                                           ctx->face_flux, ctx->vol_flux, ctx->fstar);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_volume_n(nsfr_ctx* ctx, const double* u, double* out, int epi, const RkArgs* rk,
                            cudaStream_t s) {
  constexpr int NV = N * N * N;
  constexpr int epb = vol_epb(N);
  const int eb = ctx->vol_b, ee = ctx->vol_e < 0 ? ctx->ne : ctx->vol_e;
  const int grid = (ee - eb + epb - 1) / epb;
  if (grid <= 0) return cudaSuccess;
  const size_t smem = (size_t)epb * (6 + 15 + 2) * NV * sizeof(double);
  auto kern = ctx->vol_flux == NSFR_FLUX_RANOCHA ? volume_kernel<N, NSFR_FLUX_RANOCHA>
                                                 : volume_kernel<N, NSFR_FLUX_CHANDRASHEKAR>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  RkArgs r = rk ? *rk : RkArgs{};
  nsfr_prof_begin(ctx, 2, s);
  kern<<<grid, vol_threads(N), smem, s>>>(ctx->nrec, ctx->pair_rows, ctx->face, ctx->fstar, ctx->invwj,
                                          epi == EPI_RAW ? nullptr : ctx->src_on, ctx->ops, ctx->nx, ctx->ny,
                                          ctx->nz, eb, ee, epi, r, out, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace

namespace {
// geometry-only products of the residual kernels: metric rows scaled by
// w_perp / 2 (w_perp the two GL weights transverse to the row's direction)
// and face rows scaled by the face node's w_perp
__global__ void scaled_rows_kernel(const double* __restrict__ metric, const double* __restrict__ nf_plus, OpsGL ops,
                                   int ne, double* __restrict__ metric_s, double* __restrict__ nf_s) {
  const int n = ops.n, nv = n * n * n, nfp = n * n;
  const size_t nm = (size_t)ne * 9 * nv, nf = (size_t)ne * 9 * nfp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nm + nf; t += (size_t)gridDim.x * blockDim.x) {
    if (t < nm) {
      const int node = (int)(t % nv), dd = (int)(t / nv % 9) / 3;
      const int i = node % n, j = (node / n) % n, k = node / (n * n);
      const double wp = dd == 0 ? ops.w[j] * ops.w[k] : (dd == 1 ? ops.w[i] * ops.w[k] : ops.w[i] * ops.w[j]);
      metric_s[t] = 0.5 * wp * metric[t];
    } else {
      const size_t q = t - nm;
      const int line = (int)(q % nfp);
      const double wperp = ops.w[line % n] * ops.w[line / n];
      nf_s[q] = wperp * nf_plus[q];
    }
  }
}
}  // namespace

namespace {
// The pair table of the volume kernel, from the scaled rows (geometry only): for
// element e, direction d, line l, component c, row q < n(n-1)/2 holds
// w_ab (M_a + M_b) for the q-th pair a < b of the line (the volume kernel's
// loop order), row n(n-1)/2 + s n + a holds w_sa (M_a + (w_perp C_f)/2) for
// node a and the face of side s (C_f the face's shared row), M = w_perp C / 2
// the scaled metric row of the node.  With fold the weights are the pairs'
// weights in the Hadamard sum (Eq. NSFR), w_ab = S1_ab and w_sa = t_s,a (the
// extrapolation to that face): the two-point fluxes are linear in the metric
// row, so a pair's flux on this row is its flux on the averaged row times its
// weight, which then costs the line phase nothing per step.  Without fold
// they are 1, and the line phase applies them.
__global__ void pair_rows_kernel(const double* __restrict__ metric_s, const double* __restrict__ nf_s, OpsGL ops,
                                 bool fold, int n, int nx, int ny, int nz, double* __restrict__ pm) {
  const int nv = n * n * n, nfp = n * n, np = n * (n - 1) / 2, npp = pair_rows(n);
  const size_t ne = (size_t)nx * ny * nz, total = ne * 3 * npp * 3 * nfp;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int line = (int)(t % nfp), c = (int)(t / nfp % 3), q = (int)(t / ((size_t)3 * nfp) % npp);
    const int d = (int)(t / ((size_t)3 * nfp * npp) % 3);
    const size_t e = t / ((size_t)9 * nfp * npp);
    const int l0 = line % n, l1 = line / n;
    const int base = d == 0 ? n * (l0 + n * l1) : (d == 1 ? l0 + n * n * l1 : l0 + n * l1);
    const int stride = d == 0 ? 1 : (d == 1 ? n : n * n);
    const double* M = metric_s + (e * 9 + 3 * d + c) * nv + base;
    if (q < np) {
      int a = 0, r = q;
      while (r >= n - 1 - a) {
        r -= n - 1 - a;
        ++a;
      }
      const int b = a + 1 + r;
      const double m = M[a * stride] + M[b * stride];
      pm[t] = fold ? ops.S1[a * n + b] * m : m;
    } else {
      const int side = (q - np) / n, a = (q - np) % n;
      const int en = nsfr_k::nbr_index((int)e, d, side, nx, ny, nz);
      const size_t fe = (size_t)(side ? e : en) * 3 + d;
      const double m = M[a * stride] + 0.5 * nf_s[(fe * 3 + c) * nfp + line];
      pm[t] = fold ? (side ? ops.tp[a] : ops.tm[a]) * m : m;
    }
  }
}
}  // namespace

size_t nsfr_pair_rows_count(int n, int ne) { return (size_t)ne * 9 * pair_rows(n) * n * n; }

cudaError_t nsfr_launch_scaled_rows(nsfr_ctx* ctx, cudaStream_t s) {
  scaled_rows_kernel<<<152 * 8, 256, 0, s>>>(ctx->metric, ctx->nfp_plus, ctx->ops, ctx->ne, ctx->metric_s, ctx->nf_s);
  ctx->launches++;
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess || !ctx->pair_rows) return err;
  // the weights go into the rows for Chandrashekar's flux, whose line phase
  // would otherwise multiply them into its factor s per pair; Ranocha's flux
  // takes them as plain FMA operands in its accumulation (folded, that kernel
  // measured 2% slower)
  const bool fold = ctx->vol_flux != NSFR_FLUX_RANOCHA;  // the kernel choice of nsfr_launch_volume
  pair_rows_kernel<<<152 * 8, 256, 0, s>>>(ctx->metric_s, ctx->nf_s, ctx->ops, fold, ctx->n, ctx->nx, ctx->ny,
                                           ctx->nz, ctx->pair_rows);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t nsfr_launch_face_states(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  if (ctx->precision == NSFR_FP32_BULK_FF) return nsfr_launch_face_states_bulk(ctx, u, s);
  if (ctx->uncol && ctx->n != ctx->ns) return nsfr_launch_projection(ctx, u, s);
  if (ctx->uncol) {
    // square chi (as many GL points as solution nodes): chi Pi = I, so the projected
    // state at the GL points is chi u^ itself and the face states follow from
    // E_-+ = l(-+1)^T Pi applied to v(chi u^): the collocated pass on u_q = chi u^
    cudaError_t err = nsfr_launch_interp_square(ctx, u, s);
    if (err != cudaSuccess) return err;
    u = ctx->uq;
  }
  switch (ctx->n) {
    case 2: return launch_face_n<2>(ctx, u, s);
    case 3: return launch_face_n<3>(ctx, u, s);
    case 4: return launch_face_n<4>(ctx, u, s);
    case 5: return launch_face_n<5>(ctx, u, s);
    case 6: return launch_face_n<6>(ctx, u, s);
    case 7: return launch_face_n<7>(ctx, u, s);
    case 8: return launch_face_n<8>(ctx, u, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t nsfr_launch_face_flux(nsfr_ctx* ctx, cudaStream_t s) {
  switch (ctx->n) {
    case 2: return launch_face_flux_n<2>(ctx, s);
    case 3: return launch_face_flux_n<3>(ctx, s);
    case 4: return launch_face_flux_n<4>(ctx, s);
    case 5: return launch_face_flux_n<5>(ctx, s);
    case 6: return launch_face_flux_n<6>(ctx, s);
    case 7: return launch_face_flux_n<7>(ctx, s);
    case 8: return launch_face_flux_n<8>(ctx, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t nsfr_launch_rk_first_update(nsfr_ctx* ctx, const double* u0, double* k, double* acc, double bdt,
                                        double adt, cudaStream_t s) {
  const long long n = (long long)ctx->ne * 5 * ctx->nsv;
  if (n <= 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  const int grid = (int)(want < 152 * 16 ? want : 152 * 16);
  nsfr_prof_begin(ctx, 10, s);
  rk_first_update_kernel<<<grid, 256, 0, s>>>(u0, k, acc, bdt, adt, n);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t nsfr_launch_volume(nsfr_ctx* ctx, const double* u, double* out, int epi, const RkArgs* rk,
                               cudaStream_t s) {
  switch (ctx->n) {
    case 2: return launch_volume_n<2>(ctx, u, out, epi, rk, s);
    case 3: return launch_volume_n<3>(ctx, u, out, epi, rk, s);
    case 4: return launch_volume_n<4>(ctx, u, out, epi, rk, s);
    case 5: return launch_volume_n<5>(ctx, u, out, epi, rk, s);
    case 6: return launch_volume_n<6>(ctx, u, out, epi, rk, s);
    case 7: return launch_volume_n<7>(ctx, u, out, epi, rk, s);
    case 8: return launch_volume_n<8>(ctx, u, out, epi, rk, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// nsfr_residual_static: the same kernels on caller buffers, with the working
// memory in a fixed device array of this file instead of allocations.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[NSFR_STATIC_SCRATCH_BYTES];

namespace {
// p is device (or managed) memory of device dev; host memory, memory of another
// device and unknown pointers are refused before anything is launched
bool static_dev_ptr(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}
}  // namespace

extern "C" nsfr_status nsfr_residual_static(const double* u, const double* C, const double* J, const double* Cf,
                                            int nx, int ny, int nz, int p, double c, int face_flux, double gamma,
                                            double* dudt, void* stream) {
  if (!u || !C || !J || !Cf || !dudt || nx < 1 || ny < 1 || nz < 1 || p < 1 || p > 7 || !(gamma > 1.0) ||
      !(c >= 0.0) || face_flux < NSFR_FACE_EC || face_flux > NSFR_FACE_EC_ES)
    return NSFR_ERR_ARG;
  const size_t ne = (size_t)nx * ny * nz, n = p + 1, nv = n * n * n, nfp = n * n;
  const size_t face_bytes = ne * 6 * NSFR_NFIELD * nfp * sizeof(double);
  const size_t fstar_bytes = ne * 15 * nfp * sizeof(double);
  const size_t jac_bytes = ne * nv * sizeof(double);
  const size_t ms_bytes = ne * 9 * nv * sizeof(double), nfs_bytes = ne * 9 * nfp * sizeof(double);
  const size_t pm_bytes = nsfr_pair_rows_count((int)n, (int)ne) * sizeof(double);
  // error word (padded), face states, face fluxes, 1/(wJ), wJ, node records, scaled metric and face
  // rows, the volume kernel's pair table
  const size_t need = 256 + face_bytes + fstar_bytes + (2 + NSFR_NFIELD) * jac_bytes + ms_bytes + nfs_bytes + pm_bytes;
  if (need > NSFR_STATIC_SCRATCH_BYTES || ne > (size_t)0x7fffffff) return NSFR_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NSFR_ERR_CUDA;
  if (!static_dev_ptr(u, dev) || !static_dev_ptr(C, dev) || !static_dev_ptr(J, dev) || !static_dev_ptr(Cf, dev) ||
      !static_dev_ptr(dudt, dev))
    return NSFR_ERR_ARG;
  // the array's address in the current device's context, looked up on every
  // call (no allocation: the array is part of the loaded module)
  void* addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr) return NSFR_ERR_CUDA;
  unsigned char* base = (unsigned char*)addr;
  cudaStream_t s = (cudaStream_t)stream;
  nsfr_ctx ctx;  // a view of caller buffers and the fixed array; owns nothing
  ctx.nx = nx;
  ctx.ny = ny;
  ctx.nz = nz;
  ctx.ne = (int)ne;
  ctx.p = p;
  ctx.n = (int)n;
  ctx.pg = p;
  ctx.q = (int)n;
  ctx.nv = (int)nv;
  ctx.nfp = (int)nfp;
  ctx.ns = (int)n;
  ctx.nsv = (int)nv;
  ctx.uncol = 0;
  ctx.c = c;
  ctx.gamma = gamma;
  ctx.vol_flux = NSFR_FLUX_CHANDRASHEKAR;
  ctx.face_flux = face_flux;
  ctx.precision = NSFR_FP64;
  ctx.device = dev;
  ctx.nodes = NSFR_NODES_GL;
  nsfr_build_ops(p, p, c, gamma, NSFR_NODES_GL, &ctx.ops, &ctx.gops);
  ctx.flag = (int*)base;
  ctx.face = (double*)(base + 256);
  ctx.fstar = (double*)(base + 256 + face_bytes);
  ctx.invwj = (double*)(base + 256 + face_bytes + fstar_bytes);
  ctx.wj = (double*)(base + 256 + face_bytes + fstar_bytes + jac_bytes);
  ctx.nrec = (double*)(base + 256 + face_bytes + fstar_bytes + 2 * jac_bytes);
  ctx.metric_s = (double*)(base + 256 + face_bytes + fstar_bytes + (2 + NSFR_NFIELD) * jac_bytes);
  ctx.nf_s = (double*)(base + 256 + face_bytes + fstar_bytes + (2 + NSFR_NFIELD) * jac_bytes + ms_bytes);
  ctx.pair_rows = (double*)(base + 256 + face_bytes + fstar_bytes + (2 + NSFR_NFIELD) * jac_bytes + ms_bytes +
                            nfs_bytes);
  ctx.metric = const_cast<double*>(C);
  ctx.J = const_cast<double*>(J);
  ctx.nfp_plus = const_cast<double*>(Cf);
  if (cudaMemsetAsync(ctx.flag, 0, sizeof(int), s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (nsfr_launch_jacobian_derived(&ctx, s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (nsfr_launch_scaled_rows(&ctx, s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (nsfr_launch_face_states(&ctx, u, s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (nsfr_launch_face_flux(&ctx, s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (nsfr_launch_volume(&ctx, u, dudt, EPI_DUDT, nullptr, s) != cudaSuccess) return NSFR_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, ctx.flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (flag & NSFR_FLAG_WAIT_TIMEOUT) return NSFR_ERR_CUDA;
  if (flag & 2) return NSFR_ERR_MESH;
  if (flag & 1) return NSFR_ERR_NONPHYSICAL;
  return NSFR_OK;
}
