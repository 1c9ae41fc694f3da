// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "nsfr.h"

#define NSFR_MAXN 8   // n = p+1 <= 8
#define NSFR_NFIELD 8 // per-node primitive record, see Prim below
#define NSFR_COPY_CHUNKS 8  // z-chunks of a host-state RK step (copies overlapped with kernels)

// 1D operators of the collocated GL basis, passed to kernels by value (they
// land in the constant bank).  Row-major n x n matrices.
struct OpsGL {
  int n;
  int has_K;             // c != 0: the FR projection is not the identity
  double gamma;
  double w[NSFR_MAXN];   // GL weights
  double tm[NSFR_MAXN];  // l_j(-1)
  double tp[NSFR_MAXN];  // l_j(+1)
  double S1[NSFR_MAXN * NSFR_MAXN];   // W D - D^T W
  double Pi1[NSFR_MAXN * NSFR_MAXN];  // (W + K1)^{-1} W
  double Pinv1[NSFR_MAXN * NSFR_MAXN];  // Pi1^{-1} = I + W^{-1} K1
  float S1f[NSFR_MAXN * NSFR_MAXN];
  float tmf[NSFR_MAXN];
  float tpf[NSFR_MAXN];
  // low parts: S1 = S1f + S1lo, t = tf + tlo as float-float constants
  float S1lo[NSFR_MAXN * NSFR_MAXN];
  float tmlo[NSFR_MAXN];
  float tplo[NSFR_MAXN];
  // Pi~1 = I - hv g^T (rank one: K1 = 2c g g^T), hv = alpha W^{-1} g
  double gv[NSFR_MAXN];
  double hv[NSFR_MAXN];
  float gvf[NSFR_MAXN];
  float hvf[NSFR_MAXN];
  // log-mean series coefficients (Horner order c0..c3):
  //   Gh(u) = G(u)/2 with G = f/atanh(f), F4g(u) = 2/(gamma-1) atanh(f)/f, u = f^2
  double gh[4];
  double f4g[4];
  double fr2[4];  // 2 atanh(f)/f (the FP32-bulk form's H)
  double inv_gm1;
  // the same series as FP32 corrections for the FP32-bulk kernel: with
  // P(u) = c0 + u (c1 + u c2), G = 1 + u P_g, 2 atanh(f)/f = 2 + u P_a and
  // F4g = 2/(gamma-1) + u P_b; cab = 2 + 2/(gamma-1) as float-float
  float lmg[3];
  float lma[3];
  float lmb[3];
  float cab_hi, cab_lo;
  // the series branch in float-float: {c1 hi, c1 lo, c2 hi, c2 lo, c3} of
  // G(u) - 1 = u (c1 + u (c2 + u c3)), of F4g(u) - F4g(0) and of
  // 2 atanh(f)/f - 2 (the FP32-bulk form's H); cab = 2 + 2/(gamma-1) in FP64
  float lmg_ff[5];
  float lmb_ff[5];
  float lma_ff[5];
  float lmgd_ff[5];  // G'(u) = c1 + u (c2 + u c3) (the adjoint's log-mean derivatives)
  double cab;
  // Uncollocated scheme (solution on ns Lobatto nodes, the n points above are
  // GL quadrature points, n >= ns): chi (n x ns) the solution basis at the
  // points, Pi = (chi^T W chi)^{-1} chi^T W (ns x n), ls_m / ls_p the solution
  // basis at -1 / +1, A = (chi Pi~1)^T (n x n) and Pt = Pi~1 = (M1 + K1)^{-1}
  // chi^T W (ns x n) for the weight-adjusted inverse.  uncol = 0: collocated
  // (ns = n, and none of these is used).
  int uncol;
  int lgl;  // collocated LGL nodes: t_-, t_+ are the unit vectors of the end nodes
  int ns;
  double chi[NSFR_MAXN * NSFR_MAXN];
  double Pi[NSFR_MAXN * NSFR_MAXN];
  double ls_m[NSFR_MAXN];
  double ls_p[NSFR_MAXN];
  double A[NSFR_MAXN * NSFR_MAXN];
  double Pt[NSFR_MAXN * NSFR_MAXN];
  // the same three in FP32 (the FP32-bulk epilogue of the uncollocated scheme)
  float chif[NSFR_MAXN * NSFR_MAXN];
  float Af[NSFR_MAXN * NSFR_MAXN];
  float Ptf[NSFR_MAXN * NSFR_MAXN];
};

// Operators of the metric construction (Lobatto nodes of degree p).
struct OpsGeo {
  int n;   // Lobatto nodes per direction of the metric construction (p + 1)
  int q;   // control points per direction (p_geo + 1)
  int nq;  // volume quadrature points per direction (n unless uncollocated)
  double E[NSFR_MAXN * NSFR_MAXN];   // equispaced(q) -> LGL(n), n x q
  double Eg[NSFR_MAXN * NSFR_MAXN];  // equispaced(q) -> solution nodes (n), n x q
  double Dl[NSFR_MAXN * NSFR_MAXN];  // LGL differentiation, n x n
  double I[NSFR_MAXN * NSFR_MAXN];   // LGL -> volume quadrature points, nq x n
  double w[NSFR_MAXN];               // volume quadrature weights (nq)
};

// Host construction of the operators (ops1d.cpp).
void nsfr_build_ops(int p, int p_geo, double c, double gamma, int nodes, OpsGL* gl, OpsGeo* geo);
// uncollocated: solution on the p+1 Lobatto nodes, nq >= p+1 GL quadrature points
void nsfr_build_ops_uncol(int p, int p_geo, int nq, double c, double gamma, OpsGL* gl, OpsGeo* geo);
void nsfr_gauss_legendre(int n, double* x, double* w);
void nsfr_gauss_lobatto(int n, double* x, double* w);

struct nsfr_ctx {
  // n, nv, nfp: volume quadrature points per direction / per element / per
  // face; ns, nsv: solution nodes per direction / per element (equal to n, nv
  // for the collocated schemes).  The state and the RK arrays have nsv nodes.
  int nx, ny, nz, ne, p, n, pg, q, nv, nfp;
  int ns = 0, nsv = 0, uncol = 0;
  // elements [vol_b, vol_e) get the volume pass (nsfr_rk_stage's range), elements
  // [fs_b, fs_e) the face-state pass, [ff_b, ff_e) the face-flux pass; an end < 0
  // means all
  int vol_b = 0, vol_e = -1;
  int fs_b = 0, fs_e = -1;
  int ff_b = 0, ff_e = -1;
  // host-state RK steps: a copy stream and its events (created on first use)
  cudaStream_t cs = nullptr;
  cudaEvent_t* cev = nullptr;  // [2 NSFR_COPY_CHUNKS + 1]
  // volume source (nsfr_set_source): kind, the time of the next stage 0 / residual,
  // W J q at the volume nodes [ne][5][nv] (src), and src_on = src while a source is set
  int source = 0;
  double t = 0.0;
  double* src = nullptr;
  const double* src_on = nullptr;
  double c, gamma;
  int vol_flux, face_flux, precision, nodes;
  OpsGL ops;
  OpsGeo gops;
  int device;
  double dx;  // min_d L_d / (N_d (p+1))
  // device buffers owned by the context
  double* ctrl = nullptr;     // [ne][q^3][3]
  double* metric = nullptr;   // [ne][9][nv]
  float* metric32 = nullptr;  // [ne][18][nv] float-float w_perp/2 C (FP32-bulk contexts)
  double* J = nullptr;        // [ne][nv]
  double* invwj = nullptr;    // [ne][nv] 1/(w_i w_j w_k J)
  double* wj = nullptr;       // [ne][nv] w_i w_j w_k J
  double* nfp_plus = nullptr; // [ne][3][3][nfp]
  double* metric_s = nullptr; // [ne][9][nv] metric rows scaled by w_perp / 2
  double* nf_s = nullptr;     // [ne][3][3][nfp] face rows scaled by w_perp
  double* pair_rows = nullptr; // [ne][3][n(n-1)/2 + 2n][3][nfp] averaged metric rows of the line pairs (FP64 contexts)
  float* nfp_plus32 = nullptr; // [ne][3][6][nfp] float-float w_perp C_f (FP32-bulk contexts)
  float* invwj32 = nullptr;    // [ne][nv] (FP32-bulk contexts)
  double* xyz = nullptr;      // [ne][3][nv]
  double* face = nullptr;     // [ne][6][NSFR_NFIELD][nfp] face-state scratch
  double* nrec = nullptr;     // [ne][8][nv] node records (Rec fields) of the last face-state pass
  double* uq = nullptr;       // [ne][5][nv] chi u^ (uncollocated contexts with square chi)
  double* fstar = nullptr;    // [ne][3][5][nfp] w_perp-scaled numerical flux of each + face
  double* ustage = nullptr;   // [ne][5][nv]
  double* acc = nullptr;      // [ne][5][nv]
  double* rtmp = nullptr;     // [ne][5][nv] (diagnostics / VJP scratch)
  // VJP scratch (allocated by the first nsfr_vjp call)
  double* vjp_fown = nullptr;  // [ne][6][5][nfp] face-state cotangents from the element itself
  double* vjp_fnbr = nullptr;  // [ne][6][5][nfp] cotangents for the neighbour's face state
  double* vjp_nfbar = nullptr; // [ne][6][3][nfp] face-row cotangents, per face of the element
  double* vjp_mbar = nullptr;  // [ne][9][nv] volume metric-row cotangents
  double* vjp_jbar = nullptr;  // [ne][nv] Jacobian cotangents
  double* vjp_pbq = nullptr;   // [ne][5][nv] record cotangents at the GL points (uncollocated contexts)
  double* hbuf_in = nullptr;  // staging for host pointers [ne][5][nv]
  double* hbuf_out = nullptr;
  double* red = nullptr;      // reduction scratch
  int red_cap = 0;
  double* red_host = nullptr; // pinned
  int* flag = nullptr;        // device error word
  int* flag_host = nullptr;   // pinned
  unsigned long long* umax = nullptr;  // [2]: max wave speed (FP64 bit pattern), FP32 candidate bound
  unsigned long long* umax_host = nullptr;
  long long launches = 0;
  // per-launch event pairs (nsfr_profile)
  int prof_on = 0;
  int prof_n = 0;
  cudaEvent_t* prof_ev = nullptr;  // 2 * NSFR_PROF_CAP events
  int* prof_kind = nullptr;
  cudaStream_t last_stream = nullptr;
  std::string err;
};

#define NSFR_PROF_CAP 65536
// bracket a launch with profiling events (no-op unless nsfr_profile is on)
void nsfr_prof_begin(nsfr_ctx* ctx, int kind, cudaStream_t s);
void nsfr_prof_end(nsfr_ctx* ctx, cudaStream_t s);

// Per-node record used by the flux kernels (NSFR_NFIELD doubles): rho, 2 beta,
// u/2 (3), |u|^2/4, ln rho, ln beta.  The halves make arithmetic means plain sums.
enum { P_RHO = 0, P_B2 = 1, P_UH = 2, P_QQ = 5, P_LRHO = 6, P_LBETA = 7 };

// Launchers (residual.cu)
enum { EPI_RAW = 0, EPI_DUDT = 1, EPI_RK = 2 };
struct RkArgs {
  const double* u0;   // u^n
  double* unext;      // where the next stage state goes
  double* acc;        // RK accumulator
  double a_next;      // u_next = u0 + a_next dt k
  double b;           // acc (+)= b dt k
  double dt;
  int first;          // acc = u0 + b dt k
  int last;           // unext = acc + b dt k (final update)
};
cudaError_t nsfr_launch_face_states(nsfr_ctx* ctx, const double* u, cudaStream_t s);
// the same pass in float-float for FP32-bulk contexts (residual_bulk.cu); its
// node records hold rho .. |u|^2/4 as packed float-float pairs
cudaError_t nsfr_launch_face_states_bulk(nsfr_ctx* ctx, const double* u, cudaStream_t s);
// W J q(t) of the context's source into ctx->src (source.cu)
cudaError_t nsfr_launch_source(nsfr_ctx* ctx, double t, cudaStream_t s);
// uncollocated: the entropy projection through chi and Pi (projection.cu)
cudaError_t nsfr_launch_projection(nsfr_ctx* ctx, const double* u, cudaStream_t s);
// uncollocated with square chi: u_q = chi u^ into ctx->uq (projection.cu)
cudaError_t nsfr_launch_interp_square(nsfr_ctx* ctx, const double* u, cudaStream_t s);
// w_perp-scaled metric and face rows and, where the context has one, the volume
// kernel's pair table (after the metric terms change)
cudaError_t nsfr_launch_scaled_rows(nsfr_ctx* ctx, cudaStream_t s);
// doubles of the pair table of ne elements with n points per direction
size_t nsfr_pair_rows_count(int n, int ne);
// numerical flux of every face once, from the face states (after nsfr_launch_face_states)
cudaError_t nsfr_launch_face_flux(nsfr_ctx* ctx, cudaStream_t s);
// acc = u0 + bdt k, k <- u0 + adt k over the whole state (the first RK stage)
cudaError_t nsfr_launch_rk_first_update(nsfr_ctx* ctx, const double* u0, double* k, double* acc, double bdt,
                                        double adt, cudaStream_t s);
cudaError_t nsfr_launch_volume(nsfr_ctx* ctx, const double* u, double* out, int epi, const RkArgs* rk,
                               cudaStream_t s);
// residual_bulk.cu: the FP32-bulk form of nsfr_launch_volume
cudaError_t nsfr_launch_volume_bulk(nsfr_ctx* ctx, const double* u, double* out, int epi, const RkArgs* rk,
                                    cudaStream_t s);
// float-float tables of the geometry for the bulk kernel (after the metrics change)
cudaError_t nsfr_launch_bulk_tables(nsfr_ctx* ctx, cudaStream_t s);
// geometry.cu
cudaError_t nsfr_launch_metrics(nsfr_ctx* ctx, cudaStream_t s);
cudaError_t nsfr_launch_jacobian_derived(nsfr_ctx* ctx, cudaStream_t s);
// reduce.cu
cudaError_t nsfr_launch_max_wavespeed(nsfr_ctx* ctx, const double* u, cudaStream_t s);
// the same in pieces (reduce.cu): clear, FP32 candidates over elements [e_b, e_e), FP64 pass
cudaError_t nsfr_wavespeed_begin(nsfr_ctx* ctx, cudaStream_t s);
cudaError_t nsfr_wavespeed_candidates(nsfr_ctx* ctx, const double* u, int e_b, int e_e, cudaStream_t s);
cudaError_t nsfr_wavespeed_finish(nsfr_ctx* ctx, const double* u, cudaStream_t s);
cudaError_t nsfr_launch_diagnostics(nsfr_ctx* ctx, const double* u, const double* R, double* partial,
                                    int nblocks, cudaStream_t s);
int nsfr_diag_blocks(nsfr_ctx* ctx);
// mathfn.cu
cudaError_t nsfr_launch_math_eval(int fn, const double* x, double* y, long long n, cudaStream_t s);
// vjp.cu
cudaError_t nsfr_launch_vjp(nsfr_ctx* ctx, const double* u, const double* dbar, double* ubar,
                            double* xbar, cudaStream_t s);
