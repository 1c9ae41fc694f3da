/*
 * nsfr.h -- C ABI of the GB300 (sm_103a) NSFR-EC residual library.
 *
 * Method: weight-adjusted, entropy-conserving nonlinearly stable flux
 * reconstruction (NSFR-EC) for the 3D compressible Euler equations on
 * curvilinear hexahedra (Cicchino & Nadarajah, arXiv 2312.07725).  The
 * library evaluates, once per Runge-Kutta stage,
 *   (M_m + K_m) du/dt = -R(u),           Eq. NSFR (Sec. "Nonlinearly Stable
 *                                        Flux Reconstruction")
 *   du/dt = -Pi~ (W J_m)^{-1} Pi~^T R,   Eq. weight-adj ESFR mass
 *                                        (Sec. "Weight-Adjusted Inverse ...")
 * with the solution and volume quadrature collocated on Gauss-Legendre (GL)
 * nodes, Chandrashekar's two-point flux in the volume and on faces,
 * entropy-projected face states u~_f = u(chi_f v^) (Sec. "Nonlinearly Stable
 * Flux Reconstruction", entropy projected variables), conservative-curl
 * metric terms (Sec. "Computational Space", Eq. GCL) and classic RK4
 * (Sec. "Results").
 *
 * Conventions shared by every entry point
 *   - Mesh: a structured, fully periodic block of nx*ny*nz hexahedra, element
 *     e = ex + nx*(ey + ny*ez); element-local xi, eta, zeta follow +x, +y, +z.
 *   - n = p+1 GL nodes per direction, n^3 per element, node index
 *     i + n*(j + n*k) (xi fastest).  1 <= p <= 7.
 *   - State u: conserved variables (rho, rho u, rho v, rho w, rho e) at the
 *     GL nodes, layout [N_e][5][n^3], FP64.  With the collocated basis these
 *     nodal values are the solution coefficients.
 *   - Pointers marked "host or device" may point to either; the library
 *     detects which.  Device pointers must be in the memory of the device
 *     that was current at nsfr_setup.
 *   - Every call that takes a stream is asynchronous on that stream
 *     (cudaStream_t passed as void*; NULL = legacy default stream) when all
 *     its buffers are device buffers; with a host buffer the call
 *     synchronises the stream before returning.
 *   - The caller owns every buffer it passes.  The library owns the metric
 *     terms, face buffers and its workspace, freed by nsfr_destroy.
 *   - No call aborts, traps or throws.  Errors are returned as nsfr_status;
 *     a message is kept per context (nsfr_last_error).  Non-physical states
 *     (rho <= 0, p <= 0 or NaN at a node) detected on the device set a
 *     device flag; it is reported as NSFR_ERR_NONPHYSICAL by the next call
 *     that synchronises (nsfr_rk_step with cfl > 0, nsfr_entropy,
 *     nsfr_check) and then cleared.
 */
#ifndef NSFR_H
#define NSFR_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nsfr_ctx nsfr_ctx;

typedef enum {
  NSFR_OK = 0,
  NSFR_ERR_ARG = -1,         /* invalid argument (sizes, NULL, unsupported p) */
  NSFR_ERR_MESH = -2,        /* J <= 0 at some GL node of the mesh */
  NSFR_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  NSFR_ERR_NONPHYSICAL = -4, /* rho <= 0, p <= 0 or NaN met on the device */
  NSFR_ERR_OOM = -5,         /* device allocation failed */
  NSFR_ERR_STATE = -6        /* call not valid for this context */
} nsfr_status;

typedef enum { NSFR_FLUX_CHANDRASHEKAR = 0, NSFR_FLUX_RANOCHA = 1 } nsfr_vol_flux;
typedef enum { NSFR_FACE_EC = 0, NSFR_FACE_EC_ROE = 1, NSFR_FACE_EC_ES = 2 } nsfr_face_flux;
typedef enum { NSFR_FP64 = 0, NSFR_FP32_BULK = 1, NSFR_FP32_BULK_FF = 2 } nsfr_precision;
typedef enum { NSFR_NODES_GL = 0, NSFR_NODES_LGL = 1 } nsfr_nodes;
typedef enum { NSFR_SOURCE_NONE = 0, NSFR_SOURCE_MANUFACTURED = 1 } nsfr_source;

/*
 * nsfr_setup -- build a context: 1D operators, metric terms, workspace.
 *   grid_nodes  host or device, [N_e][(p_geo+1)^3][3] FP64: control points
 *               of each element's degree-p_geo tensor-product Lagrange map
 *               x = sum_i Theta_i(xi) x_i (Sec. "Computational Space"),
 *               placed at equispaced reference nodes xi_k = -1 + 2k/p_geo,
 *               xi fastest.  Control points on shared faces must coincide
 *               (up to a constant shift across the periodic boundary).
 *   nx, ny, nz  elements per direction (each >= 1).
 *   p_geo       map degree, 1 <= p_geo <= p.
 *   p           solution degree, 1 <= p <= 7.
 *   c           ESFR parameter (c = 0: DG; Sec. "Energy Stable Flux
 *               Reconstruction", Eq. Km with c_(s,v,w) = c^{(s+v+w)/p}).
 *   vol_flux    the entropy-conserving two-point flux of the volume, hybrid
 *               and face terms: NSFR_FLUX_CHANDRASHEKAR (Chandrashekar's EC,
 *               kinetic-energy preserving flux) or NSFR_FLUX_RANOCHA (the
 *               flux the paper's EC runs use, Sec. "Results": Chandrashekar's
 *               with Ranocha's pressure terms, the arithmetic pressure mean in
 *               the momentum flux and (p_L u_R.n + p_R u_L.n)/2 as the pressure
 *               work in the energy flux).  NSFR_FLUX_RANOCHA needs precision
 *               NSFR_FP64 (else NSFR_ERR_ARG), and nsfr_vjp returns
 *               NSFR_ERR_STATE for such a context.
 *   face_flux   NSFR_FACE_EC (entropy conserving), NSFR_FACE_EC_ROE (EC
 *               flux plus Roe dissipation, Sec. "Nonlinear Stability") or
 *               NSFR_FACE_EC_ES (EC flux minus (1/2) R |Lambda| T R^T [[v]]:
 *               Roe-type dissipation written in the jump of the entropy
 *               variables with Barth's eigenvector scaling, R T R^T = du/dv,
 *               so that every face dissipates entropy).
 *   gamma       ratio of specific heats (> 1).
 *   precision   NSFR_FP64; NSFR_FP32_BULK: flux differencing and operator
 *               contractions in FP32 with FP32 accumulation (fluxes as
 *               deviations from each element's first node, the mass flux in
 *               float-float); the log means and the scalars made from them,
 *               the entropy variables and projection, the face fluxes, the
 *               state and all reductions stay FP64.  NSFR_FP32_BULK_FF: the
 *               same, but the log-mean scalars (rho_ln, p_hat, H) and the
 *               entropy projection in float-float (pairs of floats, ~48
 *               bits, with float-float log and exp; FP64 for log means
 *               across jumps wider than ~3%), so that almost nothing waits
 *               on the FP64 pipe.  Both within about 1e-5 of the FP64 path.
 *   nodes       the collocated solution / volume quadrature nodes:
 *               NSFR_NODES_GL (Gauss-Legendre; the state lives at the GL
 *               nodes) or NSFR_NODES_LGL (Gauss-Lobatto-Legendre, the paper's
 *               "LGL" integration: the face nodes are boundary volume nodes,
 *               the setting of its kinetic-energy lemma).  Everything below
 *               that says "GL nodes" means the chosen set.
 *   out         receives the context (NULL on failure).
 * Metric terms are built on the device in conservative-curl form on the
 * degree-p Lobatto nodes and interpolated to the GL nodes (Eq. GCL); the
 * face normal of each face is shared by both neighbours.  Returns
 * NSFR_ERR_MESH if J <= 0 anywhere.  Synchronises the current device.
 */
nsfr_status nsfr_setup(const double* grid_nodes, int nx, int ny, int nz, int p_geo, int p,
                       double c, int vol_flux, int face_flux, double gamma, int precision, int nodes,
                       nsfr_ctx** out);

/*
 * nsfr_setup_uncollocated -- the paper's own setting: the solution's
 * coefficients on the p+1 Lobatto (LGL) nodes, volume and face integrals on
 * nq >= p+1 Gauss-Legendre points per direction (nq > p+1: the paper's
 * "overintegration", Sec. "Results").  Arguments as in nsfr_setup, plus
 *   nq          GL points per direction, p+1 <= nq <= 8.
 * The state u, du/dt and the RK arrays are [N_e][5][(p+1)^3] values at the
 * LGL nodes (nsfr_node_coords returns those nodes); the metric terms and the
 * Jacobians (nsfr_get_metrics, nsfr_quadrature) live at the nq^3 GL points
 * and nq^2 GL face points.  Each residual evaluation projects the entropy
 * variables, v~^ = Pi v(chi u^) with chi the LGL basis at the GL points and
 * Pi = (chi^T W chi)^{-1} chi^T W, evaluates the flux differencing of Eq.
 * NSFR on the GL points with u~ = u(chi v~^) and the face states
 * u(l_f v~^), and returns chi^T R_q (nsfr_residual_raw) or the weight-
 * adjusted du/dt = -Pi~ (W J)^{-1} Pi~^T chi^T R_q, Pi~1 = (M1 + K1)^{-1}
 * chi^T W (nsfr_residual, nsfr_rk_step).  precision: NSFR_FP64, or
 * NSFR_FP32_BULK (the flux differencing in FP32 as for nsfr_setup, the
 * entropy projection and the face fluxes in FP64, and the return to the
 * solution nodes -- chi^T, or (chi Pi~1)^T, 1/(W J), Pi~1 -- as FP32 sweeps);
 * anything else is NSFR_ERR_ARG.  nsfr_vjp offers the state cotangent only
 * (x_bar NULL).  With nq = p+1 the scheme is the GL-collocated one written in
 * the LGL basis.
 */
nsfr_status nsfr_setup_uncollocated(const double* grid_nodes, int nx, int ny, int nz, int p_geo, int p, int nq,
                                    double c, int vol_flux, int face_flux, double gamma, int precision,
                                    nsfr_ctx** out);

/*
 * nsfr_residual -- du/dt = -Pi~ (W J)^{-1} Pi~^T R(u)  (Eq. NSFR with the
 * weight-adjusted inverse, Eq. weight-adj ESFR mass).
 *   u     host or device, [N_e][5][n^3] FP64, read only.
 *   dudt  host or device, [N_e][5][n^3] FP64, overwritten.
 *   stream  cudaStream_t or NULL.
 */
nsfr_status nsfr_residual(nsfr_ctx* ctx, const double* u, double* dudt, void* stream);

/*
 * nsfr_residual_raw -- R(u) of Eq. NSFR, i.e. the volume flux differencing,
 * hybrid volume-face terms and face fluxes before the mass inverse, so that
 * (M_m + K_m) du/dt = -R.  Same arguments as nsfr_residual.
 */
nsfr_status nsfr_residual_raw(nsfr_ctx* ctx, const double* u, double* R, void* stream);

/*
 * nsfr_rk_step -- one classic 4-stage, 4th-order Runge-Kutta step (Sec.
 * "Results"), u <- u + dt/6 (k1 + 2 k2 + 2 k3 + k4), each stage a fused
 * residual + stage update.
 *   u         host or device, [N_e][5][n^3] FP64, updated in place.
 *   cfl       if dt_fixed <= 0: dt = cfl * dx / max_i(|u_i| + a_i) with
 *             dx = min_d L_d/(N_d (p+1)) from the node coordinates' extent;
 *             needs one device->host read of the max (synchronises).
 *   dt_fixed  > 0: use this step and do not read anything back.
 *   dt_used   host, receives dt (may be NULL).
 * A host u (collocated contexts) is copied to the device in z-chunks while
 * stage 0 runs behind the copy (its face states, face fluxes and du/dt chunk
 * by chunk, the stage update once dt is known), and stage 3's result is
 * copied back chunk by chunk while the next is computed; the result, dt and
 * the time equal those of the same step on a device u, bit for bit.  The call
 * returns when the host u holds the new state.
 */
nsfr_status nsfr_rk_step(nsfr_ctx* ctx, double* u, double cfl, double dt_fixed, double* dt_used,
                         void* stream);

/*
 * nsfr_rk_stage -- one stage of the classic RK4 step of nsfr_rk_step, on
 * caller-owned arrays, for drivers that act between stages (a domain split
 * into slabs exchanges the ghost-layer states there).  Stage `stage`
 * (0..3) reads u for stage 0 and ustage otherwise; stages 0..2 write
 * u + a_s dt k_s (a = 1/2, 1/2, 1) to ustage and accumulate acc (stage 0
 * sets acc = u + dt/6 k_0); stage 3 writes acc + dt/6 k_3 to u.  u, ustage,
 * acc: device [N_e][5][solution nodes]; ustage may be read by the next
 * stage only.  dt > 0.  Only elements e_begin <= e < e_end are updated
 * (their entries of ustage, acc and u); the face states of every element
 * enter their face terms, and the other elements' entries are left as they
 * are (0 and N_e: all; a slab's ghost layers need no update).  Asynchronous
 * on the stream; NSFR_ERR_ARG for host or NULL buffers or a range outside
 * 0 <= e_begin <= e_end <= N_e.  Four calls (stages 0..3) over all elements
 * equal one nsfr_rk_step with dt_fixed = dt.
 */
nsfr_status nsfr_rk_stage(nsfr_ctx* ctx, double* u, double* ustage, double* acc, int stage, double dt,
                          int e_begin, int e_end, void* stream);

/*
 * nsfr_max_wavespeed -- max over the nodes of |u| + a for the device state
 * u (the CFL step of nsfr_rk_step is cfl * dx / this, dx = min_d L_d /
 * (N_d (p+1))); synchronises the stream and reports a non-physical state.
 */
nsfr_status nsfr_max_wavespeed(nsfr_ctx* ctx, const double* u, double* lam, void* stream);

/*
 * nsfr_set_source -- add a volume source q(x, t) to the semi-discrete
 * system, (M_m + K_m) du/dt = -R + W J q, i.e. du/dt = -Pi~ (W J)^{-1} Pi~^T
 * (R - W J q) with q at the volume nodes (the source integrated like the
 * residual's volume terms; the paper does not spell its discretisation out).
 *   kind  NSFR_SOURCE_NONE (remove) or NSFR_SOURCE_MANUFACTURED: the source of
 *         the manufactured solution of Sec. "Manufactured Solution
 *         Convergence", rho = 2 + sin(pi (x+y+z-2t))/10, u = v = w = 1,
 *         rho e = rho^2 (q derived from that definition; its periodic box is
 *         [-1, 1]^3).
 *   t     the context's time: nsfr_residual evaluates q at t; nsfr_rk_step
 *         and nsfr_rk_stage use the stage times t, t + dt/2, t + dt/2, t + dt
 *         and advance t by dt with the last stage (they advance it with or
 *         without a source).
 * nsfr_residual_raw returns R without the source.  Collocated contexts only
 * (NSFR_ERR_STATE otherwise); the first call with a source allocates
 * 40 B per volume node (NSFR_ERR_OOM).  Synchronous.
 */
nsfr_status nsfr_set_source(nsfr_ctx* ctx, int kind, double t);

/* nsfr_get_time -- the context's time (see nsfr_set_source). */
nsfr_status nsfr_get_time(const nsfr_ctx* ctx, double* t);

/*
 * nsfr_entropy -- diagnostics of a state (synchronises; FP64 compensated sums).
 *   u    host or device, [N_e][5][n^3].
 *   out  host, 14 doubles:
 *        [0] S       = sum W J U(u), U = -rho s/(gamma-1), s = ln p - gamma ln rho
 *        [1] dS/dt   = -sum_i v(u_i) . R_i  (semi-discrete entropy rate,
 *                      Sec. "Nonlinear Stability"; 0 to round-off for EC)
 *        [2] sum_i |v(u_i) . R_i|  (scale of [1])
 *        [3..7]  Q_k = sum W J (Pi~^{-1} u)_k, conserved by the WA scheme
 *                      (Sec. "Global Conservation")
 *        [8] KE      = sum W J rho |u|^2 / 2
 *        [9..13] sum_i R_{i,k}  (0 to round-off on a periodic mesh)
 * For an uncollocated context (nsfr_setup_uncollocated) the sums take the
 * solution at the GL points, u_q = chi u^, with the point weights W J:
 * S = sum W J U(u_q), Q_k = sum W J (u_q)_k (the GL quadrature of the
 * solution), KE = sum W J rho|u|^2/2 at the points; the entropy rate is
 * -sum_i v~^_i . R^_i at the Lobatto nodes with the projected entropy
 * variables v~^ = Pi v(u_q) and R^ = chi^T R_q (the paper's statement for
 * the uncollocated scheme), [2] its scale, and [9..13] sum_i R^_{i,k}.
 */
nsfr_status nsfr_entropy(nsfr_ctx* ctx, const double* u, double* out, void* stream);

/*
 * nsfr_vjp -- vector-Jacobian product of du/dt(u; x) (reverse mode, hand
 * written; the paper has no adjoint):
 *   u_bar += (d dudt/du)^T dudt_bar,
 *   x_bar += (d dudt/dx)^T dudt_bar  (through the metric terms and 1/J to the
 *            control points; skipped when x_bar is NULL).
 *   u, dudt_bar, u_bar  device, [N_e][5][n^3] FP64.
 *   x_bar               device or NULL, [N_e][(p_geo+1)^3][3] FP64.
 * FP64 contexts with the EC face flux and Chandrashekar's volume flux only
 * (NSFR_ERR_STATE otherwise).  For an uncollocated context (state on the
 * Lobatto nodes) the state cotangent is offered (x_bar must be NULL): the
 * flux differencing is reversed on the GL points and the entropy projection
 * (chi, v(u), Pi, u(v) at the points and the faces) back to the solution
 * nodes.  Runs the face-state pass of u (and, for x_bar, the residual R(u))
 * first; asynchronous on the stream.
 */
nsfr_status nsfr_vjp(nsfr_ctx* ctx, const double* u, const double* dudt_bar, double* u_bar,
                     double* x_bar, void* stream);

/*
 * nsfr_node_coords -- physical coordinates of the GL nodes, [N_e][3][n^3]
 * (host or device), for sampling initial states.
 */
nsfr_status nsfr_node_coords(nsfr_ctx* ctx, double* xyz, void* stream);

/*
 * nsfr_get_metrics -- copies of the metric data (host or device buffers,
 * any may be NULL):
 *   C    [N_e][9][n^3]  C[3d+c] = (J a^d)_c at GL volume nodes (row d of C^T)
 *   J    [N_e][n^3]     Jacobian determinant at GL nodes
 *   Cf   [N_e][3][3][n^2] face row (J a^d)_c on the element's xi_d = +1 face,
 *        shared with the neighbour across that face.
 */
nsfr_status nsfr_get_metrics(nsfr_ctx* ctx, double* C, double* J, double* Cf, void* stream);

/*
 * nsfr_set_metrics -- replace the context's metric terms with caller-supplied
 * ones (host or device buffers, layouts as nsfr_get_metrics; none may be
 * NULL): C [N_e][9][n^3], J [N_e][n^3], Cf [N_e][3][3][n^2].  1/(w J) and
 * w J are recomputed.  The face rows must be the ones both neighbours share
 * (row of the element's xi_d = +1 face).  Returns NSFR_ERR_MESH if some
 * J <= 0; synchronises the stream.  The control points kept for nsfr_vjp's
 * x_bar are not changed.
 */
nsfr_status nsfr_set_metrics(nsfr_ctx* ctx, const double* C, const double* J, const double* Cf, void* stream);

/*
 * nsfr_quadrature -- W J at the GL nodes, [N_e][n^3] (host or device): the
 * physical quadrature weights, so that sum_i (W J)_i f_i integrates f over the
 * domain (used for functionals such as the kinetic energy, and for the L2
 * error of Sec. "Manufactured Solution Convergence").
 */
nsfr_status nsfr_quadrature(nsfr_ctx* ctx, double* wj, void* stream);

/* nsfr_info -- sizes: out[0]=N_e, [1]=p, [2]=n^3, [3]=p_geo, [4]=precision. */
nsfr_status nsfr_info(const nsfr_ctx* ctx, long long* out);

/*
 * nsfr_check -- synchronise the context's last stream and report (then
 * clear) a device-side non-physical-state flag.
 */
nsfr_status nsfr_check(nsfr_ctx* ctx);

/*
 * Kernel ids for nsfr_profile_read: 0 metric set-up, 1 face states (entropy
 * projection), 2 volume/hybrid/surface + WA inverse (+ RK stage), 3 maximum
 * wave speed, 4 diagnostics, 5 VJP face pass, 6 VJP volume pass, 7 VJP metric
 * pass, 8 face numerical fluxes, 9 volume source, 10 the first RK stage's
 * update when it is not fused into the volume pass (a host-state step).
 */
#define NSFR_NKERNELS 11

/*
 * nsfr_profile -- on != 0: from now on record a CUDA event pair around every
 * kernel launch, on the launch's stream, and reset the totals; on == 0: stop.
 * Up to 65536 launches are recorded; later launches are not timed.
 */
nsfr_status nsfr_profile(nsfr_ctx* ctx, int on);

/*
 * nsfr_profile_read -- synchronise, then add the recorded launches' device
 * time (ms, host double[NSFR_NKERNELS]) and counts (host long long
 * [NSFR_NKERNELS]) per kernel id; either pointer may be NULL.
 */
nsfr_status nsfr_profile_read(nsfr_ctx* ctx, double* ms, long long* count);

/*
 * nsfr_residual_static -- du/dt as nsfr_residual computes it for an FP64
 * context on GL nodes with the Chandrashekar volume flux and no volume source
 * (nsfr_set_source), for callers that must not allocate device memory: code
 * running under a memory
 * manager that owns the whole device (a framework's caching allocator, an
 * application with a fixed memory budget) or code that cannot afford the
 * implicit device synchronisation of cudaMalloc/cudaFree.  It needs no
 * context and calls no cudaMalloc, cudaFree or other allocating routine; the
 * paper has no counterpart of this call.
 *   u     device [N_e][5][n^3] state (every buffer must be device memory of
 *         the current device: anything else, NULL included, is NSFR_ERR_ARG
 *         before anything runs)
 *   C     device [N_e][9][n^3] metric rows, J device [N_e][n^3] Jacobians,
 *   Cf    device [N_e][3][3][n^2] shared face rows (layouts of
 *         nsfr_get_metrics; e.g. copied once from a context)
 *   nx, ny, nz, p, c, face_flux, gamma   as in nsfr_setup (FP64 only)
 *   dudt  device [N_e][5][n^3] output
 * Its working memory (face states, node records, face fluxes, scaled metric
 * rows, the volume kernel's pair table, 1/(wJ), an error word) is a fixed
 * 16 MiB array inside the library (NSFR_STATIC_SCRATCH_BYTES), which every
 * GPU that loads the library keeps until the process exits.  A problem
 * needing more than that, 256 + N_e (36 n^4 + 260 n^3 + 576 n^2) bytes
 * (about 470 elements at p = 3, 240 at p = 4), is rejected with
 * NSFR_ERR_ARG before anything runs.  Every call looks up the array's
 * address in the current device's context (cudaGetSymbolAddress, which
 * allocates nothing).  All calls share
 * the one array and the last call's contents stay in it; the error word is
 * cleared at the start of every call.  Calls that overlap on the GPU (other
 * streams, other threads) race on the array: serialise them.  The call
 * synchronises the stream to read the error word (NSFR_ERR_NONPHYSICAL,
 * NSFR_ERR_MESH for J <= 0).
 */
#define NSFR_STATIC_SCRATCH_BYTES (16u << 20)
nsfr_status nsfr_residual_static(const double* u, const double* C, const double* J, const double* Cf, int nx,
                                 int ny, int nz, int p, double c, int face_flux, double gamma, double* dudt,
                                 void* stream);

/*
 * nsfr_math_eval -- y[i] = f(x[i]), i < n, with the library's own device
 * elementary functions, for checking them against reference values:
 *   NSFR_FN_LOG  natural logarithm (table-driven, Tang's method; about one
 *                ulp of max(|ln x|, ln 2))
 *   NSFR_FN_EXP  exponential (table-driven, Tang's method; about one ulp)
 *   NSFR_FN_RCP  1/x, FP32 seed and one third-order step (about one ulp)
 *   NSFR_FN_RCP1 1/x, FP32 seed and one Newton step (relative error <= 2^-43)
 *   NSFR_FN_LOG_FF, NSFR_FN_EXP_FF  the float-float log and exp of the
 *                FP32-bulk kernels (x split into two floats, the result
 *                summed back; about 2^-46 of max(|ln x|, 0.7), and relative
 *                2^-46; x.hi positive and normal for the log, |x| < 87 for exp)
 *   NSFR_FN_JOIN  the integer-pipe join of a float-float pair into a double:
 *                the 64 bits of x are the pair (hi in the high 32 bits, lo in
 *                the low), y = hi + lo with its bits below 2^-52 |y|
 *                truncated (exact when the sum fits 53 bits); for
 *                |lo| < |hi| / 2 or hi = 0, finite hi
 *   NSFR_FN_LOGMEAN1 the logarithmic mean (x - 1) / ln x of x > 0 and 1 as
 *                the FP64 volume kernels form the log means of Chandrashekar's
 *                flux (Sec. "Nonlinearly Stable Flux Reconstruction"): for
 *                u = ((x-1)/(x+1))^2 < 1e-4 the series of f/atanh(f) in u,
 *                its terms beyond the constant in float-float, plus one FP64
 *                FMA (about one ulp); else (x - 1) / ln x in FP64
 *   NSFR_FN_SPLIT the integer-pipe split of x into two floats: hi the
 *                nearest float (ties away from zero), lo the leading 24 bits
 *                of x - hi (truncated), returned packed as NSFR_FN_JOIN
 *                takes them (hi in the high 32 bits); for normal x with
 *                2^-100 < |x| < 2^100
 *   NSFR_FN_I2D  the integer-pipe conversion of the int in the low 32 bits of
 *                x to a double (exact)
 * The kernels compute the entropy variables, face states and two-point
 * fluxes with these.  x and y are device buffers of n doubles (n >= 0; they
 * may alias); asynchronous on the stream.  NSFR_ERR_ARG for an unknown fn, a
 * NULL or host pointer or n < 0.  No context is needed.
 */
typedef enum {
  NSFR_FN_LOG = 0,
  NSFR_FN_EXP = 1,
  NSFR_FN_RCP = 2,
  NSFR_FN_RCP1 = 3,
  NSFR_FN_LOG_FF = 4,
  NSFR_FN_EXP_FF = 5,
  NSFR_FN_JOIN = 6,
  NSFR_FN_LOGMEAN1 = 7,
  NSFR_FN_SPLIT = 8,
  NSFR_FN_I2D = 9
} nsfr_fn;
nsfr_status nsfr_math_eval(int fn, const double* x, double* y, long long n, void* stream);

/*
 * nsfr_fma_probe -- a throughput probe of the FP64 (fp32 = 0) or FP32
 * (fp32 = 1) fused multiply-add pipe, the measured denominator of the
 * kernels' ALU rooflines (the paper has no counterpart).  Launches `blocks`
 * CTAs of 256 threads, each thread running 8 independent chains
 * x <- x a + b for `iters` steps, asynchronously on `stream`; the caller
 * times the launch (CUDA events on the same stream) and divides *fmas, the
 * number of multiply-adds it performs, by the time.  sink: device buffer of
 * two doubles (written; keeps the chains live).  NSFR_ERR_ARG for iters or
 * blocks < 1 or a NULL or host pointer.  No context is needed.
 */
nsfr_status nsfr_fma_probe(int fp32, long long iters, int blocks, double* sink, long long* fmas, void* stream);

/* nsfr_kernel_launches -- kernels this context has launched so far. */
long long nsfr_kernel_launches(const nsfr_ctx* ctx);

/* nsfr_last_error -- message of the last failure on ctx ("" if none). */
const char* nsfr_last_error(const nsfr_ctx* ctx);

/* nsfr_destroy -- free everything the context owns (NULL is a no-op). */
void nsfr_destroy(nsfr_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* NSFR_H */
