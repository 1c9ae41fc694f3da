// C ABI of the library: context set-up, residual, RK4 step, diagnostics.
// See include/nsfr.h for the contract of every entry point.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "nsfr_internal.h"

size_t nsfr_metric_smem();

namespace {

nsfr_status fail(nsfr_ctx* ctx, nsfr_status st, const char* msg) {
  if (ctx) ctx->err = msg;
  return st;
}

nsfr_status cuda_fail(nsfr_ctx* ctx, cudaError_t e, const char* where) {
  if (ctx) {
    ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return NSFR_ERR_CUDA;
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(T) + 16);
}

void prof_free(nsfr_ctx* c) {
  if (c->prof_ev) {
    for (int i = 0; i < 2 * NSFR_PROF_CAP; ++i) cudaEventDestroy(c->prof_ev[i]);
    delete[] c->prof_ev;
    delete[] c->prof_kind;
    c->prof_ev = nullptr;
    c->prof_kind = nullptr;
  }
}

void free_all(nsfr_ctx* c) {
  double* dbl[] = {c->ctrl, c->metric, c->J, c->invwj, c->wj, c->nfp_plus, c->xyz, c->face, c->nrec, c->fstar,
                   c->metric_s, c->nf_s, c->pair_rows, c->uq,
                   c->ustage, c->acc, c->rtmp, c->hbuf_in, c->hbuf_out, c->red,
                   c->vjp_fown, c->vjp_fnbr, c->vjp_nfbar, c->vjp_mbar, c->vjp_jbar, c->vjp_pbq, c->src};
  for (double* p : dbl)
    if (p) cudaFree(p);
  if (c->metric32) cudaFree(c->metric32);
  if (c->nfp_plus32) cudaFree(c->nfp_plus32);
  if (c->invwj32) cudaFree(c->invwj32);
  if (c->flag) cudaFree(c->flag);
  if (c->umax) cudaFree(c->umax);
  if (c->red_host) cudaFreeHost(c->red_host);
  if (c->flag_host) cudaFreeHost(c->flag_host);
  if (c->umax_host) cudaFreeHost(c->umax_host);
  if (c->cev) {
    for (int i = 0; i < 2 * NSFR_COPY_CHUNKS + 1; ++i) cudaEventDestroy(c->cev[i]);
    delete[] c->cev;
  }
  if (c->cs) cudaStreamDestroy(c->cs);
  prof_free(c);
}

size_t state_count(const nsfr_ctx* c) { return (size_t)c->ne * 5 * c->nsv; }

nsfr_status ensure_host_buffers(nsfr_ctx* ctx) {
  if (!ctx->hbuf_in) CK(dalloc(&ctx->hbuf_in, state_count(ctx)), "cudaMalloc(staging)");
  if (!ctx->hbuf_out) CK(dalloc(&ctx->hbuf_out, state_count(ctx)), "cudaMalloc(staging)");
  return NSFR_OK;
}

// read (and clear) the device error word; synchronises the stream
nsfr_status read_flag(nsfr_ctx* ctx, cudaStream_t s) {
  CK(cudaMemcpyAsync(ctx->flag_host, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(flag)");
  CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  const int f = *ctx->flag_host;
  if (f) {
    CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), s), "cudaMemsetAsync(flag)");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (f & 4) return fail(ctx, NSFR_ERR_CUDA, "a kernel's bounded wait for its staged data timed out");
    if (f & 2) return fail(ctx, NSFR_ERR_MESH, "non-positive Jacobian at a GL node");
    return fail(ctx, NSFR_ERR_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or NaN) met on the device");
  }
  return NSFR_OK;
}

cudaError_t launch_volume_any(nsfr_ctx* ctx, const double* u, double* out, int epi, const RkArgs* rk,
                              cudaStream_t s) {
  return ctx->precision != NSFR_FP64 ? nsfr_launch_volume_bulk(ctx, u, out, epi, rk, s)
                                          : nsfr_launch_volume(ctx, u, out, epi, rk, s);
}

nsfr_status residual_device(nsfr_ctx* ctx, const double* u, double* out, int epi, cudaStream_t s) {
  if (ctx->src_on && epi != EPI_RAW) CK(nsfr_launch_source(ctx, ctx->t, s), "manufactured_source_kernel");
  CK(nsfr_launch_face_states(ctx, u, s), "face_state_kernel");
  CK(nsfr_launch_face_flux(ctx, s), "face_flux_kernel");
  CK(launch_volume_any(ctx, u, out, epi, nullptr, s), "volume_kernel");
  return NSFR_OK;
}

nsfr_status residual_any(nsfr_ctx* ctx, const double* u, double* out, int epi, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (!u || !out) return fail(ctx, NSFR_ERR_ARG, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const bool du = is_device_ptr(u), dout = is_device_ptr(out);
  if (du && dout) return residual_device(ctx, u, out, epi, s);
  nsfr_status st = ensure_host_buffers(ctx);
  if (st != NSFR_OK) return st;
  const size_t bytes = state_count(ctx) * sizeof(double);
  const double* ud = u;
  if (!du) {
    CK(cudaMemcpyAsync(ctx->hbuf_in, u, bytes, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(H2D)");
    ud = ctx->hbuf_in;
  }
  double* od = dout ? out : ctx->hbuf_out;
  st = residual_device(ctx, ud, od, epi, s);
  if (st != NSFR_OK) return st;
  if (!dout) CK(cudaMemcpyAsync(out, od, bytes, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(D2H)");
  CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return NSFR_OK;
}

// max(|u| + a) over the nodes of u (device); synchronises the stream
nsfr_status max_wavespeed(nsfr_ctx* ctx, const double* u, double* lam, cudaStream_t s) {
  CK(nsfr_launch_max_wavespeed(ctx, u, s), "max_wavespeed_kernel");
  CK(cudaMemcpyAsync(ctx->umax_host, ctx->umax, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s),
     "cudaMemcpyAsync(max)");
  nsfr_status st = read_flag(ctx, s);  // synchronises
  if (st != NSFR_OK) return st;
  std::memcpy(lam, ctx->umax_host, sizeof(double));
  if (!(*lam > 0.0)) return fail(ctx, NSFR_ERR_NONPHYSICAL, "zero or invalid wave speed");
  return NSFR_OK;
}

// one stage of classic RK4 on the caller's arrays: stage st reads
// (st == 0 ? u : ustage); u_{st+1} = u^n + a_st dt k_st goes to ustage,
// acc = u^n + sum b_st dt k_st, and the last stage writes acc + b_3 dt k_3 to u.
// `parts` selects the launches (a host-state step interleaves them with copies):
enum { PART_FACE_STATES = 1, PART_FACE_FLUX = 2, PART_SOURCE = 4, PART_VOLUME = 8, PART_TIME = 16, PART_ALL = 31 };
nsfr_status rk_stage_parts(nsfr_ctx* ctx, double* u, double* ustage, double* acc, int st, double dt,
                           cudaStream_t s, int parts) {
  const double a[3] = {0.5, 0.5, 1.0};
  const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const double* in = (st == 0) ? u : ustage;
  RkArgs rk;
  rk.u0 = u;
  rk.acc = acc;
  rk.dt = dt;
  rk.b = b[st];
  rk.first = (st == 0);
  rk.last = (st == 3);
  rk.a_next = (st < 3) ? a[st] : 0.0;
  rk.unext = (st == 3) ? u : ustage;
  const double c_stage[4] = {0.0, 0.5, 0.5, 1.0};  // stage times t + c dt
  if ((parts & PART_SOURCE) && ctx->src_on)
    CK(nsfr_launch_source(ctx, ctx->t + c_stage[st] * dt, s), "manufactured_source_kernel");
  if (parts & PART_FACE_STATES) CK(nsfr_launch_face_states(ctx, in, s), "face_state_kernel");
  if (parts & PART_FACE_FLUX) CK(nsfr_launch_face_flux(ctx, s), "face_flux_kernel");
  if (parts & PART_VOLUME) CK(launch_volume_any(ctx, in, nullptr, EPI_RK, &rk, s), "volume_kernel(rk)");
  if ((parts & PART_TIME) && st == 3) ctx->t += dt;
  return NSFR_OK;
}

nsfr_status rk_stage_device(nsfr_ctx* ctx, double* u, double* ustage, double* acc, int st, double dt,
                            cudaStream_t s) {
  return rk_stage_parts(ctx, u, ustage, acc, st, dt, s, PART_ALL);
}

nsfr_status rk_step_device(nsfr_ctx* ctx, double* u, double cfl, double dt_fixed, double* dt_used,
                           cudaStream_t s) {
  double dt = dt_fixed;
  if (!(dt_fixed > 0.0)) {
    if (!(cfl > 0.0)) return fail(ctx, NSFR_ERR_ARG, "need cfl > 0 or dt_fixed > 0");
    double lam;
    nsfr_status st = max_wavespeed(ctx, u, &lam, s);
    if (st != NSFR_OK) return st;
    dt = cfl * ctx->dx / lam;
  }
  if (dt_used) *dt_used = dt;
  // classic RK4: u_{s+1} = u^n + a_s dt k_s, acc = u^n + sum b_s dt k_s
  for (int st = 0; st < 4; ++st) {
    nsfr_status r = rk_stage_device(ctx, u, ctx->ustage, ctx->acc, st, dt, s);
    if (r != NSFR_OK) return r;
  }
  return NSFR_OK;
}

nsfr_status ensure_copy_stream(nsfr_ctx* ctx) {
  if (!ctx->cs) CK(cudaStreamCreateWithFlags(&ctx->cs, cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
  if (!ctx->cev) {
    ctx->cev = new cudaEvent_t[2 * NSFR_COPY_CHUNKS + 1];
    for (int i = 0; i < 2 * NSFR_COPY_CHUNKS + 1; ++i)
      CK(cudaEventCreateWithFlags(&ctx->cev[i], cudaEventDisableTiming), "cudaEventCreateWithFlags");
  }
  return NSFR_OK;
}

// An RK4 step of a host state (collocated contexts): the state goes to the device
// in z-chunks on a copy stream, and stage 0 runs behind it chunk by chunk without
// dt: chunk j's face states (and FP32 wave-speed candidates) as soon as it has
// arrived, then the face fluxes of chunk j-1 (whose + neighbours now have face
// states) and the volume pass of chunk j-1 (whose - neighbours' fluxes exist),
// storing k = du/dt; chunk 0 (its - neighbour is the last chunk, the mesh being
// periodic) and the last chunk follow the last copy.  With dt from the wave
// speed, one pass applies stage 0's update exactly as the fused epilogue does;
// stages 1, 2 run whole, and stage 3's volume pass runs chunk by chunk, each
// chunk copied back while the next is computed.  Same results, bit for bit, as
// copy in, rk_step_device, copy out.
nsfr_status rk_step_host(nsfr_ctx* ctx, double* uh, double cfl, double dt_fixed, double* dt_used,
                         cudaStream_t s) {
  nsfr_status st = ensure_host_buffers(ctx);
  if (st != NSFR_OK) return st;
  st = ensure_copy_stream(ctx);
  if (st != NSFR_OK) return st;
  const bool need_lam = !(dt_fixed > 0.0);
  if (need_lam && !(cfl > 0.0)) return fail(ctx, NSFR_ERR_ARG, "need cfl > 0 or dt_fixed > 0");
  const int L = ctx->nx * ctx->ny, nzc = ctx->nz < NSFR_COPY_CHUNKS ? ctx->nz : NSFR_COPY_CHUNKS;
  int cb[NSFR_COPY_CHUNKS + 1];
  for (int j = 0; j <= nzc; ++j) cb[j] = L * (int)(((long long)ctx->nz * j) / nzc);
  const size_t per = (size_t)5 * ctx->nsv;  // doubles per element
  double* ud = ctx->hbuf_in;
  cudaStream_t cs = ctx->cs;
  cudaEvent_t* ev_in = ctx->cev;
  cudaEvent_t* ev_out = ctx->cev + NSFR_COPY_CHUNKS;
  cudaEvent_t ev_start = ctx->cev[2 * NSFR_COPY_CHUNKS];
  // the copies start after the work already queued on the caller's stream
  CK(cudaEventRecord(ev_start, s), "cudaEventRecord");
  CK(cudaStreamWaitEvent(cs, ev_start, 0), "cudaStreamWaitEvent");
  for (int j = 0; j < nzc; ++j) {
    CK(cudaMemcpyAsync(ud + cb[j] * per, uh + cb[j] * per, (size_t)(cb[j + 1] - cb[j]) * per * sizeof(double),
                       cudaMemcpyHostToDevice, cs),
       "cudaMemcpyAsync(H2D)");
    CK(cudaEventRecord(ev_in[j], cs), "cudaEventRecord");
  }
  if (need_lam) CK(nsfr_wavespeed_begin(ctx, s), "cudaMemsetAsync(max)");
  // stage 0's source term (at time t) does not depend on the state
  if (ctx->src_on) CK(nsfr_launch_source(ctx, ctx->t, s), "manufactured_source_kernel");
  // stage 0 without dt: k = du/dt of chunk c into ustage
  auto stage0_chunk = [&](int c) -> nsfr_status {
    ctx->ff_b = cb[c];
    ctx->ff_e = cb[c + 1];
    cudaError_t err = nsfr_launch_face_flux(ctx, s);
    ctx->ff_b = 0;
    ctx->ff_e = -1;
    CK(err, "face_flux_kernel");
    return NSFR_OK;
  };
  auto stage0_volume = [&](int c) -> nsfr_status {
    ctx->vol_b = cb[c];
    ctx->vol_e = cb[c + 1];
    const cudaError_t err = launch_volume_any(ctx, ud, ctx->ustage, EPI_DUDT, nullptr, s);
    ctx->vol_b = 0;
    ctx->vol_e = -1;
    CK(err, "volume_kernel");
    return NSFR_OK;
  };
  for (int j = 0; j < nzc; ++j) {
    CK(cudaStreamWaitEvent(s, ev_in[j], 0), "cudaStreamWaitEvent");
    ctx->fs_b = cb[j];
    ctx->fs_e = cb[j + 1];
    const cudaError_t err = nsfr_launch_face_states(ctx, ud, s);
    ctx->fs_b = 0;
    ctx->fs_e = -1;
    CK(err, "face_state_kernel");
    if (need_lam) CK(nsfr_wavespeed_candidates(ctx, ud, cb[j], cb[j + 1], s), "max_wavespeed32_kernel");
    if (j >= 1) {
      if ((st = stage0_chunk(j - 1)) != NSFR_OK) return st;
      if (j >= 2 && (st = stage0_volume(j - 1)) != NSFR_OK) return st;
    }
  }
  if (need_lam) {
    CK(nsfr_wavespeed_finish(ctx, ud, s), "max_wavespeed_kernel");
    CK(cudaMemcpyAsync(ctx->umax_host, ctx->umax, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s),
       "cudaMemcpyAsync(max)");
  }
  if ((st = stage0_chunk(nzc - 1)) != NSFR_OK) return st;
  if (nzc >= 2 && (st = stage0_volume(nzc - 1)) != NSFR_OK) return st;
  if ((st = stage0_volume(0)) != NSFR_OK) return st;
  double dt = dt_fixed;
  if (need_lam) {
    st = read_flag(ctx, s);  // synchronises
    if (st != NSFR_OK) return st;
    double lam;
    std::memcpy(&lam, ctx->umax_host, sizeof(double));
    if (!(lam > 0.0)) return fail(ctx, NSFR_ERR_NONPHYSICAL, "zero or invalid wave speed");
    dt = cfl * ctx->dx / lam;
  }
  if (dt_used) *dt_used = dt;
  // the fused epilogue's stage-0 update: b_0 = 1/6, a_0 = 1/2
  const double b0 = 1.0 / 6.0, a0 = 0.5;
  CK(nsfr_launch_rk_first_update(ctx, ud, ctx->ustage, ctx->acc, b0 * dt, a0 * dt, s), "rk_first_update_kernel");
  for (int k = 1; k < 3 && st == NSFR_OK; ++k) st = rk_stage_device(ctx, ud, ctx->ustage, ctx->acc, k, dt, s);
  if (st == NSFR_OK)
    st = rk_stage_parts(ctx, ud, ctx->ustage, ctx->acc, 3, dt, s, PART_SOURCE | PART_FACE_STATES | PART_FACE_FLUX);
  if (st != NSFR_OK) return st;
  for (int j = 0; j < nzc; ++j) {
    ctx->vol_b = cb[j];
    ctx->vol_e = cb[j + 1];
    st = rk_stage_parts(ctx, ud, ctx->ustage, ctx->acc, 3, dt, s, PART_VOLUME);
    ctx->vol_b = 0;
    ctx->vol_e = -1;
    if (st != NSFR_OK) return st;
    CK(cudaEventRecord(ev_out[j], s), "cudaEventRecord");
    CK(cudaStreamWaitEvent(cs, ev_out[j], 0), "cudaStreamWaitEvent");
    CK(cudaMemcpyAsync(uh + cb[j] * per, ud + cb[j] * per, (size_t)(cb[j + 1] - cb[j]) * per * sizeof(double),
                       cudaMemcpyDeviceToHost, cs),
       "cudaMemcpyAsync(D2H)");
  }
  ctx->t += dt;
  CK(cudaStreamSynchronize(cs), "cudaStreamSynchronize");
  CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return NSFR_OK;
}

}  // namespace

void nsfr_prof_begin(nsfr_ctx* ctx, int kind, cudaStream_t s) {
  if (!ctx->prof_on || ctx->prof_n >= NSFR_PROF_CAP) return;
  ctx->prof_kind[ctx->prof_n] = kind;
  cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], s);
}

void nsfr_prof_end(nsfr_ctx* ctx, cudaStream_t s) {
  if (!ctx->prof_on || ctx->prof_n >= NSFR_PROF_CAP) return;
  cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], s);
  ctx->prof_n++;
}

extern "C" {

// nq = 0: collocated on ``nodes``; nq >= p+1: solution on the Lobatto nodes, nq GL points
static nsfr_status setup_common(const double* grid_nodes, int nx, int ny, int nz, int p_geo, int p, int nq,
                                double c, int vol_flux, int face_flux, double gamma, int precision, int nodes,
                                nsfr_ctx** out) {
  if (!out) return NSFR_ERR_ARG;
  *out = nullptr;
  if (!grid_nodes || nx < 1 || ny < 1 || nz < 1 || p < 1 || p > 7 || p_geo < 1 || p_geo > p || !(gamma > 1.0) ||
      (vol_flux != NSFR_FLUX_CHANDRASHEKAR && vol_flux != NSFR_FLUX_RANOCHA) ||
      (vol_flux == NSFR_FLUX_RANOCHA && precision != NSFR_FP64) || face_flux < NSFR_FACE_EC ||
      face_flux > NSFR_FACE_EC_ES ||
      (precision != NSFR_FP64 && precision != NSFR_FP32_BULK && precision != NSFR_FP32_BULK_FF) || (nodes != NSFR_NODES_GL && nodes != NSFR_NODES_LGL) ||
      !std::isfinite(c) || c < 0.0)
    return NSFR_ERR_ARG;
  nsfr_ctx* ctx = new (std::nothrow) nsfr_ctx();
  if (!ctx) return NSFR_ERR_OOM;
  ctx->nx = nx;
  ctx->ny = ny;
  ctx->nz = nz;
  ctx->ne = nx * ny * nz;
  ctx->p = p;
  ctx->uncol = nq > 0 ? 1 : 0;
  ctx->ns = p + 1;
  ctx->n = nq > 0 ? nq : p + 1;
  ctx->pg = p_geo;
  ctx->q = p_geo + 1;
  ctx->nv = ctx->n * ctx->n * ctx->n;
  ctx->nfp = ctx->n * ctx->n;
  ctx->nsv = ctx->ns * ctx->ns * ctx->ns;
  ctx->c = c;
  ctx->gamma = gamma;
  ctx->vol_flux = vol_flux;
  ctx->face_flux = face_flux;
  ctx->precision = precision;
  ctx->nodes = nodes;
  cudaGetDevice(&ctx->device);
  if (ctx->uncol) nsfr_build_ops_uncol(p, p_geo, nq, c, gamma, &ctx->ops, &ctx->gops);
  else nsfr_build_ops(p, p_geo, c, gamma, nodes, &ctx->ops, &ctx->gops);

  auto bail = [&](nsfr_status st) {
    free_all(ctx);
    delete ctx;
    return st;
  };
  const size_t ne = ctx->ne, nv = ctx->nv, nfp = ctx->nfp, nsv = ctx->nsv, q3 = (size_t)ctx->q * ctx->q * ctx->q;
  bool ok = dalloc(&ctx->ctrl, ne * q3 * 3) == cudaSuccess && dalloc(&ctx->metric, ne * 9 * nv) == cudaSuccess &&
            dalloc(&ctx->J, ne * nv) == cudaSuccess && dalloc(&ctx->invwj, ne * nv) == cudaSuccess &&
            dalloc(&ctx->wj, ne * nv) == cudaSuccess && dalloc(&ctx->nfp_plus, ne * 9 * nfp) == cudaSuccess &&
            dalloc(&ctx->xyz, ne * 3 * nsv) == cudaSuccess &&
            dalloc(&ctx->face, ne * 6 * NSFR_NFIELD * nfp) == cudaSuccess && dalloc(&ctx->nrec, ne * NSFR_NFIELD * nv) == cudaSuccess &&
            dalloc(&ctx->fstar, ne * 15 * nfp) == cudaSuccess && dalloc(&ctx->metric_s, ne * 9 * nv) == cudaSuccess &&
            dalloc(&ctx->nf_s, ne * 9 * nfp) == cudaSuccess &&
            dalloc(&ctx->ustage, ne * 5 * nsv) == cudaSuccess && dalloc(&ctx->acc, ne * 5 * nsv) == cudaSuccess &&
            dalloc(&ctx->flag, 1) == cudaSuccess && dalloc(&ctx->umax, 2) == cudaSuccess &&
            cudaMallocHost((void**)&ctx->flag_host, sizeof(int)) == cudaSuccess &&
            cudaMallocHost((void**)&ctx->umax_host, sizeof(unsigned long long)) == cudaSuccess;
  if (ok && ctx->uncol && ctx->n == ctx->ns) ok = dalloc(&ctx->uq, ne * 5 * nv) == cudaSuccess;
  if (ok && precision == NSFR_FP64)
    ok = dalloc(&ctx->pair_rows, nsfr_pair_rows_count(ctx->n, ctx->ne)) == cudaSuccess;
  if (ok && precision != NSFR_FP64)
    ok = dalloc(&ctx->metric32, ne * 18 * nv) == cudaSuccess && dalloc(&ctx->nfp_plus32, ne * 18 * nfp) == cudaSuccess &&
         dalloc(&ctx->invwj32, ne * nv) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return bail(NSFR_ERR_OOM);
  }
  if (cudaMemset(ctx->flag, 0, sizeof(int)) != cudaSuccess) return bail(NSFR_ERR_CUDA);
  const size_t cbytes = ne * q3 * 3 * sizeof(double);
  if (cudaMemcpy(ctx->ctrl, grid_nodes, cbytes, cudaMemcpyDefault) != cudaSuccess) return bail(NSFR_ERR_CUDA);
  // node spacing for the CFL step: domain extent of the control points
  {
    std::vector<double> h(ne * q3 * 3);
    if (cudaMemcpy(h.data(), ctx->ctrl, cbytes, cudaMemcpyDeviceToHost) != cudaSuccess) return bail(NSFR_ERR_CUDA);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (size_t i = 0; i < h.size(); ++i) {
      const int cc = (int)(i % 3);
      lo[cc] = std::fmin(lo[cc], h[i]);
      hi[cc] = std::fmax(hi[cc], h[i]);
    }
    const int N[3] = {nx, ny, nz};
    double dx = 1e300;
    for (int d = 0; d < 3; ++d) dx = std::fmin(dx, (hi[d] - lo[d]) / (N[d] * (p + 1.0)));
    ctx->dx = dx;
  }
  if (nsfr_launch_metrics(ctx, 0) != cudaSuccess) return bail(NSFR_ERR_CUDA);
  if (nsfr_launch_scaled_rows(ctx, 0) != cudaSuccess) return bail(NSFR_ERR_CUDA);
  if (precision != NSFR_FP64 && nsfr_launch_bulk_tables(ctx, 0) != cudaSuccess) return bail(NSFR_ERR_CUDA);
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(NSFR_ERR_CUDA);
  int f = 0;
  if (cudaMemcpy(&f, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return bail(NSFR_ERR_CUDA);
  if (f & 2) return bail(NSFR_ERR_MESH);
  *out = ctx;
  return NSFR_OK;
}

nsfr_status nsfr_setup(const double* grid_nodes, int nx, int ny, int nz, int p_geo, int p, double c,
                       int vol_flux, int face_flux, double gamma, int precision, int nodes, nsfr_ctx** out) {
  if (nodes != NSFR_NODES_GL && nodes != NSFR_NODES_LGL) {
    if (out) *out = nullptr;
    return NSFR_ERR_ARG;
  }
  return setup_common(grid_nodes, nx, ny, nz, p_geo, p, 0, c, vol_flux, face_flux, gamma, precision, nodes, out);
}

nsfr_status nsfr_setup_uncollocated(const double* grid_nodes, int nx, int ny, int nz, int p_geo, int p, int nq,
                                    double c, int vol_flux, int face_flux, double gamma, int precision,
                                    nsfr_ctx** out) {
  if (nq < p + 1 || nq > NSFR_MAXN || (precision != NSFR_FP64 && precision != NSFR_FP32_BULK)) {
    if (out) *out = nullptr;
    return NSFR_ERR_ARG;
  }
  return setup_common(grid_nodes, nx, ny, nz, p_geo, p, nq, c, vol_flux, face_flux, gamma, precision,
                      NSFR_NODES_LGL, out);
}

nsfr_status nsfr_residual(nsfr_ctx* ctx, const double* u, double* dudt, void* stream) {
  return residual_any(ctx, u, dudt, EPI_DUDT, stream);
}

nsfr_status nsfr_residual_raw(nsfr_ctx* ctx, const double* u, double* R, void* stream) {
  return residual_any(ctx, u, R, EPI_RAW, stream);
}

nsfr_status nsfr_rk_step(nsfr_ctx* ctx, double* u, double cfl, double dt_fixed, double* dt_used, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (!u) return fail(ctx, NSFR_ERR_ARG, "NULL state");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  if (is_device_ptr(u)) return rk_step_device(ctx, u, cfl, dt_fixed, dt_used, s);
  if (!ctx->uncol) return rk_step_host(ctx, u, cfl, dt_fixed, dt_used, s);
  nsfr_status st = ensure_host_buffers(ctx);
  if (st != NSFR_OK) return st;
  const size_t bytes = state_count(ctx) * sizeof(double);
  CK(cudaMemcpyAsync(ctx->hbuf_in, u, bytes, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(H2D)");
  st = rk_step_device(ctx, ctx->hbuf_in, cfl, dt_fixed, dt_used, s);
  if (st != NSFR_OK) return st;
  CK(cudaMemcpyAsync(u, ctx->hbuf_in, bytes, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(D2H)");
  CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return NSFR_OK;
}

nsfr_status nsfr_rk_stage(nsfr_ctx* ctx, double* u, double* ustage, double* acc, int stage, double dt,
                          int e_begin, int e_end, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (!u || !ustage || !acc || stage < 0 || stage > 3 || !(dt > 0.0))
    return fail(ctx, NSFR_ERR_ARG, "nsfr_rk_stage: NULL buffer, stage outside 0..3 or dt <= 0");
  if (e_begin < 0 || e_end < e_begin || e_end > ctx->ne)
    return fail(ctx, NSFR_ERR_ARG, "nsfr_rk_stage: element range outside 0 <= e_begin <= e_end <= N_e");
  if (!is_device_ptr(u) || !is_device_ptr(ustage) || !is_device_ptr(acc))
    return fail(ctx, NSFR_ERR_ARG, "nsfr_rk_stage takes device buffers");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  ctx->vol_b = e_begin;
  ctx->vol_e = e_end;
  const nsfr_status st = rk_stage_device(ctx, u, ustage, acc, stage, dt, s);
  ctx->vol_b = 0;
  ctx->vol_e = -1;
  return st;
}

nsfr_status nsfr_max_wavespeed(nsfr_ctx* ctx, const double* u, double* lam, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (!u || !lam) return fail(ctx, NSFR_ERR_ARG, "NULL buffer");
  if (!is_device_ptr(u)) return fail(ctx, NSFR_ERR_ARG, "nsfr_max_wavespeed takes a device state");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  return max_wavespeed(ctx, u, lam, s);
}

nsfr_status nsfr_entropy(nsfr_ctx* ctx, const double* u, double* out, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (!u || !out) return fail(ctx, NSFR_ERR_ARG, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  if (!ctx->rtmp) CK(dalloc(&ctx->rtmp, state_count(ctx)), "cudaMalloc(rtmp)");
  const int nb = nsfr_diag_blocks(ctx);
  if (!ctx->red || ctx->red_cap < nb) {
    if (ctx->red) cudaFree(ctx->red);
    if (ctx->red_host) cudaFreeHost(ctx->red_host);
    ctx->red = nullptr;
    ctx->red_host = nullptr;
    CK(dalloc(&ctx->red, (size_t)nb * 28), "cudaMalloc(red)");
    CK(cudaMallocHost((void**)&ctx->red_host, (size_t)nb * 28 * sizeof(double)), "cudaMallocHost(red)");
    ctx->red_cap = nb;
  }
  const double* ud = u;
  if (!is_device_ptr(u)) {
    nsfr_status st = ensure_host_buffers(ctx);
    if (st != NSFR_OK) return st;
    CK(cudaMemcpyAsync(ctx->hbuf_in, u, state_count(ctx) * sizeof(double), cudaMemcpyHostToDevice, s),
       "cudaMemcpyAsync(H2D)");
    ud = ctx->hbuf_in;
  }
  nsfr_status st = residual_device(ctx, ud, ctx->rtmp, EPI_RAW, s);
  if (st != NSFR_OK) return st;
  CK(nsfr_launch_diagnostics(ctx, ud, ctx->rtmp, ctx->red, nb, s), "diagnostics_kernel");
  CK(cudaMemcpyAsync(ctx->red_host, ctx->red, (size_t)nb * 28 * sizeof(double), cudaMemcpyDeviceToHost, s),
     "cudaMemcpyAsync(partials)");
  st = read_flag(ctx, s);
  if (st != NSFR_OK) return st;
  // finish the compensated sums over blocks (Neumaier on the leading parts)
  for (int k = 0; k < 14; ++k) {
    double sum = 0.0, comp = 0.0;
    for (int b = 0; b < nb; ++b) {
      const double x = ctx->red_host[((size_t)b * 14 + k) * 2];
      comp += ctx->red_host[((size_t)b * 14 + k) * 2 + 1];
      const double t = sum + x;
      if (std::fabs(sum) >= std::fabs(x)) comp += (sum - t) + x;
      else comp += (x - t) + sum;
      sum = t;
    }
    out[k] = sum + comp;
  }
  return NSFR_OK;
}

nsfr_status nsfr_vjp(nsfr_ctx* ctx, const double* u, const double* dudt_bar, double* u_bar, double* x_bar,
                     void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (ctx->precision != NSFR_FP64) return fail(ctx, NSFR_ERR_STATE, "nsfr_vjp needs an FP64 context");
  if (ctx->uncol && x_bar)
    return fail(ctx, NSFR_ERR_STATE, "nsfr_vjp of an uncollocated context offers the state cotangent only");
  if (ctx->face_flux != NSFR_FACE_EC) return fail(ctx, NSFR_ERR_STATE, "nsfr_vjp supports the EC face flux");
  if (ctx->vol_flux != NSFR_FLUX_CHANDRASHEKAR)
    return fail(ctx, NSFR_ERR_STATE, "nsfr_vjp supports the Chandrashekar volume flux");
  if (ctx->src_on && x_bar)
    return fail(ctx, NSFR_ERR_STATE, "nsfr_vjp with x_bar does not differentiate a volume source");
  if (!u || !dudt_bar || !u_bar) return fail(ctx, NSFR_ERR_ARG, "NULL buffer");
  if (!is_device_ptr(u) || !is_device_ptr(dudt_bar) || !is_device_ptr(u_bar) || (x_bar && !is_device_ptr(x_bar)))
    return fail(ctx, NSFR_ERR_ARG, "nsfr_vjp takes device buffers");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->last_stream = s;
  const size_t ne = ctx->ne, nv = ctx->nv, nfp = ctx->nfp;
  if (!ctx->vjp_fown) {
    CK(dalloc(&ctx->vjp_fown, ne * 30 * nfp), "cudaMalloc(vjp)");
    CK(dalloc(&ctx->vjp_fnbr, ne * 30 * nfp), "cudaMalloc(vjp)");
    CK(dalloc(&ctx->vjp_nfbar, ne * 18 * nfp), "cudaMalloc(vjp)");
    CK(dalloc(&ctx->vjp_mbar, ne * 9 * nv), "cudaMalloc(vjp)");
    CK(dalloc(&ctx->vjp_jbar, ne * nv), "cudaMalloc(vjp)");
  }
  if (ctx->uncol && !ctx->vjp_pbq) CK(dalloc(&ctx->vjp_pbq, ne * 5 * nv), "cudaMalloc(vjp)");
  if (!ctx->rtmp) CK(dalloc(&ctx->rtmp, state_count(ctx)), "cudaMalloc(rtmp)");
  CK(cudaMemsetAsync(ctx->vjp_mbar, 0, ne * 9 * nv * sizeof(double), s), "cudaMemsetAsync");
  CK(cudaMemsetAsync(ctx->vjp_jbar, 0, ne * nv * sizeof(double), s), "cudaMemsetAsync");
  CK(nsfr_launch_face_states(ctx, u, s), "face_state_kernel");
  if (x_bar) {
    CK(nsfr_launch_face_flux(ctx, s), "face_flux_kernel");
    CK(nsfr_launch_volume(ctx, u, ctx->rtmp, EPI_RAW, nullptr, s), "volume_kernel(raw)");
  }
  CK(nsfr_launch_vjp(ctx, u, dudt_bar, u_bar, x_bar, s), "vjp kernels");
  return NSFR_OK;
}

nsfr_status nsfr_set_source(nsfr_ctx* ctx, int kind, double t) {
  if (!ctx) return NSFR_ERR_ARG;
  if (kind != NSFR_SOURCE_NONE && kind != NSFR_SOURCE_MANUFACTURED)
    return fail(ctx, NSFR_ERR_ARG, "unknown source kind");
  if (!(t == t)) return fail(ctx, NSFR_ERR_ARG, "t is NaN");
  if (kind != NSFR_SOURCE_NONE && ctx->uncol)
    return fail(ctx, NSFR_ERR_STATE, "volume sources need a collocated context");
  if (kind != NSFR_SOURCE_NONE && !ctx->src) CK(dalloc(&ctx->src, state_count(ctx)), "cudaMalloc(source)");
  ctx->source = kind;
  ctx->src_on = kind == NSFR_SOURCE_NONE ? nullptr : ctx->src;
  ctx->t = t;
  return NSFR_OK;
}

nsfr_status nsfr_get_time(const nsfr_ctx* ctx, double* t) {
  if (!ctx || !t) return NSFR_ERR_ARG;
  *t = ctx->t;
  return NSFR_OK;
}

nsfr_status nsfr_node_coords(nsfr_ctx* ctx, double* xyz, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (!xyz) return fail(ctx, NSFR_ERR_ARG, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(xyz, ctx->xyz, (size_t)ctx->ne * 3 * ctx->nsv * sizeof(double), cudaMemcpyDefault, s),
     "cudaMemcpyAsync(xyz)");
  CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return NSFR_OK;
}

nsfr_status nsfr_get_metrics(nsfr_ctx* ctx, double* C, double* J, double* Cf, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ne = ctx->ne, nv = ctx->nv, nfp = ctx->nfp;
  if (C) CK(cudaMemcpyAsync(C, ctx->metric, ne * 9 * nv * sizeof(double), cudaMemcpyDefault, s), "copy C");
  if (J) CK(cudaMemcpyAsync(J, ctx->J, ne * nv * sizeof(double), cudaMemcpyDefault, s), "copy J");
  if (Cf) CK(cudaMemcpyAsync(Cf, ctx->nfp_plus, ne * 9 * nfp * sizeof(double), cudaMemcpyDefault, s), "copy Cf");
  CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return NSFR_OK;
}

nsfr_status nsfr_set_metrics(nsfr_ctx* ctx, const double* C, const double* J, const double* Cf, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (!C || !J || !Cf) return fail(ctx, NSFR_ERR_ARG, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ne = ctx->ne, nv = ctx->nv, nfp = ctx->nfp;
  CK(cudaMemcpyAsync(ctx->metric, C, ne * 9 * nv * sizeof(double), cudaMemcpyDefault, s), "copy C");
  CK(cudaMemcpyAsync(ctx->J, J, ne * nv * sizeof(double), cudaMemcpyDefault, s), "copy J");
  CK(cudaMemcpyAsync(ctx->nfp_plus, Cf, ne * 9 * nfp * sizeof(double), cudaMemcpyDefault, s), "copy Cf");
  CK(nsfr_launch_jacobian_derived(ctx, s), "jacobian_derived_kernel");
  CK(nsfr_launch_scaled_rows(ctx, s), "scaled_rows_kernel");
  if (ctx->precision != NSFR_FP64) CK(nsfr_launch_bulk_tables(ctx, s), "bulk_tables_kernel");
  return read_flag(ctx, s);
}

nsfr_status nsfr_quadrature(nsfr_ctx* ctx, double* wj, void* stream) {
  if (!ctx) return NSFR_ERR_ARG;
  if (!wj) return fail(ctx, NSFR_ERR_ARG, "NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(wj, ctx->wj, (size_t)ctx->ne * ctx->nv * sizeof(double), cudaMemcpyDefault, s), "copy wJ");
  CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
  return NSFR_OK;
}

nsfr_status nsfr_info(const nsfr_ctx* ctx, long long* out) {
  if (!ctx || !out) return NSFR_ERR_ARG;
  out[0] = ctx->ne;
  out[1] = ctx->p;
  out[2] = ctx->nsv;
  out[3] = ctx->pg;
  out[4] = ctx->precision;
  return NSFR_OK;
}

nsfr_status nsfr_check(nsfr_ctx* ctx) {
  if (!ctx) return NSFR_ERR_ARG;
  return read_flag(ctx, ctx->last_stream);
}

nsfr_status nsfr_profile(nsfr_ctx* ctx, int on) {
  if (!ctx) return NSFR_ERR_ARG;
  if (on && !ctx->prof_ev) {
    ctx->prof_ev = new (std::nothrow) cudaEvent_t[2 * NSFR_PROF_CAP];
    ctx->prof_kind = new (std::nothrow) int[NSFR_PROF_CAP];
    if (!ctx->prof_ev || !ctx->prof_kind) return fail(ctx, NSFR_ERR_OOM, "profile buffers");
    for (int i = 0; i < 2 * NSFR_PROF_CAP; ++i) CK(cudaEventCreate(&ctx->prof_ev[i]), "cudaEventCreate");
  }
  ctx->prof_on = on ? 1 : 0;
  if (on) ctx->prof_n = 0;
  return NSFR_OK;
}

nsfr_status nsfr_profile_read(nsfr_ctx* ctx, double* ms, long long* count) {
  if (!ctx) return NSFR_ERR_ARG;
  double t[NSFR_NKERNELS] = {0};
  long long c[NSFR_NKERNELS] = {0};
  for (int i = 0; i < ctx->prof_n; ++i) {
    CK(cudaEventSynchronize(ctx->prof_ev[2 * i + 1]), "cudaEventSynchronize");
    float el = 0.f;
    CK(cudaEventElapsedTime(&el, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]), "cudaEventElapsedTime");
    t[ctx->prof_kind[i]] += el;
    c[ctx->prof_kind[i]] += 1;
  }
  for (int k = 0; k < NSFR_NKERNELS; ++k) {
    if (ms) ms[k] = t[k];
    if (count) count[k] = c[k];
  }
  return NSFR_OK;
}

nsfr_status nsfr_math_eval(int fn, const double* x, double* y, long long n, void* stream) {
  if (fn < NSFR_FN_LOG || fn > NSFR_FN_I2D || n < 0) return NSFR_ERR_ARG;
  if (n == 0) return NSFR_OK;
  if (!x || !y || !is_device_ptr(x) || !is_device_ptr(y)) return NSFR_ERR_ARG;
  return nsfr_launch_math_eval(fn, x, y, n, (cudaStream_t)stream) == cudaSuccess ? NSFR_OK : NSFR_ERR_CUDA;
}

long long nsfr_kernel_launches(const nsfr_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* nsfr_last_error(const nsfr_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

void nsfr_destroy(nsfr_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
}

}  // extern "C"
