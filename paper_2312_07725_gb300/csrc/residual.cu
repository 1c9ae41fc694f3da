// NSFR-EC residual kernels (FP64 path).
//
// K1  face_state_kernel: entropy projection to the faces (Sec. "Nonlinearly
//     Stable Flux Reconstruction", entropy projected variables).  With the
//     collocated GL basis v^ = v(u) nodal, and each face state is
//     u~_f = u(t_s . v) along the line that ends on the face node.  The
//     kernel stores the primitive record of u~_f (rho, u, beta, ln rho,
//     ln beta, |u|^2), which is all the face fluxes need.
// K2  volume_kernel: Eq. NSFR with the sum-factorised Hadamard products
//     (Sec. "Scalable Evaluations"), one thread per line of an element:
//       volume:  R_a += sum_{b} w_perp S1[a,b] f_s(u_a, u_b) . (C_a + C_b)/2
//                (each unordered pair evaluated once: S1 is skew),
//       hybrid:  R_a += s w_perp t_s[a] (phi_a + f* - sum_b t_s[b] phi_b),
//                phi_a = f_s(u_a, u~_f) . (C_a + C_f)/2,
//       surface: f* = f*(u~_L, u~_R; C_f) with the shared face row C_f;
//     the three directions' line sums meet in shared memory, then the
//     epilogue applies the weight-adjusted inverse (Eq. weight-adj ESFR mass,
//     Pi~^T, 1/(w J), Pi~, each a 1D contraction per direction) and either
//     stores du/dt or performs the RK stage update in place.
#include "physics.cuh"

namespace {

// elements per CTA and CTA size (one thread per line, 3 n^2 lines per element)
constexpr int epb_for(int n) { return n == 2 ? 16 : n == 3 ? 8 : n <= 5 ? 4 : n == 6 ? 2 : 1; }
constexpr int threads_for(int n) { return epb_for(n) * 3 * n * n; }

__device__ __forceinline__ int nbr_index(int e, int d, int side, int nx, int ny, int nz) {
  int ex = e % nx, ey = (e / nx) % ny, ez = e / (nx * ny);
  const int st = side ? 1 : -1;
  if (d == 0) ex = (ex + st + nx) % nx;
  else if (d == 1) ey = (ey + st + ny) % ny;
  else ez = (ez + st + nz) % nz;
  return ex + nx * (ey + ny * ez);
}

// node index of line node a for line (d, l0, l1): base + a * stride
template <int N>
__device__ __forceinline__ void line_geometry(int d, int l0, int l1, int& base, int& stride) {
  if (d == 0) { base = N * (l0 + N * l1); stride = 1; }
  else if (d == 1) { base = l0 + N * N * l1; stride = N; }
  else { base = l0 + N * l1; stride = N * N; }
}

template <int N>
__global__ void __launch_bounds__(threads_for(N)) face_state_kernel(const double* __restrict__ u, OpsGL ops,
                                                                    double* __restrict__ face, int ne, int* flag) {
  constexpr int NV = N * N * N, NFP = N * N, NL = 3 * NFP;
  extern __shared__ double sm[];
  const int epb = blockDim.x / NL;
  const int e0 = blockIdx.x * epb;
  const double g = ops.gamma, gm1 = g - 1.0;
  // v(u) at every node of the block's elements
  for (int t = threadIdx.x; t < epb * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV, e = e0 + le;
    if (e >= ne) continue;
    const double* ue = u + (size_t)e * 5 * NV + node;
    const double r = ue[0], m0 = ue[NV], m1 = ue[2 * NV], m2 = ue[3 * NV], E = ue[4 * NV];
    const double ir = 1.0 / r;
    const double u0 = m0 * ir, u1 = m1 * ir, u2 = m2 * ir;
    const double q2 = u0 * u0 + u1 * u1 + u2 * u2;
    const double p = gm1 * (E - 0.5 * r * q2);
    if (!(r > 0.0) || !(p > 0.0)) atomicOr(flag, 1);
    const double b = 0.5 * r / p;
    const double s = log(p) - g * log(r);
    double* v = sm + (size_t)le * 5 * NV + node;
    v[0] = (g - s) / gm1 - b * q2;
    v[NV] = 2.0 * b * u0;
    v[2 * NV] = 2.0 * b * u1;
    v[3 * NV] = 2.0 * b * u2;
    v[4 * NV] = -2.0 * b;
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
      am += ops.tm[a] * x;
      ap += ops.tp[a] * x;
    }
    vm[k] = am;
    vp[k] = ap;
  }
  const double ln2 = 0.69314718055994530942;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const double* w = s ? vp : vm;
    if (!(w[4] < 0.0)) atomicOr(flag, 1);
    const double b = -0.5 * w[4];
    const double iv5 = 1.0 / w[4];
    const double u0 = -w[1] * iv5, u1 = -w[2] * iv5, u2 = -w[3] * iv5;
    const double q2 = u0 * u0 + u1 * u1 + u2 * u2;
    const double sent = g - gm1 * (w[0] + b * q2);
    const double L5 = log(-w[4]);          // ln(2 beta)
    const double lr = -(sent + L5) / gm1;  // s = (1-gamma) ln rho - ln(2 beta)
    Prim P;
    P.r = exp(lr);
    P.u0 = u0;
    P.u1 = u1;
    P.u2 = u2;
    P.b = b;
    P.lr = lr;
    P.lb = L5 - ln2;
    P.q2 = q2;
    store_prim(face + (((size_t)e * 6 + 2 * d + s) * NSFR_NFIELD) * NFP + line, NFP, P);
  }
}

// ``u`` is not __restrict__: in the middle RK stages the epilogue writes the
// next stage state over it (each CTA only over its own elements, after its
// own reads).
template <int N>
__global__ void __launch_bounds__(threads_for(N)) volume_kernel(const double* u, const double* __restrict__ metric,
                                                                const double* __restrict__ nf_plus,
                                                                const double* __restrict__ face,
                                                                const double* __restrict__ invwj, OpsGL ops, int nx,
                                                                int ny, int nz, int ne, int face_kind, int epi,
                                                                RkArgs rk, double* out, int* flag) {
  constexpr int NV = N * N * N, NFP = N * N, NL = 3 * NFP;
  extern __shared__ double sm[];
  const int epb = blockDim.x / NL;
  const int e0 = blockIdx.x * epb;
  double* P = sm;                                   // [epb][8][NV] node primitives
  double* Ms = P + (size_t)epb * NSFR_NFIELD * NV;  // [epb][9][NV] metric
  double* Rs = Ms + (size_t)epb * 9 * NV;           // [epb][5][NV] residual
  double* Ts = P;                                   // epilogue temp (aliases P)
  const double g = ops.gamma, inv2gm1 = 0.5 / (g - 1.0);

  // prologue: primitive records and metric rows of the block's elements
  for (int t = threadIdx.x; t < epb * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV, e = e0 + le;
    if (e >= ne) continue;
    const double* ue = u + (size_t)e * 5 * NV + node;
    Prim a = prim_from_conserved(ue[0], ue[NV], ue[2 * NV], ue[3 * NV], ue[4 * NV], g, flag);
    store_prim(P + (size_t)le * NSFR_NFIELD * NV + node, NV, a);
  }
  for (int t = threadIdx.x; t < epb * 9 * NV; t += blockDim.x) {
    const int le = t / (9 * NV), e = e0 + le;
    if (e >= ne) continue;
    Ms[t] = metric[(size_t)e0 * 9 * NV + t];
  }
  __syncthreads();

  const int le = threadIdx.x / NL, l = threadIdx.x % NL, e = e0 + le;
  const bool valid = (le < epb) && (e < ne);
  const int d = l / NFP, line = l % NFP, l0 = line % N, l1 = line / N;
  int base, stride;
  line_geometry<N>(d, l0, l1, base, stride);
  double R[N][5];
#pragma unroll
  for (int a = 0; a < N; ++a)
#pragma unroll
    for (int k = 0; k < 5; ++k) R[a][k] = 0.0;

  if (valid) {
    const double* Pe = P + (size_t)le * NSFR_NFIELD * NV + base;
    const double* Me = Ms + ((size_t)le * 9 + 3 * d) * NV + base;
    const double wperp = ops.w[l0] * ops.w[l1];
    // volume-volume pairs along the line
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const Prim A = load_prim(Pe + a * stride, NV);
      const double na0 = Me[a * stride], na1 = Me[NV + a * stride], na2 = Me[2 * NV + a * stride];
#pragma unroll
      for (int b = a + 1; b < N; ++b) {
        const Prim B = load_prim(Pe + b * stride, NV);
        const double n0 = 0.5 * (na0 + Me[b * stride]);
        const double n1 = 0.5 * (na1 + Me[NV + b * stride]);
        const double n2 = 0.5 * (na2 + Me[2 * NV + b * stride]);
        double F[5];
        ec_flux(A, B, n0, n1, n2, inv2gm1, F);
        const double c = wperp * ops.S1[a * N + b];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          R[a][k] += c * F[k];
          R[b][k] -= c * F[k];
        }
      }
    }
    // hybrid volume-face terms and face fluxes, both ends of the line
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int enb = nbr_index(e, d, s, nx, ny, nz);
      const double* fo = face + (((size_t)e * 6 + 2 * d + s) * NSFR_NFIELD) * NFP + line;
      const double* fn = face + (((size_t)enb * 6 + 2 * d + 1 - s) * NSFR_NFIELD) * NFP + line;
      const double* nf = nf_plus + (((size_t)(s ? e : enb) * 3 + d) * 3) * NFP + line;
      const double f0 = nf[0], f1 = nf[NFP], f2 = nf[2 * NFP];
      const Prim Fo = load_prim(fo, NFP);
      const Prim Fn = load_prim(fn, NFP);
      double fs[5];
      if (s) face_flux(Fo, Fn, f0, f1, f2, g, inv2gm1, face_kind, fs);
      else face_flux(Fn, Fo, f0, f1, f2, g, inv2gm1, face_kind, fs);
      const double* t = s ? ops.tp : ops.tm;
      const double sw = (s ? 1.0 : -1.0) * wperp;
      double tphi[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const Prim A = load_prim(Pe + a * stride, NV);
        double F[5];
        ec_flux(A, Fo, 0.5 * (Me[a * stride] + f0), 0.5 * (Me[NV + a * stride] + f1),
                0.5 * (Me[2 * NV + a * stride] + f2), inv2gm1, F);
        const double ta = t[a];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          tphi[k] += ta * F[k];
          R[a][k] += sw * ta * F[k];
        }
      }
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int k = 0; k < 5; ++k) R[a][k] += sw * t[a] * (fs[k] - tphi[k]);
    }
  }
  __syncthreads();  // P and Ms are no longer read
  // the three directions meet in shared memory (fixed order: d = 0, 1, 2)
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    if (valid && d == dd) {
      double* Re = Rs + (size_t)le * 5 * NV + base;
#pragma unroll
      for (int a = 0; a < N; ++a)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          if (dd == 0) Re[k * NV + a * stride] = R[a][k];
          else Re[k * NV + a * stride] += R[a][k];
        }
    }
    __syncthreads();
  }

  const int nel = min(epb, ne - e0);
  const int total = nel * 5 * NV;
  double* X = Rs;
  if (epi != EPI_RAW) {
    if (ops.has_K) {
      // Pi~^T along xi, eta, zeta; 1/(w J); Pi~ along xi, eta, zeta
      double* src = Rs;
      double* dst = Ts;
#pragma unroll 1
      for (int pass = 0; pass < 7; ++pass) {
        if (pass == 3) {
          for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int lq = t / (5 * NV), node = t % NV;
            src[t] *= invwj[(size_t)(e0 + lq) * NV + node];
          }
          __syncthreads();
          continue;
        }
        const int dd = (pass < 3) ? pass : pass - 4;
        const bool transpose = pass < 3;
        const int st = (dd == 0) ? 1 : (dd == 1 ? N : N * N);
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
          const int node = t % NV;
          const int r = (node / st) % N;
          const double* col = src + (t - r * st);
          double acc = 0.0;
#pragma unroll
          for (int b = 0; b < N; ++b)
            acc += (transpose ? ops.Pi1[b * N + r] : ops.Pi1[r * N + b]) * col[b * st];
          dst[t] = acc;
        }
        __syncthreads();
        double* tmp = src;
        src = dst;
        dst = tmp;
      }
      X = src;
    } else {
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int lq = t / (5 * NV), node = t % NV;
        X[t] *= invwj[(size_t)(e0 + lq) * NV + node];
      }
      __syncthreads();
    }
  }
  // store
  const size_t off = (size_t)e0 * 5 * NV;
  if (epi == EPI_RAW) {
    for (int t = threadIdx.x; t < total; t += blockDim.x) out[off + t] = X[t];
  } else if (epi == EPI_DUDT) {
    for (int t = threadIdx.x; t < total; t += blockDim.x) out[off + t] = -X[t];
  } else {
    const double bdt = rk.b * rk.dt, adt = rk.a_next * rk.dt;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const double k = -X[t];
      if (rk.last) {
        rk.unext[off + t] = rk.acc[off + t] + bdt * k;
      } else {
        const double u0 = rk.u0[off + t];
        rk.acc[off + t] = (rk.first ? u0 : rk.acc[off + t]) + bdt * k;
        rk.unext[off + t] = u0 + adt * k;
      }
    }
  }
}

template <int N>
cudaError_t launch_face_n(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  constexpr int NV = N * N * N;
  constexpr int epb = epb_for(N);
  const int grid = (ctx->ne + epb - 1) / epb;
  const size_t smem = (size_t)epb * 5 * NV * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(face_state_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  nsfr_prof_begin(ctx, 1, s);
  face_state_kernel<N><<<grid, threads_for(N), smem, s>>>(u, ctx->ops, ctx->face, ctx->ne, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_volume_n(nsfr_ctx* ctx, const double* u, double* out, int epi, const RkArgs* rk,
                            cudaStream_t s) {
  constexpr int NV = N * N * N;
  constexpr int epb = epb_for(N);
  const int grid = (ctx->ne + epb - 1) / epb;
  const size_t smem = (size_t)epb * (NSFR_NFIELD + 9 + 5) * NV * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(volume_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  RkArgs r = rk ? *rk : RkArgs{};
  nsfr_prof_begin(ctx, 2, s);
  volume_kernel<N><<<grid, threads_for(N), smem, s>>>(u, ctx->metric, ctx->nfp_plus, ctx->face, ctx->invwj,
                                                      ctx->ops, ctx->nx, ctx->ny, ctx->nz, ctx->ne, ctx->face_flux,
                                                      epi, r, out, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace

cudaError_t nsfr_launch_face_states(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
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
#include <mutex>

static __device__ __align__(256) unsigned char g_static_scratch[NSFR_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mu;
void* g_static_addr[256] = {nullptr};  // device address of g_static_scratch, per device ordinal
}  // namespace

extern "C" nsfr_status nsfr_residual_static(const double* u, const double* C, const double* J, const double* Cf,
                                            int nx, int ny, int nz, int p, double c, int face_flux, double gamma,
                                            double* dudt, void* stream) {
  if (!u || !C || !J || !Cf || !dudt || nx < 1 || ny < 1 || nz < 1 || p < 1 || p > 7 || !(gamma > 1.0) ||
      !(c >= 0.0) || (face_flux != NSFR_FACE_EC && face_flux != NSFR_FACE_EC_ROE))
    return NSFR_ERR_ARG;
  const size_t ne = (size_t)nx * ny * nz, n = p + 1, nv = n * n * n, nfp = n * n;
  const size_t face_bytes = ne * 6 * NSFR_NFIELD * nfp * sizeof(double);
  const size_t jac_bytes = ne * nv * sizeof(double);
  const size_t need = 256 + face_bytes + 2 * jac_bytes;  // error word (padded), faces, 1/(wJ), wJ
  if (need > NSFR_STATIC_SCRATCH_BYTES || ne > (size_t)0x7fffffff) return NSFR_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NSFR_ERR_CUDA;
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_static_scratch) != cudaSuccess || !addr) return NSFR_ERR_CUDA;
      g_static_addr[dev] = addr;
    }
    base = (unsigned char*)g_static_addr[dev];
  }
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
  ctx.c = c;
  ctx.gamma = gamma;
  ctx.vol_flux = NSFR_FLUX_CHANDRASHEKAR;
  ctx.face_flux = face_flux;
  ctx.precision = NSFR_FP64;
  ctx.device = dev;
  nsfr_build_ops(p, p, c, gamma, &ctx.ops, &ctx.gops);
  ctx.flag = (int*)base;
  ctx.face = (double*)(base + 256);
  ctx.invwj = (double*)(base + 256 + face_bytes);
  ctx.wj = (double*)(base + 256 + face_bytes + jac_bytes);
  ctx.metric = const_cast<double*>(C);
  ctx.J = const_cast<double*>(J);
  ctx.nfp_plus = const_cast<double*>(Cf);
  if (cudaMemsetAsync(ctx.flag, 0, sizeof(int), s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (nsfr_launch_jacobian_derived(&ctx, s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (nsfr_launch_face_states(&ctx, u, s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (nsfr_launch_volume(&ctx, u, dudt, EPI_DUDT, nullptr, s) != cudaSuccess) return NSFR_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, ctx.flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return NSFR_ERR_CUDA;
  if (flag & 2) return NSFR_ERR_MESH;
  if (flag & 1) return NSFR_ERR_NONPHYSICAL;
  return NSFR_OK;
}
