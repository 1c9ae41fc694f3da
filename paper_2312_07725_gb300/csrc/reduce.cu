// Reductions: the CFL wave speed and the scheme's diagnostics.
//
// max_i (|u_i| + a_i) sets the RK4 step (Sec. "Results": adaptive step from
// the maximum wave speed).  The diagnostics are the quantities the paper
// checks: the semi-discrete entropy rate -sum v(u_i) . R_i (Sec. "Nonlinear
// Stability"), the conserved totals Q = sum W J Pi~^{-1} u of the
// weight-adjusted scheme (Sec. "Global Conservation"), sum R, the entropy
// S = sum W J U(u) and the kinetic energy.  Sums are compensated (Neumaier)
// per thread, combined with TwoSum across the block, and the per-block
// (sum, error) pairs are finished on the host.
#include <cfloat>

#include "ffloat.cuh"
#include "kernel_common.cuh"
#include "nsfr_internal.h"

namespace {

// The maximum is found in two passes over the state.  The first evaluates
// |u| + a in FP32 (the state rounded to float by integer operations, so that
// the FP64 pipe stays free) and keeps the largest value M; a node that is not
// physical in FP32 counts as +infinity.  The second evaluates the same FP32
// value again and, only where it reaches M (1 - 1e-4), the FP64 |u| + a, whose
// maximum is the result: the FP32 values are within a few 1e-6 of the FP64
// ones (up to Mach numbers in the hundreds), so the node of the FP64 maximum is
// always among them and the result is the FP64 maximum over all nodes.  With
// M infinite every node is evaluated in FP64 (and non-physical states are
// flagged there).
__device__ __forceinline__ float wavespeed32(const double* __restrict__ ue, int nv, float g) {
  const float r = d2f_i(ue[0]), m0 = d2f_i(ue[nv]), m1 = d2f_i(ue[2 * nv]), m2 = d2f_i(ue[3 * nv]),
              E = d2f_i(ue[4 * nv]);
  const float q2 = (m0 * m0 + m1 * m1 + m2 * m2) / (r * r);
  const float p = (g - 1.0f) * (E - 0.5f * r * q2);
  const float lam = sqrtf(q2) + sqrtf(g * p / r);
  return (r > 0.0f && p > 0.0f && lam <= FLT_MAX) ? lam : INFINITY;
}

__global__ void max_wavespeed32_kernel(const double* __restrict__ u, size_t ne, int nv, float g,
                                       unsigned int* m32) {
  float m = 0.0f;
  const size_t nodes = ne * (size_t)nv;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nodes; t += (size_t)gridDim.x * blockDim.x) {
    const size_t e = t / nv, node = t % nv;
    m = fmaxf(m, wavespeed32(u + e * 5 * nv + node, nv, g));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(m32, __float_as_uint(m));  // non-negative floats order as integers
  }
}

__global__ void max_wavespeed_kernel(const double* __restrict__ u, size_t ne, int nv, double gamma,
                                     const unsigned int* __restrict__ m32, unsigned long long* out, int* flag) {
  double m = 0.0;
  const float M = __uint_as_float(*m32);
  const float T = (M <= FLT_MAX) ? M * (1.0f - 1.0e-4f) : 0.0f;
  const size_t nodes = ne * (size_t)nv;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nodes; t += (size_t)gridDim.x * blockDim.x) {
    const size_t e = t / nv, node = t % nv;
    const double* ue = u + e * 5 * nv + node;
    if (!(wavespeed32(ue, nv, (float)gamma) >= T)) continue;
    const double r = ue[0], m0 = ue[nv], m1 = ue[2 * nv], m2 = ue[3 * nv], E = ue[4 * nv];
    const double q2 = (m0 * m0 + m1 * m1 + m2 * m2) / (r * r);
    const double p = (gamma - 1.0) * (E - 0.5 * r * q2);
    if (!(r > 0.0) || !(p > 0.0)) atomicOr(flag, 1);
    const double lam = sqrt(q2) + sqrt(gamma * p / r);
    m = fmax(m, lam);  // NaN-free unless the state is non-physical (flagged)
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
  }
}

struct Comp {
  double s, c;
};

__device__ __forceinline__ void neumaier(Comp& a, double x) {
  const double t = a.s + x;
  if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x;
  else a.c += (x - t) + a.s;
  a.s = t;
}

__device__ __forceinline__ Comp comp_add(Comp a, Comp b) {
  // TwoSum of the leading parts, compensations carried along
  const double s = a.s + b.s;
  const double bb = s - a.s;
  const double err = (a.s - (s - bb)) + (b.s - bb);
  return Comp{s, a.c + b.c + err};
}

#define NDIAG 14

// one block per element (grid-stride), nv threads (<= 512) per block
__global__ void diagnostics_kernel(const double* __restrict__ u, const double* __restrict__ R,
                                   const double* __restrict__ wj, OpsGL ops, int ne, double* partial) {
  const int n = ops.n, nv = n * n * n;
  __shared__ double buf[2][5 * 512];
  __shared__ Comp red[NDIAG][32];
  // Pi~1^{-1} in shared memory: its rows differ across a warp
  __shared__ double P1[NSFR_MAXN * NSFR_MAXN];
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) P1[t] = ops.Pinv1[t];
  const double g = ops.gamma, gm1 = g - 1.0;
  Comp acc[NDIAG];
  for (int k = 0; k < NDIAG; ++k) acc[k] = Comp{0.0, 0.0};
  const int node = threadIdx.x;
  for (int e = blockIdx.x; e < ne; e += gridDim.x) {
    const double* ue = u + (size_t)e * 5 * nv;
    const double* Re = R + (size_t)e * 5 * nv;
    if (node < nv) {
      for (int k = 0; k < 5; ++k) buf[0][k * nv + node] = ue[k * nv + node];
    }
    __syncthreads();
    // Pi~^{-1} = (I + W^{-1} K1) along the three directions (identity when c = 0)
    int cur = 0;
    if (ops.has_K) {
      for (int d = 0; d < 3; ++d) {
        const int st = (d == 0) ? 1 : (d == 1 ? n : n * n);
        if (node < nv) {
          const int r = (node / st) % n;
          for (int k = 0; k < 5; ++k) {
            const double* col = buf[cur] + k * nv + node - r * st;
            double s = 0.0;
            for (int b = 0; b < n; ++b) s += P1[r * n + b] * col[b * st];
            buf[1 - cur][k * nv + node] = s;
          }
        }
        __syncthreads();
        cur = 1 - cur;
      }
    }
    if (node < nv) {
      const double w = wj[(size_t)e * nv + node];
      const double r = ue[node], m0 = ue[nv + node], m1 = ue[2 * nv + node], m2 = ue[3 * nv + node],
                   E = ue[4 * nv + node];
      const double ir = 1.0 / r;
      const double u0 = m0 * ir, u1 = m1 * ir, u2 = m2 * ir;
      const double q2 = u0 * u0 + u1 * u1 + u2 * u2;
      const double p = gm1 * (E - 0.5 * r * q2);
      const double s = log(p) - g * log(r);
      const double b = 0.5 * r / p;
      const double v[5] = {(g - s) / gm1 - b * q2, 2.0 * b * u0, 2.0 * b * u1, 2.0 * b * u2, -2.0 * b};
      double vr = 0.0;
      for (int k = 0; k < 5; ++k) vr += v[k] * Re[k * nv + node];
      neumaier(acc[0], w * (-r * s / gm1));
      neumaier(acc[1], -vr);
      neumaier(acc[2], fabs(vr));
      for (int k = 0; k < 5; ++k) neumaier(acc[3 + k], w * buf[cur][k * nv + node]);
      neumaier(acc[8], w * 0.5 * r * q2);
      for (int k = 0; k < 5; ++k) neumaier(acc[9 + k], Re[k * nv + node]);
    }
    __syncthreads();
  }
  // block reduction of the compensated pairs
  for (int k = 0; k < NDIAG; ++k) {
    Comp a = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      Comp b{__shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.c, o)};
      a = comp_add(a, b);
    }
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = a;
  }
  __syncthreads();
  if (threadIdx.x < NDIAG) {
    const int k = threadIdx.x;
    Comp a{0.0, 0.0};
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) a = comp_add(a, red[k][wi]);
    partial[((size_t)blockIdx.x * NDIAG + k) * 2 + 0] = a.s;
    partial[((size_t)blockIdx.x * NDIAG + k) * 2 + 1] = a.c;
  }
}

// the block's compensated pairs to partial[block][NDIAG][2]
__device__ __forceinline__ void diag_block_out(Comp (&acc)[NDIAG], Comp (*red)[32], double* partial) {
  for (int k = 0; k < NDIAG; ++k) {
    Comp a = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      Comp b{__shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.c, o)};
      a = comp_add(a, b);
    }
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = a;
  }
  __syncthreads();
  if (threadIdx.x < NDIAG) {
    const int k = threadIdx.x;
    Comp a{0.0, 0.0};
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) a = comp_add(a, red[k][wi]);
    partial[((size_t)blockIdx.x * NDIAG + k) * 2 + 0] = a.s;
    partial[((size_t)blockIdx.x * NDIAG + k) * 2 + 1] = a.c;
  }
}

// Diagnostics of the uncollocated scheme (solution coefficients on the ns
// Lobatto nodes, N Gauss-Legendre points per direction), one element per CTA
// (grid-stride).  With u_q = chi u^ the solution at the points and W J the
// point weights: S = sum W J U(u_q), Q = sum W J u_q and KE = sum W J rho
// |u|^2 / 2 (the GL quadrature of the solution); with the projected entropy
// variables v~^ = Pi v(u_q) at the solution nodes and R^ = chi^T R_q the raw
// residual there, the semi-discrete entropy rate -sum v~^ . R^ (Sec.
// "Nonlinear Stability": the projected variables make the volume terms
// telescope), its scale sum |v~^ . R^|, and sum R^.  Same outputs as
// diagnostics_kernel.
template <int N>
__global__ void __launch_bounds__(256) diagnostics_uncol_kernel(const double* __restrict__ u,
                                                                const double* __restrict__ R,
                                                                const double* __restrict__ wj, OpsGL ops, int ne,
                                                                double* partial) {
  constexpr int NV = N * N * N, SL = 5 * NV;
  extern __shared__ double sm[];
  double* Us = sm;  // [5][NV]: u^ (first nsv of each slab), later v~^
  double* Vq = Us + SL;
  double* T1 = Vq + SL;
  double* T2 = T1 + SL;
  __shared__ Comp red[NDIAG][32];
  const int ns = ops.ns, nsv = ns * ns * ns;
  const double g = ops.gamma, gm1 = g - 1.0;
  Comp acc[NDIAG];
  for (int k = 0; k < NDIAG; ++k) acc[k] = Comp{0.0, 0.0};
  for (int e = blockIdx.x; e < ne; e += gridDim.x) {
    for (int t = threadIdx.x; t < 5 * nsv; t += blockDim.x) Us[(t / nsv) * NV + t % nsv] = u[(size_t)e * 5 * nsv + t];
    __syncthreads();
    nsfr_k::psweep(ops.chi, ns, N, Us, T1, 5, NV, 0, ns, ns, ns);
    nsfr_k::psweep(ops.chi, ns, N, T1, T2, 5, NV, 1, N, ns, ns);
    nsfr_k::psweep(ops.chi, ns, N, T2, Vq, 5, NV, 2, N, N, ns);
    for (int t = threadIdx.x; t < NV; t += blockDim.x) {
      double* v = Vq + t;
      const double w = wj[(size_t)e * NV + t];
      const double r = v[0], m0 = v[NV], m1 = v[2 * NV], m2 = v[3 * NV], E = v[4 * NV];
      const double ir = 1.0 / r;
      const double u0 = m0 * ir, u1 = m1 * ir, u2 = m2 * ir;
      const double q2 = u0 * u0 + u1 * u1 + u2 * u2;
      const double p = gm1 * (E - 0.5 * r * q2);
      const double s = log(p) - g * log(r);
      const double b = 0.5 * r / p;
      neumaier(acc[0], w * (-r * s / gm1));
      for (int k = 0; k < 5; ++k) neumaier(acc[3 + k], w * v[k * NV]);
      neumaier(acc[8], w * 0.5 * r * q2);
      v[0] = (g - s) / gm1 - b * q2;
      v[NV] = 2.0 * b * u0;
      v[2 * NV] = 2.0 * b * u1;
      v[3 * NV] = 2.0 * b * u2;
      v[4 * NV] = -2.0 * b;
    }
    __syncthreads();
    nsfr_k::psweep(ops.Pi, N, ns, Vq, T1, 5, NV, 0, N, N, N);
    nsfr_k::psweep(ops.Pi, N, ns, T1, T2, 5, NV, 1, ns, N, N);
    nsfr_k::psweep(ops.Pi, N, ns, T2, Us, 5, NV, 2, ns, ns, N);
    for (int t = threadIdx.x; t < nsv; t += blockDim.x) {
      const double* Re = R + (size_t)e * 5 * nsv + t;
      double vr = 0.0;
      for (int k = 0; k < 5; ++k) {
        vr += Us[k * NV + t] * Re[k * nsv];
        neumaier(acc[9 + k], Re[k * nsv]);
      }
      neumaier(acc[1], -vr);
      neumaier(acc[2], fabs(vr));
    }
    __syncthreads();
  }
  diag_block_out(acc, red, partial);
}

template <int N>
cudaError_t launch_diag_uncol(nsfr_ctx* ctx, const double* u, const double* R, double* partial, int nblocks,
                              cudaStream_t s) {
  const size_t smem = (size_t)4 * 5 * N * N * N * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(diagnostics_uncol_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  diagnostics_uncol_kernel<N><<<nblocks, 256, smem, s>>>(u, R, ctx->wj, ctx->ops, ctx->ne, partial);
  return cudaGetLastError();
}

}  // namespace

int nsfr_diag_blocks(nsfr_ctx* ctx) { return ctx->ne < 1024 ? ctx->ne : 1024; }

// the two passes of the wave-speed maximum, callable piecewise: begin clears the
// results, candidates runs the FP32 pass over elements [e_b, e_e) (any number of
// calls covering the mesh), finish runs the FP64 pass over the whole state
cudaError_t nsfr_wavespeed_begin(nsfr_ctx* ctx, cudaStream_t s) {
  // umax[0]: the FP64 maximum (bit pattern), umax[1]: the FP32 candidate bound
  return cudaMemsetAsync(ctx->umax, 0, 2 * sizeof(unsigned long long), s);
}

static int wavespeed_grid(size_t nodes) {
  const size_t g = (nodes + 255) / 256;
  return g > 152 * 8 ? 152 * 8 : (int)g;
}

cudaError_t nsfr_wavespeed_candidates(nsfr_ctx* ctx, const double* u, int e_b, int e_e, cudaStream_t s) {
  if (e_e <= e_b) return cudaSuccess;
  unsigned int* m32 = reinterpret_cast<unsigned int*>(ctx->umax + 1);
  nsfr_prof_begin(ctx, 3, s);
  max_wavespeed32_kernel<<<wavespeed_grid((size_t)(e_e - e_b) * ctx->nsv), 256, 0, s>>>(
      u + (size_t)e_b * 5 * ctx->nsv, (size_t)(e_e - e_b), ctx->nsv, (float)ctx->gamma, m32);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t nsfr_wavespeed_finish(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  const unsigned int* m32 = reinterpret_cast<const unsigned int*>(ctx->umax + 1);
  nsfr_prof_begin(ctx, 3, s);
  max_wavespeed_kernel<<<wavespeed_grid((size_t)ctx->ne * ctx->nsv), 256, 0, s>>>(
      u, (size_t)ctx->ne, ctx->nsv, ctx->gamma, m32, ctx->umax, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t nsfr_launch_max_wavespeed(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  cudaError_t err = nsfr_wavespeed_begin(ctx, s);
  if (err == cudaSuccess) err = nsfr_wavespeed_candidates(ctx, u, 0, ctx->ne, s);
  if (err == cudaSuccess) err = nsfr_wavespeed_finish(ctx, u, s);
  return err;
}

cudaError_t nsfr_launch_diagnostics(nsfr_ctx* ctx, const double* u, const double* R, double* partial, int nblocks,
                                    cudaStream_t s) {
  if (ctx->uncol) {
    cudaError_t err = cudaErrorInvalidValue;
    nsfr_prof_begin(ctx, 4, s);
    switch (ctx->n) {
      case 2: err = launch_diag_uncol<2>(ctx, u, R, partial, nblocks, s); break;
      case 3: err = launch_diag_uncol<3>(ctx, u, R, partial, nblocks, s); break;
      case 4: err = launch_diag_uncol<4>(ctx, u, R, partial, nblocks, s); break;
      case 5: err = launch_diag_uncol<5>(ctx, u, R, partial, nblocks, s); break;
      case 6: err = launch_diag_uncol<6>(ctx, u, R, partial, nblocks, s); break;
      case 7: err = launch_diag_uncol<7>(ctx, u, R, partial, nblocks, s); break;
      case 8: err = launch_diag_uncol<8>(ctx, u, R, partial, nblocks, s); break;
    }
    nsfr_prof_end(ctx, s);
    ctx->launches++;
    return err;
  }
  int threads = ((ctx->nv + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  nsfr_prof_begin(ctx, 4, s);
  diagnostics_kernel<<<nblocks, threads, 0, s>>>(u, R, ctx->wj, ctx->ops, ctx->ne, partial);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}
