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
#include "nsfr_internal.h"

namespace {

__global__ void max_wavespeed_kernel(const double* __restrict__ u, size_t ne, int nv, double gamma,
                                     unsigned long long* out, int* flag) {
  double m = 0.0;
  const size_t nodes = ne * (size_t)nv;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nodes; t += (size_t)gridDim.x * blockDim.x) {
    const size_t e = t / nv, node = t % nv;
    const double* ue = u + e * 5 * nv + node;
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
            for (int b = 0; b < n; ++b) s += ops.Pinv1[r * n + b] * col[b * st];
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

}  // namespace

int nsfr_diag_blocks(nsfr_ctx* ctx) { return ctx->ne < 1024 ? ctx->ne : 1024; }

cudaError_t nsfr_launch_max_wavespeed(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  cudaError_t err = cudaMemsetAsync(ctx->umax, 0, sizeof(unsigned long long), s);
  if (err != cudaSuccess) return err;
  const size_t nodes = (size_t)ctx->ne * ctx->nsv;
  int grid = (int)((nodes + 255) / 256);
  if (grid > 152 * 8) grid = 152 * 8;
  nsfr_prof_begin(ctx, 3, s);
  max_wavespeed_kernel<<<grid, 256, 0, s>>>(u, (size_t)ctx->ne, ctx->nsv, ctx->gamma, ctx->umax, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t nsfr_launch_diagnostics(nsfr_ctx* ctx, const double* u, const double* R, double* partial, int nblocks,
                                    cudaStream_t s) {
  int threads = ((ctx->nv + 31) / 32) * 32;
  if (threads < 64) threads = 64;
  nsfr_prof_begin(ctx, 4, s);
  diagnostics_kernel<<<nblocks, threads, 0, s>>>(u, R, ctx->wj, ctx->ops, ctx->ne, partial);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}
