// Volume source terms: W J q(x, t) at the volume nodes, subtracted from the
// residual before the weight-adjusted inverse (the source is a volume
// integral beside the residual: (M_m + K_m) du/dt = -R + W J q).
//
// NSFR_SOURCE_MANUFACTURED: the manufactured solution of Sec. "Manufactured
// Solution Convergence" (Gassner et al.), rho = 2 + sin(theta)/10,
// u = v = w = 1, rho e = rho^2, theta = pi (x + y + z - 2t).  Its source
// q = du/dt + div F follows from the definition: with
// rho_t = -(pi/5) cos(theta), each rho_x = (pi/10) cos(theta) and
// p = (gamma - 1)(rho^2 - 3 rho / 2),
//   q_rho = c1 cos(theta)
//   q_m   = c2 cos(theta) + c3 sin(2 theta)          (all three components)
//   q_E   = c4 cos(theta) + c5 sin(2 theta)
//   c1 = pi/10, c2 = pi (5 gamma - 3)/20, c3 = pi (gamma - 1)/100,
//   c4 = pi (15 gamma - 7)/20, c5 = pi (3 gamma - 2)/100.
#include <algorithm>

#include "nsfr_internal.h"

namespace {

__global__ void __launch_bounds__(256) manufactured_source_kernel(const double* __restrict__ xyz,
                                                                  const double* __restrict__ wj, long long ne,
                                                                  int nv, double t, double gamma,
                                                                  double* __restrict__ src) {
  const double pi = 3.141592653589793;
  const double c1 = pi / 10.0, c2 = pi * (5.0 * gamma - 3.0) / 20.0, c3 = pi * (gamma - 1.0) / 100.0;
  const double c4 = pi * (15.0 * gamma - 7.0) / 20.0, c5 = pi * (3.0 * gamma - 2.0) / 100.0;
  const long long total = ne * nv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long e = i / nv;
    const int node = (int)(i % nv);
    const double* X = xyz + (size_t)e * 3 * nv + node;  // x, y, z are nv apart
    double s, c;
    sincospi(X[0] + X[nv] + X[2 * nv] - 2.0 * t, &s, &c);  // sin, cos of theta
    const double s2 = 2.0 * s * c;                      // sin(2 theta)
    const double w = wj[i];
    const double qm = w * fma(c3, s2, c2 * c);
    double* q = src + (size_t)e * 5 * nv + node;
    q[0] = w * (c1 * c);
    q[nv] = qm;
    q[2 * nv] = qm;
    q[3 * nv] = qm;
    q[4 * nv] = w * fma(c5, s2, c4 * c);
  }
}

}  // namespace

cudaError_t nsfr_launch_source(nsfr_ctx* ctx, double t, cudaStream_t s) {
  if (ctx->source != NSFR_SOURCE_MANUFACTURED) return cudaSuccess;
  const long long total = (long long)ctx->ne * ctx->nv;
  const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
  nsfr_prof_begin(ctx, 9, s);
  manufactured_source_kernel<<<grid, 256, 0, s>>>(ctx->xyz, ctx->wj, ctx->ne, ctx->nv, t, ctx->gamma, ctx->src);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}
