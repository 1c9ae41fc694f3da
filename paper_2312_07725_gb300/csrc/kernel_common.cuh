// Index helpers shared by the residual kernels.
#pragma once

#include "ffloat.cuh"
#include "nsfr_internal.h"

namespace nsfr_k {

// elements per CTA (one thread per line, 3 n^2 lines per element) chosen so
// that a CTA has at most 8 warps, i.e. two per SM sub-partition, which lets
// every thread keep up to 255 registers
constexpr int epb_for(int n) { return n == 2 ? 16 : n == 3 ? 8 : n == 4 ? 4 : n == 5 ? 3 : n == 6 ? 2 : 1; }
constexpr int threads_for(int n) { return epb_for(n) * 3 * n * n; }
// The FP64 volume kernel keeps 23 n^3 doubles of shared memory per element
// (records, three direction slabs of line sums) and about 110
// registers per thread; it is bound by FP64 issue, which wants as many warps
// per SM as shared memory (228 KB) and the register file (64K, split evenly
// over the four sub-partitions) allow.  Elements per CTA and CTAs per SM:
// (the n = 5 shape can be set at build time, NSFR_VOL_EPB5 / NSFR_VOL_CTAS5, to measure others)
#ifndef NSFR_VOL_EPB5
#define NSFR_VOL_EPB5 2
#endif
#ifndef NSFR_VOL_CTAS5
#define NSFR_VOL_CTAS5 3
#endif
constexpr int vol_epb(int n) {
  return n == 2 ? 16 : n == 3 ? 8 : n == 4 ? 5 : n == 5 ? NSFR_VOL_EPB5 : n == 6 ? 2 : 1;
}
constexpr int vol_ctas(int n) {
  return n == 2 ? 2 : n == 3 ? 2 : n == 4 ? 2 : n == 5 ? NSFR_VOL_CTAS5 : n == 6 ? 2 : n == 7 ? 2 : 1;
}
constexpr int vol_threads(int n) { return vol_epb(n) * 3 * n * n; }
// The FP32-bulk volume kernels: 7 n^3 doubles + 43 n^3 floats of shared memory
// per element, the same thread layout.  Both forms run their flux arithmetic
// on the FP32 pipe and are bound by latency at the 128-register cap, where 16
// warps per SM is the most the register file holds: at n = 5, 3 elements x 2
// CTAs (16 warps) measured 2% faster than 2 x 3 (15 warps) and 9% faster than
// 2 x 2 for the float-float variant.
constexpr int bulk_epb(int n, bool ff) { return n == 5 ? 3 : vol_epb(n); }
constexpr int bulk_ctas(int n, bool ff) { return n == 5 ? 2 : vol_ctas(n); }
constexpr int bulk_threads(int n, bool ff) { return bulk_epb(n, ff) * 3 * n * n; }

// neighbour of element e across face (d, side): side 0 is xi_d = -1 (periodic)
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

// w_perp of node (i, j, k) for lines of direction d: the weights of the other two
__device__ __forceinline__ double wperp_of(const double* w, int node, int n, int d) {
  const int i = node % n, j = (node / n) % n, k = node / (n * n);
  return d == 0 ? w[j] * w[k] : (d == 1 ? w[i] * w[k] : w[i] * w[j]);
}

// Y = A along direction d of X for nslab slabs of stride st (extents (ex, ey,
// ez) in, extent m along d out); A is m x k row-major.  Ends with a barrier.
__device__ inline void psweep(const double* __restrict__ A, int k, int m, const double* X, double* Y, int nslab, int st,
                       int d, int ex, int ey, int ez) {
  int ox = ex, oy = ey, oz = ez;
  if (d == 0) ox = m;
  if (d == 1) oy = m;
  if (d == 2) oz = m;
  const int per = ox * oy * oz;
  const int sx = 1, sy = ex, sz = ex * ey;
  const int sd = d == 0 ? sx : (d == 1 ? sy : sz);
  for (int t = threadIdx.x; t < nslab * per; t += blockDim.x) {
    const int sl = t / per, q = t % per;
    const int x = q % ox, y = (q / ox) % oy, z = q / (ox * oy);
    const int r = d == 0 ? x : (d == 1 ? y : z);
    const double* in = X + (size_t)sl * st + (d == 0 ? 0 : x) * sx + (d == 1 ? 0 : y) * sy + (d == 2 ? 0 : z) * sz;
    const double* a = A + r * k;
    double acc = 0.0;
    for (int b = 0; b < k; ++b) acc = fma(a[b], in[b * sd], acc);
    Y[(size_t)sl * st + q] = acc;
  }
  __syncthreads();
}

// Y = A along direction d of X for nslab slabs (stride st each, extents
// (ex, ey, ez) in, extent m along d out); A is m x k row-major, or, with
// trans, the transpose of a k x m row-major matrix.  Ends with a barrier.
__device__ inline void slab_sweep(const double* __restrict__ A, bool trans, int k, int m, const double* X, double* Y,
                           int nslab, int st, int d, int ex, int ey, int ez) {
  int ox = ex, oy = ey, oz = ez;
  if (d == 0) ox = m;
  if (d == 1) oy = m;
  if (d == 2) oz = m;
  const int per = ox * oy * oz;
  for (int t = threadIdx.x; t < nslab * per; t += blockDim.x) {
    const int sl = t / per, q = t % per;
    const int x = q % ox, y = (q / ox) % oy, z = q / (ox * oy);
    const double* in = X + (size_t)sl * st;
    double acc = 0.0;
    for (int b = 0; b < k; ++b) {
      int xi = x, yi = y, zi = z, r;
      if (d == 0) { r = x; xi = b; }
      else if (d == 1) { r = y; yi = b; }
      else { r = z; zi = b; }
      const double a = trans ? A[b * m + r] : A[r * k + b];
      acc = fma(a, in[xi + ex * (yi + ey * zi)], acc);
    }
    Y[(size_t)sl * st + q] = acc;
  }
  __syncthreads();
}

// Epilogue of the uncollocated scheme for the nel elements of a CTA, R_q (the
// line-wise residual at the N^3 GL points) in X[nel*5][NV]; Y is a second
// buffer of the same size.  R^ = chi^T R_q (raw residual) or
// du^/dt = -Pi~ (W J)^{-1} Pi~^T chi^T R_q = -Pi~ (W J)^{-1} A R_q with
// A = (chi Pi~1)^T per direction, on the ns^3 solution nodes; then the store
// or the RK stage update as in the collocated epilogue.
template <int N>
__device__ void uncol_epilogue(double* X, double* Y, int nel, int e0, const OpsGL& ops,
                               const double* __restrict__ invwj, int epi, const RkArgs& rk, double* out) {
  constexpr int NV = N * N * N;
  const int ns = ops.ns, nsv = ns * ns * ns, nsl = nel * 5;
  double* res;
  if (epi == EPI_RAW) {
    slab_sweep(ops.chi, true, N, ns, X, Y, nsl, NV, 0, N, N, N);
    slab_sweep(ops.chi, true, N, ns, Y, X, nsl, NV, 1, ns, N, N);
    slab_sweep(ops.chi, true, N, ns, X, Y, nsl, NV, 2, ns, ns, N);
    res = Y;
  } else {
    slab_sweep(ops.A, false, N, N, X, Y, nsl, NV, 0, N, N, N);
    slab_sweep(ops.A, false, N, N, Y, X, nsl, NV, 1, N, N, N);
    slab_sweep(ops.A, false, N, N, X, Y, nsl, NV, 2, N, N, N);
    for (int t = threadIdx.x; t < nsl * NV; t += blockDim.x) Y[t] *= invwj[(size_t)(e0 + t / (5 * NV)) * NV + t % NV];
    __syncthreads();
    slab_sweep(ops.Pt, false, N, ns, Y, X, nsl, NV, 0, N, N, N);
    slab_sweep(ops.Pt, false, N, ns, X, Y, nsl, NV, 1, ns, N, N);
    slab_sweep(ops.Pt, false, N, ns, Y, X, nsl, NV, 2, ns, ns, N);
    res = X;
  }
  const size_t off = (size_t)e0 * 5 * nsv;
  for (int t = threadIdx.x; t < nsl * nsv; t += blockDim.x) {
    const double r = res[(size_t)(t / nsv) * NV + t % nsv];
    if (epi == EPI_RAW) {
      out[off + t] = r;
    } else if (epi == EPI_DUDT) {
      out[off + t] = neg_i(r);
    } else {
      const double k = neg_i(r);
      if (rk.last) {
        rk.unext[off + t] = fma(rk.b * rk.dt, k, rk.acc[off + t]);
      } else {
        const double u0 = rk.u0[off + t];
        rk.acc[off + t] = fma(rk.b * rk.dt, k, rk.first ? u0 : rk.acc[off + t]);
        rk.unext[off + t] = fma(rk.a_next * rk.dt, k, u0);
      }
    }
  }
}

}  // namespace nsfr_k
