// Metric terms of the curvilinear hexahedra (setup, run once per context).
//
// Sec. "Computational Space": J = a_1 . (a_2 x a_3), C^T rows J a^i, built in
// Kopriva's conservative-curl form so the discrete GCL (Eq. GCL) holds:
//   (J a^i)_n = -[curl_xi (X_l grad_xi X_m)]_i,  (n, m, l) cyclic.
// The map (control points at equispaced reference nodes) is evaluated on the
// degree-p Lobatto nodes, the products X_l d_k X_m are formed there (X_l
// relative to the element's first control point: curl(c grad X_m) = 0 for a
// constant c because derivatives along different directions commute, so the
// shift changes only rounding, which would otherwise grow like |X|/h), the
// curl is the exact derivative of their Lobatto interpolant, and the result (a
// degree <= p polynomial per direction) is interpolated to the GL volume
// nodes and, layer by layer, to the GL nodes of each face.  Because the
// Lobatto layer on a face depends only on the face's control points, the
// face rows are watertight; the row of each element's xi_d = +1 face is the
// one both neighbours use.  One CTA per element; every step is a 1D
// contraction along one direction (sum factorisation) on shared memory.
#include "nsfr_internal.h"

namespace {

// out[z][y][x] = sum_b A[r][b] in[..b..] along direction d.  ``ext`` are the
// input extents (x, y, z); the output has extent m along d.
__device__ void sweep(const double* __restrict__ A, int k, int m, const double* in, double* out, int d,
                      int ex, int ey, int ez) {
  int ox = ex, oy = ey, oz = ez;
  if (d == 0) ox = m;
  if (d == 1) oy = m;
  if (d == 2) oz = m;
  const int total = ox * oy * oz;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int x = t % ox, y = (t / ox) % oy, z = t / (ox * oy);
    double s = 0.0;
    for (int b = 0; b < k; ++b) {
      int xi = x, yi = y, zi = z, r;
      if (d == 0) { r = x; xi = b; }
      else if (d == 1) { r = y; yi = b; }
      else { r = z; zi = b; }
      s += A[r * k + b] * in[xi + ex * (yi + ey * zi)];
    }
    out[t] = s;
  }
  __syncthreads();
}

// three sweeps of the same (m x k) matrix: (k,k,k) -> (m,m,m), via two temps
__device__ void sweep3(const double* A, int k, int m, const double* in, double* out, double* t1,
                       double* t2) {
  sweep(A, k, m, in, t1, 0, k, k, k);
  sweep(A, k, m, t1, t2, 1, m, k, k);
  sweep(A, k, m, t2, out, 2, m, m, k);
}

__global__ void metric_kernel(const double* __restrict__ ctrl, OpsGeo g, double* __restrict__ metric,
                              double* __restrict__ Jout, double* __restrict__ invwj,
                              double* __restrict__ wj, double* __restrict__ nf_plus,
                              double* __restrict__ xyz, int* flag) {
  extern __shared__ double sm[];
  // n: Lobatto nodes of the construction (and solution nodes, whose coordinates
  // are returned); m: volume quadrature points the metric is evaluated at
  const int n = g.n, q = g.q, m = g.nq, nv = n * n * n, q3 = q * q * q;
  const int mv = m * m * m, mfp = m * m;
  const int S = 512;  // stride of the shared arrays (>= n^3, q^3)
  double* Xe = sm;             // 3 arrays: control points
  double* X = Xe + 3 * S;      // 3: map at LGL nodes
  double* dX = X + 3 * S;      // 9: dX[k*3+m] = d_k X_m at LGL
  double* Cl = dX + 9 * S;     // 9: Cl[i*3+c] = (J a^i)_c at LGL
  double* V = Cl + 9 * S;      // 3
  double* T1 = V + 3 * S;      // temps
  double* T2 = T1 + S;
  double* T3 = T2 + S;
  double* T4 = T3 + S;
  const int e = blockIdx.x;

  for (int t = threadIdx.x; t < 3 * q3; t += blockDim.x) {
    const int node = t / 3, c = t % 3;
    Xe[c * S + node] = ctrl[(size_t)e * q3 * 3 + t];
  }
  __syncthreads();
  // 1. the map at the LGL nodes
  for (int c = 0; c < 3; ++c) sweep3(g.E, q, n, Xe + c * S, X + c * S, T1, T2);
  // 2. exact derivatives at the LGL nodes
  for (int k = 0; k < 3; ++k)
    for (int m = 0; m < 3; ++m) sweep(g.Dl, n, n, X + m * S, dX + (k * 3 + m) * S, k, n, n, n);
  // 3. conservative curl: (J a^i)_c = -(curl V)_i, V_k = X_l d_k X_m, (c, m, l) cyclic
  for (int c = 0; c < 3; ++c) {
    const int m = (c + 1) % 3, l = (c + 2) % 3;
    for (int t = threadIdx.x; t < nv; t += blockDim.x)
      for (int k = 0; k < 3; ++k) V[k * S + t] = (X[l * S + t] - Xe[l * S]) * dX[(k * 3 + m) * S + t];
    __syncthreads();
    // i = 0: d_eta V_3 - d_zeta V_2 ; i = 1: d_zeta V_1 - d_xi V_3 ; i = 2: d_xi V_2 - d_eta V_1
    const int da[3] = {1, 2, 0}, va[3] = {2, 0, 1};
    const int db[3] = {2, 0, 1}, vb[3] = {1, 2, 0};
    for (int i = 0; i < 3; ++i) {
      sweep(g.Dl, n, n, V + va[i] * S, T1, da[i], n, n, n);
      sweep(g.Dl, n, n, V + vb[i] * S, T2, db[i], n, n, n);
      for (int t = threadIdx.x; t < nv; t += blockDim.x) Cl[(i * 3 + c) * S + t] = -(T1[t] - T2[t]);
      __syncthreads();
    }
  }
  // 4. to the volume quadrature points
  for (int r = 0; r < 9; ++r) {
    sweep3(g.I, n, m, Cl + r * S, T3, T1, T2);
    for (int t = threadIdx.x; t < mv; t += blockDim.x) metric[((size_t)e * 9 + r) * mv + t] = T3[t];
    __syncthreads();
  }
  // face rows: Lobatto layer xi_d = +1 of (J a^d)_c, interpolated tangentially
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) {
      const double* src = Cl + (d * 3 + c) * S;
      for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int f0 = t % n, f1 = t / n;  // remaining directions, fast then slow
        int x, y, z;
        if (d == 0) { x = n - 1; y = f0; z = f1; }
        else if (d == 1) { x = f0; y = n - 1; z = f1; }
        else { x = f0; y = f1; z = n - 1; }
        T3[t] = src[x + n * (y + n * z)];
      }
      __syncthreads();
      sweep(g.I, n, m, T3, T4, 0, n, n, 1);
      sweep(g.I, n, m, T4, T3, 1, m, n, 1);
      for (int t = threadIdx.x; t < mfp; t += blockDim.x)
        nf_plus[(((size_t)e * 3 + d) * 3 + c) * mfp + t] = T3[t];
      __syncthreads();
    }
  // 5. J = a_1 . (a_2 x a_3) from the map's exact derivative at the quadrature points
  for (int r = 0; r < 9; ++r) {
    sweep3(g.I, n, m, dX + r * S, T3, T1, T2);
    for (int t = threadIdx.x; t < mv; t += blockDim.x) Cl[r * S + t] = T3[t];  // reuse Cl: a there
    __syncthreads();
  }
  for (int t = threadIdx.x; t < mv; t += blockDim.x) {
    const double* a = Cl;
    double a00 = a[0 * S + t], a01 = a[1 * S + t], a02 = a[2 * S + t];
    double a10 = a[3 * S + t], a11 = a[4 * S + t], a12 = a[5 * S + t];
    double a20 = a[6 * S + t], a21 = a[7 * S + t], a22 = a[8 * S + t];
    double Jv = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) + a02 * (a10 * a21 - a11 * a20);
    const int i = t % m, j = (t / m) % m, k = t / (m * m);
    const double w3 = g.w[i] * g.w[j] * g.w[k];
    Jout[(size_t)e * mv + t] = Jv;
    wj[(size_t)e * mv + t] = w3 * Jv;
    invwj[(size_t)e * mv + t] = 1.0 / (w3 * Jv);
    if (!(Jv > 0.0)) atomicOr(flag, 2);
  }
  // physical coordinates of the solution nodes
  for (int c = 0; c < 3; ++c) {
    sweep3(g.Eg, q, n, Xe + c * S, T3, T1, T2);
    for (int t = threadIdx.x; t < nv; t += blockDim.x) xyz[((size_t)e * 3 + c) * nv + t] = T3[t];
    __syncthreads();
  }
}

__global__ void jacobian_derived_kernel(const double* __restrict__ J, OpsGeo g, size_t total,
                                        double* __restrict__ invwj, double* __restrict__ wj, int* flag) {
  const int n = g.nq, nv = n * n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int node = (int)(t % nv);
    const int i = node % n, j = (node / n) % n, k = node / (n * n);
    const double w3 = g.w[i] * g.w[j] * g.w[k];
    const double Jv = J[t];
    if (!(Jv > 0.0)) atomicOr(flag, 2);
    wj[t] = w3 * Jv;
    invwj[t] = 1.0 / (w3 * Jv);
  }
}

}  // namespace

cudaError_t nsfr_launch_jacobian_derived(nsfr_ctx* ctx, cudaStream_t s) {
  const size_t total = (size_t)ctx->ne * ctx->nv;
  int grid = (int)((total + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  jacobian_derived_kernel<<<grid, 256, 0, s>>>(ctx->J, ctx->gops, total, ctx->invwj, ctx->wj, ctx->flag);
  ctx->launches++;
  return cudaGetLastError();
}

size_t nsfr_metric_smem() { return (size_t)(3 + 3 + 9 + 9 + 3 + 4) * 512 * sizeof(double); }

cudaError_t nsfr_launch_metrics(nsfr_ctx* ctx, cudaStream_t s) {
  const size_t smem = nsfr_metric_smem();
  cudaError_t err = cudaFuncSetAttribute(metric_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  metric_kernel<<<ctx->ne, 256, smem, s>>>(ctx->ctrl, ctx->gops, ctx->metric, ctx->J, ctx->invwj, ctx->wj,
                                           ctx->nfp_plus, ctx->xyz, ctx->flag);
  ctx->launches++;
  return cudaGetLastError();
}
