// Entropy projection of the uncollocated scheme (solution coefficients on the
// ns Lobatto nodes, volume and face quadrature on the N GL points; Sec.
// "Nonlinearly Stable Flux Reconstruction", entropy projected variables):
//
//   u_q = chi u^            the state at the GL points,
//   v~^ = Pi v(u_q)         the L2 projection of the entropy variables,
//   u~  = u(chi v~^)        the projected state at the GL points,
//   u~_f = u(l_s v~^)       at the GL points of each face (l_s: the solution
//                           basis at xi_d = -1 / +1, chi along the face).
//
// One CTA per element; every step is a 1D contraction along one direction
// (sum factorisation) on shared memory.  The kernel writes the node records
// of u~ at the GL points (rho, 2 beta, u/2, |u|^2/4, ln rho, ln beta) and the
// face records, the two inputs of the face-flux and volume kernels, exactly
// as the collocated face-state kernel does for its nodes.
#include "kernel_common.cuh"
#include "mathfn.cuh"
#include "physics.cuh"

namespace {
using namespace nsfr_k;

// out = A along direction d of in; A is (m x k) row-major, in has extents
// (ex, ey, ez) with extent k along d, out has extent m along d
__device__ void psweep(const double* __restrict__ A, int k, int m, const double* in, double* out, int d, int ex,
                       int ey, int ez) {
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
      s = fma(A[r * k + b], in[xi + ex * (yi + ey * zi)], s);
    }
    out[t] = s;
  }
  __syncthreads();
}

// three sweeps of the same (m x k) matrix: (k,k,k) -> (m,m,m)
__device__ void psweep3(const double* A, int k, int m, const double* in, double* out, double* t1, double* t2) {
  psweep(A, k, m, in, t1, 0, k, k, k);
  psweep(A, k, m, t1, t2, 1, m, k, k);
  psweep(A, k, m, t2, out, 2, m, m, k);
}

// the record of u(w), w entropy variables (the face-state conversion); flags
// 2 beta <= 0 or NaN
__device__ __forceinline__ Rec rec_from_entropy(const double w[5], const OpsGL& ops, const MathTables& T, int* flag) {
  const double g = ops.gamma, gm1 = g - 1.0, ln2 = 0.69314718055994530942;
  if (!(w[4] < 0.0)) atomicOr(flag, 1);
  const double b2 = -w[4];
  const double iv5 = rcp_full(w[4]);
  const double u0 = -w[1] * iv5, u1 = -w[2] * iv5, u2 = -w[3] * iv5;
  const double q2 = fma(u0, u0, fma(u1, u1, u2 * u2));
  const double sent = g - gm1 * fma(0.5 * b2, q2, w[0]);
  const double L5 = nsfr_log(b2, T);
  const double lr = -(sent + L5) * ops.inv_gm1;
  Rec P;
  P.r = nsfr_exp(lr, T);
  P.b2 = b2;
  P.u0 = 0.5 * u0;
  P.u1 = 0.5 * u1;
  P.u2 = 0.5 * u2;
  P.qq = 0.25 * q2;
  P.lr = lr;
  P.lb = L5 - ln2;
  return P;
}

// shared memory: Us [5][S] solution-node values, Vq [5][S] point values, two temps
constexpr int PS = NSFR_MAXN * NSFR_MAXN * NSFR_MAXN;

__global__ void projection_kernel(const double* __restrict__ u, OpsGL ops, double* __restrict__ face,
                                  double* __restrict__ nrec, int* flag) {
  extern __shared__ double sm[];
  const int N = ops.n, ns = ops.ns, NV = N * N * N, NFP = N * N, nsv = ns * ns * ns;
  double* Us = sm;             // [5][PS]
  double* Vq = Us + 5 * PS;    // [5][PS]
  double* T1 = Vq + 5 * PS;
  double* T2 = T1 + PS;
  const MathTables T = nsfr_stage_tables(T2 + PS);
  const int e = blockIdx.x;
  const double g = ops.gamma, gm1 = g - 1.0;
  for (int t = threadIdx.x; t < 5 * nsv; t += blockDim.x) Us[(t / nsv) * PS + t % nsv] = u[(size_t)e * 5 * nsv + t];
  __syncthreads();
  // u_q = chi u^
  for (int k = 0; k < 5; ++k) psweep3(ops.chi, ns, N, Us + k * PS, Vq + k * PS, T1, T2);
  // v(u_q) in place
  for (int t = threadIdx.x; t < NV; t += blockDim.x) {
    const double r = Vq[t], m0 = Vq[PS + t], m1 = Vq[2 * PS + t], m2 = Vq[3 * PS + t], E = Vq[4 * PS + t];
    const double ir = rcp_full(r);
    const double u0 = m0 * ir, u1 = m1 * ir, u2 = m2 * ir;
    const double q2 = fma(u0, u0, fma(u1, u1, u2 * u2));
    const double p = gm1 * fma(-0.5 * r, q2, E);
    if (!(r > 0.0) || !(p > 0.0)) atomicOr(flag, 1);
    const double b = 0.5 * r * rcp_full(p);
    const double s = nsfr_log(p, T) - g * nsfr_log(r, T);
    Vq[t] = (g - s) * ops.inv_gm1 - b * q2;
    Vq[PS + t] = 2.0 * b * u0;
    Vq[2 * PS + t] = 2.0 * b * u1;
    Vq[3 * PS + t] = 2.0 * b * u2;
    Vq[4 * PS + t] = -2.0 * b;
  }
  __syncthreads();
  // v~^ = Pi v(u_q), into Us
  for (int k = 0; k < 5; ++k) psweep3(ops.Pi, N, ns, Vq + k * PS, Us + k * PS, T1, T2);
  // chi v~^ at the GL points -> node records of u~
  for (int k = 0; k < 5; ++k) psweep3(ops.chi, ns, N, Us + k * PS, Vq + k * PS, T1, T2);
  for (int t = threadIdx.x; t < NV; t += blockDim.x) {
    double w[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) w[k] = Vq[k * PS + t];
    store_rec(nrec + (size_t)e * NSFR_NFIELD * NV + t, NV, rec_from_entropy(w, ops, T, flag));
  }
  __syncthreads();
  // faces: l_s along d, chi along the two face directions
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) {
      const double* ls = s ? ops.ls_p : ops.ls_m;
      for (int k = 0; k < 5; ++k) {
        // contract along d: (ns,ns,ns) -> the face layer (f0, f1) over the two other directions
        for (int t = threadIdx.x; t < ns * ns; t += blockDim.x) {
          const int f0 = t % ns, f1 = t / ns;
          double acc = 0.0;
          for (int a = 0; a < ns; ++a) {
            int x, y, z;
            if (d == 0) { x = a; y = f0; z = f1; }
            else if (d == 1) { x = f0; y = a; z = f1; }
            else { x = f0; y = f1; z = a; }
            acc = fma(ls[a], Us[k * PS + x + ns * (y + ns * z)], acc);
          }
          T1[t] = acc;
        }
        __syncthreads();
        psweep(ops.chi, ns, N, T1, T2, 0, ns, ns, 1);
        psweep(ops.chi, ns, N, T2, Vq + k * PS, 1, N, ns, 1);
      }
      for (int t = threadIdx.x; t < NFP; t += blockDim.x) {
        double w[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = Vq[k * PS + t];
        store_rec(face + (((size_t)e * 6 + 2 * d + s) * NSFR_NFIELD) * NFP + t, NFP, rec_from_entropy(w, ops, T, flag));
      }
      __syncthreads();
    }
}

}  // namespace

cudaError_t nsfr_launch_projection(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  const size_t smem = ((size_t)12 * PS + NSFR_MATH_TABLE_DOUBLES) * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(projection_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  nsfr_prof_begin(ctx, 1, s);
  projection_kernel<<<ctx->ne, 256, smem, s>>>(u, ctx->ops, ctx->face, ctx->nrec, ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}
