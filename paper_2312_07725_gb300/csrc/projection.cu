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
// A CTA takes a batch of elements; every step is a 1D contraction along one
// direction (sum factorisation) over all of the batch's elements and
// variables at once, on shared memory.  The kernel writes the node records
// of u~ at the GL points (rho, 2 beta, u/2, |u|^2/4, ln rho, ln beta) and the
// face records, the two inputs of the face-flux and volume kernels, exactly
// as the collocated face-state kernel does for its nodes.
#include "kernel_common.cuh"
#include "mathfn.cuh"
#include "physics.cuh"

namespace {
using namespace nsfr_k;

// the record of u(w), w entropy variables (the face-state conversion, with its
// constants ngig = -gamma/(gamma-1), nigm1 = -1/(gamma-1)); flags 2 beta <= 0 or
// NaN.  As in the face-state kernel: ln rho = (w_1 + beta |u|^2) - (gamma +
// ln(2 beta))/(gamma-1), the negations and the sign test on the integer pipe.
__device__ __forceinline__ Rec rec_from_entropy(const double w[5], double ngig, double nigm1, const MathTables& T,
                                                int* flag) {
  const double ln2 = 0.69314718055994530942;
  const double b2 = neg_i(w[4]);
  if (!pos_i(b2)) atomicOr(flag, 1);
  const double iv = rcp_ff(b2);
  const double u0 = w[1] * iv, u1 = w[2] * iv, u2 = w[3] * iv;  // u = -w_{2..4} / w_5
  const double q2 = fma(u0, u0, fma(u1, u1, u2 * u2));
  const double L5 = nsfr_log(b2, T);
  const double lr = fma(nigm1, L5, fma(mul_pow2<-1>(b2), q2, w[0] + ngig));
  Rec P;
  P.r = nsfr_exp(lr, T);
  P.b2 = b2;
  P.u0 = mul_pow2<-1>(u0);
  P.u1 = mul_pow2<-1>(u1);
  P.u2 = mul_pow2<-1>(u2);
  P.qq = mul_pow2<-2>(q2);
  P.lr = lr;
  P.lb = L5 - ln2;
  return P;
}

// elements per CTA: four arrays of 5 N^3 doubles per element in shared memory
__host__ __device__ constexpr int proj_epb(int n) { return n <= 4 ? 8 : n == 5 ? 4 : n == 6 ? 2 : 1; }

template <int N>
__global__ void __launch_bounds__(256) projection_kernel(const double* __restrict__ u, OpsGL ops,
                                                         double* __restrict__ face, double* __restrict__ nrec,
                                                         int ne, int* flag) {
  constexpr int NV = N * N * N, NFP = N * N, SL = 5 * NV, EPB = proj_epb(N);
  extern __shared__ double sm[];
  const int ns = ops.ns, nsv = ns * ns * ns;
  const int e0 = blockIdx.x * EPB, nel = min(EPB, ne - e0), nsl = 5 * nel;
  double* Us = sm;                  // [EPB*5][NV] solution-node values (first nsv of each slab)
  double* Vq = Us + EPB * SL;       // [EPB*5][NV] point values
  double* T1 = Vq + EPB * SL;
  double* T2 = T1 + EPB * SL;
  const MathTables T = nsfr_stage_tables(T2 + EPB * SL);
  const double g = ops.gamma, gm1 = g - 1.0, igm1 = ops.inv_gm1, ln2 = 0.69314718055994530942;
  const double cv0 = (g + ln2) * igm1, ngig = -g * igm1, nigm1 = -igm1;
  for (int t = threadIdx.x; t < nsl * nsv; t += blockDim.x)
    Us[(size_t)(t / nsv) * NV + t % nsv] = u[(size_t)e0 * 5 * nsv + t];
  __syncthreads();
  // u_q = chi u^ (all elements and variables at once)
  psweep(ops.chi, ns, N, Us, T1, nsl, NV, 0, ns, ns, ns);
  psweep(ops.chi, ns, N, T1, T2, nsl, NV, 1, N, ns, ns);
  psweep(ops.chi, ns, N, T2, Vq, nsl, NV, 2, N, N, ns);
  // v(u_q) in place
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    double* v = Vq + (size_t)(t / NV) * SL + t % NV;
    const double r = v[0], m0 = v[NV], m1 = v[2 * NV], m2 = v[3 * NV], E = v[4 * NV];
    const double ir = rcp_ff(r);
    const double u0 = m0 * ir, u1 = m1 * ir, u2 = m2 * ir;
    const double q2 = fma(u0, u0, fma(u1, u1, u2 * u2));
    const double p = gm1 * fma(neg_i(mul_pow2<-1>(r)), q2, E);
    if (!pos_i(r) || !pos_i(p)) atomicOr(flag, 1);
    const double b2 = r * rcp_ff(p);  // 2 beta
    // v_1 = (gamma - s)/(gamma-1) - beta |u|^2, s = ln 2p - ln 2 - gamma ln rho
    v[0] = fma(neg_i(mul_pow2<-1>(b2)), q2,
               fma(igm1, fma(g, nsfr_log(r, T), neg_i(nsfr_log(mul_pow2<1>(p), T))), cv0));
    v[NV] = b2 * u0;
    v[2 * NV] = b2 * u1;
    v[3 * NV] = b2 * u2;
    v[4 * NV] = neg_i(b2);
  }
  __syncthreads();
  // v~^ = Pi v(u_q), into Us
  psweep(ops.Pi, N, ns, Vq, T1, nsl, NV, 0, N, N, N);
  psweep(ops.Pi, N, ns, T1, T2, nsl, NV, 1, ns, N, N);
  psweep(ops.Pi, N, ns, T2, Us, nsl, NV, 2, ns, ns, N);
  // chi v~^ at the GL points -> node records of u~
  psweep(ops.chi, ns, N, Us, T1, nsl, NV, 0, ns, ns, ns);
  psweep(ops.chi, ns, N, T1, T2, nsl, NV, 1, N, ns, ns);
  psweep(ops.chi, ns, N, T2, Vq, nsl, NV, 2, N, N, ns);
  for (int t = threadIdx.x; t < nel * NV; t += blockDim.x) {
    const int le = t / NV, node = t % NV;
    const double* v = Vq + (size_t)le * SL + node;
    const double w[5] = {v[0], v[NV], v[2 * NV], v[3 * NV], v[4 * NV]};
    store_rec(nrec + (size_t)(e0 + le) * NSFR_NFIELD * NV + node, NV, rec_from_entropy(w, ngig, nigm1, T, flag));
  }
  __syncthreads();
  // faces: l_s along d (to extent 1), then chi along the two face directions
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) {
      const double* ls = s ? ops.ls_p : ops.ls_m;
      psweep(ls, ns, 1, Us, T1, nsl, NV, d, ns, ns, ns);
      if (d == 0) {
        psweep(ops.chi, ns, N, T1, T2, nsl, NV, 1, 1, ns, ns);
        psweep(ops.chi, ns, N, T2, Vq, nsl, NV, 2, 1, N, ns);
      } else if (d == 1) {
        psweep(ops.chi, ns, N, T1, T2, nsl, NV, 0, ns, 1, ns);
        psweep(ops.chi, ns, N, T2, Vq, nsl, NV, 2, N, 1, ns);
      } else {
        psweep(ops.chi, ns, N, T1, T2, nsl, NV, 0, ns, ns, 1);
        psweep(ops.chi, ns, N, T2, Vq, nsl, NV, 1, N, ns, 1);
      }
      for (int t = threadIdx.x; t < nel * NFP; t += blockDim.x) {
        const int le = t / NFP, fn = t % NFP;
        const double* v = Vq + (size_t)le * SL + fn;
        const double w[5] = {v[0], v[NV], v[2 * NV], v[3 * NV], v[4 * NV]};
        store_rec(face + (((size_t)(e0 + le) * 6 + 2 * d + s) * NSFR_NFIELD) * NFP + fn, NFP,
                  rec_from_entropy(w, ngig, nigm1, T, flag));
      }
      __syncthreads();
    }
}

template <int N>
cudaError_t launch_projection_n(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  constexpr int NV = N * N * N, EPB = proj_epb(N);
  const size_t smem = ((size_t)EPB * 20 * NV + NSFR_MATH_TABLE_DOUBLES) * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(projection_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  nsfr_prof_begin(ctx, 1, s);
  projection_kernel<N><<<(ctx->ne + EPB - 1) / EPB, 256, smem, s>>>(u, ctx->ops, ctx->face, ctx->nrec, ctx->ne,
                                                                   ctx->flag);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace

// u_q = chi u^ for every element (square chi: the GL points carry as many
// nodes as the solution), written to uq[N_e][5][N^3]
template <int N>
__global__ void __launch_bounds__(256) interp_kernel(const double* __restrict__ u, OpsGL ops,
                                                     double* __restrict__ uq, int ne) {
  constexpr int NV = N * N * N, SL = 5 * NV, EPB = proj_epb(N);
  extern __shared__ double sm[];
  const int ns = ops.ns, nsv = ns * ns * ns;
  const int e0 = blockIdx.x * EPB, nel = min(EPB, ne - e0), nsl = 5 * nel;
  double* Us = sm;
  double* T1 = Us + EPB * SL;
  double* T2 = T1 + EPB * SL;
  for (int t = threadIdx.x; t < nsl * nsv; t += blockDim.x)
    Us[(size_t)(t / nsv) * NV + t % nsv] = u[(size_t)e0 * 5 * nsv + t];
  __syncthreads();
  psweep(ops.chi, ns, N, Us, T1, nsl, NV, 0, ns, ns, ns);
  psweep(ops.chi, ns, N, T1, T2, nsl, NV, 1, N, ns, ns);
  psweep(ops.chi, ns, N, T2, Us, nsl, NV, 2, N, N, ns);
  for (int t = threadIdx.x; t < nsl * NV; t += blockDim.x) uq[(size_t)e0 * SL + t] = Us[t];
}

template <int N>
cudaError_t launch_interp_n(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  constexpr int NV = N * N * N, EPB = proj_epb(N);
  const size_t smem = (size_t)EPB * 15 * NV * sizeof(double);
  cudaError_t err = cudaFuncSetAttribute(interp_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  nsfr_prof_begin(ctx, 1, s);
  interp_kernel<N><<<(ctx->ne + EPB - 1) / EPB, 256, smem, s>>>(u, ctx->ops, ctx->uq, ctx->ne);
  nsfr_prof_end(ctx, s);
  ctx->launches++;
  return cudaGetLastError();
}

cudaError_t nsfr_launch_interp_square(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  switch (ctx->n) {
    case 2: return launch_interp_n<2>(ctx, u, s);
    case 3: return launch_interp_n<3>(ctx, u, s);
    case 4: return launch_interp_n<4>(ctx, u, s);
    case 5: return launch_interp_n<5>(ctx, u, s);
    case 6: return launch_interp_n<6>(ctx, u, s);
    case 7: return launch_interp_n<7>(ctx, u, s);
    case 8: return launch_interp_n<8>(ctx, u, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t nsfr_launch_projection(nsfr_ctx* ctx, const double* u, cudaStream_t s) {
  switch (ctx->n) {
    case 2: return launch_projection_n<2>(ctx, u, s);
    case 3: return launch_projection_n<3>(ctx, u, s);
    case 4: return launch_projection_n<4>(ctx, u, s);
    case 5: return launch_projection_n<5>(ctx, u, s);
    case 6: return launch_projection_n<6>(ctx, u, s);
    case 7: return launch_projection_n<7>(ctx, u, s);
    case 8: return launch_projection_n<8>(ctx, u, s);
  }
  return cudaErrorInvalidValue;
}
