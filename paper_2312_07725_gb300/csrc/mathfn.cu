// Elementwise evaluation of the library's own device elementary functions
// (nsfr_math_eval): the FP64 log and exp of mathfn.cuh, the float-float ones
// of mathfn_ff.cuh and the reciprocals of physics.cuh, so that they can be
// checked against reference values.
#include "mathfn.cuh"
#include "mathfn_ff.cuh"
#include "physics.cuh"

namespace {

__global__ void math_eval_kernel(int fn, const double* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    double r;
    switch (fn) {
      case NSFR_FN_LOG: r = nsfr_log(v); break;
      case NSFR_FN_EXP: r = nsfr_exp(v); break;
      case NSFR_FN_RCP: r = rcp_full(v); break;
      case NSFR_FN_LOG_FF: r = ff_to_double(ff_log(ff_from_double(v), nsfr_global_tables_f())); break;
      case NSFR_FN_EXP_FF: r = ff_to_double(ff_exp(ff_from_double(v), nsfr_global_tables_f())); break;
      default: r = rcp_newton1(v); break;
    }
    y[i] = r;
  }
}

}  // namespace

cudaError_t nsfr_launch_math_eval(int fn, const double* x, double* y, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  math_eval_kernel<<<(int)blocks, 256, 0, s>>>(fn, x, y, n);
  return cudaGetLastError();
}
