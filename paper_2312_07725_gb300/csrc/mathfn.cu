// Elementwise evaluation of the library's own device elementary functions
// (nsfr_math_eval): the FP64 log and exp of mathfn.cuh, the float-float ones
// of mathfn_ff.cuh, the reciprocals of physics.cuh, the integer-pipe split,
// join and int-to-double conversion of ffloat.cuh and the volume kernels'
// logarithmic mean, so that they can be checked against reference values.
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
      case NSFR_FN_JOIN: {  // the 64 bits of v as two floats, hi in the high word
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        r = ff_join_i(ff{__uint_as_float((unsigned int)(b >> 32)), __uint_as_float((unsigned int)b)});
        break;
      }
      case NSFR_FN_SPLIT: {  // the integer-pipe split of v, hi in the high 32 bits, lo in the low
        const ff q = ff_split_i(v);
        r = __hiloint2double((int)__float_as_uint(q.hi), (int)__float_as_uint(q.lo));
        break;
      }
      case NSFR_FN_I2D: r = i2d_i(__double2loint(v)); break;  // the low 32 bits of v as an int
      case NSFR_FN_LOGMEAN1: {  // logarithmic mean of v and 1 as the volume kernels form it
        // G(u) - 1 = u (c1 + u (c2 + u c3)): c1 = -1/3, c2 = -4/45 (hi, lo), c3 = -44/945
        const double c1 = -1.0 / 3.0, c2 = -4.0 / 45.0;
        const float c[5] = {d2f_i(c1), d2f_i(c1 - f2d_i(d2f_i(c1))), d2f_i(c2), d2f_i(c2 - f2d_i(d2f_i(c2))),
                            d2f_i(-44.0 / 945.0)};
        double eps;
        if (lm_series_ff(ff_from_double(v), ff{1.0f, 0.0f}, c, eps)) {
          const double sh = mul_pow2<-1>(v + 1.0);
          r = fma(sh, eps, sh);
        } else {
          r = (v - 1.0) / nsfr_log(v);
        }
        break;
      }
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
