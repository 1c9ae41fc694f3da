// FMA-throughput probe: the measured denominator of the kernels' ALU rooflines.
//
// Every thread runs NSFR_PROBE_CHAINS independent multiply-add chains
// x <- x a + b (FP64 or FP32), each step depending on the one before, so the
// pipe sees NSFR_PROBE_CHAINS independent instructions per thread between
// dependent ones; the grid fills every SM several times.  The caller times the
// launch; the FMA count is threads x chains x iters.  The chains converge to
// b / (1 - a) and never overflow; the sum of their end values is written so
// that nothing is optimised away.
#include "nsfr_internal.h"

#define NSFR_PROBE_CHAINS 8

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(long long iters, T a, T b, double* sink) {
  T x[NSFR_PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < NSFR_PROBE_CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < NSFR_PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < NSFR_PROBE_CHAINS; ++c) s += x[c];
  if (s == (T)-1) sink[0] = (double)s;  // never true for these chains; keeps them live
  if (threadIdx.x == 0 && blockIdx.x == 0) sink[1] = (double)s;
}

}  // namespace

extern "C" nsfr_status nsfr_fma_probe(int fp32, long long iters, int blocks, double* sink, long long* fmas,
                                      void* stream) {
  if (iters < 1 || blocks < 1 || !sink || !fmas) return NSFR_ERR_ARG;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, sink) != cudaSuccess) {
    cudaGetLastError();
    return NSFR_ERR_ARG;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return NSFR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (fp32)
    fma_probe_kernel<float><<<blocks, 256, 0, s>>>(iters, 0.999999f, 1.0e-6f, sink);
  else
    fma_probe_kernel<double><<<blocks, 256, 0, s>>>(iters, 0.999999999, 1.0e-9, sink);
  *fmas = (long long)blocks * 256 * NSFR_PROBE_CHAINS * iters;
  return cudaGetLastError() == cudaSuccess ? NSFR_OK : NSFR_ERR_CUDA;
}
