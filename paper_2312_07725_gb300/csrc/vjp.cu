// Reverse-mode (VJP) kernels of the residual: not built yet in this file.
#include "nsfr_internal.h"

cudaError_t nsfr_launch_vjp(nsfr_ctx*, const double*, const double*, double*, double*, cudaStream_t) {
  return cudaErrorNotSupported;
}
