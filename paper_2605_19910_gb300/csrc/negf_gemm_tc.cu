// Split-precision complex block products on the tcgen05 tensor cores.
#include "negf_common.cuh"
#include "negf_kernels.h"

namespace negf {

cudaError_t zinv_init();

bool zgemm_tc_available() { return false; }

cudaError_t zgemm_tc(const ZGemm& g, cudaStream_t st) {
  (void)g; (void)st;
  return cudaErrorNotSupported;
}

cudaError_t kernels_init() {
  cudaError_t e = zinv_init();
  return e;
}

}  // namespace negf
