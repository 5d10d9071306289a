// Mixed-precision sigma (tcgen05 tensor-core path): placeholder until the
// kernels land; fails loudly instead of falling back.
#include "internal.cuh"

namespace ea {
void sigma_mixed(cudaStream_t, State&, int, const double*, double*) {
  fail(EAADC_ERR_ARG, "mixed-precision sigma is not available in this build");
}
}  // namespace ea
