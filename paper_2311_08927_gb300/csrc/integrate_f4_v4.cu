// Integrator kernel instance: form 4 (mixed with S_h2 algebraic), 256 threads per block, at least
// 1 resident blocks per SM, W_d in per-thread arrays (variant 4 of
// kernel_variant in kernels.h).  See integrate_mx.cuh.
#include "integrate_mx.cuh"

namespace chad {
cudaError_t launch_integrate_f4_v4(const StepArgs& a, cudaStream_t s) {
  return launch_variant_mx<256, 1, false>(a, s);
}
}  // namespace chad
