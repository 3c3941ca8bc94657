// Integrator kernel instance: form 2, 128 threads per block, at least
// 3 resident blocks per SM, W_d in per-thread arrays (variant 1 of
// kernel_variant in kernels.h).  See integrate_impl.cuh.
#include "integrate_impl.cuh"

namespace chad {
cudaError_t launch_integrate_f2_v1(const StepArgs& a, cudaStream_t s) {
  return launch_variant<2, 128, 3, false>(a, s);
}
}  // namespace chad
