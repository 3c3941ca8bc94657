// Integrator kernel instance: form 0, 64 threads per block, at least
// 2 resident blocks per SM, W_d in shared memory (variant 6 of
// kernel_variant in kernels.h).  See integrate_impl.cuh.
#include "integrate_impl.cuh"

namespace chad {
cudaError_t launch_integrate_f0_v6(const StepArgs& a, cudaStream_t s) {
  return launch_variant<0, 64, 2, true>(a, s);
}
}  // namespace chad
