// Integrator kernel instance: precision form 1, at least 3 resident
// 128-thread blocks per SM (sets the register budget).  See integrate_impl.cuh.
#include "integrate_impl.cuh"

namespace chad {
cudaError_t launch_integrate_f1_v1(const StepArgs& a, cudaStream_t s) {
  return launch_variant<1, 3>(a, s);
}
}  // namespace chad
