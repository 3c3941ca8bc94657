// Integrator kernel instance: precision form 1, at least 4 resident
// 128-thread blocks per SM (sets the register budget).  See integrate_impl.cuh.
#include "integrate_impl.cuh"

namespace chad {
cudaError_t launch_integrate_f1_v2(const StepArgs& a, cudaStream_t s) {
  return launch_variant<1, 4>(a, s);
}
}  // namespace chad
