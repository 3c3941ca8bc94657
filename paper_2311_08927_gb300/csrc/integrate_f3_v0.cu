// Integrator kernel instance: form 3 (FP64, S_h2 algebraic), at least 2 resident
// 128-thread blocks per SM (sets the register budget).  See integrate_impl.cuh.
#include "integrate_impl.cuh"

namespace chad {
cudaError_t launch_integrate_f3_v0(const StepArgs& a, cudaStream_t s) {
  return launch_variant<3, 2>(a, s);
}
}  // namespace chad
