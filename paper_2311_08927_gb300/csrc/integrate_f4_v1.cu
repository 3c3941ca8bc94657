// Integrator kernel instance: form 4 (mixed with S_h2 algebraic), at least
// 3 resident 128-thread blocks per SM (sets the register budget).  See
// integrate_mx.cuh.
#include "integrate_mx.cuh"

namespace chad {
cudaError_t launch_integrate_f4_v1(const StepArgs& a, cudaStream_t s) {
  return launch_variant_mx<3>(a, s);
}
}  // namespace chad
