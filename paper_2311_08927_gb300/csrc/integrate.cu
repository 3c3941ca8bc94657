// Dispatch of the integrator over kernel forms (0 FP64, 1 mixed, 2 mixed with
// FP32 stage rates, 3 FP64 with S_h2 algebraic, 4 mixed with S_h2 algebraic)
// and tuned kernel variants
// (each instance lives in its own translation unit so they build in parallel).
#include "kernels.h"

namespace chad {

#define CHAD_DECL(f, v) cudaError_t launch_integrate_f##f##_v##v(const StepArgs& a, cudaStream_t s);
CHAD_DECL(0, 0) CHAD_DECL(0, 1) CHAD_DECL(0, 2)
CHAD_DECL(1, 0) CHAD_DECL(1, 1) CHAD_DECL(1, 2)
CHAD_DECL(2, 0) CHAD_DECL(2, 1) CHAD_DECL(2, 2)
CHAD_DECL(3, 0) CHAD_DECL(3, 1) CHAD_DECL(3, 2)
CHAD_DECL(4, 0) CHAD_DECL(4, 1) CHAD_DECL(4, 2)
#undef CHAD_DECL

cudaError_t launch_integrate(const StepArgs& a, int precision, int variant, cudaStream_t s) {
  using Fn = cudaError_t (*)(const StepArgs&, cudaStream_t);
  static const Fn table[5][kNumVariants] = {
      {launch_integrate_f0_v0, launch_integrate_f0_v1, launch_integrate_f0_v2},
      {launch_integrate_f1_v0, launch_integrate_f1_v1, launch_integrate_f1_v2},
      {launch_integrate_f2_v0, launch_integrate_f2_v1, launch_integrate_f2_v2},
      {launch_integrate_f3_v0, launch_integrate_f3_v1, launch_integrate_f3_v2},
      {launch_integrate_f4_v0, launch_integrate_f4_v1, launch_integrate_f4_v2}};
  if (a.n <= 0) return cudaSuccess;
  if (variant < 0 || variant >= kNumVariants) variant = kDefaultVariant;
  if (precision < 0 || precision > 4) precision = 0;
  return table[precision][variant](a, s);
}

}  // namespace chad
