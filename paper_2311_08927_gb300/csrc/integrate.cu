// Dispatch of the integrator over kernel forms (0 FP64, 1 mixed, 2 mixed with
// FP32 stage rates, 3 FP64 with S_h2 algebraic, 4 mixed with S_h2 algebraic)
// and tuned kernel variants
// (each instance lives in its own translation unit so they build in parallel).
#include "kernels.h"

namespace chad {

#define CHAD_DECL(f, v) cudaError_t launch_integrate_f##f##_v##v(const StepArgs& a, cudaStream_t s);
#define CHAD_FORM(f) CHAD_DECL(f, 0) CHAD_DECL(f, 1) CHAD_DECL(f, 2) CHAD_DECL(f, 3) \
  CHAD_DECL(f, 4) CHAD_DECL(f, 5) CHAD_DECL(f, 6)
CHAD_FORM(0) CHAD_FORM(1) CHAD_FORM(2) CHAD_FORM(3) CHAD_FORM(4)
#undef CHAD_FORM
#undef CHAD_DECL

cudaError_t launch_integrate(const StepArgs& a, int precision, int variant, cudaStream_t s) {
  using Fn = cudaError_t (*)(const StepArgs&, cudaStream_t);
#define CHAD_ROW(f) {launch_integrate_f##f##_v0, launch_integrate_f##f##_v1, \
  launch_integrate_f##f##_v2, launch_integrate_f##f##_v3, launch_integrate_f##f##_v4, \
  launch_integrate_f##f##_v5, launch_integrate_f##f##_v6}
  static const Fn table[5][kNumVariants] = {CHAD_ROW(0), CHAD_ROW(1), CHAD_ROW(2), CHAD_ROW(3),
                                            CHAD_ROW(4)};
#undef CHAD_ROW
  if (a.n <= 0) return cudaSuccess;
  if (variant < 0 || variant >= kNumVariants) variant = kDefaultVariant;
  if (precision < 0 || precision > 4) precision = 0;
  return table[precision][variant](a, s);
}

}  // namespace chad
