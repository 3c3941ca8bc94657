// Diagnostic evaluation of the library's own model for one particle: rate
// vector f, analytic Jacobian J and the Eq. 7 root S_H, on the host or on the
// GPU (the same source compiled for both).  Used to generate the Jacobian's
// sparsity pattern at build time and to compare J with an independent
// differentiation in the tests.
#include <cuda_runtime.h>

#include <cstring>

#include "adm1_device.cuh"
#include "chad.h"
#include "model.h"

namespace chad {
namespace {

struct EvalIn {
  DigConst c;
  double T, D, SH_guess;
  double y[NS];
};
struct EvalOut {
  double f[NS];
  double J[NS * NS];
  double SH;
  int newton_failed;
};

__host__ __device__ void eval_one(const EvalIn& in, EvalOut& out) {
  PartConst q;
  part_const(in.c, in.T, q);
  AcidBase ab;
  NewtonCounters nc{0, 0, 0};
  solve_SH(in.c, q, in.y, in.SH_guess, 50, ab, nc);
  Rates<double> o;
  rates<double, true>(in.c, q, in.y, ab, o);
  balances<double>(in.c, in.y, in.D, o, out.f);
  jacobian<DenseIdx, double>(in.c, q, in.y, in.D, ab, o, out.J);
  out.SH = ab.SH;
  out.newton_failed = nc.failed;
}

__global__ void eval_kernel(const EvalIn* in, EvalOut* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) eval_one(*in, *out);
}

}  // namespace
}  // namespace chad

using namespace chad;

extern "C" chad_status chad_eval_model(const double* params, double V_liq, double V_gas, double D,
                                       const double* y_in, double T, const double* y,
                                       double SH_guess, double* f, double* J, double* SH,
                                       int on_device) {
  if (!params || !y || !f || !J || !SH) return CHAD_E_INVALID;
  if (!(T > 0.0)) return CHAD_E_INVALID;
  EvalIn in;
  std::memset(&in, 0, sizeof(in));
  const char* why = "";
  if (!derive_digester(params, V_liq, V_gas, D, y_in, in.c, &why)) return CHAD_E_INVALID;
  in.T = T;
  in.D = D;
  in.SH_guess = SH_guess;
  for (int i = 0; i < NS; ++i) in.y[i] = y[i];
  EvalOut out;
  if (on_device) {
    EvalIn* din = nullptr;
    EvalOut* dout = nullptr;
    if (cudaMalloc(&din, sizeof(EvalIn)) != cudaSuccess) return CHAD_E_NOMEM;
    if (cudaMalloc(&dout, sizeof(EvalOut)) != cudaSuccess) { cudaFree(din); return CHAD_E_NOMEM; }
    cudaError_t e = cudaMemcpy(din, &in, sizeof(in), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      eval_kernel<<<1, 32>>>(din, dout);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&out, dout, sizeof(out), cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
    if (e != cudaSuccess) return CHAD_E_CUDA;
  } else {
    eval_one(in, out);
  }
  std::memcpy(f, out.f, sizeof(out.f));
  std::memcpy(J, out.J, sizeof(out.J));
  *SH = out.SH;
  return out.newton_failed ? CHAD_E_PARTICLE : CHAD_OK;
}
