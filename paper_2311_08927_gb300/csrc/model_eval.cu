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
  double x[NS];  // direction of the Jacobian-vector product (split only)
};
struct EvalOut {
  double f[NS];
  double J[NS * NS];  // full J, or J_d when split
  double u[NS], v[NS];
  double Jx[NS];  // J x from the rate partials (split only)
  double SH;
  int newton_failed;
};

// split = false: full J; split = true: J_d, u = df/dS_H, v = dS_H/dy.
__host__ __device__ void eval_one(const EvalIn& in, EvalOut& out, bool split) {
  PartConst q;
  part_const(in.c, in.T, q);
  AcidBase ab;
  NewtonCounters nc{0, 0, 0};
  solve_SH(in.c, q, in.y, in.SH_guess, 50, ab, nc);
  Rates<double> o;
  rates<double, true>(in.c, q, in.y, ab, o);
  balances<double>(in.c, in.y, in.D, o, out.f);
  for (int i = 0; i < NS; ++i) out.u[i] = out.v[i] = 0.0;
  if (split) {
    jacobian<DenseIdx, double>(in.c, q, in.y, in.D, ab, o, out.J, out.u);
    double vd[8];
    sh_tangent(in.c, q, ab, vd);
    const int hc[8] = {iS_va, iS_bu, iS_pro, iS_ac, iS_IC, iS_IN, iS_cat, iS_an};
    for (int k = 0; k < 8; ++k) out.v[hc[k]] = vd[k];
    double s = 0.0;
    for (int k = 0; k < 8; ++k) s += vd[k] * in.x[hc[k]];
    jvp<double, double>(in.c, in.y, in.D, o, in.x, s, out.Jx);
  } else {
    jacobian<DenseIdx, double>(in.c, q, in.y, in.D, ab, o, out.J);
  }
  out.SH = ab.SH;
  out.newton_failed = nc.failed;
}

__global__ void eval_kernel(const EvalIn* in, EvalOut* out, bool split) {
  if (threadIdx.x == 0 && blockIdx.x == 0) eval_one(*in, *out, split);
}

chad_status eval_common(const double* params, double V_liq, double V_gas, double D,
                        const double* y_in, double T, const double* y, double SH_guess,
                        const double* x, bool split, int on_device, EvalOut& out) {
  if (!params || !y) return CHAD_E_INVALID;
  if (!(T > 0.0)) return CHAD_E_INVALID;
  EvalIn in;
  std::memset(&in, 0, sizeof(in));
  const char* why = "";
  if (!derive_digester(params, V_liq, V_gas, D, y_in, in.c, &why)) return CHAD_E_INVALID;
  in.T = T;
  in.D = D;
  in.SH_guess = SH_guess;
  for (int i = 0; i < NS; ++i) {
    in.y[i] = y[i];
    in.x[i] = x ? x[i] : 0.0;
  }
  if (on_device) {
    EvalIn* din = nullptr;
    EvalOut* dout = nullptr;
    if (cudaMalloc(&din, sizeof(EvalIn)) != cudaSuccess) return CHAD_E_NOMEM;
    if (cudaMalloc(&dout, sizeof(EvalOut)) != cudaSuccess) { cudaFree(din); return CHAD_E_NOMEM; }
    cudaError_t e = cudaMemcpy(din, &in, sizeof(in), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      eval_kernel<<<1, 32>>>(din, dout, split);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&out, dout, sizeof(out), cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
    if (e != cudaSuccess) return CHAD_E_CUDA;
  } else {
    eval_one(in, out, split);
  }
  return out.newton_failed ? CHAD_E_PARTICLE : CHAD_OK;
}

}  // namespace
}  // namespace chad

using namespace chad;

extern "C" chad_status chad_eval_model(const double* params, double V_liq, double V_gas, double D,
                                       const double* y_in, double T, const double* y,
                                       double SH_guess, double* f, double* J, double* SH,
                                       int on_device) {
  if (!f || !J || !SH) return CHAD_E_INVALID;
  EvalOut out;
  const chad_status st =
      eval_common(params, V_liq, V_gas, D, y_in, T, y, SH_guess, nullptr, false, on_device, out);
  if (st != CHAD_OK && st != CHAD_E_PARTICLE) return st;
  std::memcpy(f, out.f, sizeof(out.f));
  std::memcpy(J, out.J, sizeof(out.J));
  *SH = out.SH;
  return st;
}

extern "C" chad_status chad_eval_model_split(const double* params, double V_liq, double V_gas,
                                             double D, const double* y_in, double T,
                                             const double* y, double SH_guess, const double* x,
                                             double* f, double* J_d, double* u, double* v,
                                             double* Jx, double* SH, int on_device) {
  if (!f || !J_d || !u || !v || !SH) return CHAD_E_INVALID;
  if ((x == nullptr) != (Jx == nullptr)) return CHAD_E_INVALID;
  EvalOut out;
  const chad_status st =
      eval_common(params, V_liq, V_gas, D, y_in, T, y, SH_guess, x, true, on_device, out);
  if (st != CHAD_OK && st != CHAD_E_PARTICLE) return st;
  std::memcpy(f, out.f, sizeof(out.f));
  std::memcpy(J_d, out.J, sizeof(out.J));
  std::memcpy(u, out.u, sizeof(out.u));
  std::memcpy(v, out.v, sizeof(out.v));
  if (Jx) std::memcpy(Jx, out.Jx, sizeof(out.Jx));
  *SH = out.SH;
  return st;
}

namespace chad {
namespace {
__global__ void numerics_kernel(const double* x, int n, float* narrow, double* widen,
                                double* recip) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = x[i];
  narrow[i] = cvt<float, double>(d);
  widen[i] = cvt<double, float>(__double2float_rn(d));
  recip[i] = rcp<double>(d);
}
}  // namespace
}  // namespace chad

extern "C" chad_status chad_probe_numerics(const double* x, int n, float* narrow, double* widen,
                                           double* recip) {
  if (!x || !narrow || !widen || !recip || n < 0) return CHAD_E_INVALID;
  if (n == 0) return CHAD_OK;
  const size_t nb = (size_t)n;
  double* dx = nullptr;
  float* dn = nullptr;
  double* dw = nullptr;
  double* dr = nullptr;
  cudaError_t e = cudaMalloc(&dx, nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dn, nb * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dw, nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dr, nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, nb * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    numerics_kernel<<<(unsigned)((nb + 255) / 256), 256>>>(dx, n, dn, dw, dr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(narrow, dn, nb * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(widen, dw, nb * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(recip, dr, nb * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dn);
  cudaFree(dw);
  cudaFree(dr);
  return e == cudaSuccess ? CHAD_OK : CHAD_E_CUDA;
}
