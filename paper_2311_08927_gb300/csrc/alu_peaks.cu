// FMA-chain throughput probe used as the roofline denominator of the
// ALU-bound integrator: FP64 DFMA and FP32 FFMA rates of the current GPU
// with every SM busy (8 independent chains per thread, 16 warps per SM).
#include <cuda_runtime.h>

#include "chad.h"

namespace {

template <class R, int ILP>
__global__ void fma_chain(R* out, int iters, R a, R b) {
  R x[ILP];
#pragma unroll
  for (int k = 0; k < ILP; ++k) x[k] = R(threadIdx.x) * R(1e-3) + R(k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < ILP; ++k) x[k] = fma(x[k], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int k = 0; k < ILP; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" chad_status chad_probe_alu_peak(int fp64, double* tflops) {
  if (!tflops) return CHAD_E_INVALID;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CHAD_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CHAD_E_CUDA;
  const int threads = 512, blocks = sms;  // 16 warps per SM
  const int iters = fp64 ? 20000 : 200000;
  void* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess) return CHAD_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    if (fp64)
      fma_chain<double, 8><<<blocks, threads>>>((double*)out, iters, 1.0000001, 1e-9);
    else
      fma_chain<float, 8><<<blocks, threads>>>((float*)out, iters, 1.0000001f, 1e-9f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return CHAD_E_CUDA;
  *tflops = 2.0 * 8.0 * (double)iters * threads * blocks / (best * 1e-3) / 1e12;
  return CHAD_OK;
}
