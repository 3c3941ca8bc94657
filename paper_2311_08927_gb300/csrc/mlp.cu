// Learned initial guesses: a 32 -> 64 -> 64 -> 2 multilayer perceptron with
// SiLU activations, BF16 weights and activations, FP32 accumulation, run on
// the tensor cores with warp-level mma.sync (m16n8k16, BF16 inputs, FP32
// accumulators).  It predicts the standardised log10 S_H+ (Eq. 7 root) and
// log10 of the next accepted step size from the log-scaled ADM1 state and the
// temperature; the Newton solver and the step controller stay the judges.
//
// Kernels: feature extraction, inference, fused forward + backward of the
// mean-squared loss with deterministic per-block gradient partials, a
// fixed-order reduction of those partials, FP32 Adam, and the guess kernel
// that runs on the particle state of a context.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "chad.h"
#include "kernels.h"
#include "model.h"

namespace chad {
namespace mlp {

constexpr int IN = 32, HID = 64, OUT = 2, OUTP = 8;  // OUT padded to one n8 tile
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * IN, OFF_W2 = OFF_B1 + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + OUT * HID;
constexpr int NPARAM = OFF_B3 + OUT;
static_assert(NPARAM == CHAD_MLP_NPARAM, "parameter count");
constexpr float kLogFloor = 1e-20f;

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Warp-level C(+)= A B with A(m,k) = As[m*sam + k*sak], B(k,n) = Bs[k*sbk + n*sbn]
// (BF16, shared memory) and C(m,n) = Cs[m*ldc + n] (FP32, shared memory).
// M % 16 == 0, N % 8 == 0, K % 16 == 0.  Fragments follow the m16n8k16
// layouts: A rows g and g+8, columns 2t..2t+1 and 2t+8..2t+9; B columns g,
// rows 2t..2t+1 and 2t+8..2t+9; C rows g and g+8, columns 2t..2t+1
// (g = lane / 4, t = lane % 4).
__device__ void warp_gemm(const __nv_bfloat16* As, int sam, int sak, const __nv_bfloat16* Bs,
                          int sbk, int sbn, float* Cs, int ldc, int M, int N, int K,
                          bool accumulate) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int mt = 0; mt < M; mt += 16) {
    for (int nt = 0; nt < N; nt += 8) {
      float acc[4];
      const int r0 = mt + g, r1 = mt + g + 8, c0 = nt + 2 * t;
      if (accumulate) {
        acc[0] = Cs[r0 * ldc + c0];
        acc[1] = Cs[r0 * ldc + c0 + 1];
        acc[2] = Cs[r1 * ldc + c0];
        acc[3] = Cs[r1 * ldc + c0 + 1];
      } else {
        acc[0] = acc[1] = acc[2] = acc[3] = 0.0f;
      }
      for (int kt = 0; kt < K; kt += 16) {
        const int k0 = kt + 2 * t, k1 = kt + 2 * t + 8;
        uint32_t a[4], b[2];
        a[0] = pack2(As[r0 * sam + k0 * sak], As[r0 * sam + (k0 + 1) * sak]);
        a[1] = pack2(As[r1 * sam + k0 * sak], As[r1 * sam + (k0 + 1) * sak]);
        a[2] = pack2(As[r0 * sam + k1 * sak], As[r0 * sam + (k1 + 1) * sak]);
        a[3] = pack2(As[r1 * sam + k1 * sak], As[r1 * sam + (k1 + 1) * sak]);
        const int n = nt + g;
        b[0] = pack2(Bs[k0 * sbk + n * sbn], Bs[(k0 + 1) * sbk + n * sbn]);
        b[1] = pack2(Bs[k1 * sbk + n * sbn], Bs[(k1 + 1) * sbk + n * sbn]);
        mma_bf16(acc, a, b);
      }
      Cs[r0 * ldc + c0] = acc[0];
      Cs[r0 * ldc + c0 + 1] = acc[1];
      Cs[r1 * ldc + c0] = acc[2];
      Cs[r1 * ldc + c0 + 1] = acc[3];
    }
  }
  __syncwarp();
}

// Shared-memory image of the weights (BF16) and biases (FP32).
struct WeightsSmem {
  __nv_bfloat16 W1[HID * IN];
  __nv_bfloat16 W2[HID * HID];
  __nv_bfloat16 W3[OUTP * HID];  // rows OUT..OUTP-1 are zero
  float b1[HID], b2[HID], b3[OUTP];
};

__device__ void load_weights(const float* P, WeightsSmem& w) {
  for (int i = threadIdx.x; i < HID * IN; i += blockDim.x) w.W1[i] = __float2bfloat16_rn(P[OFF_W1 + i]);
  for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) w.W2[i] = __float2bfloat16_rn(P[OFF_W2 + i]);
  for (int i = threadIdx.x; i < OUTP * HID; i += blockDim.x)
    w.W3[i] = __float2bfloat16_rn(i < OUT * HID ? P[OFF_W3 + i] : 0.0f);
  for (int i = threadIdx.x; i < HID; i += blockDim.x) {
    w.b1[i] = P[OFF_B1 + i];
    w.b2[i] = P[OFF_B2 + i];
  }
  for (int i = threadIdx.x; i < OUTP; i += blockDim.x) w.b3[i] = i < OUT ? P[OFF_B3 + i] : 0.0f;
}

// Per-warp activation buffers for 32 samples.
struct WarpBufs {
  __nv_bfloat16 X[32 * IN];
  float Z1[32 * HID];
  __nv_bfloat16 A1[32 * HID];
  float Z2[32 * HID];
  __nv_bfloat16 A2[32 * HID];
  float O[32 * OUTP];
};

// Forward pass of 32 samples whose features are in b.X.
__device__ void forward32(const WeightsSmem& w, WarpBufs& b) {
  const int lane = threadIdx.x & 31;
  // Z1 = X W1^T: A(i,k) = X[i][k]; B(k,n) = W1[n][k]
  warp_gemm(b.X, IN, 1, w.W1, 1, IN, b.Z1, HID, 32, HID, IN, false);
  for (int e = lane; e < 32 * HID; e += 32) {
    const float z = b.Z1[e] + w.b1[e % HID];
    b.Z1[e] = z;
    b.A1[e] = __float2bfloat16_rn(silu(z));
  }
  __syncwarp();
  warp_gemm(b.A1, HID, 1, w.W2, 1, HID, b.Z2, HID, 32, HID, HID, false);
  for (int e = lane; e < 32 * HID; e += 32) {
    const float z = b.Z2[e] + w.b2[e % HID];
    b.Z2[e] = z;
    b.A2[e] = __float2bfloat16_rn(silu(z));
  }
  __syncwarp();
  warp_gemm(b.A2, HID, 1, w.W3, 1, HID, b.O, OUTP, 32, OUTP, HID, false);
  for (int e = lane; e < 32 * OUTP; e += 32) b.O[e] += w.b3[e % OUTP];
  __syncwarp();
}

// Features of one particle: (log10 max(y_i, floor) - mu_i) * inv_sigma_i for
// the 29 states, (T/100 - mu) * inv_sigma for the temperature, zero padding.
__device__ __forceinline__ void features(const double* y, int64_t ld, int64_t p, double T,
                                         const float* norm, __nv_bfloat16* row) {
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    const float v = fmaxf((float)y[(int64_t)i * ld + p], kLogFloor);
    row[i] = __float2bfloat16_rn((log10f(v) - norm[i]) * norm[IN + i]);
  }
  row[NS] = __float2bfloat16_rn(((float)T * 0.01f - norm[NS]) * norm[IN + NS]);
  row[NS + 1] = __float2bfloat16_rn(0.0f);
  row[NS + 2] = __float2bfloat16_rn(0.0f);
}

__global__ void features_kernel(const double* y, int64_t ld, const double* T, int64_t n,
                                const float* norm, __nv_bfloat16* X) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  features(y, ld, p, T[p], norm, X + p * IN);
}

// Inference: out[p][0..1] = MLP(X[p]) (standardised outputs).
__global__ void __launch_bounds__(128) forward_kernel(const __nv_bfloat16* X, int64_t n,
                                                      const float* P, float* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  WeightsSmem& w = *reinterpret_cast<WeightsSmem*>(smem);
  WarpBufs& b = reinterpret_cast<WarpBufs*>(smem + sizeof(WeightsSmem))[threadIdx.x >> 5];
  load_weights(P, w);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
       base += warps * 32) {
    for (int e = lane; e < 32 * IN; e += 32) {
      const int64_t p = base + e / IN;
      b.X[e] = p < n ? X[p * IN + e % IN] : __float2bfloat16_rn(0.0f);
    }
    __syncwarp();
    forward32(w, b);
    const int64_t p = base + lane;
    if (p < n) {
      out[p * OUT + 0] = b.O[lane * OUTP + 0];
      out[p * OUT + 1] = b.O[lane * OUTP + 1];
    }
    __syncwarp();
  }
}

// Learned guesses for the particles of a context: S_H = 10^(o0 s0 + m0) kmol/m^3
// and h = 10^(o1 s1 + m1) days, clamped to [1e-14, 1] and [1e-10, 1].
__global__ void __launch_bounds__(128) guess_kernel(const double* y, int64_t ld, const double* T,
                                                    int64_t n, const float* P, const float* norm,
                                                    const float* onorm, double* SH_out,
                                                    double* h_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  WeightsSmem& w = *reinterpret_cast<WeightsSmem*>(smem);
  WarpBufs& b = reinterpret_cast<WarpBufs*>(smem + sizeof(WeightsSmem))[threadIdx.x >> 5];
  load_weights(P, w);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
       base += warps * 32) {
    const int64_t p = base + lane;
    if (p < n) {
      features(y, ld, p, T[p], norm, b.X + lane * IN);
    } else {
      for (int i = 0; i < IN; ++i) b.X[lane * IN + i] = __float2bfloat16_rn(0.0f);
    }
    __syncwarp();
    forward32(w, b);
    if (p < n) {
      const float l0 = b.O[lane * OUTP + 0] * onorm[2] + onorm[0];
      const float l1 = b.O[lane * OUTP + 1] * onorm[3] + onorm[1];
      SH_out[p] = fmin(1.0, fmax(1e-14, exp10((double)l0)));
      h_out[p] = fmin(1.0, fmax(1e-10, exp10((double)l1)));
    }
    __syncwarp();
  }
}

// Fused forward + backward of L = (1/n_total) sum_i sum_j (O_ij - Y_ij)^2 over
// the block's samples; writes the block's gradient partial (NPARAM floats)
// and loss partial.  One warp per block, samples in chunks of 32.
struct GradSmem {
  WeightsSmem w;
  WarpBufs b;
  __nv_bfloat16 dZ2[32 * HID];
  float dA[32 * HID];
  __nv_bfloat16 dZ1[32 * HID];
  float gW1[HID * IN], gW2[HID * HID], gW3[OUTP * HID], gb1[HID], gb2[HID], gb3[OUTP];
  float dO[32 * OUTP];
  float loss;
};

__global__ void __launch_bounds__(32) grad_kernel(const __nv_bfloat16* X, const float* Y, int64_t n,
                                                  int64_t per_block, float inv_n, const float* P,
                                                  float* partial, float* loss_partial) {
  extern __shared__ __align__(16) unsigned char smem[];
  GradSmem& s = *reinterpret_cast<GradSmem*>(smem);
  const int lane = threadIdx.x;
  load_weights(P, s.w);
  for (int i = lane; i < HID * IN; i += 32) s.gW1[i] = 0.0f;
  for (int i = lane; i < HID * HID; i += 32) s.gW2[i] = 0.0f;
  for (int i = lane; i < OUTP * HID; i += 32) s.gW3[i] = 0.0f;
  for (int i = lane; i < HID; i += 32) s.gb1[i] = s.gb2[i] = 0.0f;
  if (lane < OUTP) s.gb3[lane] = 0.0f;
  if (lane == 0) s.loss = 0.0f;
  __syncwarp();
  const int64_t beg = (int64_t)blockIdx.x * per_block;
  const int64_t end = min(n, beg + per_block);
  for (int64_t base = beg; base < end; base += 32) {
    for (int e = lane; e < 32 * IN; e += 32) {
      const int64_t p = base + e / IN;
      s.b.X[e] = p < end ? X[p * IN + e % IN] : __float2bfloat16_rn(0.0f);
    }
    __syncwarp();
    forward32(s.w, s.b);
    // dO = 2 (O - Y) / n_total (rows beyond the block's range contribute 0)
    float lsum = 0.0f;
    for (int e = lane; e < 32 * OUTP; e += 32) {
      const int i = e / OUTP, j = e % OUTP;
      const int64_t p = base + i;
      float d = 0.0f;
      if (j < OUT && p < end) {
        d = s.b.O[e] - Y[p * OUT + j];
        lsum += d * d;
        d *= 2.0f * inv_n;
      }
      s.dO[e] = d;
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) s.loss += lsum * inv_n;
    __syncwarp();
    // layer 3: gW3[j][c] += sum_i dO[i][j] A2[i][c]; gb3 += sum_i dO; dA2 = dO W3
    for (int e = lane; e < OUT * HID; e += 32) {
      const int j = e / HID, cc = e % HID;
      float acc = 0.0f;
      for (int i = 0; i < 32; ++i) acc += s.dO[i * OUTP + j] * __bfloat162float(s.b.A2[i * HID + cc]);
      s.gW3[e] += acc;
    }
    if (lane < OUT) {
      float acc = 0.0f;
      for (int i = 0; i < 32; ++i) acc += s.dO[i * OUTP + lane];
      s.gb3[lane] += acc;
    }
    for (int e = lane; e < 32 * HID; e += 32) {
      const int i = e / HID, cc = e % HID;
      float d = 0.0f;
      for (int j = 0; j < OUT; ++j) d += s.dO[i * OUTP + j] * __bfloat162float(s.w.W3[j * HID + cc]);
      s.dZ2[e] = __float2bfloat16_rn(d * dsilu(s.b.Z2[e]));
    }
    __syncwarp();
    // layer 2: gW2 += dZ2^T A1 (A(m=o,k=i) = dZ2[i][o], B(k=i,n=c) = A1[i][c])
    warp_gemm(s.dZ2, 1, HID, s.b.A1, HID, 1, s.gW2, HID, HID, HID, 32, true);
    for (int cc = lane; cc < HID; cc += 32) {
      float acc = 0.0f;
      for (int i = 0; i < 32; ++i) acc += __bfloat162float(s.dZ2[i * HID + cc]);
      s.gb2[cc] += acc;
    }
    // dA1 = dZ2 W2 (A(m=i,k=o) = dZ2[i][o], B(k=o,n=c) = W2[o][c])
    warp_gemm(s.dZ2, HID, 1, s.w.W2, HID, 1, s.dA, HID, 32, HID, HID, false);
    for (int e = lane; e < 32 * HID; e += 32) s.dZ1[e] = __float2bfloat16_rn(s.dA[e] * dsilu(s.b.Z1[e]));
    __syncwarp();
    // layer 1: gW1 += dZ1^T X (A(m=o,k=i) = dZ1[i][o], B(k=i,n=c) = X[i][c])
    warp_gemm(s.dZ1, 1, HID, s.b.X, IN, 1, s.gW1, IN, HID, IN, 32, true);
    for (int cc = lane; cc < HID; cc += 32) {
      float acc = 0.0f;
      for (int i = 0; i < 32; ++i) acc += __bfloat162float(s.dZ1[i * HID + cc]);
      s.gb1[cc] += acc;
    }
    __syncwarp();
  }
  float* out = partial + (int64_t)blockIdx.x * NPARAM;
  for (int i = lane; i < HID * IN; i += 32) out[OFF_W1 + i] = s.gW1[i];
  for (int i = lane; i < HID; i += 32) out[OFF_B1 + i] = s.gb1[i];
  for (int i = lane; i < HID * HID; i += 32) out[OFF_W2 + i] = s.gW2[i];
  for (int i = lane; i < HID; i += 32) out[OFF_B2 + i] = s.gb2[i];
  for (int i = lane; i < OUT * HID; i += 32) out[OFF_W3 + i] = s.gW3[i];
  if (lane < OUT) out[OFF_B3 + lane] = s.gb3[lane];
  if (lane == 0) loss_partial[blockIdx.x] = s.loss;
}

// grad[k] = sum over blocks of partial[b][k] in block order (deterministic).
__global__ void reduce_kernel(const float* partial, int nb, float* grad, const float* loss_partial,
                              float* loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < NPARAM) {
    float acc = 0.0f;
    for (int b = 0; b < nb; ++b) acc += partial[(int64_t)b * NPARAM + k];
    grad[k] = acc;
  }
  if (k == 0 && loss) {
    float l = 0.0f;
    for (int b = 0; b < nb; ++b) l += loss_partial[b];
    *loss = l;
  }
}

// Adam (Kingma & Ba 2015) with bias correction, FP32 master weights.
__global__ void adam_kernel(float* P, const float* g, float* m, float* v, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk;
  const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  P[k] -= lr * (mk * c1) / (sqrtf(vk * c2) + eps);
}

constexpr int kFwdThreads = 128;
size_t fwd_smem() { return sizeof(WeightsSmem) + (kFwdThreads / 32) * sizeof(WarpBufs); }

}  // namespace mlp

cudaError_t launch_mlp_guess(const double* y, int64_t ld, const double* T, int64_t n,
                             const float* params, const float* norm, const float* onorm,
                             double* SH_out, double* h_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mlp::guess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)mlp::fwd_smem());
    attr = true;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (n + mlp::kFwdThreads - 1) / mlp::kFwdThreads;
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  mlp::guess_kernel<<<(unsigned)blocks, mlp::kFwdThreads, mlp::fwd_smem(), s>>>(
      y, ld, T, n, params, norm, onorm, SH_out, h_out);
  return cudaGetLastError();
}

}  // namespace chad

using namespace chad;

extern "C" {

chad_status chad_mlp_features(const double* y, int64_t ld, const double* T, int64_t n,
                              const float* norm, uint16_t* X, void* stream) {
  if (n < 0 || (n > 0 && (!y || !T || !norm || !X)) || ld < n) return CHAD_E_INVALID;
  if (n == 0) return CHAD_OK;
  mlp::features_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      y, ld, T, n, norm, reinterpret_cast<__nv_bfloat16*>(X));
  return cudaGetLastError() == cudaSuccess ? CHAD_OK : CHAD_E_CUDA;
}

chad_status chad_mlp_forward(const uint16_t* X, int64_t n, const float* params, float* out,
                             void* stream) {
  if (n < 0 || (n > 0 && (!X || !params || !out))) return CHAD_E_INVALID;
  if (n == 0) return CHAD_OK;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(mlp::forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mlp::fwd_smem()) != cudaSuccess)
      return CHAD_E_CUDA;
    attr = true;
  }
  int64_t blocks = (n + mlp::kFwdThreads - 1) / mlp::kFwdThreads;
  if (blocks > 65535) blocks = 65535;
  mlp::forward_kernel<<<(unsigned)blocks, mlp::kFwdThreads, mlp::fwd_smem(), (cudaStream_t)stream>>>(
      reinterpret_cast<const __nv_bfloat16*>(X), n, params, out);
  return cudaGetLastError() == cudaSuccess ? CHAD_OK : CHAD_E_CUDA;
}

size_t chad_mlp_grad_scratch_bytes(int64_t n) {
  const int64_t per = 256;
  const int64_t nb = (n + per - 1) / per;
  return (size_t)nb * (mlp::NPARAM + 1) * sizeof(float);
}

chad_status chad_mlp_grad(const uint16_t* X, const float* Y, int64_t n, const float* params,
                          float* grad, float* loss, void* scratch, size_t scratch_bytes,
                          void* stream) {
  if (n <= 0 || !X || !Y || !params || !grad || !scratch) return CHAD_E_INVALID;
  if (scratch_bytes < chad_mlp_grad_scratch_bytes(n)) return CHAD_E_INVALID;
  const int64_t per = 256;
  const int nb = (int)((n + per - 1) / per);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(mlp::grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(mlp::GradSmem)) != cudaSuccess)
      return CHAD_E_CUDA;
    attr = true;
  }
  float* partial = static_cast<float*>(scratch);
  float* lpart = partial + (int64_t)nb * mlp::NPARAM;
  cudaStream_t s = (cudaStream_t)stream;
  mlp::grad_kernel<<<nb, 32, sizeof(mlp::GradSmem), s>>>(
      reinterpret_cast<const __nv_bfloat16*>(X), Y, n, per, 1.0f / (float)n, params, partial, lpart);
  mlp::reduce_kernel<<<(mlp::NPARAM + 255) / 256, 256, 0, s>>>(partial, nb, grad, lpart, loss);
  return cudaGetLastError() == cudaSuccess ? CHAD_OK : CHAD_E_CUDA;
}

chad_status chad_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t t,
                          float lr, float beta1, float beta2, float eps, void* stream) {
  if (!params || !grad || !m || !v || t < 1) return CHAD_E_INVALID;
  const float c1 = 1.0f / (1.0f - powf(beta1, (float)t));
  const float c2 = 1.0f / (1.0f - powf(beta2, (float)t));
  mlp::adam_kernel<<<(mlp::NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      params, grad, m, v, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? CHAD_OK : CHAD_E_CUDA;
}

}  // extern "C"
