// Shared-headspace mean without any device allocation.
//
// Some callers cannot call cudaMalloc: a host application that hands this
// library a fixed device memory budget and forbids allocation after start-up,
// a real-time coupling loop where an allocation could stall or fail midway,
// or a caller running under an allocator that owns the whole device.  For
// them this entry point computes the per-digester volume-weighted mean of
// the three headspace states -- the reduction that chad_step performs with a
// shared headspace -- using a scratch array that lives in this file as a
// static device symbol instead of a buffer allocated per context.
//
// The arithmetic is the same as the allocating reduction of chad_step: chunks
// of 4096 particles that never span two digesters, per-thread strided sums
// over 256 threads and a fixed shared-memory tree per chunk, then a second
// fixed tree over the chunk partials of each digester.  The results are
// therefore bit-identical.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "chad.h"
#include "kernels.h"

namespace chad {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxDigesters = 1024;
constexpr int kNoallocMaxChunks = 16384;  // 3 doubles each: 384 KiB

// Scratch for the chunk partial sums.  Every GPU that loads the library
// holds it until the process exits.  All calls share it: each call writes
// every partial it reads, so nothing needs clearing, but calls that overlap
// on the GPU (different streams, or host threads racing) corrupt each other.
static __device__ __align__(256) double g_headspace_scratch[kNoallocMaxChunks * 3];

struct NoallocParams {
  const double* y;  // [29][ld] states (device)
  int64_t ld;
  int n_dig;
  int n_chunks;
  double* scratch;  // device address of g_headspace_scratch
  double* mean;     // [n_dig][3] output (device)
  int64_t off[kNoallocMaxDigesters + 1];
  int chunk0[kNoallocMaxDigesters + 1];
};
// Passed by value as the kernels' parameter block (about 12 KB with the
// offset tables inline, so no device buffer is needed for them either).
// Parameter blocks above 4 KB need CUDA 12.1 or later, which allows up to
// 32,764 bytes.
static_assert(sizeof(NoallocParams) <= 32764, "kernel parameter block too large");

__global__ void __launch_bounds__(kNoallocThreads) noalloc_partial(const NoallocParams P) {
  __shared__ double s[3][kNoallocThreads];
  const int c = blockIdx.x;
  int lo = 0, hi = P.n_dig;  // digester d with chunk0[d] <= c < chunk0[d+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (P.chunk0[mid] <= c) lo = mid; else hi = mid;
  }
  const int d = lo;
  const int64_t beg = P.off[d] + (int64_t)(c - P.chunk0[d]) * kHeadspaceChunk;
  const int64_t end = min(P.off[d + 1], beg + (int64_t)kHeadspaceChunk);
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t p = beg + threadIdx.x; p < end; p += kNoallocThreads) {
#pragma unroll
    for (int g = 0; g < 3; ++g) acc[g] += P.y[(iG_h2 + g) * P.ld + p];
  }
#pragma unroll
  for (int g = 0; g < 3; ++g) s[g][threadIdx.x] = acc[g];
  __syncthreads();
  for (int w = kNoallocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int g = 0; g < 3; ++g) s[g][threadIdx.x] += s[g][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) P.scratch[c * 3 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void __launch_bounds__(kNoallocThreads) noalloc_mean(const NoallocParams P) {
  __shared__ double s[3][kNoallocThreads];
  const int d = blockIdx.x;
  const int c0 = P.chunk0[d], c1 = P.chunk0[d + 1];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int c = c0 + threadIdx.x; c < c1; c += kNoallocThreads)
#pragma unroll
    for (int g = 0; g < 3; ++g) acc[g] += P.scratch[c * 3 + g];
#pragma unroll
  for (int g = 0; g < 3; ++g) s[g][threadIdx.x] = acc[g];
  __syncthreads();
  for (int w = kNoallocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int g = 0; g < 3; ++g) s[g][threadIdx.x] += s[g][threadIdx.x + w];
    __syncthreads();
  }
  const int64_t n = P.off[d + 1] - P.off[d];
  if (threadIdx.x < 3 && n > 0) P.mean[d * 3 + threadIdx.x] = s[threadIdx.x][0] / (double)n;
}

// Device address of the scratch symbol, looked up once per device with that
// device current (in host code the symbol's name is only a host stand-in).
constexpr int kMaxDevices = 64;
std::mutex g_sym_mutex;
double* g_sym_addr[kMaxDevices] = {nullptr};

cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_sym_mutex);
  if (!g_sym_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_headspace_scratch);
    if (e != cudaSuccess) return e;
    g_sym_addr[dev] = static_cast<double*>(p);
  }
  *out = g_sym_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace chad

using namespace chad;

extern "C" chad_status chad_headspace_mean_noalloc(const double* y, int64_t ld, int n_digesters,
                                                   const int64_t* dig_offset, double* mean,
                                                   void* cuda_stream) {
  if (!y || !dig_offset || !mean) return CHAD_E_INVALID;
  if (n_digesters < 1 || n_digesters > kNoallocMaxDigesters) return CHAD_E_INVALID;
  if (dig_offset[0] != 0) return CHAD_E_INVALID;
  NoallocParams P;
  P.y = y;
  P.ld = ld;
  P.n_dig = n_digesters;
  P.mean = mean;
  int64_t chunks = 0;
  P.off[0] = 0;
  for (int d = 0; d < n_digesters; ++d) {
    const int64_t n = dig_offset[d + 1] - dig_offset[d];
    if (n < 0) return CHAD_E_INVALID;
    P.off[d + 1] = dig_offset[d + 1];
    P.chunk0[d] = (int)chunks;
    chunks += (n + kHeadspaceChunk - 1) / kHeadspaceChunk;
    if (chunks > kNoallocMaxChunks) return CHAD_E_INVALID;
  }
  P.chunk0[n_digesters] = (int)chunks;
  if (ld < dig_offset[n_digesters]) return CHAD_E_INVALID;
  P.n_chunks = (int)chunks;
  cudaError_t e = scratch_address(&P.scratch);
  if (e != cudaSuccess) return CHAD_E_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (chunks > 0) noalloc_partial<<<(unsigned)chunks, kNoallocThreads, 0, s>>>(P);
  noalloc_mean<<<(unsigned)n_digesters, kNoallocThreads, 0, s>>>(P);
  return cudaGetLastError() == cudaSuccess ? CHAD_OK : CHAD_E_CUDA;
}
