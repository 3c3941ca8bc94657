// Advection of the AD particles through the prescribed swirl (Sec. 2.3) and
// the shared-headspace reduction of the gas states (Table 1 gas volume).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "bounds.h"
#include "adm1_device.cuh"
#include "kernels.h"

namespace chad {

namespace {

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based generator
// with the 4x64 S-box multipliers and Weyl key increments of the publication.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
    const uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// Irwin-Hall(12) normal deviate from one Philox block: 12 uniforms
// (b + 1/2)/2^16 from 16-bit chunks, summed as integers, minus 6.
__device__ __forceinline__ double gauss(uint64_t seed, uint64_t pid, uint64_t interval,
                                        uint64_t sub, uint64_t axis) {
  uint64_t c[4] = {interval, sub, axis, 0};
  philox4x64_10(c, seed, pid);
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < 12; ++k) s += (c[k >> 2] >> (16 * (k & 3))) & 0xFFFFull;
  return __dsub_rn(__ddiv_rn(__dadd_rn((double)s, 6.0), 65536.0), 6.0);
}

// Explicit IEEE operations (no contraction) keep positions bit-identical to
// any IEEE implementation of the same sequence, so slab membership cannot
// flip by a rounding difference.
__global__ void advect_kernel(AdvectArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const int d = a.dig[p];
  const FlowConst& f = a.fl[d];
  if (!f.has_flow) return;
  double x = a.pos[p], y = a.pos[a.ld + p], z = a.pos[2 * a.ld + p];
  a.D[p] = (z >= f.slab_zmin) ? f.D_slab : 0.0;  // slab membership at interval start
  const uint64_t pid = (uint64_t)(p - a.dig_offset[d]);
  const uint64_t interval = *a.interval;
  const double twoR = __dmul_rn(2.0, f.R), twoH = __dmul_rn(2.0, f.H);
#pragma unroll 1
  for (int k = 0; k < f.n_sub; ++k) {
    const double xr = __dsub_rn(__dmul_rn(f.cw, x), __dmul_rn(f.sw, y));
    const double yr = __dadd_rn(__dmul_rn(f.sw, x), __dmul_rn(f.cw, y));
    x = __dadd_rn(xr, __dmul_rn(f.amp, gauss(f.seed, pid, interval, (uint64_t)k, 0)));
    y = __dadd_rn(yr, __dmul_rn(f.amp, gauss(f.seed, pid, interval, (uint64_t)k, 1)));
    z = __dadd_rn(z, __dmul_rn(f.amp, gauss(f.seed, pid, interval, (uint64_t)k, 2)));
    const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
    if (r > f.R) {
      const double g = __ddiv_rn(__dsub_rn(twoR, r), r);
      x = __dmul_rn(x, g);
      y = __dmul_rn(y, g);
    }
    if (z < 0.0) z = -z;
    if (z > f.H) z = __dsub_rn(twoH, z);
  }
  a.pos[p] = x;
  a.pos[a.ld + p] = y;
  a.pos[2 * a.ld + p] = z;
}

constexpr int kRedThreads = 256;

// Stage 1: each block sums the three gas states of one chunk (a contiguous
// range of one digester) in a fixed order: strided per-thread sums, then a
// fixed shared-memory tree.  Deterministic run to run.
__global__ void __launch_bounds__(kRedThreads) headspace_partial(HeadspaceArgs a) {
  __shared__ double s[3][kRedThreads];
  const int b = blockIdx.x;
  const int64_t beg = a.chunk_begin[b], end = a.chunk_end[b];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int64_t p = beg + threadIdx.x; p < end; p += kRedThreads) {
#pragma unroll
    for (int g = 0; g < 3; ++g) acc[g] += a.y[(iG_h2 + g) * a.ld + p];
  }
#pragma unroll
  for (int g = 0; g < 3; ++g) s[g][threadIdx.x] = acc[g];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int g = 0; g < 3; ++g) s[g][threadIdx.x] += s[g][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) a.partial[b * 3 + threadIdx.x] = s[threadIdx.x][0];
}

// Stage 2: one block per digester adds its chunk partials (fixed tree) and
// writes the volume-weighted mean (equal particle volumes within a digester).
__global__ void __launch_bounds__(kRedThreads) headspace_mean(HeadspaceArgs a) {
  __shared__ double s[3][kRedThreads];
  const int d = blockIdx.x;
  const int c0 = a.dig_chunk0[d], c1 = a.dig_chunk0[d + 1];
  double acc[3] = {0.0, 0.0, 0.0};
  for (int c = c0 + threadIdx.x; c < c1; c += kRedThreads)
#pragma unroll
    for (int g = 0; g < 3; ++g) acc[g] += a.partial[c * 3 + g];
#pragma unroll
  for (int g = 0; g < 3; ++g) s[g][threadIdx.x] = acc[g];
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int g = 0; g < 3; ++g) s[g][threadIdx.x] += s[g][threadIdx.x + w];
    __syncthreads();
  }
  const int64_t n = a.dig_offset[d + 1] - a.dig_offset[d];
  if (threadIdx.x < 3 && n > 0) a.mean[d * 3 + threadIdx.x] = s[threadIdx.x][0] / (double)n;
}

// Stage 3: broadcast the digester mean back to every particle.
__global__ void headspace_broadcast(HeadspaceArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const int d = a.dig[p];
#pragma unroll
  for (int g = 0; g < 3; ++g) a.y[(iG_h2 + g) * a.ld + p] = a.mean[d * 3 + g];
}

__global__ void bump_kernel(unsigned long long* interval) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *interval += 1ull;
}

__global__ void part_const_kernel(const DigConst* dc, const int* dig, const double* T, double* pc,
                                  int64_t ld, int64_t begin, int64_t end) {
  const int64_t p = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= end) return;
  PartConst q;
  part_const(dc[dig[p]], T[p], q);
  pc_store(q, pc, ld, p);
}

// Cost bucket of a particle, 0 = most expensive: floor(log2(dt / h)) from the
// IEEE-754 exponent fields of dt and h (no FP64 division), clamped to the
// buckets; h <= 0 or not finite (no history) -> bucket 0.
__device__ __forceinline__ int order_bucket(double h, double dt) {
  const long long hb = __double_as_longlong(h);
  if (hb <= 0 || hb >= 0x7ff0000000000000ll) return 0;
  const int eh = (int)((hb >> 52) & 0x7ff);
  const int ed = (int)((__double_as_longlong(dt) >> 52) & 0x7ff);
  const int k = (kOrderBuckets - 1) - (ed - eh);
  return k < 0 ? 0 : (k > kOrderBuckets - 1 ? kOrderBuckets - 1 : k);
}

CHAD_BOUNDS_WORD(aux)

__global__ void order_count(const double* h, int64_t n, double dt, int* counts) {
  __shared__ int loc[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) loc[threadIdx.x] = 0;
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) atomicAdd(&loc[order_bucket(h[p], dt)], 1);
  __syncthreads();
  if (threadIdx.x < kOrderBuckets && loc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], loc[threadIdx.x]);
}

// Each block reserves a contiguous range of every bucket for its particles
// (counts[kOrderBuckets + b] is the running cursor of bucket b).
__global__ void order_scatter(const double* h, int64_t n, double dt, int* counts, int* order) {
  __shared__ int loc[kOrderBuckets], base[kOrderBuckets], rank[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) {
    loc[threadIdx.x] = 0;
    rank[threadIdx.x] = 0;
  }
  __syncthreads();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = p < n ? order_bucket(h[p], dt) : 0;
  if (!CHAD_IN_BOUNDS(aux, b >= 0 && b < kOrderBuckets, kBoundsBucket)) b = 0;
  if (p < n) atomicAdd(&loc[b], 1);
  __syncthreads();
  if (threadIdx.x < kOrderBuckets) {
    const int k = threadIdx.x;
    int start = 0;
    for (int j = 0; j < k; ++j) start += counts[j];
    base[k] = loc[k] ? start + atomicAdd(&counts[kOrderBuckets + k], loc[k]) : 0;
  }
  __syncthreads();
  if (p < n) {
    const int at = base[b] + atomicAdd(&rank[b], 1);
    if (CHAD_IN_BOUNDS(aux, at >= 0 && at < n, kBoundsOrder)) order[at] = (int)p;
  }
}

__global__ void check_load_kernel(const double* y, int64_t ld, const double* T, int64_t o,
                                  int64_t n, int* flag) {
  int bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < (int64_t)NS * n; k += stride) {
    const int64_t i = k / n, p = k - i * n;
    const double v = y[i * ld + o + p];
    if (!(v >= 0.0) || !isfinite(v)) bad |= 1;
  }
  if (T)
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
      const double t = T[o + p];
      if (!(t > 200.0 && t < 400.0)) bad |= 2;
    }
  if (bad) atomicOr(flag, bad);
}

__global__ void fill_kernel(double* dst, int64_t n, double value) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) dst[p] = value;
}

__global__ void count_status_kernel(const int* status, int64_t o, int64_t n,
                                    unsigned long long* count) {
  unsigned c = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
    c += status[o + p] != 0;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

}  // namespace

cudaError_t launch_check_load(const double* y, int64_t ld, const double* T, int64_t o, int64_t n,
                              int* flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  check_load_kernel<<<(unsigned)(sms > 0 ? 4 * sms : 256), 256, 0, s>>>(y, ld, T, o, n, flag);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* dst, int64_t n, double value, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, n, value);
  return cudaGetLastError();
}

cudaError_t launch_count_status(const int* status, int64_t o, int64_t n,
                                unsigned long long* count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1024);
  count_status_kernel<<<(unsigned)blocks, 256, 0, s>>>(status, o, n, count);
  return cudaGetLastError();
}

cudaError_t launch_order(const double* h, int64_t n, double dt_days, int* counts, int* order,
                         cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * 2 * kOrderBuckets, s);
  if (e != cudaSuccess || n <= 0) return e;
  const int block = 256;
  const unsigned grid = (unsigned)((n + block - 1) / block);
  order_count<<<grid, block, 0, s>>>(h, n, dt_days, counts);
  order_scatter<<<grid, block, 0, s>>>(h, n, dt_days, counts, order);
  return cudaGetLastError();
}

cudaError_t launch_part_const(const DigConst* dc, const int* dig, const double* T, double* pc,
                              int64_t ld, int64_t begin, int64_t end, cudaStream_t s) {
  if (end <= begin) return cudaSuccess;
  const int block = 256;
  part_const_kernel<<<(unsigned)((end - begin + block - 1) / block), block, 0, s>>>(dc, dig, T, pc, ld,
                                                                                   begin, end);
  return cudaGetLastError();
}

cudaError_t launch_bump(unsigned long long* interval, cudaStream_t s) {
  bump_kernel<<<1, 32, 0, s>>>(interval);
  return cudaGetLastError();
}

cudaError_t launch_advect(const AdvectArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int block = 128;
  advect_kernel<<<(unsigned)((a.n + block - 1) / block), block, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_headspace(const HeadspaceArgs& a, cudaStream_t s) {
  if (a.n <= 0 || a.n_chunks <= 0) return cudaSuccess;
  headspace_partial<<<a.n_chunks, kRedThreads, 0, s>>>(a);
  headspace_mean<<<a.n_dig, kRedThreads, 0, s>>>(a);
  headspace_broadcast<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

CHAD_BOUNDS_ACCESSOR(aux)

}  // namespace chad
