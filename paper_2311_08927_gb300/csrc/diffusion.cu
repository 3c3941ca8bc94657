// Diffusion between the particles of a digester: the extension the paper
// plans (Sec. 2.3 and its future developments: an SPH discretisation of the
// diffusion equation with a neighbour search).  Each coupling interval,
// after advection, n_sub explicit Euler steps of
//   dC_i/dt = sum_{j != i, r_ij < 2h} 2 D V (C_i - C_j) r_ij W'(r_ij) / (r_ij^2 + 0.01 h^2)
// (Cleary & Monaghan's SPH form of the diffusion operator, Wendland C2
// kernel of smoothing length h in the form of Eq. 1, equal particle volumes
// V = V_liq / N) for the soluble species and the lumped ions.  The fluxes are
// pairwise antisymmetric, so every species' total is conserved.
//
// The particles do not move during the substeps, so the operator is fixed
// for the interval: with a_ij = -w_ij >= 0 and S_i = sum_j a_ij each substep
// is C_i <- C_i + dt (sum_j a_ij C_j - S_i C_i), a sparse product with 14
// right-hand sides.  Per interval:
//   1. neighbour grid: cells 2h wide over the digester's cylinder, a
//      counting sort (count, scan, scatter), each cell's particles ordered by
//      index -- the slot order; sums run in it, so reruns are bitwise equal;
//   2. gather: positions and species into slot order (species as 128-B rows);
//   3. rows: per slot, the 27 surrounding cells (contiguous slot ranges) give
//      the entries a_ij, stored as one CSR row reserved by an atomic add; a
//      row beyond the capacity is marked and recomputed in each substep;
//   4. plan: S_max = max_i S_i; dt_sub S_max <= 1 keeps every update a convex
//      combination of the old values, so n_sub = ceil(dt S_max), capped at the
//      substep kernels the host enqueues (8 times the continuum estimate
//      dt 7 D / h^2, at least 8; a capped plan flags the particles);
//   5. n_sub substeps (the kernels past the plan return at once, so the
//      interval's graph is static), then the species are stored back.
#include <cuda_runtime.h>

#include <cstdint>

#include "bounds.h"
#include "diffusion.h"
#include "model.h"

namespace chad {
namespace {

CHAD_BOUNDS_WORD(diffusion)

__constant__ int kDiffStates[kNumDiffusing] = {iS_su, iS_aa, iS_fa, iS_va, iS_bu,  iS_pro, iS_ac,
                                               iS_h2, iS_ch4, iS_IC, iS_IN, iS_I, iS_cat, iS_an};

__device__ __forceinline__ int cell_of(const DiffConst& g, double x, double y, double z, int& cx,
                                       int& cy, int& cz) {
  const double inv = 1.0 / g.cell;
  cx = (int)floor((x + g.R) * inv);
  cy = (int)floor((y + g.R) * inv);
  cz = (int)floor(z * inv);
  cx = cx < 0 ? 0 : (cx >= g.nx ? g.nx - 1 : cx);
  cy = cy < 0 ? 0 : (cy >= g.ny ? g.ny - 1 : cy);
  cz = cz < 0 ? 0 : (cz >= g.nz ? g.nz - 1 : cz);
  return g.cell0 + (cz * g.ny + cy) * g.nx + cx;
}

__global__ void diff_count(DiffArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const int d = a.dig[p];
  const DiffConst& g = a.dc[d];
  if (!g.on) return;
  int cx, cy, cz;
  const int c = cell_of(g, a.pos[p], a.pos[a.ld + p], a.pos[2 * a.ld + p], cx, cy, cz);
  if (!CHAD_IN_BOUNDS(diffusion, c >= 0 && c < a.n_cells, kBoundsCell)) return;
  atomicAdd(&a.cell_count[c], 1);
}

// Exclusive scan of the cell counts into cell_start[0 .. n_cells] by one
// block: each thread scans a contiguous run, then the run totals are scanned.
__global__ void diff_scan(DiffArgs a) {
  __shared__ int tot[1024];
  const int T = blockDim.x, t = threadIdx.x;
  const int per = (a.n_cells + T - 1) / T;
  const int b = t * per, e = min(a.n_cells, b + per);
  int s = 0;
  for (int c = b; c < e; ++c) s += a.cell_count[c];
  tot[t] = s;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int k = 0; k < T; ++k) {
      const int v = tot[k];
      tot[k] = acc;
      acc += v;
    }
    a.cell_start[a.n_cells] = acc;
  }
  __syncthreads();
  int acc = tot[t];
  for (int c = b; c < e; ++c) {
    a.cell_start[c] = acc;
    acc += a.cell_count[c];
    a.cell_count[c] = 0;  // reused as the scatter cursor
  }
}

__global__ void diff_scatter(DiffArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const DiffConst& g = a.dc[a.dig[p]];
  if (!g.on) return;
  int cx, cy, cz;
  const int c = cell_of(g, a.pos[p], a.pos[a.ld + p], a.pos[2 * a.ld + p], cx, cy, cz);
  if (!CHAD_IN_BOUNDS(diffusion, c >= 0 && c < a.n_cells, kBoundsCell)) return;
  const int slot = a.cell_start[c] + atomicAdd(&a.cell_count[c], 1);
  if (!CHAD_IN_BOUNDS(diffusion, slot >= 0 && slot < a.n, kBoundsScatter)) return;
  a.cell_list[slot] = (int)p;
}

// Order each cell's list by particle index (insertion sort; cells hold a few
// dozen particles), which fixes the summation order.
__global__ void diff_sort_cells(DiffArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.n_cells) return;
  int* L = a.cell_list + a.cell_start[c];
  const int m = a.cell_start[c + 1] - a.cell_start[c];
  for (int i = 1; i < m; ++i) {
    const int v = L[i];
    int j = i - 1;
    while (j >= 0 && L[j] > v) {
      L[j + 1] = L[j];
      --j;
    }
    L[j + 1] = v;
  }
}

__device__ __forceinline__ double wendland_dwdr(double r, const DiffConst& g) {
  const double q = r * g.inv_h;
  const double t = 1.0 - 0.5 * q;
  return q < 2.0 ? g.dw_coef * q * t * t * t : 0.0;  // -5 alpha q t^3 / h
}


// Visit the neighbours of slot i (position xi..zi, FP32 copy pi, digester
// constants g): every slot m != i of the 27 surrounding cells with r < 2h,
// in slot order; f(m, r2).  Candidates are first tested in FP32 against a
// bound that admits every pair within 2h, then exactly: r2 < r2_lim is the
// same decision as sqrt(r2) < 2h, so no square root is taken for it.
template <class F>
__device__ __forceinline__ void for_each_neighbour(const DiffArgs& a, const DiffConst& g, int i,
                                                   double xi, double yi, double zi, float4 pi,
                                                   F&& f) {
  int cx, cy, cz;
  cell_of(g, xi, yi, zi, cx, cy, cz);
  const int64_t n = a.n;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = cy + dy;
      if (yy < 0 || yy >= g.ny) continue;
      const int x0 = max(cx - 1, 0), x1 = min(cx + 1, g.nx - 1);
      const int c0 = g.cell0 + (z * g.ny + yy) * g.nx;
      // the x-neighbours are adjacent cells, so their slots are one range
      if (!CHAD_IN_BOUNDS(diffusion, c0 + x1 + 1 <= a.n_cells, kBoundsRange)) continue;
      const int b = a.cell_start[c0 + x0], e = a.cell_start[c0 + x1 + 1];
      if (!CHAD_IN_BOUNDS(diffusion, b >= 0 && e <= a.n, kBoundsRange)) continue;
      for (int m = b; m < e; ++m) {
        const float4 pm = a.sposf[m];
        const float fx = pi.x - pm.x, fy = pi.y - pm.y, fz = pi.z - pm.z;
        if (!(fx * fx + fy * fy + fz * fz < g.r2f_max) || m == i) continue;
        const double ex = xi - a.spos[m], ey = yi - a.spos[n + m], ez = zi - a.spos[2 * n + m];
        // no contraction: every inlined copy takes the same decisions
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
        if (!(r2 < g.r2_lim)) continue;
        f(m, r2);
      }
    }
  }
}

// The operator's entry a_ij = -2 D V r W'(r) / (r^2 + 0.01 h^2) >= 0 for a
// neighbour at squared distance r2.
__device__ __forceinline__ double entry(const DiffConst& g, double r2) {
  const double r = sqrt(r2);
  return -(g.two_DV * r * wendland_dwdr(r, g) / (r2 + 0.01 * g.h * g.h));
}

__device__ __forceinline__ int n_slots(const DiffArgs& a) { return a.cell_start[a.n_cells]; }

// Slot order copies of positions, digester and species.
__global__ void diff_gather(DiffArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots(a)) return;
  const int p = a.cell_list[s];
  const double x = a.pos[p], y = a.pos[a.ld + p], z = a.pos[2 * a.ld + p];
  a.spos[s] = x;
  a.spos[a.n + s] = y;
  a.spos[2 * a.n + s] = z;
  a.sposf[s] = make_float4((float)x, (float)y, (float)z, 0.f);
  a.sdig[s] = a.dig[p];
  double* row = a.sc[0] + s * kDiffRow;
#pragma unroll
  for (int k = 0; k < kNumDiffusing; ++k) row[k] = a.y[(int64_t)kDiffStates[k] * a.ld + p];
  for (int k = kNumDiffusing; k < kDiffRow; ++k) row[k] = 0.0;
}

// The operator's rows, one warp per slot.  Pass 1 counts the candidates that
// pass the FP32 pre-test (a bound on the row length) and reserves that many
// entries with one atomic add.  Pass 2 compacts the passing candidates, in
// slot order, into a per-warp queue (ballot + rank) and drains it 32 at a
// time, one candidate per lane: the exact test, the entry, and its place in
// the row by rank, so the row holds the neighbours in slot order (the order
// the per-thread scan of a row that did not fit also takes).  S_i is reduced
// over the warp; its maximum goes to *a.smax (positive doubles order like
// their bit patterns).
constexpr int kRowsBlock = 128;
__global__ void __launch_bounds__(kRowsBlock) diff_rows(DiffArgs a) {
  __shared__ int queue[kRowsBlock / 32][64];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int* q = queue[threadIdx.x >> 5];
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n_slots(a)) return;  // the whole warp
  const DiffConst& g = a.dc[a.sdig[i]];
  const int64_t n = a.n;
  const double xi = a.spos[i], yi = a.spos[n + i], zi = a.spos[2 * n + i];
  const float4 pi = a.sposf[i];
  int cx, cy, cz;
  cell_of(g, xi, yi, zi, cx, cy, cz);
  const int x0 = max(cx - 1, 0), x1 = min(cx + 1, g.nx - 1);
  auto pretest = [&](int m, int e) {
    if (m >= e || m == (int)i) return false;
    const float4 pm = a.sposf[m];
    const float fx = pi.x - pm.x, fy = pi.y - pm.y, fz = pi.z - pm.z;
    // no contraction: both passes take the same decisions
    return __fadd_rn(__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)), __fmul_rn(fz, fz)) < g.r2f_max;
  };
  // pass 1: bound on the row length, reservation
  int bound = 0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = cy + dy;
      if (yy < 0 || yy >= g.ny) continue;
      const int c0 = g.cell0 + (z * g.ny + yy) * g.nx;
      if (!CHAD_IN_BOUNDS(diffusion, c0 + x1 + 1 <= a.n_cells, kBoundsRange)) continue;
      const int b = a.cell_start[c0 + x0], e = a.cell_start[c0 + x1 + 1];
      if (!CHAD_IN_BOUNDS(diffusion, b >= 0 && e <= a.n, kBoundsRange)) continue;
      for (int m0 = b; m0 < e; m0 += 32) bound += __popc(__ballot_sync(full, pretest(m0 + lane, e)));
    }
  }
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(a.nnz, (unsigned long long)bound);
  base = __shfl_sync(full, base, 0);
  const bool fits = base + (unsigned long long)bound <= (unsigned long long)a.cap;
  // pass 2: entries
  const unsigned below = (1u << lane) - 1u;
  int queued = 0, len = 0;
  double S = 0.0;
  auto drain = [&](int k) {
    int m = -1;
    double w = 0.0;
    bool ok = false;
    if (lane < k) {
      m = q[lane];
      const double ex = xi - a.spos[m], ey = yi - a.spos[n + m], ez = zi - a.spos[2 * n + m];
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
      ok = r2 < g.r2_lim;
      if (ok) w = entry(g, r2);
    }
    const unsigned got = __ballot_sync(full, ok);
    if (ok) {
      S += w;
      const int k = len + __popc(got & below);
      if (fits && k < bound) {
        a.cols[base + (unsigned long long)k] = m;
        a.vals[base + (unsigned long long)k] = w;
      }
    }
    len += __popc(got);
  };
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = cy + dy;
      if (yy < 0 || yy >= g.ny) continue;
      const int c0 = g.cell0 + (z * g.ny + yy) * g.nx;
      if (!CHAD_IN_BOUNDS(diffusion, c0 + x1 + 1 <= a.n_cells, kBoundsRange)) continue;
      const int b = a.cell_start[c0 + x0], e = a.cell_start[c0 + x1 + 1];
      if (!CHAD_IN_BOUNDS(diffusion, b >= 0 && e <= a.n, kBoundsRange)) continue;
      for (int m0 = b; m0 < e; m0 += 32) {
        const int m = m0 + lane;
        const bool pass = pretest(m, e);
        const unsigned got = __ballot_sync(full, pass);
        const int at = queued + __popc(got & below);
        if (pass && CHAD_IN_BOUNDS(diffusion, at < 64, kBoundsQueue)) q[at] = m;
        queued += __popc(got);
        __syncwarp();
        if (queued >= 32) {
          drain(32);
          const int rest = lane < queued - 32 ? q[32 + lane] : 0;
          __syncwarp();
          if (lane < queued - 32) q[lane] = rest;
          queued -= 32;
          __syncwarp();
        }
      }
    }
  }
  drain(queued);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) S += __shfl_xor_sync(full, S, off);
  if (lane == 0) {
    a.srow[i] = S;
    a.row_len[i] = fits ? min(len, bound) : len;
    a.row_start[i] = fits ? (int64_t)base : -1;
    atomicMax(a.smax, (unsigned long long)__double_as_longlong(S));
  }
}

// Substep plan: n_sub = ceil(dt S_max), at least 1, at most max_sub (a capped
// plan sets *a.capped); records the largest CSR request.
__global__ void diff_plan(DiffArgs a) {
  const double smax = __longlong_as_double((long long)*a.smax);
  double want = ceil(a.dt_s * smax);
  if (!(want >= 1.0)) want = 1.0;
  int n = a.max_sub;
  if (want <= (double)a.max_sub) n = (int)want; else *a.capped = 1;
  *a.nsub = n;
  *a.dt_sub = a.dt_s / n;
  if (*a.nnz > *a.nnz_peak) *a.nnz_peak = *a.nnz;
}

// One explicit Euler step in slot order, sc[sub & 1] -> sc[(sub + 1) & 1]:
// a half-warp per slot, lane k holding species k (lanes 14 and 15 idle), so
// each neighbour's species row is one 128-byte load and its column index and
// entry are broadcasts.  Rows that did not fit are formed on the fly (every
// lane forms the same entries).
constexpr int kStepBlock = 256;
__global__ void __launch_bounds__(kStepBlock) diff_step(DiffArgs a, int sub) {
  if (sub >= *a.nsub) return;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const int k = threadIdx.x & 15;
  if (i >= n_slots(a)) return;
  const bool on = k < kNumDiffusing;
  const double* __restrict__ src = a.sc[sub & 1];
  double* __restrict__ dst = a.sc[(sub + 1) & 1];
  double acc = 0.0;
  const int64_t b = a.row_start[i];
  if (b >= 0) {
    const int len = a.row_len[i];
    const int* __restrict__ col = a.cols + b;
    const double* __restrict__ val = a.vals + b;
    int e = 0;
    for (; e + 4 <= len; e += 4) {
      const int m0 = col[e], m1 = col[e + 1], m2 = col[e + 2], m3 = col[e + 3];
      const double w0 = val[e], w1 = val[e + 1], w2 = val[e + 2], w3 = val[e + 3];
      double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
#ifdef CHAD_DEBUG_BOUNDS
      const int ns = n_slots(a);
      if (!CHAD_IN_BOUNDS(diffusion, m0 >= 0 && m0 < ns && m1 >= 0 && m1 < ns && m2 >= 0 && m2 < ns &&
                                         m3 >= 0 && m3 < ns, kBoundsColumn))
        continue;
#endif
      if (on) {
        c0 = src[(int64_t)m0 * kDiffRow + k];
        c1 = src[(int64_t)m1 * kDiffRow + k];
        c2 = src[(int64_t)m2 * kDiffRow + k];
        c3 = src[(int64_t)m3 * kDiffRow + k];
      }
      acc = fma(w0, c0, acc);
      acc = fma(w1, c1, acc);
      acc = fma(w2, c2, acc);
      acc = fma(w3, c3, acc);
    }
    for (; e < len; ++e) {
      if (!CHAD_IN_BOUNDS(diffusion, col[e] >= 0 && col[e] < n_slots(a), kBoundsColumn)) continue;
      acc = fma(val[e], on ? src[(int64_t)col[e] * kDiffRow + k] : 0.0, acc);
    }
  } else {
    const DiffConst& g = a.dc[a.sdig[i]];
    for_each_neighbour(a, g, (int)i, a.spos[i], a.spos[a.n + i], a.spos[2 * a.n + i], a.sposf[i],
                       [&](int m, double r2) {
                         acc = fma(entry(g, r2), on ? src[(int64_t)m * kDiffRow + k] : 0.0, acc);
                       });
  }
  if (on) {
    const double dt = *a.dt_sub, S = a.srow[i];
    const double c = src[i * kDiffRow + k];
    dst[i * kDiffRow + k] = c + dt * (acc - S * c);
  }
}

// Species back to the particles; a capped plan flags them.
__global__ void diff_store(DiffArgs a) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots(a)) return;
  const int p = a.cell_list[s];
  const double* row = a.sc[*a.nsub & 1] + s * kDiffRow;
#pragma unroll
  for (int k = 0; k < kNumDiffusing; ++k) a.y[(int64_t)kDiffStates[k] * a.ld + p] = row[k];
  if (*a.capped) a.status[p] |= 32;  // CHAD_P_DIFFUSION
}

}  // namespace

cudaError_t launch_diffusion(const DiffArgs& a, cudaStream_t s) {
  if (a.n <= 0 || a.n_cells <= 0 || a.max_sub <= 0) return cudaSuccess;
  const int block = 256;
  const unsigned grid = (unsigned)((a.n + block - 1) / block);
  cudaError_t e = cudaMemsetAsync(a.cell_count, 0, sizeof(int) * a.n_cells, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.smax, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.nnz, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.capped, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  diff_count<<<grid, block, 0, s>>>(a);
  diff_scan<<<1, 1024, 0, s>>>(a);
  diff_scatter<<<grid, block, 0, s>>>(a);
  diff_sort_cells<<<(unsigned)((a.n_cells + block - 1) / block), block, 0, s>>>(a);
  diff_gather<<<grid, block, 0, s>>>(a);
  diff_rows<<<(unsigned)((a.n * 32 + kRowsBlock - 1) / kRowsBlock), kRowsBlock, 0, s>>>(a);
  diff_plan<<<1, 1, 0, s>>>(a);
  const unsigned step_grid = (unsigned)((a.n * 16 + kStepBlock - 1) / kStepBlock);
  for (int k = 0; k < a.max_sub; ++k) diff_step<<<step_grid, kStepBlock, 0, s>>>(a, k);
  diff_store<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

CHAD_BOUNDS_ACCESSOR(diffusion)

cudaError_t time_diffusion_kernels(const DiffArgs& a, int reps, float* ms_rows, float* ms_step,
                                   cudaStream_t s) {
  if (a.n <= 0 || a.n_cells <= 0 || reps <= 0) return cudaErrorInvalidValue;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
  float tr = 0.f, ts = 0.f;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaMemsetAsync(a.nnz, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    if (e != cudaSuccess) break;
    diff_rows<<<(unsigned)((a.n * 32 + kRowsBlock - 1) / kRowsBlock), kRowsBlock, 0, s>>>(a);
    e = cudaEventRecord(ev[1], s);
    if (e != cudaSuccess) break;
    diff_step<<<(unsigned)((a.n * 16 + kStepBlock - 1) / kStepBlock), kStepBlock, 0, s>>>(a, 0);
    e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
    float t0 = 0.f, t1 = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t1, ev[1], ev[2]);
    tr += t0;
    ts += t1;
  }
  for (int k = 0; k < 4; ++k)
    if (ev[k]) cudaEventDestroy(ev[k]);
  if (e != cudaSuccess) return e;
  *ms_rows = tr / reps;
  *ms_step = ts / reps;
  return cudaGetLastError();
}

}  // namespace chad
