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
// Substeps: explicit Euler keeps every concentration a convex combination
// of the old ones (positive, stable) when dt_sub sum_j w_ij <= 1; each
// interval a kernel takes S_max = max_i sum_j w_ij over the current
// positions and the substep count is ceil(2 dt S_max) (half that limit),
// capped at the substep kernels the host enqueues (8 times the continuum
// estimate 2 dt 7 D / h^2, at least 8; a capped plan flags the particles).
// The substep kernels are all in the interval's graph and return at once
// past the planned count.
//
// Neighbour search: a uniform grid of cells 2h wide over the digester's
// cylinder, built per interval by a counting sort (count, scan, scatter);
// each cell's particle list is then ordered by particle index, so the sums
// run in a fixed order and reruns are bitwise identical.  The flux kernel
// runs one thread per particle over the 27 surrounding cells and writes the
// new concentrations to a second buffer.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "model.h"

namespace chad {
namespace {

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
  a.cell_list[a.cell_start[c] + atomicAdd(&a.cell_count[c], 1)] = (int)p;
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

// Row sum S_i = sum_j |w_ij| of particle i, maximum over particles into
// *a.smax (positive doubles order like their bit patterns).
__global__ void diff_rowsum(DiffArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const DiffConst& g = a.dc[a.dig[i]];
  if (!g.on) return;
  const double xi = a.pos[i], yi = a.pos[a.ld + i], zi = a.pos[2 * a.ld + i];
  int cx, cy, cz;
  cell_of(g, xi, yi, zi, cx, cy, cz);
  const double two_h = 2.0 * g.h, eta = 0.01 * g.h * g.h;
  double S = 0.0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = cy + dy;
      if (yy < 0 || yy >= g.ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = cx + dx;
        if (x < 0 || x >= g.nx) continue;
        const int c = g.cell0 + (z * g.ny + yy) * g.nx + x;
        for (int m = a.cell_start[c]; m < a.cell_start[c + 1]; ++m) {
          const int j = a.cell_list[m];
          if (j == i) continue;
          const double ex = xi - a.pos[j], ey = yi - a.pos[a.ld + j], ez = zi - a.pos[2 * a.ld + j];
          const double r2 = ex * ex + ey * ey + ez * ez;
          const double r = sqrt(r2);
          if (!(r < two_h)) continue;
          S -= g.two_DV * r * wendland_dwdr(r, g) / (r2 + eta);
        }
      }
    }
  }
  atomicMax(a.smax, (unsigned long long)__double_as_longlong(S));
}

// Substep plan: n_sub = ceil(2 dt S_max), at least 1, at most max_sub (a
// capped plan sets *a.capped).
__global__ void diff_plan(DiffArgs a) {
  const double smax = __longlong_as_double((long long)*a.smax);
  double want = ceil(2.0 * a.dt_s * smax);
  if (!(want >= 1.0)) want = 1.0;
  int n = a.max_sub;
  if (want <= (double)a.max_sub) n = (int)want; else *a.capped = 1;
  *a.nsub = n;
  *a.dt_sub = a.dt_s / n;
}

// One explicit Euler step: out[k][i] = C_k,i + dt sum_j w_ij (C_k,i - C_k,j).
__global__ void diff_flux(DiffArgs a, int sub) {
  if (sub >= *a.nsub) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const DiffConst& g = a.dc[a.dig[i]];
  if (!g.on) return;
  const double xi = a.pos[i], yi = a.pos[a.ld + i], zi = a.pos[2 * a.ld + i];
  int cx, cy, cz;
  cell_of(g, xi, yi, zi, cx, cy, cz);
  double ci[kNumDiffusing], acc[kNumDiffusing];
#pragma unroll
  for (int k = 0; k < kNumDiffusing; ++k) {
    ci[k] = a.y[(int64_t)kDiffStates[k] * a.ld + i];
    acc[k] = 0.0;
  }
  const double two_h = 2.0 * g.h, eta = 0.01 * g.h * g.h;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = cy + dy;
      if (yy < 0 || yy >= g.ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = cx + dx;
        if (x < 0 || x >= g.nx) continue;
        const int c = g.cell0 + (z * g.ny + yy) * g.nx + x;
        const int b = a.cell_start[c], e = a.cell_start[c + 1];
        for (int m = b; m < e; ++m) {
          const int j = a.cell_list[m];
          if (j == i) continue;
          const double ex = xi - a.pos[j], ey = yi - a.pos[a.ld + j], ez = zi - a.pos[2 * a.ld + j];
          const double r2 = ex * ex + ey * ey + ez * ez;
          const double r = sqrt(r2);
          if (!(r < two_h)) continue;
          const double w = g.two_DV * r * wendland_dwdr(r, g) / (r2 + eta);
#pragma unroll
          for (int k = 0; k < kNumDiffusing; ++k)
            acc[k] += w * (ci[k] - a.y[(int64_t)kDiffStates[k] * a.ld + j]);
        }
      }
    }
  }
  const double dt = *a.dt_sub;
#pragma unroll
  for (int k = 0; k < kNumDiffusing; ++k) a.buf[(int64_t)k * a.ld + i] = ci[k] + dt * acc[k];
}

__global__ void diff_copy_back(DiffArgs a, int sub) {
  if (sub >= *a.nsub) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  if (!a.dc[a.dig[i]].on) return;
  if (sub == 0 && *a.capped) a.status[i] |= 32;  // CHAD_P_DIFFUSION
#pragma unroll
  for (int k = 0; k < kNumDiffusing; ++k)
    a.y[(int64_t)kDiffStates[k] * a.ld + i] = a.buf[(int64_t)k * a.ld + i];
}

}  // namespace

cudaError_t launch_diffusion(const DiffArgs& a, cudaStream_t s) {
  if (a.n <= 0 || a.n_cells <= 0 || a.max_sub <= 0) return cudaSuccess;
  const int block = 256;
  const unsigned grid = (unsigned)((a.n + block - 1) / block);
  cudaError_t e = cudaMemsetAsync(a.cell_count, 0, sizeof(int) * a.n_cells, s);
  if (e != cudaSuccess) return e;
  diff_count<<<grid, block, 0, s>>>(a);
  diff_scan<<<1, 1024, 0, s>>>(a);
  diff_scatter<<<grid, block, 0, s>>>(a);
  diff_sort_cells<<<(unsigned)((a.n_cells + block - 1) / block), block, 0, s>>>(a);
  e = cudaMemsetAsync(a.smax, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.capped, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  diff_rowsum<<<grid, block, 0, s>>>(a);
  diff_plan<<<1, 1, 0, s>>>(a);
  for (int k = 0; k < a.max_sub; ++k) {
    diff_flux<<<grid, block, 0, s>>>(a, k);
    diff_copy_back<<<grid, block, 0, s>>>(a, k);
  }
  return cudaGetLastError();
}

}  // namespace chad
