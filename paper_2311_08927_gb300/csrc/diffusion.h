// Diffusion between particles: the interface of diffusion.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace chad {

// Diffusion between particles (diffusion.cu): per-digester grid and
// coefficients, and the arguments of one interval's diffusion.
constexpr int kNumDiffusing = 14;  // S_su .. S_I, S_cat, S_an
constexpr int kDiffRow = 16;       // doubles per slot row of the species buffers (128 B)
struct DiffConst {
  int on;                 // D > 0 and particles present
  int nx, ny, nz, cell0;  // grid of cells 2h wide over [-R, R]^2 x [0, H]; first cell id
  int pad;
  double R, H, h, inv_h, cell;
  double two_DV;          // 2 D V (m^5/s), V = V_liq / particles
  double dw_coef;         // W'(r) = dw_coef q (1 - q/2)^3, q = r/h (Wendland C2)
  double r2_lim;          // sqrt(r2) < 2h exactly when r2 < r2_lim (correctly rounded sqrt)
  float r2f_max;          // FP32 pre-test: every pair with r < 2h has r2 (in FP32) below it
  float pad2;
};
struct DiffArgs {
  int64_t n, ld;
  const int* dig;
  const DiffConst* dc;
  const double* pos;  // [3][ld]
  double* y;          // [NS][ld]
  int* cell_count;    // [n_cells]
  int* cell_start;    // [n_cells + 1]; cell_start[n_cells] = diffusing particles
  int* cell_list;     // [n] particle of each slot (slots grouped by cell, by index within)
  int n_cells;
  // per slot, in cell order (built each interval)
  double* spos;       // [3][n] positions
  float4* sposf;      // [n] positions in FP32 (x, y, z, 0) for the neighbour pre-test
  int* sdig;          // [n] digester
  double* sc[2];      // [n][kDiffRow] diffusing species, ping-pong between substeps
  double* srow;       // [n] row sum S_i = sum_j a_ij
  int64_t* row_start; // [n] first entry of the slot's row, -1 if it did not fit
  int* row_len;       // [n]
  // the operator's off-diagonal entries a_ij = -w_ij >= 0 (rows in any order)
  int* cols;          // [cap] neighbour slot
  double* vals;       // [cap]
  int64_t cap;
  unsigned long long* nnz;       // entries requested this interval
  unsigned long long* nnz_peak;  // largest request so far (not reset)
  int* status;                // [n] status bits (a capped substep plan is recorded)
  unsigned long long* smax;   // largest row sum of the diffusion operator (bit pattern)
  int* nsub;                  // planned substeps of this interval
  int* capped;                // 1 if the plan hit max_sub
  double* dt_sub;             // seconds per substep
  double dt_s;                // interval length, seconds
  int max_sub;                // substep kernels in the interval's launch sequence
};
cudaError_t launch_diffusion(const DiffArgs& a, cudaStream_t s);

// Times the two dominant diffusion kernels (operator rows, one substep) with
// CUDA events on stream s, re-running them reps times on the last interval's
// slot-order buffers (scratch: the particles' states are not touched).
cudaError_t time_diffusion_kernels(const DiffArgs& a, int reps, float* ms_rows, float* ms_step,
                                   cudaStream_t s);

}  // namespace chad
