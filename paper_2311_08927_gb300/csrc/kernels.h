// Internal launch interface of the CUDA kernels (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "model.h"

namespace chad {

// Per-particle status bits (same values as the public CHAD_P_* bits)
enum : int { ST_NEWTON = 1, ST_STEPS = 2, ST_HMIN = 4, ST_NEG = 8, ST_NAN = 16 };

// Device counters accumulated by the integrator (reset by the host)
struct DevCounters {
  unsigned long long accepted, rejected, newton_iters, newton_fallbacks, pivot_rejects, mlp_redo;
  int min_steps, max_steps;
  unsigned long long h2_iters;  // Eq. 8 Newton iterations (S_h2 algebraic)
};

struct StepArgs {
  int64_t n;            // particles
  int64_t ld;           // leading dimension of the SoA arrays
  const int* dig;       // [n] digester of each particle
  const DigConst* dc;   // [n_dig]
  const DigConstF* dcf; // [n_dig] float copy (mixed form's FP32 Jacobian evaluation)
  double* y;            // [NS][ld]
  const double* T;      // [n] K
  const double* pc;     // [kPartConstFields][ld] per-particle constants (part_const of T)
  const double* D;      // [n] dilution rate 1/d for this interval
  double* SH;           // [n] running S_H (guess in, root out)
  double* h;            // [n] next step size (days)
  int* status;          // [n] OR-accumulated bits
  const double* atol;   // [NS]
  double rtol;
  double dt_days;
  int max_steps;
  int max_newton;
  int fixed_n;          // 0: adaptive
  DevCounters* counters;
  unsigned long long* queue;  // particle queue head (reset before each launch)
  const int* order;           // [n] queue position -> particle (null: identity)
  const double* SH_learned;   // learned guesses for particles without history (or null)
  const double* h_learned;
  int n_dig;                  // digesters of the context
};

struct AdvectArgs {
  int64_t n, ld;
  const int* dig;
  const int64_t* dig_offset;  // [n_dig + 1]
  const FlowConst* fl;
  double* pos;                // [3][ld]
  double* D;                  // [n] written for particles of digesters with flow
  const unsigned long long* interval;  // device copy of the global interval index
};

struct HeadspaceArgs {
  int64_t ld;
  int n_chunks;
  const int* chunk_dig;       // [n_chunks]
  const int64_t* chunk_begin; // [n_chunks]
  const int64_t* chunk_end;   // [n_chunks]
  const int64_t* dig_offset;  // [n_dig + 1]
  const int* dig_chunk0;      // [n_dig + 1] first chunk of each digester
  int n_dig;
  double* y;                  // [NS][ld]
  double* partial;            // [n_chunks][3] scratch
  double* mean;               // [n_dig][3] scratch
  const int* dig;             // [n]
  int64_t n;
};

// Integrator kernel variants, chosen per context and kernel form by the
// autotuner: threads per block, minimum resident blocks per SM (which sets
// the register budget, 65536 / (threads x blocks) up to 255) and where the
// factored matrix W_d lives (0: per-thread arrays, i.e. registers spilling to
// local memory; 1: the thread's column of a shared-memory tile, 128 threads
// for the float forms, 64 for the FP64 forms, 2 blocks per SM).
constexpr int kNumVariants = 7;
constexpr int kDefaultVariant = 0;
struct KernelVariant {
  int threads, min_blocks, w_shared;
};
// form: 0-4 (FP64 forms 0 and 3 keep W_d in double)
constexpr KernelVariant kernel_variant(int form, int v) {
  return v == 0   ? KernelVariant{128, 2, 0}
         : v == 1 ? KernelVariant{128, 3, 0}
         : v == 2 ? KernelVariant{128, 4, 0}
         : v == 3 ? KernelVariant{64, 4, 0}
         : v == 4 ? KernelVariant{256, 1, 0}
         : v == 5 ? KernelVariant{32, 8, 0}
                  : KernelVariant{(form == 0 || form == 3) ? 64 : 128, 2, 1};
}
cudaError_t launch_integrate(const StepArgs& a, int precision, int variant, cudaStream_t s);
cudaError_t launch_advect(const AdvectArgs& a, cudaStream_t s);
// MLP guesses for every particle of a context (see mlp.cu)
cudaError_t launch_mlp_guess(const double* y, int64_t ld, const double* T, int64_t n,
                             const float* params, const float* norm, const float* onorm,
                             double* SH_out, double* h_out, cudaStream_t s);
// interval index += 1 (last node of every interval)
cudaError_t launch_bump(unsigned long long* interval, cudaStream_t s);
// Queue order of the integrator: particles by decreasing expected cost, the
// steps of the coming interval estimated as dt / h from each particle's last
// step size (no history counts as the most expensive), bucketed by powers of
// two.  Long particles then start first and the interval does not end on a
// tail of them.  Order within a bucket is arbitrary; results do not depend
// on it.  counts: [2 * kOrderBuckets] scratch, zeroed here; order: [n].
constexpr int kOrderBuckets = 16;
// Input check of a load on the device: flag |= 1 if a state y[i][o + p]
// (p < n) is negative or not finite, |= 2 if T[o + p] is outside (200, 400) K
// (T may be null).  The caller zeroes *flag.
cudaError_t launch_check_load(const double* y, int64_t ld, const double* T, int64_t o, int64_t n,
                              int* flag, cudaStream_t s);
// dst[p] = value for p < n.
cudaError_t launch_fill(double* dst, int64_t n, double value, cudaStream_t s);
// *count += number of nonzero status[o + p], p < n.  The caller zeroes *count.
cudaError_t launch_count_status(const int* status, int64_t o, int64_t n,
                                unsigned long long* count, cudaStream_t s);
cudaError_t launch_order(const double* h, int64_t n, double dt_days, int* counts, int* order,
                         cudaStream_t s);
// pc[.][p] = part_const(dc[dig[p]], T[p]) for p in [begin, end)
cudaError_t launch_part_const(const DigConst* dc, const int* dig, const double* T, double* pc,
                              int64_t ld, int64_t begin, int64_t end, cudaStream_t s);
cudaError_t launch_headspace(const HeadspaceArgs& a, cudaStream_t s);

constexpr int kHeadspaceChunk = 4096;  // particles per partial sum

}  // namespace chad
