/*
 * chad.h -- C ABI of the GB300 per-particle ADM1 integrator.
 *
 * Each Lagrangian (SPH) particle is an "AD particle", a small CSTR of volume
 * V/N that carries the 29 ADM1 states (Sec. 2.3).  Over every synchronised
 * coupling interval the library advects the particles through a prescribed
 * velocity field (Sec. 2.3: positions and velocities are supplied per CFD
 * step), integrates ADM1 on every particle independently (Sec. 2.2, Eq. 2-6)
 * with the acid-base charge balance of Eq. 7 solved for S_H+ by Newton, and
 * couples the particles of one digester through a shared headspace where
 * that is configured (Table 1 gas volume).
 *
 * Conventions
 *   - Every call returns chad_status; nothing is thrown across the ABI and
 *     the library never exits or traps.  chad_last_error() describes the
 *     last failure of a context.
 *   - Pointers passed in are owned by the caller and are not retained after
 *     the call returns.  Inputs are copied into the context's device buffers.
 *   - `mem` selects whether a caller pointer is host memory (CHAD_MEM_HOST)
 *     or device memory of the context's GPU (CHAD_MEM_DEVICE).
 *   - State arrays are structure-of-arrays: y is [29][n] (species-major,
 *     particle index fastest), positions are [3][n] (x, y, z in metres).
 *   - ADM1 units: kgCOD/m^3, except S_IC, S_IN, S_cat, S_an, S_gas_co2 in
 *     kmol/m^3.  Rates are per day; the coupling interval is in seconds.
 *   - Call order: chad_create -> chad_load_particles (every digester) ->
 *     [chad_set_flow] -> chad_step* -> chad_read_states -> chad_destroy.
 *     Out-of-order calls return CHAD_E_STATE.
 *   - Calls on one context are not thread-safe; use one context per thread.
 */
#ifndef CHAD_H
#define CHAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHAD_NS 29        /* differential states per particle (Sec. 2.2) */
#define CHAD_NPARAM 113   /* length of one digester's parameter vector */
#define CHAD_ABI_VERSION 3

/* Learned initial guesses: a 32 -> 64 -> 64 -> 2 MLP with SiLU activations.
   FP32 parameter vector layout: W1[64][32], b1[64], W2[64][64], b2[64],
   W3[2][64], b3[2] (weights row-major [out][in]). */
#define CHAD_MLP_IN 32
#define CHAD_MLP_HID 64
#define CHAD_MLP_OUT 2
#define CHAD_MLP_NPARAM (64 * 32 + 64 + 64 * 64 + 64 + 2 * 64 + 2)

typedef struct chad_ctx chad_ctx; /* opaque, library-owned */

typedef enum {
  CHAD_OK = 0,
  CHAD_E_INVALID = 1,  /* bad argument: null pointer, size, range, NaN */
  CHAD_E_NOMEM = 2,    /* device or host allocation failed */
  CHAD_E_CUDA = 3,     /* a CUDA call failed; see chad_last_error */
  CHAD_E_STATE = 4,    /* call out of order (e.g. step before load) */
  CHAD_E_PARTICLE = 5  /* >= 1 particle ended an interval with status != 0 */
} chad_status;

enum { CHAD_MEM_HOST = 0, CHAD_MEM_DEVICE = 1 };
/* Precision forms of the integrator:
   FP64        rates, Jacobian, LU and solves in FP64;
   MIXED       Jacobian and LU in FP32, one FP64 refinement step per linear
               solve; stage rates, Eq. 7 Newton, state accumulation and the
               error estimate in FP64;
   MIXED_F32RATES  as MIXED with the stage rates also in FP32 (their rounding
               noise enters the embedded error estimate and costs rejected
               steps; kept for comparison). */
enum { CHAD_PREC_FP64 = 0, CHAD_PREC_MIXED = 1, CHAD_PREC_MIXED_F32RATES = 2 };
enum { CHAD_HEADSPACE_PARTICLE = 0, CHAD_HEADSPACE_SHARED = 1 };

/* Per-particle status bits (OR-accumulated across intervals until read). */
enum {
  CHAD_P_NEWTON = 1,  /* Eq. 7: Newton and its bisection fallback found no root */
  CHAD_P_STEPS = 2,   /* max_steps_per_interval reached before the interval end */
  CHAD_P_HMIN = 4,    /* step size fell below 1e-12 d after rejections */
  CHAD_P_NEG = 8,     /* a state ended the interval below -atol_i */
  CHAD_P_NAN = 16,    /* non-finite state or singular iteration matrix */
  CHAD_P_DIFFUSION = 32  /* diffusion needed more substeps than planned (see
                            chad_set_diffusion); the diffusion step may be unstable */
};

/* Library configuration (copied at chad_create). */
typedef struct {
  int n_digesters;             /* >= 1 */
  const int64_t* n_particles;  /* [n_digesters] particle count per digester (>= 0) */
  const double* V_liq;         /* [n_digesters] liquid volume, m^3 (> 0) */
  const double* V_gas;         /* [n_digesters] headspace volume, m^3 (> 0) */
  const double* params;        /* [n_digesters][CHAD_NPARAM]; names: chad_param_name */
  const double* D_uniform;     /* [n_digesters] dilution rate 1/d for digesters without a
                                  flow field (Eq. 2 with q_in = q_out); NULL = all 0 */
  const double* y_in;          /* [n_digesters][29] influent; NULL = zeros */
  int precision;               /* CHAD_PREC_FP64, CHAD_PREC_MIXED or CHAD_PREC_MIXED_F32RATES */
  int learned;                 /* 1: particles loaded without a step-size history take
                                  their first S_H and h from the MLP (chad_set_mlp) */
  int headspace;               /* CHAD_HEADSPACE_PARTICLE or CHAD_HEADSPACE_SHARED */
  double rtol;                 /* relative tolerance of the step controller (> 0) */
  const double* atol;          /* [29] absolute tolerances (> 0) */
  int max_steps_per_interval;  /* step attempts per particle and interval (>= 1) */
  int max_newton_iters;        /* Newton iterations per Eq. 7 solve (>= 1) */
  int fixed_substeps;          /* 0: adaptive; k > 0: k equal steps per interval */
  void* cuda_stream;           /* cudaStream_t to run on; NULL = legacy default stream */
  int h2_algebraic;            /* 1: S_h2 from its mass balance (Eq. 8) at every rate
                                  evaluation, as the paper does, instead of as a
                                  differential state.  With CHAD_PREC_FP64 the root is
                                  FP64; with CHAD_PREC_MIXED the stage rates and the
                                  root are FP32, the refinement residual two-float,
                                  the Eq. 7 Newton and the state FP64 (not available
                                  with CHAD_PREC_MIXED_F32RATES).  The S_h2 entry of y
                                  then holds the root at the current state. */
} chad_config;

/* Prescribed flow of one digester (Sec. 2.3).  Rigid swirl u_theta = U r/R
   about the z axis plus Gaussian velocity noise of std sigma (m/s) per
   1-second sub-step, reflecting walls at r = R, z = 0, z = H.  Particles
   with z >= slab_zmin at the start of an interval form the inlet slab and
   receive the influent at dilution rate q_in / (pi R^2 (H - slab_zmin)). */
typedef struct {
  int has_flow;      /* 0: particles do not move (D_uniform applies) */
  double U;          /* swirl speed at r = R, m/s */
  double R, H;       /* cylinder radius and height, m (> 0) */
  double sigma;      /* velocity noise std, m/s (>= 0) */
  double slab_zmin;  /* inlet slab lower bound, m */
  double q_in;       /* inflow, m^3/d (>= 0) */
  const double* y_in;/* [29] influent of the slab; NULL keeps the config's y_in */
  uint64_t seed;     /* noise stream key */
} chad_flow;

/* Counters accumulated since the last chad_read_states of the context. */
typedef struct {
  int64_t accepted_steps;    /* accepted W-method steps, all particles */
  int64_t rejected_steps;
  int64_t newton_iters;      /* Eq. 7 Newton iterations (charge balance, FP64) */
  int64_t newton_fallbacks;  /* bisection fallbacks */
  int64_t min_steps;         /* fewest accepted steps of one particle in one interval */
  int64_t max_steps;         /* most accepted steps of one particle in one interval */
  int64_t failed_particles;  /* particles with status != 0 */
  int64_t mlp_redo;          /* learned guesses rejected and redone plainly */
  int64_t pivot_rejects;     /* attempts rejected by the static-pivot threshold test */
  int64_t intervals;         /* coupling intervals integrated */
  double sim_days;           /* particle-days integrated */
  int64_t h2_newton_iters;   /* with h2_algebraic: Eq. 8 Newton iterations (FP64 in the
                                FP64 form, FP32 in the mixed form); else 0 */
} chad_stats;

/* ---- introspection ------------------------------------------------------ */
int chad_abi_version(void);
int chad_n_params(void);
/* Name of parameter i (0 <= i < CHAD_NPARAM), or NULL.  Static storage. */
const char* chad_param_name(int i);

/* ---- lifecycle ---------------------------------------------------------- */

/* Create a context on the current CUDA device.  Validates cfg, derives the
   per-digester model constants (Sec. 2.2; temperature-independent part), and
   allocates the particle buffers (about 280 bytes per particle in FP64 SoA).
   On error *out is NULL and nothing is leaked. */
chad_status chad_create(const chad_config* cfg, chad_ctx** out);

/* Free every resource of ctx (NULL is a no-op).  Synchronises its stream. */
void chad_destroy(chad_ctx* ctx);

/* Description of the last error of ctx (or of the last failed chad_create
   when ctx is NULL).  Valid until the next call on ctx. */
const char* chad_last_error(const chad_ctx* ctx);

/* ---- data in ------------------------------------------------------------ */

/* Load the n particles of one digester (Sec. 2.3: one AD particle per SPH
   particle).  n must equal cfg->n_particles[digester].
     pos [3][n] m (NULL: all zero), y [29][n] (required), T [n] K (NULL: the
     digester's T_op = 308.15 K), S_H [n] kmol/m^3 and h [n] days (NULL:
     cold start, S_H guess 1e-7 and h 1e-6 d).
   Resets the particles' status bits.  Host pointers are copied synchronously;
   device pointers are copied on the context's stream.  Host arrays are
   checked on the GPU after the copy (y finite and >= 0, T in (200, 400) K;
   CHAD_E_INVALID otherwise); device arrays are not checked.  A load that
   fails after its argument checks leaves the digester not loaded (chad_step
   returns CHAD_E_STATE until it is loaded again). */
chad_status chad_load_particles(chad_ctx* ctx, int digester, int64_t n, const double* pos,
                                const double* y, const double* T, const double* S_H,
                                const double* h, int mem);

/* Replace the positions of one digester's particles and keep their states:
   the coupling step of an external CFD solver, which supplies the particles'
   positions at every coupling step (Sec. 2.3).  pos [3][n] m, n =
   cfg->n_particles[digester].  The next chad_step advects from these
   positions with the digester's flow; a flow with U = 0 and noise_sigma = 0
   leaves them where the caller put them, while its geometry, inlet slab and
   any diffusion still apply.  Host arrays must be finite (else
   CHAD_E_INVALID and the positions are unchanged); device arrays are copied
   on the context's stream unchecked.  CHAD_E_STATE before the digester is
   loaded. */
chad_status chad_set_positions(chad_ctx* ctx, int digester, int64_t n, const double* pos, int mem);

/* As chad_set_positions for positions listed in another order: pos [3][n]
   holds the frame's entries and id [n] the library particle (0 .. n-1 within
   the digester) each entry belongs to -- an SPH code re-sorts its particles
   every step and writes them with their ids.  The ids must name every
   particle exactly once; otherwise CHAD_E_INVALID (checked on the GPU) and
   the positions are unchanged.  Host positions must be finite.  Blocks until
   the check is done. */
chad_status chad_set_positions_by_id(chad_ctx* ctx, int digester, int64_t n, const double* pos,
                                     const int64_t* id, int mem);

/* Particle frame files, one per CFD step (the paper's coupling reads the
   particles of every CFD step from files, Sec. 2.3).  Little-endian layout:
     64-byte header: char magic[8] = "CHADFRM\0"; uint32 version = 1;
       uint32 dtype = 4 or 8 (bytes per position/velocity value); uint64 n;
       uint64 step; double time_s; uint32 fields (bit 0 positions, required;
       bit 1 velocities; bit 2 ids); uint32 reserved[5] = 0;
     then x[n], y[n], z[n] (dtype); u[n], v[n], w[n] (dtype, if bit 1; not
     used by the library); id[n] (uint32, if bit 2; without ids the entries
     are in the library's particle order).
   chad_load_frame reads one into the positions of one digester through
   chad_set_positions_by_id (FP32 values widened exactly); the frame's n must
   equal the digester's particle count.  step and time_s (may be NULL)
   receive the header's values.  A missing, short or malformed file, or bad
   ids: CHAD_E_INVALID with the reason in chad_last_error, positions
   unchanged. */
chad_status chad_load_frame(chad_ctx* ctx, int digester, const char* path, uint64_t* step,
                            double* time_s);

/* Read a frame file on the host without a context: *n, *step, *time_s and
   *has_id (each may be NULL) from the header; pos [3][n] (doubles) and id [n]
   filled when non-NULL and n <= n_max (id untouched without ids).
   CHAD_E_INVALID on any I/O or format error or n > n_max.  Needs no GPU. */
chad_status chad_read_frame(const char* path, int64_t n_max, double* pos, int64_t* id, int64_t* n,
                            uint64_t* step, double* time_s, int32_t* has_id);

/* The bounds-check build (libchad_debug.so, compiled with
   -DCHAD_DEBUG_BOUNDS): the kernels with data-dependent indices (the
   diffusion cell lists, neighbour ranges and stored columns, the ordering
   scatter) check each index, record a failed check as a bit in *status
   (one bit per check site) and skip the access instead of trapping.
   *enabled = 1 in that build, 0 in the normal one (whose *status is always
   0).  reset != 0 clears the bits after reading.  Needs no context. */
chad_status chad_debug_bounds(int32_t* enabled, uint32_t* status, int reset);

/* Checkpoint and resume.  The coupling-interval index keys the advection
   noise (0 after chad_create, +1 per interval), so a run restored from a
   checkpoint continues bit for bit when it is put back: save y, pos, S_H, h
   (chad_read_states), T and this index; restore with chad_load_particles
   (with S_H and h) for every digester, then chad_set_interval.  Both wait
   for the context's stream. */
chad_status chad_get_interval(chad_ctx* ctx, uint64_t* interval);
chad_status chad_set_interval(chad_ctx* ctx, uint64_t interval);

/* Set (or clear, has_flow = 0) the flow field of one digester. */
chad_status chad_set_flow(chad_ctx* ctx, int digester, const chad_flow* flow);

/* ---- the hot path ------------------------------------------------------- */

/* Diffusion between the particles of one digester, the extension the paper
   plans (Sec. 2.3 and its future developments): every coupling interval,
   after advection, explicit substeps of the SPH discretisation of the
   diffusion equation (Cleary-Monaghan form of Eq. 1 with the Wendland C2
   kernel, smoothing length h in m, support 2h; equal particle volumes
   V_liq / n) move the soluble species (S_su .. S_I) and the lumped ions
   S_cat, S_an between particles closer than 2h; particulates and gases do
   not diffuse.  D is the diffusivity in m^2/s (0 switches it off).  The
   substep count follows the particles: each interval the largest row sum
   S of the discrete operator (over all diffusing particles) is taken and
   ceil(dt S) substeps are made (every update stays a convex combination),
   at most 8 times the continuum estimate dt 7 D / h^2 (at least 8, at most
   4096); a
   plan above that runs the maximum and sets CHAD_P_DIFFUSION on the
   diffusing particles.  Needs the digester's flow geometry (chad_set_flow with has_flow, else
   CHAD_E_STATE).  Allocates the neighbour-grid buffers on first use; the
   operator's entries (12 bytes each, about the particles times their
   neighbours within 2h) are allocated by chad_step and grown to the largest
   need seen (rows that do not fit are recomputed in every substep). */
chad_status chad_set_diffusion(chad_ctx* ctx, int digester, double D, double h);

/* The last interval's diffusion plan: entries reserved for the operator (an
   upper bound on its non-zeros, those beyond the capacity included), the
   substeps taken, 1 if the plan was capped (see chad_set_diffusion), and
   the largest row sum S_max (1/s) over the diffusing particles.  Waits for
   the context's stream.  Any output pointer may be NULL.  CHAD_E_STATE
   before diffusion was first set. */
chad_status chad_diffusion_info(chad_ctx* ctx, int64_t* entries, int32_t* n_sub, int32_t* capped,
                                double* s_max);

/* Measurement: the two dominant diffusion kernels (the operator's rows, one
   substep) timed with CUDA events on the context's stream, each re-run reps
   times on the last interval's slot-order buffers (scratch: the particles'
   states are not touched); mean milliseconds per launch.  Blocks until done.
   CHAD_E_STATE before a diffusion interval has run. */
chad_status chad_diffusion_kernel_times(chad_ctx* ctx, int reps, double* ms_rows, double* ms_step);

/* Integrate n_intervals coupling intervals of dt_coupling_s seconds each:
   per interval, advect (digesters with flow), integrate every particle
   (Eq. 2-7) and, with a shared headspace, average the three gas states of
   each digester.  Asynchronous on the context's stream; particle failures
   are reported by chad_read_states / chad_synchronize.  On a non-default
   stream the launch sequence of one interval is captured once as a CUDA
   graph and replayed for every interval.
   dt_coupling_s > 0, n_intervals >= 0. */
chad_status chad_step(chad_ctx* ctx, double dt_coupling_s, int n_intervals);

/* Number of integrator kernel variants the autotuner chooses from. */
#define CHAD_NUM_VARIANTS 7

/* Pick the fastest integrator kernel variant for this population and
   interval length: the particle state is snapshot, two intervals are run
   and timed with each of the CHAD_NUM_VARIANTS variants, and the state is
   restored, so results are unaffected.  The variants span threads per block
   (32, 64, 128, 256), the register budget per thread (255, 168, 128: at
   least 2, 3 or 4 resident 128-thread blocks per SM) and where the factored
   matrix I - g J_d lives (per-thread arrays, or a shared-memory tile); see
   chad_kernel_variant.  The choice is kept by the context for its kernel
   form; *chosen (may be NULL) receives the variant index and ms (may be
   NULL, else CHAD_NUM_VARIANTS doubles) the time of two intervals with each
   variant.  Temporarily allocates about 290 bytes per particle of device
   memory.  Synchronous. */
chad_status chad_autotune(chad_ctx* ctx, double dt_coupling_s, int32_t* chosen, double* ms);

/* Use kernel variant v (0 <= v < CHAD_NUM_VARIANTS) for this context's
   kernel form from the next chad_step on, in place of the default (0) or
   the autotuner's choice: a fixed launch shape, e.g. for reproducible
   timing.  Results do not depend on the variant. */
chad_status chad_set_kernel_variant(chad_ctx* ctx, int variant);

/* The launch shape of kernel variant v (0 <= v < CHAD_NUM_VARIANTS) for a
   context's configuration (precision and h2_algebraic as in chad_config):
   threads per block, minimum resident blocks per SM (the register budget
   is 65536 / (threads x blocks), at most 255) and w_shared = 1 when the
   factored matrix lives in shared memory.  Any output may be NULL. */
chad_status chad_kernel_variant(int precision, int h2_algebraic, int v, int32_t* threads,
                                int32_t* min_blocks, int32_t* w_shared);

/* Wait for the context's stream.  CHAD_E_PARTICLE if any particle has a
   status bit set, CHAD_E_CUDA if a kernel failed. */
chad_status chad_synchronize(chad_ctx* ctx);

/* ---- data out ----------------------------------------------------------- */

/* Copy one digester's particles out (any pointer may be NULL to skip it):
   y [29][n], pos [3][n], S_H [n], h [n] (next step size, days), status [n].
   stats (may be NULL) receives and clears the context's counters.
   Synchronises the stream.  Returns CHAD_E_PARTICLE if any particle of the
   digester has a status bit set (the data is still copied). */
chad_status chad_read_states(chad_ctx* ctx, int digester, double* y, double* pos, double* S_H,
                             double* h, int32_t* status, chad_stats* stats, int mem);

/* ---- learned guesses (an extension; the paper has no counterpart) -------- */

/* Install a trained MLP into a context with learned = 1.  params [NPARAM]
   FP32 (layout above), feat_norm [2][32]: per-feature mean and 1/std of the
   features (log10 max(y_i, 1e-20) for the 29 states, T/100 K, 2 zero pads),
   out_norm [4]: mean of log10 S_H, mean of log10 h, std of each.  Host
   pointers, copied.  Particles loaded without h then start their first
   interval from S_H = 10^(o0 s0 + m0) and h = 10^(o1 s1 + m1): Newton runs
   at most 4 iterations from the learned S_H; if it has not converged the
   particle restarts from the plain guess (counted in chad_stats.mlp_redo). */
chad_status chad_set_mlp(chad_ctx* ctx, const float* params, const float* feat_norm,
                         const float* out_norm);

/* Features of n particles (device pointers): X [n][32] BF16 (uint16 bits)
   from y [29][ld], T [n]; feat_norm [2][32] device.  Asynchronous. */
chad_status chad_mlp_features(const double* y, int64_t ld, const double* T, int64_t n,
                              const float* feat_norm, uint16_t* X, void* cuda_stream);

/* Inference on the tensor cores (tcgen05, accumulators in tensor memory):
   out [n][2] FP32 standardised outputs for X [n][32] BF16 (16-byte aligned),
   params [NPARAM] FP32 (device pointers).  Waits for the stream and returns
   CHAD_E_CUDA if a tensor-core completion wait timed out. */
chad_status chad_mlp_forward(const uint16_t* X, int64_t n, const float* params, float* out,
                             void* cuda_stream);

/* Bytes of scratch chad_mlp_grad needs for a batch of n samples. */
size_t chad_mlp_grad_scratch_bytes(int64_t n);

/* Gradient of L = (1/n) sum_i sum_j (MLP(X_i)_j - Y_ij)^2 w.r.t. params
   (forward and backward on the tensor cores with tcgen05, BF16 operands,
   FP32 accumulation in tensor memory; per-CTA partials reduced in a fixed
   order, so the result is deterministic).  X [n][32] BF16 (16-byte
   aligned), Y [n][2] FP32, params and grad [NPARAM] FP32, loss (may be NULL)
   one FP32; all device pointers; scratch is caller-owned device memory of
   chad_mlp_grad_scratch_bytes(n) bytes.  Waits for the stream and returns
   CHAD_E_CUDA if a tensor-core completion wait timed out. */
chad_status chad_mlp_grad(const uint16_t* X, const float* Y, int64_t n, const float* params,
                          float* grad, float* loss, void* scratch, size_t scratch_bytes,
                          void* cuda_stream);

/* As chad_mlp_grad, without waiting: a tensor-core wait that timed out is
   recorded on the device and reported by the next chad_mlp_wait.  A training
   loop can then queue an epoch of batches (chad_mlp_gather, this,
   chad_mlp_adam) and wait once. */
chad_status chad_mlp_grad_async(const uint16_t* X, const float* Y, int64_t n,
                                const float* params, float* grad, float* loss, void* scratch,
                                size_t scratch_bytes, void* cuda_stream);

/* Wait for the stream; CHAD_E_CUDA if a tensor-core wait of an MLP kernel
   timed out since the last check (the record is then cleared). */
chad_status chad_mlp_wait(void* cuda_stream);

/* Bytes of scratch chad_mlp_feature_norm and chad_mlp_targets need. */
size_t chad_mlp_prep_scratch_bytes(void);

/* Standardisation of the MLP features over n >= 2 samples (device
   pointers): y [29][ld], T [n] -> norm [2][32]: the mean and 1 / sample
   standard deviation (floored at 1e-6) of log10 max(y_i, 1e-20) for the 29
   states and of T/100; the padding features get mean 0, 1/std 1.  Sums in
   FP64, reduced in a fixed order (deterministic).  Asynchronous. */
chad_status chad_mlp_feature_norm(const double* y, int64_t ld, const double* T, int64_t n,
                                  float* norm, void* scratch, size_t scratch_bytes,
                                  void* cuda_stream);

/* Training targets of n >= 2 samples (device pointers; S_H and h positive,
   as the integrator stores them): out_norm [4] = mean of log10 S_H, mean of
   log10 h, their sample standard deviations (floored at 1e-6); Y [n][2] =
   the standardised targets.  Asynchronous. */
chad_status chad_mlp_targets(const double* S_H, const double* h, int64_t n, float* Y,
                             float* out_norm, void* scratch, size_t scratch_bytes,
                             void* cuda_stream);

/* One shuffled mini-batch (device pointers): rows k = 0 .. count-1 are
   sample P_s(offset + P_e(start + k)) of X [M][32] BF16 (16-byte aligned)
   and Y [M][2], written to Xb [count][32] and Yb [count][2].  P_s is a
   keyed permutation of [0, M) (split_key): its positions [offset, offset +
   n_part) form one split (training, validation, test); P_e a keyed
   permutation of [0, n_part) (epoch_key), so each epoch visits the split in
   a new order without a stored index array.  The permutations are
   four-round Feistel networks walked to the range (bijections).
   Requires offset + n_part <= M and start + count <= n_part.  Asynchronous. */
chad_status chad_mlp_gather(const uint16_t* X, const float* Y, int64_t M, uint64_t split_key,
                            int64_t offset, int64_t n_part, uint64_t epoch_key, int64_t start,
                            int64_t count, uint16_t* Xb, float* Yb, void* cuda_stream);

/* One Adam step (Kingma & Ba 2015, bias-corrected, step t >= 1) on the FP32
   master parameters: params, grad, m, v [NPARAM] device.  Asynchronous. */
chad_status chad_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t t,
                          float lr, float beta1, float beta2, float eps, void* cuda_stream);

/* ---- allocation-free entry point ----------------------------------------- */

/* Per-digester volume-weighted mean of the three headspace states (the
   shared-headspace reduction that chad_step applies at every interval end)
   for callers that must not allocate device memory -- e.g. a host program
   with a fixed device memory budget that forbids allocation after start-up,
   a real-time coupling loop where an allocation could stall or fail midway,
   or a process whose allocator owns the whole device.  The paper has no
   counterpart: this is a property of the library, not of the method.
     y          [29][ld] particle states in device memory (gas states are
                rows 26..28), particles of digester d at dig_offset[d] ..
                dig_offset[d+1]-1
     dig_offset host array [n_digesters + 1], dig_offset[0] = 0,
                non-decreasing, dig_offset[n_digesters] <= ld
     mean       device output [n_digesters][3] (digesters without particles
                are left untouched)
     cuda_stream  stream to run on (NULL: legacy default stream)
   It calls no cudaMalloc, cudaFree or allocating routine: its scratch is a
   static device array of this library (384 KiB, held by every GPU that
   loads the library until the process exits).  Limits: n_digesters <= 1024
   and sum_d ceil(n_d / 4096) <= 16384 (67,108,864 particles in a single
   digester); larger inputs return CHAD_E_INVALID.  The first call on each
   device looks up the scratch's device address with that device current;
   make that first call before any stream capture.  The array keeps the
   last call's partial sums; every call rewrites all it reads, so nothing
   needs clearing, but calls that overlap on the GPU (other streams or host
   threads) race on it.  Asynchronous on the stream; results are
   bit-identical to chad_step's reduction. */
chad_status chad_headspace_mean_noalloc(const double* y, int64_t ld, int n_digesters,
                                        const int64_t* dig_offset, double* mean,
                                        void* cuda_stream);

/* ---- diagnostics ------------------------------------------------------- */

/* Measure the dense FMA throughput of the current GPU (fp64 = 1: FP64 DFMA,
   0: FP32 FFMA), in TFLOP/s, with FMA chains on every SM (about 0.2 s).
   These are the roofline denominators of the integrator, whose path is
   bound by plain ALU arithmetic.  Allocates and frees a small buffer. */
chad_status chad_probe_alu_peak(int fp64, double* tflops);

/* Algorithmic operation counts of the integrator's building blocks, taken
   from the kernel source (its templated routines run on the host with an
   operation-counting scalar; +, -, *, / count 1, an FMA 2): out[0] one rate
   vector, out[1] rate vector + J_d and u (the split Jacobian of
   chad_eval_model_split), out[2] one Eq. 7 evaluation, out[3] formation of
   I - g J_d, out[4] its sparse LU, out[5] one sparse solve, out[6] J x from
   the rate partials,
   out[7] stage combinations and error norm of one step attempt, out[8]
   refinement update of one mixed solve (with its rank-1 term), out[9]
   Sherman-Morrison set-up of one attempt (q = (I - g J_d)^-1 g u and its
   denominator, besides the sparse solve), out[10] Sherman-Morrison update
   of one solve, out[11] move of the Eq. 7 reciprocals and slope to a
   converged root, out[12] scaling of the rate partials by -g (the FP64
   form's formation of I - g J_d, with one add per diagonal).  n >= 13.
   With n >= 18 also the mixed form with S_h2 algebraic: out[13] J x from
   the FP32 rate partials in two-float arithmetic (in FP32 flops), out[14]
   the Eq. 8 balance coefficients, out[15] one Eq. 8 Newton iteration,
   out[16] the rest of one attempt's FP32 work (two-float stage arithmetic,
   residuals, second Sherman-Morrison level), out[17] the rest of its FP64
   work (evaluation points, S_H guesses); with n >= 19 out[18] the rates
   with their partials alone; with n >= 22 out[19] W formation, out[20]
   LU and out[21] one solve of the LU without S_h2's row and column, which
   the forms with S_h2 algebraic factor. */
chad_status chad_flop_counts(int64_t* out, int n);

/* The integrator's device arithmetic helpers applied to x [n] (host
   memory) on the current GPU: narrow [n] = x converted to float by the
   integer bit-pattern conversion (significand truncated), widen [n] = the
   round-to-nearest float of x converted back to double by the integer
   conversion (exact for normal floats), recip [n] = the FP64 reciprocal
   1/x as the kernels compute it.  Allocates and frees device buffers. */
chad_status chad_probe_numerics(const double* x, int n, float* narrow, double* widen,
                                double* recip);

/* Evaluate the library's model for one particle: f = dy/dt (Eq. 2-6) [29],
   the analytic Jacobian J = df/dy [29][29] row-major (with S_H(y) from Eq. 7
   differentiated implicitly), and the Eq. 7 root *SH, for the digester
   described by params [CHAD_NPARAM], V_liq, V_gas (m^3), dilution rate D
   (1/d), influent y_in [29] (NULL: zeros), temperature T (K) and state y
   [29], starting Newton from SH_guess.  on_device = 0 runs the code on the
   host CPU (no GPU needed), 1 runs the identical source as a one-thread
   kernel on the current GPU.  All pointers are host memory.
   CHAD_E_PARTICLE if Eq. 7 had no root in [1e-14, 1]. */
chad_status chad_eval_model(const double* params, double V_liq, double V_gas, double D,
                            const double* y_in, double T, const double* y, double SH_guess,
                            double* f, double* J, double* SH, int on_device);

/* The same evaluation with the Jacobian split the way the integrator uses it
   (Sec. 2.2 with Eq. 7 solved inside every rate evaluation): J = J_d + u v^T,
   where J_d [29][29] (row-major) is df/dy with S_H held fixed, u [29] =
   df/dS_H at fixed y and v [29] = dS_H/dy from Eq. 7 differentiated
   implicitly (nonzero only in the eight states that enter Eq. 7).  The
   integrator factors I - g J_d and applies the rank-1 term by the
   Sherman-Morrison formula.  If x [29] is given, Jx [29] receives J x as the
   mixed form's refinement forms it, from the rate partials without a matrix
   (x and Jx both NULL or both set).  Arguments and errors otherwise as
   chad_eval_model; f and SH are as there. */
chad_status chad_eval_model_split(const double* params, double V_liq, double V_gas, double D,
                                  const double* y_in, double T, const double* y,
                                  double SH_guess, const double* x, double* f, double* J_d,
                                  double* u, double* v, double* Jx, double* SH, int on_device);

#ifdef __cplusplus
}
#endif
#endif /* CHAD_H */
