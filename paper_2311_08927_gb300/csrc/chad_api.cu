// Host implementation of the C ABI declared in include/chad.h.
//
// Owns the device buffers of one particle population (structure-of-arrays,
// particle index fastest), validates every argument, and issues the
// per-interval sequence advect -> integrate -> headspace on the caller's
// stream.  Nothing here computes the model: it derives constants once
// (model_host.cpp) and launches the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bounds.h"
#include "chad.h"
#include "diffusion.h"
#include "frames.h"
#include "kernels.h"
#include "model.h"

using namespace chad;

static_assert(CHAD_NS == chad::NS, "state count");
static_assert(CHAD_NPARAM == chad::kNumParams, "parameter count");

struct chad_ctx {
  std::string err;
  int n_dig = 0;
  std::vector<int64_t> count, offset;  // per digester
  int64_t N = 0, ld = 0;
  int precision = 0, learned = 0, headspace = 0;
  int h2_alg = 0;  // S_h2 algebraic (Eq. 8): kernel form 3
  double rtol = 1e-6;
  int max_steps = 100000, max_newton = 50, fixed_n = 0;
  cudaStream_t stream = nullptr;
  std::vector<DigConst> hdc;
  std::vector<FlowConst> hfl;
  // diffusion between particles (chad_set_diffusion)
  std::vector<double> diff_D, diff_h, V_liq;  // V_liq per digester (m^3)
  bool any_diff = false, diff_dirty = false;
  double diff_dt = -1.0;
  int n_cells = 0, cells_cap = 0;
  DiffConst* d_diffc = nullptr;
  int* d_cell_count = nullptr;
  int* d_cell_start = nullptr;
  int* d_cell_list = nullptr;
  // slot-order copies and the operator's rows (see diffusion.cu)
  double* d_spos = nullptr;       // [3][N]
  float4* d_sposf = nullptr;      // [N]
  int* d_sdig = nullptr;          // [N]
  double* d_sc = nullptr;         // 2 x [N][kDiffRow]
  double* d_srow = nullptr;       // [N]
  int64_t* d_row_start = nullptr; // [N]
  int* d_row_len = nullptr;       // [N]
  int* d_cols = nullptr;          // [diff_cap]
  double* d_vals = nullptr;       // [diff_cap]
  int64_t diff_cap = 0;
  // plan scratch: smax, dt_sub, nnz, nnz_peak (8 B each), nsub, capped (4 B each)
  unsigned char* d_diff_plan = nullptr;
  int diff_max_sub = 0;
  // positions by particle id (chad_set_positions_by_id, chad_load_frame):
  // frame positions [3][m], scattered positions [3][m], ids [m], counts [m],
  // flag; m = the largest digester
  unsigned char* d_frame = nullptr;
  std::vector<char> loaded;
  bool any_flow = false;
  double sim_days = 0.0;
  int64_t intervals = 0;
  // headspace chunking
  int n_chunks = 0;
  // device buffers
  DigConst* d_dc = nullptr;
  DigConstF* d_dcf = nullptr;
  FlowConst* d_fl = nullptr;
  int* d_dig = nullptr;
  int64_t* d_off = nullptr;
  double* d_y = nullptr;
  double* d_pos = nullptr;
  double* d_T = nullptr;
  double* d_pc = nullptr;  // [kPartConstFields][ld] temperature-dependent constants
  double* d_D = nullptr;
  double* d_SH = nullptr;
  double* d_h = nullptr;
  int* d_status = nullptr;
  double* d_atol = nullptr;
  DevCounters* d_cnt = nullptr;
  unsigned long long* d_queue = nullptr;
  int* d_order = nullptr;      // [N] queue position -> particle, heaviest first
  int* d_order_cnt = nullptr;  // [2 * kOrderBuckets] bucket counts and cursors
  unsigned long long* d_misc = nullptr;  // [2]: load check flag, failed-particle count
  unsigned long long* d_interval = nullptr;  // global interval index (noise counter)
  int variant[5] = {kDefaultVariant, kDefaultVariant, kDefaultVariant, kDefaultVariant,
                    kDefaultVariant};
  double flow_dt = -1.0;        // interval length the device flow constants hold
  // CUDA graph of one interval (captured on first use, replayed per interval)
  cudaGraphExec_t gexec = nullptr;
  // learned guesses
  bool has_mlp = false;
  bool cold_pending = false;  // some particles were loaded without h
  float* d_mlp = nullptr;     // params [NPARAM], feature norm [64], output norm [4]
  double* d_SH_learned = nullptr;
  double* d_h_learned = nullptr;
  double g_dt = -1.0;
  int g_variant = -1;
  bool use_graph = true;
  int* d_chunk_dig = nullptr;
  int64_t* d_chunk_beg = nullptr;
  int64_t* d_chunk_end = nullptr;
  int* d_dig_chunk0 = nullptr;
  double* d_partial = nullptr;
  double* d_mean = nullptr;
};

static thread_local std::string g_create_err;

static chad_status fail(chad_ctx* c, chad_status s, const std::string& msg) {
  if (c) c->err = msg; else g_create_err = msg;
  return s;
}

static chad_status cuda_fail(chad_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, CHAD_E_CUDA, m);
}

#define CK(ctx, call, what)                                     \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, (what)); \
  } while (0)

template <class T>
static cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

// The arguments of the diffusion kernels for the context's current buffers.
static DiffArgs diff_args(const chad_ctx* c) {
  DiffArgs da;
  da.n = c->N;
  da.ld = c->ld;
  da.dig = c->d_dig;
  da.dc = c->d_diffc;
  da.pos = c->d_pos;
  da.y = c->d_y;
  da.spos = c->d_spos;
  da.sposf = c->d_sposf;
  da.sdig = c->d_sdig;
  da.sc[0] = c->d_sc;
  da.sc[1] = c->d_sc + (size_t)kDiffRow * c->N;
  da.srow = c->d_srow;
  da.row_start = c->d_row_start;
  da.row_len = c->d_row_len;
  da.cols = c->d_cols;
  da.vals = c->d_vals;
  da.cap = c->diff_cap;
  da.cell_count = c->d_cell_count;
  da.cell_start = c->d_cell_start;
  da.cell_list = c->d_cell_list;
  da.n_cells = c->n_cells;
  da.status = c->d_status;
  da.smax = reinterpret_cast<unsigned long long*>(c->d_diff_plan);
  da.dt_sub = reinterpret_cast<double*>(c->d_diff_plan + 8);
  da.nnz = reinterpret_cast<unsigned long long*>(c->d_diff_plan + 16);
  da.nnz_peak = reinterpret_cast<unsigned long long*>(c->d_diff_plan + 24);
  da.nsub = reinterpret_cast<int*>(c->d_diff_plan + 32);
  da.capped = reinterpret_cast<int*>(c->d_diff_plan + 36);
  da.dt_s = c->diff_dt;  // the interval in seconds, as chad_step received it
  da.max_sub = c->diff_max_sub;
  return da;
}

static void free_all(chad_ctx* c) {
  void* ptrs[] = {c->d_dc, c->d_dcf, c->d_fl, c->d_dig, c->d_off, c->d_y, c->d_pos, c->d_T, c->d_pc, c->d_D,
                  c->d_SH, c->d_h, c->d_status, c->d_atol, c->d_cnt, c->d_queue, c->d_order, c->d_order_cnt, c->d_misc, c->d_interval, c->d_chunk_dig,
                  c->d_chunk_beg, c->d_chunk_end, c->d_dig_chunk0, c->d_partial, c->d_mean};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* lp[] = {c->d_mlp, c->d_SH_learned, c->d_h_learned, c->d_diffc, c->d_cell_count,
                c->d_cell_start, c->d_cell_list, c->d_spos, c->d_sposf, c->d_sdig, c->d_sc, c->d_srow,
                c->d_row_start, c->d_row_len, c->d_cols, c->d_vals, c->d_diff_plan, c->d_frame};
  for (void* p : lp)
    if (p) cudaFree(p);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
}

static void drop_graph(chad_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->g_dt = -1.0;
  c->g_variant = -1;
}

extern "C" {

int chad_abi_version(void) { return CHAD_ABI_VERSION; }
int chad_n_params(void) { return kNumParams; }
const char* chad_param_name(int i) { return (i >= 0 && i < kNumParams) ? kParamNames[i] : nullptr; }

const char* chad_last_error(const chad_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

chad_status chad_create(const chad_config* cfg, chad_ctx** out) {
  if (!out) return fail(nullptr, CHAD_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, CHAD_E_INVALID, "cfg is NULL");
  if (cfg->n_digesters < 1 || cfg->n_digesters > (1 << 20))
    return fail(nullptr, CHAD_E_INVALID, "n_digesters must be in [1, 2^20]");
  if (!cfg->n_particles || !cfg->V_liq || !cfg->V_gas || !cfg->params || !cfg->atol)
    return fail(nullptr, CHAD_E_INVALID, "n_particles, V_liq, V_gas, params and atol are required");
  if (cfg->precision != CHAD_PREC_FP64 && cfg->precision != CHAD_PREC_MIXED &&
      cfg->precision != CHAD_PREC_MIXED_F32RATES)
    return fail(nullptr, CHAD_E_INVALID, "precision must be one of CHAD_PREC_*");
  if (cfg->h2_algebraic != 0 && cfg->h2_algebraic != 1)
    return fail(nullptr, CHAD_E_INVALID, "h2_algebraic must be 0 or 1");
  if (cfg->h2_algebraic && cfg->precision == CHAD_PREC_MIXED_F32RATES)
    return fail(nullptr, CHAD_E_INVALID,
                "h2_algebraic takes CHAD_PREC_FP64 or CHAD_PREC_MIXED (whose stage rates are "
                "then FP32)");
  if (cfg->headspace != CHAD_HEADSPACE_PARTICLE && cfg->headspace != CHAD_HEADSPACE_SHARED)
    return fail(nullptr, CHAD_E_INVALID, "invalid headspace mode");
  if (cfg->learned != 0 && cfg->learned != 1)
    return fail(nullptr, CHAD_E_INVALID, "learned must be 0 or 1");
  if (!(cfg->rtol > 0.0) || !std::isfinite(cfg->rtol))
    return fail(nullptr, CHAD_E_INVALID, "rtol must be > 0");
  for (int i = 0; i < NS; ++i)
    if (!(cfg->atol[i] > 0.0) || !std::isfinite(cfg->atol[i]))
      return fail(nullptr, CHAD_E_INVALID, "atol entries must be > 0");
  if (cfg->max_steps_per_interval < 1 || cfg->max_newton_iters < 1 || cfg->fixed_substeps < 0)
    return fail(nullptr, CHAD_E_INVALID, "max_steps_per_interval, max_newton_iters >= 1, fixed_substeps >= 0");

  chad_ctx* c = new (std::nothrow) chad_ctx();
  if (!c) return fail(nullptr, CHAD_E_NOMEM, "host allocation failed");
  c->n_dig = cfg->n_digesters;
  c->count.resize(c->n_dig);
  c->offset.resize(c->n_dig + 1);
  c->offset[0] = 0;
  for (int d = 0; d < c->n_dig; ++d) {
    if (cfg->n_particles[d] < 0 || cfg->n_particles[d] > (int64_t(1) << 34)) {
      delete c;
      return fail(nullptr, CHAD_E_INVALID, "n_particles out of range");
    }
    c->count[d] = cfg->n_particles[d];
    c->V_liq.push_back(cfg->V_liq[d]);
    c->offset[d + 1] = c->offset[d] + c->count[d];
  }
  c->N = c->offset[c->n_dig];
  c->ld = ((c->N + 31) / 32) * 32;
  if (c->N >= (int64_t(1) << 31)) {
    delete c;
    return fail(nullptr, CHAD_E_INVALID, "total particle count must be < 2^31");
  }
  c->precision = cfg->precision;
  c->h2_alg = cfg->h2_algebraic ? 1 : 0;
  c->learned = cfg->learned;
  c->headspace = cfg->headspace;
  c->rtol = cfg->rtol;
  c->max_steps = cfg->max_steps_per_interval;
  c->max_newton = cfg->max_newton_iters;
  c->fixed_n = cfg->fixed_substeps;
  c->stream = (cudaStream_t)cfg->cuda_stream;
  c->hdc.resize(c->n_dig);
  c->hfl.resize(c->n_dig);
  c->diff_D.assign(c->n_dig, 0.0);
  c->diff_h.assign(c->n_dig, 0.0);
  c->loaded.assign(c->n_dig, 0);
  for (int d = 0; d < c->n_dig; ++d) {
    const char* why = "";
    const double Du = cfg->D_uniform ? cfg->D_uniform[d] : 0.0;
    const double* yin = cfg->y_in ? cfg->y_in + (size_t)d * NS : nullptr;
    if (!derive_digester(cfg->params + (size_t)d * kNumParams, cfg->V_liq[d], cfg->V_gas[d], Du,
                         yin, c->hdc[d], &why)) {
      std::string m = "digester " + std::to_string(d) + ": " + why;
      delete c;
      return fail(nullptr, CHAD_E_INVALID, m);
    }
    std::memset(&c->hfl[d], 0, sizeof(FlowConst));
  }
  // headspace chunks: contiguous ranges never spanning digesters
  std::vector<int> chunk_dig, dig_chunk0(c->n_dig + 1);
  std::vector<int64_t> chunk_beg, chunk_end;
  for (int d = 0; d < c->n_dig; ++d) {
    dig_chunk0[d] = (int)chunk_dig.size();
    for (int64_t b = c->offset[d]; b < c->offset[d + 1]; b += kHeadspaceChunk) {
      chunk_dig.push_back(d);
      chunk_beg.push_back(b);
      chunk_end.push_back(std::min(c->offset[d + 1], b + (int64_t)kHeadspaceChunk));
    }
  }
  dig_chunk0[c->n_dig] = (int)chunk_dig.size();
  c->n_chunks = (int)chunk_dig.size();

  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  A(dalloc(&c->d_dc, c->n_dig));
  A(dalloc(&c->d_dcf, c->n_dig));
  A(dalloc(&c->d_fl, c->n_dig));
  A(dalloc(&c->d_dig, c->N));
  A(dalloc(&c->d_off, c->n_dig + 1));
  A(dalloc(&c->d_y, (size_t)NS * c->ld));
  A(dalloc(&c->d_pos, (size_t)3 * c->ld));
  A(dalloc(&c->d_T, c->ld));
  A(dalloc(&c->d_pc, (size_t)kPartConstFields * c->ld));
  A(dalloc(&c->d_D, c->ld));
  A(dalloc(&c->d_SH, c->ld));
  A(dalloc(&c->d_h, c->ld));
  A(dalloc(&c->d_status, c->ld));
  A(dalloc(&c->d_atol, NS));
  A(dalloc(&c->d_cnt, 1));
  A(dalloc(&c->d_queue, 1));
  A(dalloc(&c->d_order, c->N));
  A(dalloc(&c->d_order_cnt, 2 * kOrderBuckets));
  A(dalloc(&c->d_misc, 2));
  A(dalloc(&c->d_interval, 1));
  if (c->learned) {
    A(dalloc(&c->d_mlp, (size_t)CHAD_MLP_NPARAM + 2 * CHAD_MLP_IN + 4));
    A(dalloc(&c->d_SH_learned, c->ld));
    A(dalloc(&c->d_h_learned, c->ld));
  }
  A(dalloc(&c->d_chunk_dig, c->n_chunks));
  A(dalloc(&c->d_chunk_beg, c->n_chunks));
  A(dalloc(&c->d_chunk_end, c->n_chunks));
  A(dalloc(&c->d_dig_chunk0, c->n_dig + 1));
  A(dalloc(&c->d_partial, (size_t)3 * c->n_chunks));
  A(dalloc(&c->d_mean, (size_t)3 * c->n_dig));
  if (e != cudaSuccess) {
    free_all(c);
    std::string m = std::string("device allocation: ") + cudaGetErrorString(e);
    delete c;
    cudaGetLastError();
    return fail(nullptr, CHAD_E_NOMEM, m);
  }
  std::vector<int> dig(c->N > 0 ? c->N : 1);
  for (int d = 0; d < c->n_dig; ++d)
    for (int64_t p = c->offset[d]; p < c->offset[d + 1]; ++p) dig[p] = d;
  A(cudaMemcpy(c->d_dc, c->hdc.data(), sizeof(DigConst) * c->n_dig, cudaMemcpyHostToDevice));
  {
    std::vector<DigConstF> hf(c->n_dig);
    for (int d = 0; d < c->n_dig; ++d) narrow_digester(c->hdc[d], hf[d]);
    A(cudaMemcpy(c->d_dcf, hf.data(), sizeof(DigConstF) * c->n_dig, cudaMemcpyHostToDevice));
  }
  A(cudaMemcpy(c->d_fl, c->hfl.data(), sizeof(FlowConst) * c->n_dig, cudaMemcpyHostToDevice));
  A(cudaMemcpy(c->d_dig, dig.data(), sizeof(int) * (c->N > 0 ? c->N : 1), cudaMemcpyHostToDevice));
  A(cudaMemcpy(c->d_off, c->offset.data(), sizeof(int64_t) * (c->n_dig + 1), cudaMemcpyHostToDevice));
  A(cudaMemcpy(c->d_atol, cfg->atol, sizeof(double) * NS, cudaMemcpyHostToDevice));
  if (c->n_chunks > 0) {
    A(cudaMemcpy(c->d_chunk_dig, chunk_dig.data(), sizeof(int) * c->n_chunks, cudaMemcpyHostToDevice));
    A(cudaMemcpy(c->d_chunk_beg, chunk_beg.data(), sizeof(int64_t) * c->n_chunks, cudaMemcpyHostToDevice));
    A(cudaMemcpy(c->d_chunk_end, chunk_end.data(), sizeof(int64_t) * c->n_chunks, cudaMemcpyHostToDevice));
  }
  A(cudaMemcpy(c->d_dig_chunk0, dig_chunk0.data(), sizeof(int) * (c->n_dig + 1), cudaMemcpyHostToDevice));
  A(cudaMemset(c->d_y, 0, sizeof(double) * NS * c->ld));
  A(cudaMemset(c->d_pos, 0, sizeof(double) * 3 * c->ld));
  A(cudaMemset(c->d_status, 0, sizeof(int) * c->ld));
  A(cudaMemset(c->d_mean, 0, sizeof(double) * 3 * c->n_dig));
  A(cudaMemset(c->d_interval, 0, sizeof(unsigned long long)));
  A(cudaMemset(c->d_queue, 0, sizeof(unsigned long long)));
  DevCounters z{0, 0, 0, 0, 0, 0, 0x7fffffff, 0, 0};
  A(cudaMemcpy(c->d_cnt, &z, sizeof(z), cudaMemcpyHostToDevice));
  if (e != cudaSuccess) {
    free_all(c);
    std::string m = std::string("device setup: ") + cudaGetErrorString(e);
    delete c;
    cudaGetLastError();
    return fail(nullptr, CHAD_E_CUDA, m);
  }
  *out = c;
  return CHAD_OK;
}

void chad_destroy(chad_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
}

static cudaMemcpyKind kind_in(int mem) { return mem == CHAD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
static cudaMemcpyKind kind_out(int mem) { return mem == CHAD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

chad_status chad_load_particles(chad_ctx* c, int digester, int64_t n, const double* pos,
                                const double* y, const double* T, const double* S_H,
                                const double* h, int mem) {
  if (!c) return CHAD_E_INVALID;
  if (digester < 0 || digester >= c->n_dig) return fail(c, CHAD_E_INVALID, "digester out of range");
  if (n != c->count[digester]) return fail(c, CHAD_E_INVALID, "n differs from cfg->n_particles[digester]");
  if (!y && n > 0) return fail(c, CHAD_E_INVALID, "y is required");
  if (mem != CHAD_MEM_HOST && mem != CHAD_MEM_DEVICE) return fail(c, CHAD_E_INVALID, "mem must be HOST or DEVICE");
  const int64_t o = c->offset[digester];
  cudaStream_t s = c->stream;
  c->loaded[digester] = 0;
  const cudaMemcpyKind k = kind_in(mem);
  if (n > 0) {
    for (int i = 0; i < NS; ++i)
      CK(c, cudaMemcpyAsync(c->d_y + (size_t)i * c->ld + o, y + (size_t)i * n, sizeof(double) * n, k, s), "load y");
    if (pos) {
      for (int i = 0; i < 3; ++i)
        CK(c, cudaMemcpyAsync(c->d_pos + (size_t)i * c->ld + o, pos + (size_t)i * n, sizeof(double) * n, k, s), "load pos");
    } else {
      for (int i = 0; i < 3; ++i)
        CK(c, cudaMemsetAsync(c->d_pos + (size_t)i * c->ld + o, 0, sizeof(double) * n, s), "zero pos");
    }
    auto fill = [&](double* dst, const double* src, double dflt) -> cudaError_t {
      if (src) return cudaMemcpyAsync(dst + o, src, sizeof(double) * n, k, s);
      return launch_fill(dst + o, n, dflt, s);
    };
    CK(c, fill(c->d_T, T, 308.15), "load T");
    if (mem == CHAD_MEM_HOST) {
      // y >= 0 and finite, T in (200, 400) K: checked on the GPU after the copy
      int* flag = reinterpret_cast<int*>(c->d_misc);
      CK(c, cudaMemsetAsync(flag, 0, sizeof(int), s), "load check");
      CK(c, launch_check_load(c->d_y, c->ld, T ? c->d_T : nullptr, o, n, flag, s), "load check");
      int bad = 0;
      CK(c, cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, s), "load check");
      CK(c, cudaStreamSynchronize(s), "load check");
      if (bad & 1) return fail(c, CHAD_E_INVALID, "y must be finite and >= 0");
      if (bad & 2) return fail(c, CHAD_E_INVALID, "T must be in (200, 400) K");
    }
    CK(c, launch_part_const(c->d_dc, c->d_dig, c->d_T, c->d_pc, c->ld, o, o + n, s), "part constants");
    CK(c, fill(c->d_SH, S_H, 1e-7), "load S_H");
    CK(c, fill(c->d_h, h, 0.0), "load h");
    if (!h) c->cold_pending = true;
    CK(c, fill(c->d_D, nullptr, c->hdc[digester].D_uniform), "init D");
    CK(c, cudaMemsetAsync(c->d_status + o, 0, sizeof(int) * n, s), "reset status");
    if (mem == CHAD_MEM_HOST) CK(c, cudaStreamSynchronize(s), "load sync");
  }
  c->loaded[digester] = 1;
  return CHAD_OK;
}

chad_status chad_debug_bounds(int32_t* enabled, uint32_t* status, int reset) {
#ifdef CHAD_DEBUG_BOUNDS
  if (enabled) *enabled = 1;
#else
  if (enabled) *enabled = 0;
#endif
  const unsigned int v = bounds_status_diffusion(reset != 0) | bounds_status_aux(reset != 0);
  if (status) *status = v;
  return v == ~0u ? CHAD_E_CUDA : CHAD_OK;
}

chad_status chad_get_interval(chad_ctx* c, uint64_t* interval) {
  if (!c || !interval) return CHAD_E_INVALID;
  unsigned long long v = 0;
  CK(c, cudaMemcpyAsync(&v, c->d_interval, sizeof(v), cudaMemcpyDeviceToHost, c->stream), "interval");
  CK(c, cudaStreamSynchronize(c->stream), "interval");
  *interval = (uint64_t)v;
  return CHAD_OK;
}

chad_status chad_set_interval(chad_ctx* c, uint64_t interval) {
  if (!c) return CHAD_E_INVALID;
  const unsigned long long v = (unsigned long long)interval;
  CK(c, cudaMemcpyAsync(c->d_interval, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream), "interval");
  CK(c, cudaStreamSynchronize(c->stream), "interval");
  return CHAD_OK;
}

chad_status chad_set_positions(chad_ctx* c, int digester, int64_t n, const double* pos, int mem) {
  if (!c) return CHAD_E_INVALID;
  if (digester < 0 || digester >= c->n_dig) return fail(c, CHAD_E_INVALID, "digester out of range");
  if (n != c->count[digester]) return fail(c, CHAD_E_INVALID, "n differs from cfg->n_particles[digester]");
  if (mem != CHAD_MEM_HOST && mem != CHAD_MEM_DEVICE) return fail(c, CHAD_E_INVALID, "mem must be HOST or DEVICE");
  if (!c->loaded[digester]) return fail(c, CHAD_E_STATE, "load the digester before setting positions");
  if (n == 0) return CHAD_OK;
  if (!pos) return fail(c, CHAD_E_INVALID, "pos is required");
  if (mem == CHAD_MEM_HOST)
    for (int64_t i = 0; i < 3 * n; ++i)
      if (!std::isfinite(pos[i])) return fail(c, CHAD_E_INVALID, "positions must be finite");
  const int64_t o = c->offset[digester];
  const cudaMemcpyKind k = kind_in(mem);
  for (int i = 0; i < 3; ++i)
    CK(c, cudaMemcpyAsync(c->d_pos + (size_t)i * c->ld + o, pos + (size_t)i * n, sizeof(double) * n, k,
                          c->stream), "set positions");
  if (mem == CHAD_MEM_HOST) CK(c, cudaStreamSynchronize(c->stream), "set positions");
  return CHAD_OK;
}

chad_status chad_set_positions_by_id(chad_ctx* c, int digester, int64_t n, const double* pos,
                                     const int64_t* id, int mem) {
  if (!c) return CHAD_E_INVALID;
  if (digester < 0 || digester >= c->n_dig) return fail(c, CHAD_E_INVALID, "digester out of range");
  if (n != c->count[digester]) return fail(c, CHAD_E_INVALID, "n differs from cfg->n_particles[digester]");
  if (mem != CHAD_MEM_HOST && mem != CHAD_MEM_DEVICE) return fail(c, CHAD_E_INVALID, "mem must be HOST or DEVICE");
  if (!c->loaded[digester]) return fail(c, CHAD_E_STATE, "load the digester before setting positions");
  if (n == 0) return CHAD_OK;
  if (!pos || !id) return fail(c, CHAD_E_INVALID, "pos and id are required");
  if (mem == CHAD_MEM_HOST)
    for (int64_t i = 0; i < 3 * n; ++i)
      if (!std::isfinite(pos[i])) return fail(c, CHAD_E_INVALID, "positions must be finite");
  cudaStream_t s = c->stream;
  if (!c->d_frame) {
    int64_t m = 0;
    for (int d = 0; d < c->n_dig; ++d) m = std::max(m, c->count[d]);
    const size_t bytes = (size_t)m * (6 * sizeof(double) + sizeof(int64_t) + sizeof(int)) + 16;
    if (cudaMalloc(&c->d_frame, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->d_frame = nullptr;
      return fail(c, CHAD_E_NOMEM, "frame buffers");
    }
  }
  int64_t m = 0;
  for (int d = 0; d < c->n_dig; ++d) m = std::max(m, c->count[d]);
  double* fpos = reinterpret_cast<double*>(c->d_frame);
  double* tmp = fpos + 3 * m;
  int64_t* fid = reinterpret_cast<int64_t*>(tmp + 3 * m);
  int* seen = reinterpret_cast<int*>(fid + m);
  int* bad = seen + m;
  const cudaMemcpyKind k = kind_in(mem);
  for (int i = 0; i < 3; ++i)
    CK(c, cudaMemcpyAsync(fpos + (size_t)i * n, pos + (size_t)i * n, sizeof(double) * n, k, s), "frame positions");
  CK(c, cudaMemcpyAsync(fid, id, sizeof(int64_t) * n, k, s), "frame ids");
  CK(c, cudaMemsetAsync(bad, 0, sizeof(int), s), "frame check");
  CK(c, launch_scatter_by_id(fpos, fid, n, tmp, seen, bad, s), "frame scatter");
  int h_bad = 0;
  CK(c, cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s), "frame check");
  CK(c, cudaStreamSynchronize(s), "frame check");
  if (h_bad & 1) return fail(c, CHAD_E_INVALID, "particle id outside [0, n)");
  if (h_bad & 2) return fail(c, CHAD_E_INVALID, "particle ids are not a permutation of 0 .. n-1");
  const int64_t o = c->offset[digester];
  for (int i = 0; i < 3; ++i)
    CK(c, cudaMemcpyAsync(c->d_pos + (size_t)i * c->ld + o, tmp + (size_t)i * n, sizeof(double) * n,
                          cudaMemcpyDeviceToDevice, s), "frame positions");
  return CHAD_OK;
}

chad_status chad_read_frame(const char* path, int64_t n_max, double* pos, int64_t* id,
                            int64_t* n, uint64_t* step, double* time_s, int32_t* has_id) {
  if (!path) return CHAD_E_INVALID;
  FrameHeader h;
  std::vector<double> p;
  std::vector<int64_t> ids;
  std::string err;
  if (!read_frame_file(path, h, p, ids, err)) return CHAD_E_INVALID;
  if (n) *n = (int64_t)h.n;
  if (step) *step = h.step;
  if (time_s) *time_s = h.time_s;
  if (has_id) *has_id = ids.empty() ? 0 : 1;
  if ((pos || id) && (int64_t)h.n > n_max) return CHAD_E_INVALID;
  if (pos) std::memcpy(pos, p.data(), sizeof(double) * p.size());
  if (id && !ids.empty()) std::memcpy(id, ids.data(), sizeof(int64_t) * ids.size());
  return CHAD_OK;
}

chad_status chad_load_frame(chad_ctx* c, int digester, const char* path, uint64_t* step,
                            double* time_s) {
  if (!c) return CHAD_E_INVALID;
  if (!path) return fail(c, CHAD_E_INVALID, "path is required");
  if (digester < 0 || digester >= c->n_dig) return fail(c, CHAD_E_INVALID, "digester out of range");
  FrameHeader h;
  std::vector<double> p;
  std::vector<int64_t> ids;
  std::string err;
  if (!read_frame_file(path, h, p, ids, err)) return fail(c, CHAD_E_INVALID, err);
  const int64_t n = (int64_t)h.n;
  if (n != c->count[digester]) return fail(c, CHAD_E_INVALID, "frame particle count differs from the digester's");
  if (ids.empty()) {
    ids.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) ids[(size_t)i] = i;
  }
  const chad_status st = chad_set_positions_by_id(c, digester, n, p.data(), ids.data(), CHAD_MEM_HOST);
  if (st != CHAD_OK) return st;
  if (step) *step = h.step;
  if (time_s) *time_s = h.time_s;
  return CHAD_OK;
}

chad_status chad_set_diffusion(chad_ctx* c, int digester, double D, double h) {
  if (!c) return CHAD_E_INVALID;
  if (digester < 0 || digester >= c->n_dig) return fail(c, CHAD_E_INVALID, "digester out of range");
  if (!(D >= 0.0) || !std::isfinite(D)) return fail(c, CHAD_E_INVALID, "D must be finite and >= 0");
  if (D > 0.0 && (!(h > 0.0) || !std::isfinite(h))) return fail(c, CHAD_E_INVALID, "h must be > 0");
  if (D > 0.0 && !c->hfl[digester].has_flow)
    return fail(c, CHAD_E_STATE, "diffusion needs the digester's flow geometry (chad_set_flow)");
  if (D > 0.0 && !c->d_diffc) {
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    A(dalloc(&c->d_diffc, c->n_dig));
    A(dalloc(&c->d_cell_list, c->N));
    A(dalloc(&c->d_spos, (size_t)3 * c->N));
    A(dalloc(&c->d_sposf, (size_t)c->N));
    A(dalloc(&c->d_sdig, (size_t)c->N));
    A(dalloc(&c->d_sc, (size_t)2 * kDiffRow * c->N));
    A(dalloc(&c->d_srow, (size_t)c->N));
    A(dalloc(&c->d_row_start, (size_t)c->N));
    A(dalloc(&c->d_row_len, (size_t)c->N));
    A(dalloc(&c->d_diff_plan, 64));
    if (e == cudaSuccess) e = cudaMemset(c->d_diff_plan, 0, 64);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CHAD_E_NOMEM, "diffusion buffers");
    }
  }
  c->diff_D[digester] = D;
  c->diff_h[digester] = D > 0.0 ? h : 0.0;
  c->any_diff = false;
  for (int d = 0; d < c->n_dig; ++d) c->any_diff |= c->diff_D[d] > 0.0;
  c->diff_dirty = true;
  drop_graph(c);
  return CHAD_OK;
}

chad_status chad_diffusion_info(chad_ctx* c, int64_t* entries, int32_t* n_sub, int32_t* capped,
                                double* s_max) {
  if (!c) return CHAD_E_INVALID;
  if (!c->d_diff_plan) return fail(c, CHAD_E_STATE, "diffusion was never set");
  unsigned char h[40];
  CK(c, cudaMemcpyAsync(h, c->d_diff_plan, sizeof(h), cudaMemcpyDeviceToHost, c->stream),
     "diffusion plan");
  CK(c, cudaStreamSynchronize(c->stream), "diffusion plan");
  unsigned long long smax_bits, nnz;
  int32_t ns, cap;
  std::memcpy(&smax_bits, h, 8);
  std::memcpy(&nnz, h + 16, 8);
  std::memcpy(&ns, h + 32, 4);
  std::memcpy(&cap, h + 36, 4);
  if (entries) *entries = (int64_t)nnz;
  if (n_sub) *n_sub = ns;
  if (capped) *capped = cap;
  if (s_max) std::memcpy(s_max, &smax_bits, 8);
  return CHAD_OK;
}

chad_status chad_diffusion_kernel_times(chad_ctx* c, int reps, double* ms_rows, double* ms_step) {
  if (!c || reps <= 0) return CHAD_E_INVALID;
  if (!c->any_diff || c->n_cells <= 0 || c->diff_cap <= 0)
    return fail(c, CHAD_E_STATE, "no diffusion interval has run");
  float r = 0.f, t = 0.f;
  CK(c, time_diffusion_kernels(diff_args(c), reps, &r, &t, c->stream), "diffusion kernel timing");
  if (ms_rows) *ms_rows = r;
  if (ms_step) *ms_step = t;
  return CHAD_OK;
}

chad_status chad_set_flow(chad_ctx* c, int digester, const chad_flow* f) {
  if (!c) return CHAD_E_INVALID;
  if (digester < 0 || digester >= c->n_dig) return fail(c, CHAD_E_INVALID, "digester out of range");
  if (!f) return fail(c, CHAD_E_INVALID, "flow is NULL");
  FlowConst fc;
  std::memset(&fc, 0, sizeof(fc));
  if (f->has_flow) {
    if (!(f->R > 0.0) || !(f->H > 0.0) || !(f->sigma >= 0.0) || !(f->q_in >= 0.0) ||
        !std::isfinite(f->U) || !std::isfinite(f->slab_zmin) || !(f->slab_zmin < f->H))
      return fail(c, CHAD_E_INVALID, "flow: need R, H > 0, sigma, q_in >= 0, finite U, slab_zmin < H");
    fc.has_flow = 1;
    fc.R = f->R;
    fc.H = f->H;
    fc.slab_zmin = f->slab_zmin;
    fc.D_slab = f->q_in / (M_PI * f->R * f->R * (f->H - f->slab_zmin));
    fc.seed = f->seed;
    fc.U = f->U;
    fc.sigma = f->sigma;
    fc.cw = 1.0;  // rotation and noise amplitude are expanded per dt in chad_step
    fc.sw = 0.0;
    fc.amp = 0.0;
    fc.n_sub = 0;
    c->hfl[digester] = fc;
    if (f->y_in) {
      for (int i = 0; i < NS; ++i) {
        if (!std::isfinite(f->y_in[i])) return fail(c, CHAD_E_INVALID, "flow y_in must be finite");
        c->hdc[digester].y_in[i] = f->y_in[i];
      }
      CK(c, cudaMemcpyAsync(c->d_dc + digester, &c->hdc[digester], sizeof(DigConst),
                            cudaMemcpyHostToDevice, c->stream), "update influent");
      CK(c, cudaStreamSynchronize(c->stream), "flow sync");
    }
  } else {
    c->hfl[digester] = fc;
  }
  c->any_flow = false;
  for (int d = 0; d < c->n_dig; ++d) c->any_flow |= (c->hfl[d].has_flow != 0);
  c->flow_dt = -1.0;
  drop_graph(c);
  return CHAD_OK;
}

// Expand the per-digester flow constants for an interval length (1-s
// sub-steps) and upload them; no-op when they already hold this length.
static chad_status prepare_flow(chad_ctx* c, double dt_coupling_s) {
  if (!c->any_flow || c->flow_dt == dt_coupling_s) return CHAD_OK;
  int n_sub = (int)std::lround(dt_coupling_s);
  if (n_sub < 1) n_sub = 1;
  const double dsub = dt_coupling_s / n_sub;
  std::vector<FlowConst> fl = c->hfl;
  for (int d = 0; d < c->n_dig; ++d) {
    if (!fl[d].has_flow) continue;
    const double w = fl[d].U / fl[d].R;
    fl[d].cw = std::cos(w * dsub);
    fl[d].sw = std::sin(w * dsub);
    fl[d].amp = fl[d].sigma * dsub;
    fl[d].n_sub = n_sub;
  }
  CK(c, cudaMemcpyAsync(c->d_fl, fl.data(), sizeof(FlowConst) * c->n_dig, cudaMemcpyHostToDevice,
                        c->stream), "flow upload");
  CK(c, cudaStreamSynchronize(c->stream), "flow upload sync");
  c->flow_dt = dt_coupling_s;
  drop_graph(c);
  return CHAD_OK;
}

// Grid, coefficients and buffers of the diffusion for an interval of dt
// seconds: cells 2h wide; room for the operator's entries from the continuum
// neighbour count, twice over, grown to the largest request of earlier
// intervals (rows that did not fit were recomputed in every substep); and
// the substep kernels to enqueue: 8 times the continuum estimate
// dt 7 D / h^2 of the substep count (largest over the digesters), at least 8.
constexpr int64_t kDiffMaxEntries = int64_t(1) << 29;  // 6 GiB of entries at most
constexpr int64_t kMaxDiffusionSubsteps = 4096;

// Smallest x >= 0 whose correctly rounded square root is >= t: for r2 >= 0,
// sqrt(r2) < t exactly when r2 < x.
static double sqrt_threshold(double t) {
  double x = t * t;
  while (x > 0.0 && std::sqrt(x) >= t) x = std::nextafter(x, 0.0);
  while (std::sqrt(x) < t) x = std::nextafter(x, HUGE_VAL);
  return x;
}
static chad_status prepare_diffusion(chad_ctx* c, double dt_s) {
  if (!c->any_diff) return CHAD_OK;
  int64_t grow = 0;
  if (c->diff_cap > 0 && c->diff_cap < kDiffMaxEntries) {
    unsigned long long peak = 0;
    CK(c, cudaMemcpyAsync(&peak, c->d_diff_plan + 24, sizeof(peak), cudaMemcpyDeviceToHost, c->stream),
       "diffusion request");
    CK(c, cudaStreamSynchronize(c->stream), "diffusion request");
    if ((int64_t)peak > c->diff_cap) grow = (int64_t)peak + (int64_t)peak / 4;
  }
  if (!c->diff_dirty && c->diff_dt == dt_s && grow == 0) return CHAD_OK;
  std::vector<DiffConst> g(c->n_dig);
  int64_t cells = 0;
  int nsub = 1;
  double entries = 0.0;
  for (int d = 0; d < c->n_dig; ++d) {
    DiffConst& q = g[d];
    std::memset(&q, 0, sizeof(q));
    const double D = c->diff_D[d], h = c->diff_h[d];
    if (!(D > 0.0) || c->count[d] == 0) continue;
    q.on = 1;
    q.R = c->hfl[d].R;
    q.H = c->hfl[d].H;
    q.h = h;
    q.inv_h = 1.0 / h;
    q.cell = 2.0 * h;
    q.nx = q.ny = std::max(1, (int)std::ceil(2.0 * q.R / q.cell));
    q.nz = std::max(1, (int)std::ceil(q.H / q.cell));
    q.cell0 = (int)cells;
    cells += (int64_t)q.nx * q.ny * q.nz;
    const double V = c->V_liq[d] / (double)c->count[d];  // equal particle volumes
    q.two_DV = 2.0 * D * V;
    q.dw_coef = -5.0 * (21.0 / (16.0 * M_PI * h * h * h)) / h;
    q.r2_lim = sqrt_threshold(2.0 * h);
    // FP32 positions are within 2^-24 max(R, H) of the FP64 ones, so an FP32
    // distance is within a few 1e-7 max(R, H) of the true one: a margin of
    // 2^-16 (max(R, H) + 2h) admits every pair closer than 2h
    const double margin = std::ldexp(std::max(q.R, q.H) + 2.0 * h, -16);
    q.r2f_max = std::nextafter((float)((2.0 * h + margin) * (2.0 * h + margin)), HUGE_VALF);
    // continuum estimates: 7 D / h^2 for the row sum (Wendland C2), the
    // support's share of the cylinder for the neighbours
    nsub = (int)std::min(1.0e6, std::max((double)nsub, std::ceil(dt_s * 7.0 * D / (h * h))));
    const double n_d = (double)c->count[d];
    const double share = (4.0 / 3.0) * (8.0 * h * h * h) / (q.R * q.R * q.H);
    entries += n_d * std::min(n_d - 1.0, n_d * share);
  }
  int64_t cap = std::max<int64_t>(grow, (int64_t)std::min(2.0 * entries + 1024.0, (double)kDiffMaxEntries));
  cap = std::min(cap, kDiffMaxEntries);
  if (cap > c->diff_cap) {
    if (c->d_cols) cudaFree(c->d_cols);
    if (c->d_vals) cudaFree(c->d_vals);
    c->d_cols = nullptr;
    c->d_vals = nullptr;
    c->diff_cap = 0;
    if (dalloc(&c->d_cols, (size_t)cap) != cudaSuccess || dalloc(&c->d_vals, (size_t)cap) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CHAD_E_NOMEM, "diffusion operator");
    }
    c->diff_cap = cap;
  }
  if (cells > (int64_t(1) << 26))
    return fail(c, CHAD_E_INVALID, "diffusion grid too fine (more than 2^26 cells): raise h");
  if (cells > c->cells_cap) {
    if (c->d_cell_count) cudaFree(c->d_cell_count);
    if (c->d_cell_start) cudaFree(c->d_cell_start);
    c->d_cell_count = nullptr;
    c->d_cell_start = nullptr;
    c->cells_cap = 0;
    if (cudaMalloc(&c->d_cell_count, sizeof(int) * cells) != cudaSuccess ||
        cudaMalloc(&c->d_cell_start, sizeof(int) * (cells + 1)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, CHAD_E_NOMEM, "diffusion grid");
    }
    c->cells_cap = (int)cells;
  }
  CK(c, cudaMemcpy(c->d_diffc, g.data(), sizeof(DiffConst) * c->n_dig, cudaMemcpyHostToDevice),
     "diffusion constants");
  c->n_cells = (int)cells;
  // at most kMaxDiffusionSubsteps kernels in an interval's graph; a plan
  // above them runs that many and flags the particles (CHAD_P_DIFFUSION)
  c->diff_max_sub = (int)std::min<int64_t>(kMaxDiffusionSubsteps, std::max<int64_t>(8, 8 * (int64_t)nsub));
  c->diff_dt = dt_s;
  c->diff_dirty = false;
  drop_graph(c);
  return CHAD_OK;
}

// Kernel form of a context: 0-2 = precision form, 3 = FP64 with S_h2
// algebraic, 4 = mixed with S_h2 algebraic (FP32 stage rates, two-float
// refinement residual).
static int kernel_form(const chad_ctx* c) {
  if (c->h2_alg) return c->precision == CHAD_PREC_MIXED ? 4 : 3;
  return c->precision;
}

// The launch sequence of one coupling interval: advect (digesters with
// flow) -> integrate every particle -> shared-headspace mean -> interval += 1.
static cudaError_t enqueue_interval(chad_ctx* c, double dt_days, int variant, cudaStream_t s,
                                    bool learned_now = false) {
  StepArgs a;
  a.n = c->N;
  a.ld = c->ld;
  a.dig = c->d_dig;
  a.dc = c->d_dc;
  a.dcf = c->d_dcf;
  a.y = c->d_y;
  a.T = c->d_T;
  a.pc = c->d_pc;
  a.D = c->d_D;
  a.SH = c->d_SH;
  a.h = c->d_h;
  a.status = c->d_status;
  a.atol = c->d_atol;
  a.rtol = c->rtol;
  a.dt_days = dt_days;
  a.max_steps = c->max_steps;
  a.max_newton = c->max_newton;
  a.fixed_n = c->fixed_n;
  a.counters = c->d_cnt;
  a.queue = c->d_queue;
  a.order = nullptr;
  a.SH_learned = learned_now ? c->d_SH_learned : nullptr;
  a.h_learned = learned_now ? c->d_h_learned : nullptr;
  a.n_dig = c->n_dig;
  cudaError_t e;
  if (learned_now) {
    const float* P = c->d_mlp;
    e = launch_mlp_guess(c->d_y, c->ld, c->d_T, c->N, P, P + CHAD_MLP_NPARAM,
                         P + CHAD_MLP_NPARAM + 2 * CHAD_MLP_IN, c->d_SH_learned, c->d_h_learned, s);
    if (e != cudaSuccess) return e;
  }
  if (c->any_flow) {
    AdvectArgs v;
    v.n = c->N;
    v.ld = c->ld;
    v.dig = c->d_dig;
    v.dig_offset = c->d_off;
    v.fl = c->d_fl;
    v.pos = c->d_pos;
    v.D = c->d_D;
    v.interval = c->d_interval;
    if ((e = launch_advect(v, s)) != cudaSuccess) return e;
  }
  if (c->any_diff && c->n_cells > 0) {
    const DiffArgs da = diff_args(c);
    if ((e = launch_diffusion(da, s)) != cudaSuccess) return e;
  }
  if (c->fixed_n == 0 && c->N > 0) {
    if ((e = launch_order(c->d_h, c->N, dt_days, c->d_order_cnt, c->d_order, s)) != cudaSuccess)
      return e;
    a.order = c->d_order;
  }
  if ((e = launch_integrate(a, kernel_form(c), variant, s)) != cudaSuccess) return e;
  if (c->headspace == CHAD_HEADSPACE_SHARED) {
    HeadspaceArgs hs;
    hs.ld = c->ld;
    hs.n_chunks = c->n_chunks;
    hs.chunk_dig = c->d_chunk_dig;
    hs.chunk_begin = c->d_chunk_beg;
    hs.chunk_end = c->d_chunk_end;
    hs.dig_offset = c->d_off;
    hs.dig_chunk0 = c->d_dig_chunk0;
    hs.n_dig = c->n_dig;
    hs.y = c->d_y;
    hs.partial = c->d_partial;
    hs.mean = c->d_mean;
    hs.dig = c->d_dig;
    hs.n = c->N;
    if ((e = launch_headspace(hs, s)) != cudaSuccess) return e;
  }
  return launch_bump(c->d_interval, s);
}

chad_status chad_set_mlp(chad_ctx* c, const float* params, const float* feat_norm,
                         const float* out_norm) {
  if (!c) return CHAD_E_INVALID;
  if (!c->learned) return fail(c, CHAD_E_STATE, "context created with learned = 0");
  if (!params || !feat_norm || !out_norm) return fail(c, CHAD_E_INVALID, "null MLP input");
  for (int i = 0; i < CHAD_MLP_NPARAM; ++i)
    if (!std::isfinite(params[i])) return fail(c, CHAD_E_INVALID, "non-finite MLP parameter");
  for (int i = 0; i < 2 * CHAD_MLP_IN; ++i)
    if (!std::isfinite(feat_norm[i])) return fail(c, CHAD_E_INVALID, "non-finite feature norm");
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(out_norm[i])) return fail(c, CHAD_E_INVALID, "non-finite output norm");
  float* P = c->d_mlp;
  CK(c, cudaMemcpyAsync(P, params, sizeof(float) * CHAD_MLP_NPARAM, cudaMemcpyHostToDevice, c->stream), "mlp upload");
  CK(c, cudaMemcpyAsync(P + CHAD_MLP_NPARAM, feat_norm, sizeof(float) * 2 * CHAD_MLP_IN, cudaMemcpyHostToDevice, c->stream), "mlp upload");
  CK(c, cudaMemcpyAsync(P + CHAD_MLP_NPARAM + 2 * CHAD_MLP_IN, out_norm, sizeof(float) * 4, cudaMemcpyHostToDevice, c->stream), "mlp upload");
  CK(c, cudaStreamSynchronize(c->stream), "mlp upload sync");
  c->has_mlp = true;
  return CHAD_OK;
}

chad_status chad_step(chad_ctx* c, double dt_coupling_s, int n_intervals) {
  if (!c) return CHAD_E_INVALID;
  if (!(dt_coupling_s > 0.0) || !std::isfinite(dt_coupling_s) || n_intervals < 0)
    return fail(c, CHAD_E_INVALID, "dt_coupling_s must be > 0 and n_intervals >= 0");
  for (int d = 0; d < c->n_dig; ++d)
    if (!c->loaded[d]) return fail(c, CHAD_E_STATE, "every digester must be loaded before chad_step");
  if (n_intervals == 0 || c->N == 0) return CHAD_OK;
  cudaStream_t s = c->stream;
  chad_status st = prepare_flow(c, dt_coupling_s);
  if (st != CHAD_OK) return st;
  st = prepare_diffusion(c, dt_coupling_s);
  if (st != CHAD_OK) return st;
  const double dt_days = dt_coupling_s / 86400.0;
  const int variant = c->variant[kernel_form(c)];
  // one graph per interval: capture once, replay per interval (not possible
  // on the legacy default stream)
  if (c->use_graph && s != nullptr &&
      (c->gexec == nullptr || c->g_dt != dt_coupling_s || c->g_variant != variant)) {
    drop_graph(c);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_interval(c, dt_days, variant, s);
      e = cudaStreamEndCapture(s, &g);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->gexec = nullptr;
      c->use_graph = false;  // capture unavailable: launch directly from now on
    } else {
      c->g_dt = dt_coupling_s;
      c->g_variant = variant;
    }
  }
  if (c->learned && !c->has_mlp)
    return fail(c, CHAD_E_STATE, "learned = 1 needs chad_set_mlp before chad_step");
  for (int it = 0; it < n_intervals; ++it) {
    if (c->learned && c->cold_pending) {
      // first interval after a load without step-size history: learned guesses
      CK(c, enqueue_interval(c, dt_days, variant, s, true), "interval launch");
      c->cold_pending = false;
    } else if (c->gexec) {
      CK(c, cudaGraphLaunch(c->gexec, s), "graph launch");
    } else {
      CK(c, enqueue_interval(c, dt_days, variant, s), "interval launch");
    }
    c->intervals++;
    c->sim_days += dt_days * (double)c->N;
  }
  return CHAD_OK;
}

chad_status chad_set_kernel_variant(chad_ctx* c, int variant) {
  if (!c) return CHAD_E_INVALID;
  if (variant < 0 || variant >= kNumVariants)
    return fail(c, CHAD_E_INVALID, "variant must be in [0, CHAD_NUM_VARIANTS)");
  c->variant[kernel_form(c)] = variant;
  drop_graph(c);
  return CHAD_OK;
}

chad_status chad_autotune(chad_ctx* c, double dt_coupling_s, int32_t* chosen, double* ms) {
  if (!c) return CHAD_E_INVALID;
  if (!(dt_coupling_s > 0.0) || !std::isfinite(dt_coupling_s))
    return fail(c, CHAD_E_INVALID, "dt_coupling_s must be > 0");
  for (int d = 0; d < c->n_dig; ++d)
    if (!c->loaded[d]) return fail(c, CHAD_E_STATE, "every digester must be loaded before chad_autotune");
  cudaStream_t s = c->stream;
  chad_status st = prepare_flow(c, dt_coupling_s);
  if (st != CHAD_OK) return st;
  st = prepare_diffusion(c, dt_coupling_s);
  if (st != CHAD_OK) return st;
  const size_t nd = (size_t)c->ld;
  // snapshot of everything an interval modifies
  const size_t dbl = (size_t)(NS + 3 + 3) * nd;  // y, pos, SH, h, D
  double* snap = nullptr;
  int* snap_st = nullptr;
  if (cudaMalloc(&snap, sizeof(double) * dbl) != cudaSuccess) { cudaGetLastError(); return fail(c, CHAD_E_NOMEM, "autotune snapshot"); }
  if (cudaMalloc(&snap_st, sizeof(int) * nd) != cudaSuccess) { cudaFree(snap); cudaGetLastError(); return fail(c, CHAD_E_NOMEM, "autotune snapshot"); }
  DevCounters cnt_saved;
  unsigned long long int_saved = 0;
  auto save = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(snap, c->d_y, sizeof(double) * NS * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(snap + NS * nd, c->d_pos, sizeof(double) * 3 * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(snap + (NS + 3) * nd, c->d_SH, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(snap + (NS + 4) * nd, c->d_h, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(snap + (NS + 5) * nd, c->d_D, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(snap_st, c->d_status, sizeof(int) * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt_saved, c->d_cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&int_saved, c->d_interval, sizeof(int_saved), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  };
  auto restore = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(c->d_y, snap, sizeof(double) * NS * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_pos, snap + NS * nd, sizeof(double) * 3 * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_SH, snap + (NS + 3) * nd, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_h, snap + (NS + 4) * nd, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_D, snap + (NS + 5) * nd, sizeof(double) * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_status, snap_st, sizeof(int) * nd, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_cnt, &cnt_saved, sizeof(DevCounters), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_interval, &int_saved, sizeof(int_saved), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
  };
  cudaError_t e = save();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int best = c->variant[kernel_form(c)];
  float best_ms = 1e30f;
  for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) {
    // two consecutive intervals per variant: one interval alone is too noisy
    // to separate variants that differ by a few per cent
    e = restore();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = enqueue_interval(c, dt_coupling_s / 86400.0, v, s);
    if (e == cudaSuccess) e = enqueue_interval(c, dt_coupling_s / 86400.0, v, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (ms) ms[v] = t;
    if (e == cudaSuccess && t < best_ms) { best_ms = t; best = v; }
  }
  if (e == cudaSuccess) e = restore();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(snap);
  cudaFree(snap_st);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
  c->variant[kernel_form(c)] = best;
  drop_graph(c);
  if (chosen) *chosen = best;
  return CHAD_OK;
}

chad_status chad_kernel_variant(int precision, int h2_algebraic, int v, int32_t* threads,
                                int32_t* min_blocks, int32_t* w_shared) {
  if (v < 0 || v >= kNumVariants) return CHAD_E_INVALID;
  if (precision < CHAD_PREC_FP64 || precision > CHAD_PREC_MIXED_F32RATES) return CHAD_E_INVALID;
  const int form = h2_algebraic ? (precision == CHAD_PREC_MIXED ? 4 : 3) : precision;
  const KernelVariant k = kernel_variant(form, v);
  if (threads) *threads = k.threads;
  if (min_blocks) *min_blocks = k.min_blocks;
  if (w_shared) *w_shared = k.w_shared;
  return CHAD_OK;
}

chad_status chad_synchronize(chad_ctx* c) {
  if (!c) return CHAD_E_INVALID;
  CK(c, cudaStreamSynchronize(c->stream), "synchronize");
  CK(c, cudaGetLastError(), "kernel");
  return CHAD_OK;
}

chad_status chad_read_states(chad_ctx* c, int digester, double* y, double* pos, double* S_H,
                             double* h, int32_t* status, chad_stats* stats, int mem) {
  if (!c) return CHAD_E_INVALID;
  if (digester < 0 || digester >= c->n_dig) return fail(c, CHAD_E_INVALID, "digester out of range");
  if (!c->loaded[digester]) return fail(c, CHAD_E_STATE, "digester not loaded");
  if (mem != CHAD_MEM_HOST && mem != CHAD_MEM_DEVICE) return fail(c, CHAD_E_INVALID, "mem must be HOST or DEVICE");
  cudaStream_t s = c->stream;
  const int64_t o = c->offset[digester], n = c->count[digester];
  const cudaMemcpyKind k = kind_out(mem);
  CK(c, cudaStreamSynchronize(s), "read sync");
  CK(c, cudaGetLastError(), "kernel");
  if (n > 0) {
    if (y)
      for (int i = 0; i < NS; ++i)
        CK(c, cudaMemcpyAsync(y + (size_t)i * n, c->d_y + (size_t)i * c->ld + o, sizeof(double) * n, k, s), "read y");
    if (pos)
      for (int i = 0; i < 3; ++i)
        CK(c, cudaMemcpyAsync(pos + (size_t)i * n, c->d_pos + (size_t)i * c->ld + o, sizeof(double) * n, k, s), "read pos");
    if (S_H) CK(c, cudaMemcpyAsync(S_H, c->d_SH + o, sizeof(double) * n, k, s), "read S_H");
    if (h) CK(c, cudaMemcpyAsync(h, c->d_h + o, sizeof(double) * n, k, s), "read h");
  }
  if (status && n > 0)
    CK(c, cudaMemcpyAsync(status, c->d_status + o, sizeof(int32_t) * n, k, s), "read status");
  unsigned long long* d_failed = c->d_misc + 1;
  CK(c, cudaMemsetAsync(d_failed, 0, sizeof(unsigned long long), s), "count failed");
  CK(c, launch_count_status(c->d_status, o, n, d_failed, s), "count failed");
  unsigned long long nfailed = 0;
  CK(c, cudaMemcpyAsync(&nfailed, d_failed, sizeof(nfailed), cudaMemcpyDeviceToHost, s), "count failed");
  DevCounters dc;
  CK(c, cudaMemcpyAsync(&dc, c->d_cnt, sizeof(dc), cudaMemcpyDeviceToHost, s), "read counters");
  CK(c, cudaStreamSynchronize(s), "read sync");
  const int64_t failed = (int64_t)nfailed;
  if (stats) {
    stats->accepted_steps = (int64_t)dc.accepted;
    stats->rejected_steps = (int64_t)dc.rejected;
    stats->newton_iters = (int64_t)dc.newton_iters;
    stats->newton_fallbacks = (int64_t)dc.newton_fallbacks;
    stats->min_steps = dc.min_steps == 0x7fffffff ? 0 : dc.min_steps;
    stats->max_steps = dc.max_steps;
    stats->failed_particles = failed;
    stats->mlp_redo = (int64_t)dc.mlp_redo;
    stats->pivot_rejects = (int64_t)dc.pivot_rejects;
    stats->h2_newton_iters = (int64_t)dc.h2_iters;
    stats->intervals = c->intervals;
    stats->sim_days = c->sim_days;
    DevCounters z{0, 0, 0, 0, 0, 0, 0x7fffffff, 0, 0};
    CK(c, cudaMemcpy(c->d_cnt, &z, sizeof(z), cudaMemcpyHostToDevice), "reset counters");
    c->intervals = 0;
    c->sim_days = 0.0;
  }
  return failed ? fail(c, CHAD_E_PARTICLE, std::to_string(failed) + " particle(s) with status != 0")
                : CHAD_OK;
}

}  // extern "C"
