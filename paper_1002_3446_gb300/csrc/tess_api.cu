// C ABI of the generator (declared in include/tess.h): argument validation,
// error reporting, launch sequencing.  Allocates no device memory.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tess.h"
#include "tess_grad.cuh"
#include "tess_kernels.cuh"
#include "tess_persist.cuh"
#include "tess_pipe_launch.cuh"

namespace tess {
cudaError_t launch_generate_f64(int n, bool sum, const EventParams &P, double *partials, int grid, cudaStream_t s);
cudaError_t launch_generate_f32(int n, bool sum, const EventParams &P, double *partials, int grid, cudaStream_t s);
cudaError_t peak_probe(int kind, int sms, int reps, cudaStream_t s, float *best_ms, double *flop);
cudaError_t persist_launch(const PersistParams &Q, const PersistFold &F, int nmax, int max_hist_bins, int sm_count,
                           cudaStream_t s, int *grid_out);
int grid_generate_f64(int n, bool sum, int sm_count, uint64_t n_events, int hist_bins);
int grid_generate_f32(int n, bool sum, int sm_count, uint64_t n_events, int hist_bins);
cudaError_t launch_me2_f64(int n, uint64_t n_events, const double *k, const uint8_t *order, const uint32_t *hel,
                           double *me2, cudaStream_t s, bool gauge = false);
cudaError_t launch_me2_f32(int n, uint64_t n_events, const double *k, const uint8_t *order, const uint32_t *hel,
                           double *me2, cudaStream_t s, bool gauge = false);
cudaError_t launch_grad_a(int n, bool fp64, const GradParams &G, void *ws, cudaStream_t s,
                           const GradStreams &gs);
cudaError_t launch_grad_b(int n, bool fp64, const GradParams &G, void *ws, cudaStream_t s,
                           const GradStreams &gs);
cudaError_t launch_grad_c(int n, bool fp64, const GradParams &G, void *ws, cudaStream_t s,
                           const GradStreams &gs);
size_t grad_workspace_a(int n, uint64_t n_events, size_t chunk_bytes);
size_t grad_workspace_b(int n, uint64_t n_events, size_t chunk_bytes);
size_t grad_workspace_c(int n, uint64_t n_events, size_t chunk_bytes);
cudaError_t launch_draws_a(int n, const EventParams &P, double *u, uint32_t *hel, uint8_t *order, cudaStream_t s);
cudaError_t launch_draws_b(int n, const EventParams &P, double *u, uint32_t *hel, uint8_t *order, cudaStream_t s);
cudaError_t launch_draws_c(int n, const EventParams &P, double *u, uint32_t *hel, uint8_t *order, cudaStream_t s);
int plan_pipeline_f64(int n, int sm_count, uint64_t n_events, int hist_bins, int form, int sched,
                      unsigned caps, PipePlan *pl);
int plan_pipeline_f32a(int n, int sm_count, uint64_t n_events, int hist_bins, int form, int sched,
                      unsigned caps, PipePlan *pl);
int plan_pipeline_f32b(int n, int sm_count, uint64_t n_events, int hist_bins, int form, int sched,
                      unsigned caps, PipePlan *pl);
int plan_pipeline_f32c(int n, int sm_count, uint64_t n_events, int hist_bins, int form, int sched,
                      unsigned caps, PipePlan *pl);
cudaError_t run_pipeline_f64(int n, const EventParams &P, const PipePlan &pl, char *ws, cudaStream_t s,
                             const StageHook *hook, const OverlapRes *ov);
cudaError_t run_pipeline_f32a(int n, const EventParams &P, const PipePlan &pl, char *ws, cudaStream_t s,
                             const StageHook *hook, const OverlapRes *ov);
cudaError_t run_pipeline_f32b(int n, const EventParams &P, const PipePlan &pl, char *ws, cudaStream_t s,
                             const StageHook *hook, const OverlapRes *ov);
cudaError_t run_pipeline_f32c(int n, const EventParams &P, const PipePlan &pl, char *ws, cudaStream_t s,
                             const StageHook *hook, const OverlapRes *ov);
// Neumaier-compensated addition (s, c) += x.
__device__ __forceinline__ void comp_add(double &s, double &c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

// Adds the total of partial-row column q into the caller's running
// accumulators (acc, hist), which carry their own compensation terms.
__device__ __forceinline__ void fold_column(int q, double tot, int nb2, double *acc, double *hist) {
  if (q == 0 || q == 1) {
    double hs = acc[q], hc = acc[4 + q];
    comp_add(hs, hc, tot);
    acc[q] = hs;
    acc[4 + q] = hc;
  } else if (q == 2) {
    acc[2] += tot;
  } else if (q == 3) {
    acc[6] += tot;
  } else if (q == 4) {
    acc[7] += tot;
  } else {
    const int h = q - kPartialHead;  // 0..2 nb2 - 1: w bins then w^2 bins
    double hs = hist[h], hc = hist[2 * nb2 + h];
    comp_add(hs, hc, tot);
    hist[h] = hs;
    hist[2 * nb2 + h] = hc;
  }
}

// Folds the per-block partials, in block order with compensation, into the
// caller's running accumulators (acc, hist), which carry their own
// compensation terms between calls.
__global__ void finalize_kernel(const double *__restrict__ partials, int nblocks, int hist_bins, uint64_t n_events,
                                double *acc, double *hist) {
  const int stride = partial_stride(hist_bins);
  const int nb2 = hist_bins > 0 ? hist_bins + 2 : 0;
  const int nq = kPartialHead + 2 * nb2;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double s = 0.0, c = 0.0;
    for (int b = 0; b < nblocks; ++b) comp_add(s, c, partials[(size_t)b * stride + q]);
    fold_column(q, s + c, nb2, acc, hist);
  }
  if (threadIdx.x == 0) acc[3] += (double)n_events;
}

// The same fold with the work spread over the GPU: block q sums column q,
// its kFinThreads threads each over the rows t, t + kFinThreads, ... with
// compensation, then a fixed-shape compensated tree.  Deterministic (fixed
// assignment and order); FP64 issue is 1/64 rate here, so a single thread
// per column would spend ~64 cycles per row.
constexpr int kFinThreads = 64;

__global__ void __launch_bounds__(kFinThreads) finalize_cols_kernel(const double *__restrict__ partials, int nrows,
                                                                    int hist_bins, uint64_t n_events, double *acc,
                                                                    double *hist) {
  const int stride = partial_stride(hist_bins);
  const int nb2 = hist_bins > 0 ? hist_bins + 2 : 0;
  const int q = blockIdx.x, t = threadIdx.x;
  double s = 0.0, c = 0.0;
  for (int r = t; r < nrows; r += kFinThreads) comp_add(s, c, partials[(size_t)r * stride + q]);
  __shared__ double ss[kFinThreads], cc[kFinThreads];
  ss[t] = s;
  cc[t] = c;
  __syncthreads();
  for (int w = kFinThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
      double a = ss[t], ac = cc[t];
      comp_add(a, ac, ss[t + w]);
      ss[t] = a;
      cc[t] = ac + cc[t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    fold_column(q, ss[0] + cc[0], nb2, acc, hist);
    if (q == 0) acc[3] += (double)n_events;
  }
}

}  // namespace tess

constexpr int kMaxBranches = 16;
constexpr int kGradSlot = kMaxBranches + 1;

struct tess_ctx {
  int device = 0;
  int sm_count = 1;
  // tuned amplitude-kernel variant and chunk schedule per (precision,
  // polarisation kind, cut-first, n) -- see variant_slot; -1 = built-in default
  int form[8][TESS_MAX_N + 1];
  int sched[8][TESS_MAX_N + 1];
  // streams/events of the overlapped pipelines: [0] plain calls, [1 + i] batch
  // branch i, [kGradSlot] the gradient pipeline
  tess::OverlapRes ovl[kMaxBranches + 2];
  // batched generation: capture streams, fork/join events, cached graph
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t fork_ev = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned char> graph_key;
  // pipeline plans already made on this context, keyed by what sizes them
  // (n, precision, polarisation kind, flags, histogram bins, events, variant,
  // schedule): planning queries the runtime (function attributes, occupancy)
  // for every candidate kernel, and sizing a workspace plans every variant
  mutable std::mutex plan_mu;
  mutable std::map<std::array<int64_t, 9>, tess::PipePlan> plans;
  // bytes of per-event intermediate data per generation chunk (0 = default)
  size_t chunk_bytes = 0;
  // opt-in stage timing: event pairs recorded around each launch
  bool timing = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_marks;
  cudaEvent_t ev_open[4] = {};
  tess_ctx() {
    for (auto &row : form)
      for (int &f : row) f = -1;
    for (auto &row : sched)
      for (int &f : row) f = -1;
  }
};

namespace {

thread_local std::string g_error;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

int ok() {
  g_error.clear();
  return TESS_OK;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(TESS_E_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Makes ctx's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) {
      err = cudaSetDevice(dev);
      changed = (err == cudaSuccess);
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int check_process(const tess_process *p) {
  if (!p) return fail(TESS_E_INVALID, "process is NULL");
  if (p->n_gluons < TESS_MIN_N || p->n_gluons > TESS_MAX_N)
    return fail(TESS_E_UNSUPPORTED, "n_gluons = %d outside %d..%d", p->n_gluons, TESS_MIN_N, TESS_MAX_N);
  if (p->precision != TESS_FP64 && p->precision != TESS_FP32_CURRENTS && p->precision != TESS_FP32_DS)
    return fail(TESS_E_INVALID, "precision = %d is not TESS_FP64, TESS_FP32_CURRENTS or TESS_FP32_DS",
                p->precision);
  if (p->helicity_mode != TESS_HEL_SUM && p->helicity_mode != TESS_HEL_SAMPLE && p->helicity_mode != TESS_POL_RANDOM)
    return fail(TESS_E_INVALID, "helicity_mode = %d is not TESS_HEL_SUM, TESS_HEL_SAMPLE or TESS_POL_RANDOM",
                p->helicity_mode);
  if (p->helicity_mode == TESS_HEL_SUM && p->n_gluons > 5)
    return fail(TESS_E_UNSUPPORTED, "TESS_HEL_SUM is built for n <= 5 (n = %d)", p->n_gluons);
  if ((p->flags & ~(TESS_FLAG_CUT_FIRST | TESS_FLAG_PDF_GRID)) != 0 || p->reserved != 0)
    return fail(TESS_E_INVALID, "flags = %d / reserved = %d: only TESS_FLAG_CUT_FIRST and TESS_FLAG_PDF_GRID are defined",
                p->flags, p->reserved);
  if (p->flags != 0 && (p->precision == TESS_FP64 || p->helicity_mode == TESS_HEL_SUM))
    return fail(TESS_E_UNSUPPORTED, "TESS_FLAG_* are built for the FP32 forms with sampled events");
  if (!finite_pos(p->sqrt_s)) return fail(TESS_E_INVALID, "sqrt_s must be finite and > 0");
  if (!finite_pos(p->pt_min)) return fail(TESS_E_INVALID, "pt_min must be finite and > 0");
  if (!finite_pos(p->eta_max)) return fail(TESS_E_INVALID, "eta_max must be finite and > 0");
  if (!(std::isfinite(p->dr_min) && p->dr_min >= 0.0)) return fail(TESS_E_INVALID, "dr_min must be finite and >= 0");
  if (!finite_pos(p->alphas_mz)) return fail(TESS_E_INVALID, "alphas_mz must be finite and > 0");
  if (!finite_pos(p->mz)) return fail(TESS_E_INVALID, "mz must be finite and > 0");
  if (!finite_pos(p->mu_r_factor)) return fail(TESS_E_INVALID, "mu_r_factor must be finite and > 0");
  if (p->nf < 0 || p->nf > 6) return fail(TESS_E_INVALID, "nf = %d outside 0..6", p->nf);
  if ((p->n_gluons - 2) * p->pt_min >= p->sqrt_s)
    return fail(TESS_E_INVALID, "(n-2) * pt_min must be below sqrt_s (no phase space passes the cuts)");
  if (p->hist_bins < 0 || p->hist_bins > TESS_MAX_BINS)
    return fail(TESS_E_INVALID, "hist_bins = %d outside 0..%d", p->hist_bins, TESS_MAX_BINS);
  if (p->hist_bins > 0) {
    if (p->hist_observable < 0 || p->hist_observable > 2)
      return fail(TESS_E_INVALID, "hist_observable = %d is not a TESS_OBS_* value", p->hist_observable);
    if (!(std::isfinite(p->hist_lo) && std::isfinite(p->hist_hi) && p->hist_lo < p->hist_hi))
      return fail(TESS_E_INVALID, "histogram range must satisfy finite hist_lo < hist_hi");
  }
  return TESS_OK;
}

// Rejects host or foreign-device pointers before any kernel dereferences them.
int check_device_ptr(const void *p, int device, const char *name) {
  if (!p) return TESS_OK;
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TESS_E_INVALID, "%s: not a CUDA pointer (%s)", name, cudaGetErrorName(e));
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(TESS_E_INVALID, "%s: must be device memory", name);
  if (a.type == cudaMemoryTypeDevice && a.device != device)
    return fail(TESS_E_INVALID, "%s: lives on device %d, context is on device %d", name, a.device, device);
  return TESS_OK;
}

// A per-event output array: device memory, or pinned host memory mapped into
// the device's address space (cudaHostAlloc / cudaHostRegister), which the
// kernels then store into directly (over NVLink-C2C on Grace-Blackwell).
// *dev receives the pointer the kernels use.
int output_ptr(void *p, int device, const char *name, void **dev) {
  *dev = p;
  if (!p) return TESS_OK;
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TESS_E_INVALID, "%s: not a CUDA pointer (%s)", name, cudaGetErrorName(e));
  }
  if (a.type == cudaMemoryTypeHost) {
    if (!a.devicePointer) return fail(TESS_E_INVALID, "%s: pinned host memory not mapped for the device", name);
    *dev = a.devicePointer;
    return TESS_OK;
  }
  return check_device_ptr(p, device, name);
}

int grid_for(const tess_ctx *ctx, const tess_process *p, uint64_t n_events) {
  const bool sum = p->helicity_mode == TESS_HEL_SUM;
  const uint64_t ne = n_events ? n_events : 1;
  return p->precision == TESS_FP64 ? tess::grid_generate_f64(p->n_gluons, sum, ctx->sm_count, ne, p->hist_bins)
                                   : tess::grid_generate_f32(p->n_gluons, sum, ctx->sm_count, ne, p->hist_bins);
}

double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

// Sampled helicity/ordering runs the two-kernel pipeline; the exact sum runs
// the fused kernel.
bool uses_pipeline(const tess_process *p) { return p->helicity_mode != TESS_HEL_SUM; }

// Variant-table row of a process: precision (FP64 / FP32) x polarisation
// kind (complex helicity vectors / random real vectors, which admit the
// real-current amplitude forms) x cut-first (which the staged forms lack).
int variant_slot(const tess_process *p) {
  return (p->precision == TESS_FP64 ? 0 : 1) + (p->helicity_mode == TESS_POL_RANDOM ? 2 : 0) +
         ((p->flags & TESS_FLAG_CUT_FIRST) ? 4 : 0);
}

int plan_with_form(const tess_ctx *ctx, const tess_process *p, uint64_t n_events, int form, int sched,
                   tess::PipePlan *pl) {
  const int n = p->n_gluons;
  const std::array<int64_t, 9> key = {n,    p->precision, p->helicity_mode == TESS_POL_RANDOM, p->flags,
                                      p->hist_bins, (int64_t)n_events, form, sched, (int64_t)ctx->chunk_bytes};
  {
    std::lock_guard<std::mutex> lock(ctx->plan_mu);
    const auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
      *pl = it->second;
      return TESS_OK;
    }
  }
  const unsigned caps = (p->helicity_mode == TESS_POL_RANDOM ? tess::CAP_REAL_EPS : 0u) |
                        ((p->flags & TESS_FLAG_CUT_FIRST) ? tess::CAP_CUT_FIRST : 0u) |
                        ((p->flags & TESS_FLAG_PDF_GRID) ? tess::CAP_PDF_GRID : 0u) |
                        (p->precision == TESS_FP32_DS ? tess::CAP_KIN_DS : 0u);
  int rc;
  *pl = tess::PipePlan();
  pl->chunk_target = ctx->chunk_bytes;
  if (p->precision == TESS_FP64)
    rc = tess::plan_pipeline_f64(n, ctx->sm_count, n_events, p->hist_bins, form, sched, caps, pl);
  else if (n <= 7)
    rc = tess::plan_pipeline_f32a(n, ctx->sm_count, n_events, p->hist_bins, form, sched, caps, pl);
  else if (n <= 10)
    rc = tess::plan_pipeline_f32b(n, ctx->sm_count, n_events, p->hist_bins, form, sched, caps, pl);
  else
    rc = tess::plan_pipeline_f32c(n, ctx->sm_count, n_events, p->hist_bins, form, sched, caps, pl);
  if (rc)
    return fail(TESS_E_CUDA, "could not size the pipeline kernels (n %d, amplitude variant %d, schedule %d: %s)", n,
                form, sched,
                rc == tess::kPlanNoResidentBlock ? "no block fits on an SM" : cudaGetErrorString((cudaError_t)rc));
  std::lock_guard<std::mutex> lock(ctx->plan_mu);
  if (ctx->plans.size() >= 4096) ctx->plans.clear();
  ctx->plans.emplace(key, *pl);
  return TESS_OK;
}

int pipeline_plan(const tess_ctx *ctx, const tess_process *p, uint64_t n_events, tess::PipePlan *pl) {
  const int pi = variant_slot(p);
  return plan_with_form(ctx, p, n_events, ctx->form[pi][p->n_gluons], ctx->sched[pi][p->n_gluons], pl);
}

// Workspace of the largest amplitude-kernel variant and schedule (the
// overlapped ones hold two chunk buffers), so that tuning never needs a larger
// workspace than the one sized before it.
int pipeline_bytes_any_form(const tess_ctx *ctx, const tess_process *p, uint64_t n_events, size_t *bytes) {
  size_t best = 0;
  for (int f = 0; f < tess::K2_NFORMS; ++f)
    for (int o = 0; o < tess::SCHED_N; ++o) {
      tess::PipePlan pl;
      const int rc = plan_with_form(ctx, p, n_events, f, o, &pl);
      if (rc) return rc;
      if (pl.bytes > best) best = pl.bytes;
    }
  *bytes = best;
  return TESS_OK;
}

// Lazily created streams and events of the overlapped pipeline.
int overlap_res(tess_ctx *ctx, int slot, tess::OverlapRes **out) {
  tess::OverlapRes &o = ctx->ovl[slot];
  if (!o.aux) {
    cudaError_t e = cudaStreamCreateWithFlags(&o.aux, cudaStreamNonBlocking);
    cudaEvent_t *evs[] = {&o.fork, &o.join, &o.k1done[0], &o.k1done[1], &o.k2done[0], &o.k2done[1]};
    for (cudaEvent_t *ev : evs)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "overlap stream/event creation");
  }
  *out = &o;
  return TESS_OK;
}

cudaError_t pipeline_run(const tess_process *p, const tess::EventParams &P, const tess::PipePlan &pl, char *ws,
                         cudaStream_t s, const tess::StageHook *hook, const tess::OverlapRes *ov) {
  const int n = p->n_gluons;
  if (p->precision == TESS_FP64) return tess::run_pipeline_f64(n, P, pl, ws, s, hook, ov);
  if (n <= 7) return tess::run_pipeline_f32a(n, P, pl, ws, s, hook, ov);
  if (n <= 10) return tess::run_pipeline_f32b(n, P, pl, ws, s, hook, ov);
  return tess::run_pipeline_f32c(n, P, pl, ws, s, hook, ov);
}

// Stage timing hook: records an event before and after each launch.
void stage_mark(void *self, int kind, bool begin, cudaStream_t s) {
  tess_ctx *ctx = (tess_ctx *)self;
  cudaEvent_t e = nullptr;
  if (!ctx->ev_free.empty()) {
    e = ctx->ev_free.back();
    ctx->ev_free.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return;
  }
  cudaEventRecord(e, s);
  if (begin) {
    ctx->ev_open[kind] = e;
  } else if (ctx->ev_open[kind]) {
    ctx->ev_marks.push_back({kind, {ctx->ev_open[kind], e}});
    ctx->ev_open[kind] = nullptr;
  } else {
    ctx->ev_free.push_back(e);
  }
}

// Launch constants of one generation call.
void fill_params(const tess_process *proc, uint64_t seed, uint64_t first_event, uint64_t n_events,
                 const tess_outputs *out, tess::EventParams *Pp) {
  tess::EventParams &P = *Pp;
  const int n = proc->n_gluons, m = n - 2;
  const bool sum = proc->helicity_mode == TESS_HEL_SUM;
  memset(&P, 0, sizeof P);
  P.seed = seed;
  P.first_event = first_event;
  P.n_events = n_events;
  P.S = proc->sqrt_s * proc->sqrt_s;
  P.lnxmin = std::log((m * proc->pt_min) * (m * proc->pt_min) / P.S);
  P.pt_min = proc->pt_min;
  P.eta_max = proc->eta_max;
  P.dr2_min = proc->dr_min * proc->dr_min;
  P.alphas_mz = proc->alphas_mz;
  P.ln_mz2 = std::log(proc->mz * proc->mz);
  P.b0 = (33.0 - 2.0 * proc->nf) / (12.0 * M_PI);
  P.mu_r_factor = proc->mu_r_factor;
  const double nc = 3.0;
  P.wconst = std::pow(nc, n - 2) * (nc * nc - 1.0) / (256.0 * factorial(m)) * 0.3893793721e9;
  P.phiconst = std::pow(2.0 * M_PI, 4.0 - 3.0 * m) * std::pow(M_PI / 2.0, m - 1.0) / (factorial(m - 1) * factorial(m - 2));
  P.efac = sum ? 1.0 / std::ldexp(1.0, n - 2) : std::ldexp(1.0, n) * factorial(n - 1) / std::ldexp(1.0, n - 2);
  P.hist_bins = proc->hist_bins;
  P.hist_obs = proc->hist_observable;
  P.hist_lo = proc->hist_lo;
  P.hist_inv_width = proc->hist_bins > 0 ? proc->hist_bins / (proc->hist_hi - proc->hist_lo) : 0.0;
  P.weight = out->weight;
  P.me2 = out->me2;
  P.pass = out->pass;
  P.ht = out->ht;
  P.ptlead = out->ptlead;
  P.rmin = out->rmin;
  P.kin_ds = proc->precision == TESS_FP32_DS;
  P.pol_random = proc->helicity_mode == TESS_POL_RANDOM;
  P.cut_first = (proc->flags & TESS_FLAG_CUT_FIRST) != 0;
  P.pdf_grid = (proc->flags & TESS_FLAG_PDF_GRID) != 0;
  {  // alpha_s table range: ln mu^2 from the smallest H_T that passes the cuts to sqrt(S)
    const double vlo = 2.0 * std::log(proc->mu_r_factor * m * proc->pt_min);
    const double vhi = 2.0 * std::log(proc->mu_r_factor * proc->sqrt_s);
    P.as_vlo = vlo;
    P.as_vhi = vhi;
    P.f_as_vlo = (float)vlo;
    P.f_as_inv = (float)(tess::kAsSegments / (vhi - vlo));
  }
  P.S_hi = (float)P.S;
  P.S_lo = (float)(P.S - (double)P.S_hi);
  P.wk = P.wconst * P.lnxmin * P.lnxmin * P.phiconst * 0.5;
  tess::philox_round_keys(seed, P.rk);
  P.f_lnxmin = (float)P.lnxmin;
  P.f_pt_min = (float)P.pt_min;
  P.f_eta_max = (float)P.eta_max;
  P.f_dr2_min = (float)P.dr2_min;
  P.f_alphas_mz = (float)P.alphas_mz;
  P.f_asb0 = (float)P.alphas_mz * (float)P.b0;
  P.f_ln_mz2 = (float)P.ln_mz2;
  P.f_mu_r_factor = (float)P.mu_r_factor;
}

}  // namespace

extern "C" {

const char *tess_version(void) { return "tess-gb300 0.1"; }

const char *tess_last_error(void) { return g_error.c_str(); }

int tess_init(int device, tess_ctx **ctx) {
  if (!ctx) return fail(TESS_E_INVALID, "ctx is NULL");
  *ctx = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) return fail(TESS_E_INVALID, "device %d outside 0..%d", device, count - 1);
  int major = 0, minor = 0, sms = 0;
  if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
    return cuda_fail(e, "cudaDeviceGetAttribute");
  if (major != 10 || minor != 3)
    return fail(TESS_E_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a (GB300) only", device,
                major, minor);
  tess_ctx *c = new tess_ctx();
  c->device = device;
  c->sm_count = sms;
  *ctx = c;
  return ok();
}

void tess_destroy(tess_ctx *ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  for (auto &o : ctx->ovl) {
    if (o.aux) cudaStreamDestroy(o.aux);
    cudaEvent_t evs[] = {o.fork, o.join, o.k1done[0], o.k1done[1], o.k2done[0], o.k2done[1]};
    for (cudaEvent_t e : evs)
      if (e) cudaEventDestroy(e);
  }
  for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
  for (auto &m : ctx->ev_marks) {
    cudaEventDestroy(m.second.first);
    cudaEventDestroy(m.second.second);
  }
  delete ctx;
}

int tess_workspace_size(const tess_ctx *ctx, const tess_process *proc, uint64_t n_events, size_t *bytes) {
  if (!ctx || !bytes) return fail(TESS_E_INVALID, "ctx and bytes must not be NULL");
  int rc = check_process(proc);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if (uses_pipeline(proc)) {
    if ((rc = pipeline_bytes_any_form(ctx, proc, n_events, bytes))) return rc;
    return ok();
  }
  const int grid = grid_for(ctx, proc, n_events);
  *bytes = (size_t)grid * (size_t)tess::partial_stride(proc->hist_bins) * sizeof(double);
  return ok();
}

int tess_kernel_launches(const tess_ctx *ctx, const tess_process *proc, uint64_t n_events, int *launches) {
  if (!ctx || !launches) return fail(TESS_E_INVALID, "ctx and launches must not be NULL");
  int rc = check_process(proc);
  if (rc) return rc;
  if (n_events == 0) {
    *launches = 0;
    return ok();
  }
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if (uses_pipeline(proc)) {
    tess::PipePlan pl;
    if ((rc = pipeline_plan(ctx, proc, n_events, &pl))) return rc;
    *launches = 2 * pl.chunks + 1;  // (kinematics, amplitude) per chunk + finalize
  } else {
    *launches = 2;  // fused event kernel + finalize
  }
  return ok();
}

}  // extern "C"

namespace {

// A validated, planned generation call: everything tess_generate needs except
// the stream.  Built outside any stream capture; launching it only enqueues
// memsets and kernels.
struct Prepared {
  tess::EventParams P;
  bool pipeline = false;
  bool sum = false;
  tess::PipePlan pl;
  int grid = 1;
  const tess_process *proc = nullptr;
  void *workspace = nullptr;
  double *acc = nullptr, *hist = nullptr;
};

int prepare(tess_ctx *ctx, const tess_process *proc, uint64_t seed, uint64_t first_event, uint64_t n_events,
            const tess_outputs *out, void *workspace, size_t workspace_bytes, Prepared *pr) {
  int rc = check_process(proc);
  if (rc) return rc;
  if (!out || !out->acc) return fail(TESS_E_INVALID, "outputs and outputs->acc must not be NULL");
  if (proc->hist_bins > 0 && !out->hist) return fail(TESS_E_INVALID, "hist_bins > 0 needs outputs->hist");
  if (n_events > (UINT64_MAX - first_event)) return fail(TESS_E_INVALID, "event range overflows 64 bits");
  const void *ptrs[] = {out->acc, out->hist, workspace};
  const char *names[] = {"acc", "hist", "workspace"};
  for (int i = 0; i < 3; ++i)
    if ((rc = check_device_ptr(ptrs[i], ctx->device, names[i]))) return rc;
  if (((uintptr_t)workspace) % 256 != 0) return fail(TESS_E_WORKSPACE, "workspace must be 256-byte aligned");
  tess_outputs o = *out;  // per-event arrays as the kernels address them
  void *dev = nullptr;
  if ((rc = output_ptr(out->weight, ctx->device, "weight", &dev))) return rc;
  o.weight = (double *)dev;
  if ((rc = output_ptr(out->me2, ctx->device, "me2", &dev))) return rc;
  o.me2 = (double *)dev;
  if ((rc = output_ptr(out->pass, ctx->device, "pass", &dev))) return rc;
  o.pass = (uint8_t *)dev;
  if ((rc = output_ptr(out->ht, ctx->device, "ht", &dev))) return rc;
  o.ht = (double *)dev;
  if ((rc = output_ptr(out->ptlead, ctx->device, "ptlead", &dev))) return rc;
  o.ptlead = (double *)dev;
  if ((rc = output_ptr(out->rmin, ctx->device, "rmin", &dev))) return rc;
  o.rmin = (double *)dev;
  fill_params(proc, seed, first_event, n_events, &o, &pr->P);
  pr->proc = proc;
  pr->workspace = workspace;
  pr->acc = out->acc;
  pr->hist = out->hist;
  pr->sum = proc->helicity_mode == TESS_HEL_SUM;
  pr->pipeline = uses_pipeline(proc);
  size_t need;
  if (pr->pipeline) {
    if ((rc = pipeline_plan(ctx, proc, n_events, &pr->pl))) return rc;
    pr->grid = pr->pl.grid;
    need = pr->pl.bytes;
  } else {
    pr->grid = grid_for(ctx, proc, n_events);
    need = (size_t)pr->grid * (size_t)tess::partial_stride(proc->hist_bins) * sizeof(double);
  }
  if (!workspace || workspace_bytes < need)
    return fail(TESS_E_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, workspace ? workspace_bytes : 0);
  return TESS_OK;
}

// fold = false: leave the sums in the workspace's partial rows (timing runs).
int launch_prepared(const Prepared &pr, cudaStream_t s, const tess::StageHook *hook = nullptr,
                    const tess::OverlapRes *ov = nullptr, bool fold = true) {
  if (pr.P.n_events == 0) return TESS_OK;
  const int n = pr.proc->n_gluons;
  double *partials = (double *)pr.workspace;
  cudaError_t e;
  if (pr.pipeline) {
    e = pipeline_run(pr.proc, pr.P, pr.pl, (char *)pr.workspace, s, hook, ov);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline launch");
  } else {
    if (hook) (*hook)(tess::STAGE_FUSED, true, s);
    e = pr.proc->precision == TESS_FP64 ? tess::launch_generate_f64(n, pr.sum, pr.P, partials, pr.grid, s)
                                        : tess::launch_generate_f32(n, pr.sum, pr.P, partials, pr.grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "event kernel launch");
    if (hook) (*hook)(tess::STAGE_FUSED, false, s);
  }
  if (!fold) return TESS_OK;
  if (hook) (*hook)(tess::STAGE_FINAL, true, s);
  tess::finalize_cols_kernel<<<tess::kPartialHead + 2 * (pr.proc->hist_bins > 0 ? pr.proc->hist_bins + 2 : 0),
                                tess::kFinThreads, 0, s>>>(partials, pr.grid, pr.proc->hist_bins, pr.P.n_events, pr.acc,
                                                           pr.hist);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel launch");
  if (hook) (*hook)(tess::STAGE_FINAL, false, s);
  return TESS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

int tess_generate(tess_ctx *ctx, const tess_process *proc, uint64_t seed, uint64_t first_event, uint64_t n_events,
                  const tess_outputs *out, void *workspace, size_t workspace_bytes, void *stream) {
  if (!ctx) return fail(TESS_E_INVALID, "ctx is NULL");
  int rc = check_process(proc);
  if (rc) return rc;
  if (!out || !out->acc) return fail(TESS_E_INVALID, "outputs and outputs->acc must not be NULL");
  if (n_events == 0) return ok();
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  Prepared pr;
  if ((rc = prepare(ctx, proc, seed, first_event, n_events, out, workspace, workspace_bytes, &pr))) return rc;
  tess::OverlapRes *ov = nullptr;
  if (pr.pipeline && pr.pl.overlap && (rc = overlap_res(ctx, 0, &ov))) return rc;
  tess::StageHook hook{stage_mark, ctx};
  if ((rc = launch_prepared(pr, (cudaStream_t)stream, ctx->timing ? &hook : nullptr, ov))) return rc;
  return ok();
}

int tess_stage_timing(tess_ctx *ctx, int enable) {
  if (!ctx) return fail(TESS_E_INVALID, "ctx is NULL");
  ctx->timing = enable != 0;
  return ok();
}

int tess_stage_times(tess_ctx *ctx, double *ms, int *launches) {
  if (!ctx || !ms || !launches) return fail(TESS_E_INVALID, "NULL argument");
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  for (int k = 0; k < tess::STAGE_NKINDS; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  cudaError_t e = cudaSuccess;
  for (auto &m : ctx->ev_marks) {
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventSynchronize(m.second.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, m.second.first, m.second.second);
    ms[m.first] += t;
    launches[m.first] += 1;
    ctx->ev_free.push_back(m.second.first);
    ctx->ev_free.push_back(m.second.second);
  }
  ctx->ev_marks.clear();
  if (e != cudaSuccess) return cuda_fail(e, "stage timing events");
  return ok();
}

int tess_workspace_size_batched(const tess_ctx *ctx, int n_proc, const tess_process *procs,
                                const uint64_t *n_events, size_t *bytes) {
  if (!ctx || !procs || !n_events || !bytes) return fail(TESS_E_INVALID, "NULL argument");
  if (n_proc < 1 || n_proc > kMaxBranches) return fail(TESS_E_INVALID, "n_proc must be 1..%d", kMaxBranches);
  size_t tot = 0;
  for (int i = 0; i < n_proc; ++i) {
    size_t b = 0;
    const int rc = tess_workspace_size(ctx, &procs[i], n_events[i], &b);
    if (rc) return rc;
    tot += align256(b);
  }
  *bytes = tot;
  return ok();
}

int tess_generate_batched(tess_ctx *ctx, int n_proc, const tess_process *procs, const uint64_t *seeds,
                          const uint64_t *first_events, const uint64_t *n_events, const tess_outputs *outs,
                          void *workspace, size_t workspace_bytes, void *stream) {
  if (!ctx || !procs || !seeds || !first_events || !n_events || !outs) return fail(TESS_E_INVALID, "NULL argument");
  if (n_proc < 1 || n_proc > kMaxBranches) return fail(TESS_E_INVALID, "n_proc must be 1..%d", kMaxBranches);
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  // validate and plan every process before anything is captured
  std::vector<Prepared> prs(n_proc);
  char *ws = (char *)workspace;
  size_t left = workspace ? workspace_bytes : 0;
  int rc;
  for (int i = 0; i < n_proc; ++i) {
    size_t b = 0;
    if ((rc = tess_workspace_size(ctx, &procs[i], n_events[i], &b))) return rc;
    b = align256(b);
    if (b > left) return fail(TESS_E_WORKSPACE, "batched workspace too small at process %d", i);
    if ((rc = prepare(ctx, &procs[i], seeds[i], first_events[i], n_events[i], &outs[i], ws, b, &prs[i]))) return rc;
    ws += b;
    left -= b;
  }
  // graph key: every argument that is baked into the captured launches
  std::vector<unsigned char> key;
  auto put = [&](const void *p, size_t n) {
    const unsigned char *c = (const unsigned char *)p;
    key.insert(key.end(), c, c + n);
  };
  put(&n_proc, sizeof n_proc);
  put(procs, sizeof(tess_process) * n_proc);
  put(seeds, sizeof(uint64_t) * n_proc);
  put(first_events, sizeof(uint64_t) * n_proc);
  put(n_events, sizeof(uint64_t) * n_proc);
  put(outs, sizeof(tess_outputs) * n_proc);
  put(&workspace, sizeof workspace);
  put(ctx->form, sizeof ctx->form);
  put(ctx->sched, sizeof ctx->sched);
  cudaError_t e = cudaSuccess;
  if (!ctx->graph_exec || key != ctx->graph_key) {
    if (!ctx->cap_stream) {
      if ((e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "stream/event creation");
    }
    for (int i = 0; i < n_proc; ++i) {
      tess::OverlapRes *ov = nullptr;
      if (prs[i].pipeline && prs[i].pl.overlap && (rc = overlap_res(ctx, 1 + i, &ov))) return rc;
    }
    // the processes one after another in a single chain (concurrent branches
    // measured slower than sequential launches); the graph removes the launch
    // gaps, and a process with an overlapped schedule keeps its own second
    // stream inside the chain
    cudaGraph_t graph = nullptr;
    if ((e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamBeginCapture");
    int lrc = TESS_OK;
    for (int i = 0; i < n_proc && lrc == TESS_OK; ++i) {
      const tess::OverlapRes *ov = (prs[i].pipeline && prs[i].pl.overlap) ? &ctx->ovl[1 + i] : nullptr;
      lrc = launch_prepared(prs[i], ctx->cap_stream, nullptr, ov);
    }
    const cudaError_t ee = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (lrc != TESS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return lrc;
    }
    if (e == cudaSuccess) e = ee;
    if (e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(e, "graph capture");
    }
    if (ctx->graph_exec) {
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
    e = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->graph_exec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    ctx->graph_key = key;
  }
  if ((e = cudaGraphLaunch(ctx->graph_exec, (cudaStream_t)stream)) != cudaSuccess)
    return cuda_fail(e, "cudaGraphLaunch");
  return ok();
}

int tess_set_chunk_bytes(tess_ctx *ctx, size_t bytes) {
  if (!ctx) return fail(TESS_E_INVALID, "ctx is NULL");
  if (bytes != 0 && bytes < ((size_t)1 << 20))
    return fail(TESS_E_INVALID, "chunk size %zu bytes is below 1 MiB", bytes);
  std::lock_guard<std::mutex> lock(ctx->plan_mu);
  ctx->chunk_bytes = bytes;
  ctx->graph_key.clear();  // the batched graph's pipelines were planned with the old size
  return ok();
}

int tess_select_variant(tess_ctx *ctx, const tess_process *proc, int form, int schedule) {
  if (!ctx || !proc) return fail(TESS_E_INVALID, "NULL argument");
  int rc = check_process(proc);
  if (rc) return rc;
  if (form < -1 || form >= tess::K2_NFORMS) return fail(TESS_E_INVALID, "form out of range");
  if (schedule < -1 || schedule >= tess::SCHED_N) return fail(TESS_E_INVALID, "schedule out of range");
  const int pi = variant_slot(proc);
  ctx->form[pi][proc->n_gluons] = form;
  ctx->sched[pi][proc->n_gluons] = schedule;
  return ok();
}

int tess_plan_info(const tess_ctx *ctx, const tess_process *proc, uint64_t n_events, int *info) {
  if (!ctx || !proc || !info) return fail(TESS_E_INVALID, "NULL argument");
  int rc = check_process(proc);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if (!uses_pipeline(proc)) {
    info[0] = -1;
    info[1] = tess::SCHED_SERIAL;
    info[2] = 1;
    info[3] = grid_for(ctx, proc, n_events);
    return ok();
  }
  tess::PipePlan pl;
  if ((rc = pipeline_plan(ctx, proc, n_events, &pl))) return rc;
  info[0] = pl.form;
  // the schedule in effect: an overlapped one runs serially on a single chunk,
  // the deferred-histogram one serially where it does not apply
  if (pl.sched == tess::SCHED_SERIAL_HIST)
    info[1] = pl.defer_hist ? tess::SCHED_SERIAL_HIST : tess::SCHED_SERIAL;
  else
    info[1] = pl.overlap || pl.sched == tess::SCHED_SERIAL || pl.sched == tess::SCHED_SERIAL_TILES
                  ? pl.sched
                  : (pl.sched == tess::SCHED_OVERLAP ? tess::SCHED_SERIAL : tess::SCHED_SERIAL_TILES);
  info[2] = pl.chunks;
  info[3] = pl.grid;
  return ok();
}

constexpr int kTuneReps = 5;  // timed runs per candidate (median)

static int autotune(tess_ctx *ctx, const tess_process *proc, uint64_t probe_events, const tess_outputs &out,
                    void *workspace, size_t workspace_bytes, void *stream, int *form_out);

int tess_autotune(tess_ctx *ctx, const tess_process *proc, uint64_t probe_events, double *acc_scratch,
                  void *workspace, size_t workspace_bytes, void *stream, int *form_out) {
  if (!ctx || !proc || !acc_scratch || !form_out) return fail(TESS_E_INVALID, "NULL argument");
  tess_outputs out;
  memset(&out, 0, sizeof out);
  out.acc = acc_scratch;
  out.hist = acc_scratch;  // never written: no fold
  return autotune(ctx, proc, probe_events, out, workspace, workspace_bytes, stream, form_out);
}

int tess_autotune_outputs(tess_ctx *ctx, const tess_process *proc, uint64_t probe_events,
                          const tess_outputs *out, void *workspace, size_t workspace_bytes, void *stream,
                          int *form_out) {
  if (!ctx || !proc || !out || !out->acc || !form_out) return fail(TESS_E_INVALID, "NULL argument");
  tess_outputs o = *out;
  if (!o.hist) o.hist = o.acc;  // never written: no fold
  return autotune(ctx, proc, probe_events, o, workspace, workspace_bytes, stream, form_out);
}

static int autotune(tess_ctx *ctx, const tess_process *proc, uint64_t probe_events, const tess_outputs &out,
                    void *workspace, size_t workspace_bytes, void *stream, int *form_out) {
  int rc = check_process(proc);
  if (rc) return rc;
  if (probe_events == 0) return fail(TESS_E_INVALID, "probe_events must be > 0");
  const int pi = variant_slot(proc);
  const int n = proc->n_gluons;
  if (!uses_pipeline(proc)) {  // the exact-sum mode has a single kernel
    *form_out = -1;
    return ok();
  }
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  // timed with the process's own histogram settings (the epilogue cost
  // differs between variants); the runs stop before the final fold, so
  // nothing is written through `out` beyond the per-event outputs it names
  const tess_process pp = *proc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return cuda_fail(e, "cudaEventCreate");
  }
  const int saved = ctx->form[pi][n], saved_sched = ctx->sched[pi][n];
  int best = -1, best_sched = 0;
  float best_ms = 0.f;
  for (int f = 0; f < tess::K2_NFORMS && !rc; ++f) {
    for (int o = 0; o < tess::SCHED_N && !rc; ++o) {
      tess::PipePlan pl;
      if ((rc = plan_with_form(ctx, &pp, probe_events, f, o, &pl))) break;
      if (pl.form != f) continue;  // not built for (precision, n)
      const bool wants_overlap = o == tess::SCHED_OVERLAP || o == tess::SCHED_OVERLAP_TILES;
      if (wants_overlap && !pl.overlap) continue;  // a single chunk: nothing to overlap
      if (o == tess::SCHED_SERIAL_HIST && !pl.defer_hist) continue;  // the serial schedule again
      ctx->form[pi][n] = f;
      ctx->sched[pi][n] = o;
      Prepared pr;
      if ((rc = prepare(ctx, &pp, 1, 0, probe_events, &out, workspace, workspace_bytes, &pr))) break;
      tess::OverlapRes *ov = nullptr;
      if (pl.overlap && (rc = overlap_res(ctx, 0, &ov))) break;
      if ((rc = launch_prepared(pr, s, nullptr, ov, false))) break;  // warm-up
      float t[kTuneReps];
      for (int r = 0; r < kTuneReps && !rc; ++r) {
        cudaEventRecord(a, s);
        if ((rc = launch_prepared(pr, s, nullptr, ov, false))) break;
        cudaEventRecord(b, s);
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
          rc = cuda_fail(e, "autotune timing");
          break;
        }
        t[r] = 0.f;
        cudaEventElapsedTime(&t[r], a, b);
      }
      if (rc) break;
      std::sort(t, t + kTuneReps);
      const float ms = t[kTuneReps / 2];  // median
      if (best < 0 || ms < best_ms) {
        best = f;
        best_sched = o;
        best_ms = ms;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) {
    ctx->form[pi][n] = saved;
    ctx->sched[pi][n] = saved_sched;
    return rc;
  }
  ctx->sched[pi][n] = best_sched;
  ctx->form[pi][n] = best;
  *form_out = best;
  return ok();
}

int tess_draws(tess_ctx *ctx, int n, uint64_t seed, uint64_t first_event, uint64_t n_events, double *u,
               uint32_t *hel, uint8_t *order, void *stream) {
  if (!ctx) return fail(TESS_E_INVALID, "ctx is NULL");
  if (n < TESS_MIN_N || n > TESS_MAX_N) return fail(TESS_E_UNSUPPORTED, "n = %d outside %d..%d", n, TESS_MIN_N, TESS_MAX_N);
  if (n_events == 0) return ok();
  if (!u || !hel || !order) return fail(TESS_E_INVALID, "u, hel and order must not be NULL");
  if (n_events > (uint64_t)INT32_MAX * 128ull || n_events > (UINT64_MAX - first_event))
    return fail(TESS_E_INVALID, "event range too large for one call");
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  int rc;
  if ((rc = check_device_ptr(u, ctx->device, "u")) || (rc = check_device_ptr(hel, ctx->device, "hel")) ||
      (rc = check_device_ptr(order, ctx->device, "order")))
    return rc;
  tess::EventParams P;
  memset(&P, 0, sizeof P);
  P.seed = seed;
  P.first_event = first_event;
  P.n_events = n_events;
  tess::philox_round_keys(seed, P.rk);
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = n <= 8 ? tess::launch_draws_a(n, P, u, hel, order, s)
                               : (n <= 10 ? tess::launch_draws_b(n, P, u, hel, order, s)
                                          : tess::launch_draws_c(n, P, u, hel, order, s));
  if (e != cudaSuccess) return cuda_fail(e, "draws kernel launch");
  return ok();
}

int tess_gradients_workspace_size(const tess_ctx *ctx, const tess_process *proc, uint64_t n_events, size_t *bytes) {
  if (!ctx || !bytes) return fail(TESS_E_INVALID, "ctx and bytes must not be NULL");
  int rc = check_process(proc);
  if (rc) return rc;
  const int n = proc->n_gluons;
  if (proc->precision == TESS_FP64) {
    *bytes = 0;
  } else {
    const size_t cb = ctx->chunk_bytes;
    *bytes = n <= 8 ? tess::grad_workspace_a(n, n_events, cb)
                    : (n <= 10 ? tess::grad_workspace_b(n, n_events, cb) : tess::grad_workspace_c(n, n_events, cb));
  }
  return ok();
}

int tess_gradients(tess_ctx *ctx, const tess_process *proc, uint64_t n_events, const double *u, const uint32_t *hel,
                   const uint8_t *order, const double *dL_dw, double *w, double *dw_du, double *dw_dk,
                   double *dw_dlnmu, void *workspace, size_t workspace_bytes, void *stream) {
  if (!ctx) return fail(TESS_E_INVALID, "ctx is NULL");
  int rc = check_process(proc);
  if (rc) return rc;
  if (proc->helicity_mode != TESS_HEL_SAMPLE || proc->flags != 0)
    return fail(TESS_E_UNSUPPORTED,
                "gradients are built for sampled helicity and ordering (TESS_HEL_SAMPLE, no TESS_FLAG_CUT_FIRST)");
  if (n_events == 0) return ok();
  if (!u || !hel || !order) return fail(TESS_E_INVALID, "u, hel and order must not be NULL");
  if (n_events > (uint64_t)INT32_MAX * 128ull) return fail(TESS_E_INVALID, "n_events too large for one call");
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  const void *ptrs[] = {u, hel, order, dL_dw, w, dw_du, dw_dk, dw_dlnmu};
  const char *names[] = {"u", "hel", "order", "dL_dw", "w", "dw_du", "dw_dk", "dw_dlnmu"};
  for (int i = 0; i < 8; ++i)
    if ((rc = check_device_ptr(ptrs[i], ctx->device, names[i]))) return rc;
  tess::GradParams G;
  memset(&G, 0, sizeof G);
  tess_outputs none;
  memset(&none, 0, sizeof none);
  fill_params(proc, 0, 0, n_events, &none, &G.P);
  G.u = u;
  G.hel = hel;
  G.order = order;
  G.dL_dw = dL_dw;
  G.w = w;
  G.dw_du = dw_du;
  G.dw_dk = dw_dk;
  G.dw_dlnmu = dw_dlnmu;
  G.n_events = n_events;
  G.chunk_bytes = ctx->chunk_bytes;
  const int n = proc->n_gluons;
  const bool fp64 = proc->precision == TESS_FP64;
  size_t need = 0;
  if ((rc = tess_gradients_workspace_size(ctx, proc, n_events, &need))) return rc;
  if (need) {
    if (!workspace || workspace_bytes < need)
      return fail(TESS_E_WORKSPACE, "gradient workspace of %zu bytes needed, %zu given", need,
                  workspace ? workspace_bytes : 0);
    if ((rc = check_device_ptr(workspace, ctx->device, "workspace"))) return rc;
    if (((uintptr_t)workspace) % 256 != 0) return fail(TESS_E_WORKSPACE, "workspace must be 256-byte aligned");
  }
  cudaStream_t s = (cudaStream_t)stream;
  tess::GradStreams gs;
  if (!fp64) {
    tess::OverlapRes *ov = nullptr;
    if ((rc = overlap_res(ctx, kGradSlot, &ov))) return rc;
    gs.aux = ov->aux;
    gs.fork = ov->fork;
    gs.join = ov->join;
    for (int b = 0; b < 2; ++b) {
      gs.g2done[b] = ov->k1done[b];
      gs.g3done[b] = ov->k2done[b];
    }
  }
  const cudaError_t e = n <= 8 ? tess::launch_grad_a(n, fp64, G, workspace, s, gs)
                               : (n <= 10 ? tess::launch_grad_b(n, fp64, G, workspace, s, gs)
                                          : tess::launch_grad_c(n, fp64, G, workspace, s, gs));
  if (e != cudaSuccess) return cuda_fail(e, "gradient kernel launch");
  return ok();
}

namespace {
int me2_or_gauge(tess_ctx *ctx, int n, int precision, uint64_t n_events, const double *k, const uint8_t *order,
                 const uint32_t *hel, double *me2, void *stream, bool gauge) {
  if (!ctx) return fail(TESS_E_INVALID, "ctx is NULL");
  if (n < TESS_MIN_N || n > TESS_MAX_N) return fail(TESS_E_UNSUPPORTED, "n = %d outside %d..%d", n, TESS_MIN_N, TESS_MAX_N);
  if (precision != TESS_FP64 && precision != TESS_FP32_CURRENTS && precision != TESS_FP32_DS)
    return fail(TESS_E_INVALID, "bad precision %d", precision);
  if (n_events == 0) return ok();
  if (!k || !order || !hel || !me2) return fail(TESS_E_INVALID, "k, order, hel and me2 must not be NULL");
  if (n_events > (uint64_t)INT32_MAX * 128ull) return fail(TESS_E_INVALID, "n_events too large for one call");
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  int rc;
  if ((rc = check_device_ptr(k, ctx->device, "k")) || (rc = check_device_ptr(order, ctx->device, "order")) ||
      (rc = check_device_ptr(hel, ctx->device, "hel")) || (rc = check_device_ptr(me2, ctx->device, "me2")))
    return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = precision == TESS_FP64 ? tess::launch_me2_f64(n, n_events, k, order, hel, me2, s, gauge)
                                               : tess::launch_me2_f32(n, n_events, k, order, hel, me2, s, gauge);
  if (e != cudaSuccess) return cuda_fail(e, gauge ? "gauge kernel launch" : "me2 kernel launch");
  return ok();
}
}  // namespace

int tess_me2(tess_ctx *ctx, int n, int precision, uint64_t n_events, const double *k, const uint8_t *order,
             const uint32_t *hel, double *me2, void *stream) {
  return me2_or_gauge(ctx, n, precision, n_events, k, order, hel, me2, stream, false);
}

int tess_gauge_ratio(tess_ctx *ctx, int n, int precision, uint64_t n_events, const double *k, const uint8_t *order,
                     const uint32_t *hel, double *ratio, void *stream) {
  return me2_or_gauge(ctx, n, precision, n_events, k, order, hel, ratio, stream, true);
}

int tess_result(tess_ctx *ctx, const double *acc, double *out, void *stream) {
  if (!ctx || !acc || !out) return fail(TESS_E_INVALID, "ctx, acc and out must not be NULL");
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  int rc = check_device_ptr(acc, ctx->device, "acc");
  if (rc) return rc;
  double h[TESS_ACC_LEN];
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "copy of acc");
  const double n = h[3];
  const double sw = h[0] + h[4], sw2 = h[1] + h[5];
  const double mean = n > 0 ? sw / n : 0.0;
  const double var = n > 1 ? (sw2 / n - mean * mean) / (n - 1.0) : 0.0;
  out[0] = mean;
  out[1] = std::sqrt(var > 0 ? var : 0.0);
  out[2] = h[2];
  out[3] = n;
  if (h[7] > 0)
    return fail(TESS_E_CUDA, "%.0f amplitude blocks timed out waiting for a staged input copy (sums incomplete)",
                h[7]);
  if (h[6] > 0) return fail(TESS_E_NUMERICAL, "%.0f events had non-finite weights (counted as 0)", h[6]);
  return ok();
}

int tess_weights(tess_ctx *ctx, const tess_outputs *dev, uint64_t n_events, double *host_weight, uint8_t *host_pass,
                 double *host_me2, void *stream) {
  if (!ctx || !dev) return fail(TESS_E_INVALID, "ctx and dev must not be NULL");
  if (n_events == 0) return ok();
  if ((host_weight && !dev->weight) || (host_pass && !dev->pass) || (host_me2 && !dev->me2))
    return fail(TESS_E_INVALID, "a requested host output has no device array");
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (host_weight && e == cudaSuccess)
    e = cudaMemcpyAsync(host_weight, dev->weight, n_events * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (host_pass && e == cudaSuccess)
    e = cudaMemcpyAsync(host_pass, dev->pass, n_events, cudaMemcpyDeviceToHost, s);
  if (host_me2 && e == cudaSuccess)
    e = cudaMemcpyAsync(host_me2, dev->me2, n_events * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "copy of per-event outputs");
  return ok();
}

int tess_histograms(tess_ctx *ctx, const tess_process *proc, const double *hist, double *host_sumw,
                    double *host_sumw2, void *stream) {
  if (!ctx || !hist || !host_sumw || !host_sumw2) return fail(TESS_E_INVALID, "NULL argument");
  int rc = check_process(proc);
  if (rc) return rc;
  if (proc->hist_bins <= 0) return fail(TESS_E_INVALID, "process has no histogram");
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if ((rc = check_device_ptr(hist, ctx->device, "hist"))) return rc;
  const int nb2 = proc->hist_bins + 2;
  double *h = new double[4 * nb2];
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h, hist, 4 * nb2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete[] h;
    return cuda_fail(e, "copy of hist");
  }
  for (int b = 0; b < nb2; ++b) {
    host_sumw[b] = h[b] + h[2 * nb2 + b];
    host_sumw2[b] = h[nb2 + b] + h[3 * nb2 + b];
  }
  delete[] h;
  return ok();
}

}  // extern "C"

// ===========================================================================
// Batched mixed multiplicities in one persistent launch (tess_persist.cuh).
// ===========================================================================
namespace {

// Workspace: the work counter, then each process's tile rows of partial sums.
int persistent_layout(int n_proc, const tess_process *procs, const uint64_t *n_events, size_t *offsets,
                      size_t *total) {
  if (n_proc < 1 || n_proc > tess::kPersistMaxProc)
    return fail(TESS_E_INVALID, "n_proc must be 1..%d", tess::kPersistMaxProc);
  size_t off = 256;  // the counter
  uint64_t items = 0;
  for (int i = 0; i < n_proc; ++i) {
    int rc = check_process(&procs[i]);
    if (rc) return rc;
    const tess_process &p = procs[i];
    if (p.precision != TESS_FP32_DS || p.helicity_mode != TESS_HEL_SAMPLE || p.flags != 0)
      return fail(TESS_E_UNSUPPORTED,
                  "persistent batched form: process %d must be TESS_FP32_DS, TESS_HEL_SAMPLE, no flags", i);
    const uint64_t tiles = (n_events[i] + tess::kBlock - 1) / tess::kBlock;
    items += tiles;
    if (items > (uint64_t)INT32_MAX) return fail(TESS_E_INVALID, "too many events for one persistent launch");
    offsets[i] = off;
    off = align256(off + (size_t)tiles * tess::partial_stride(p.hist_bins) * sizeof(double));
  }
  *total = off;
  return TESS_OK;
}

}  // namespace

extern "C" int tess_workspace_size_persistent(const tess_ctx *ctx, int n_proc, const tess_process *procs,
                                              const uint64_t *n_events, size_t *bytes) {
  if (!ctx || !procs || !n_events || !bytes) return fail(TESS_E_INVALID, "NULL argument");
  size_t offs[tess::kPersistMaxProc];
  const int rc = persistent_layout(n_proc, procs, n_events, offs, bytes);
  return rc ? rc : ok();
}

extern "C" int tess_generate_persistent(tess_ctx *ctx, int n_proc, const tess_process *procs, const uint64_t *seeds,
                                        const uint64_t *first_events, const uint64_t *n_events,
                                        const tess_outputs *outs, void *workspace, size_t workspace_bytes,
                                        void *stream) {
  if (!ctx || !procs || !seeds || !first_events || !n_events || !outs) return fail(TESS_E_INVALID, "NULL argument");
  size_t offs[tess::kPersistMaxProc], need = 0;
  int rc = persistent_layout(n_proc, procs, n_events, offs, &need);
  if (rc) return rc;
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if ((rc = check_device_ptr(workspace, ctx->device, "workspace"))) return rc;
  if (!workspace || workspace_bytes < need)
    return fail(TESS_E_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, workspace ? workspace_bytes : 0);
  if (((uintptr_t)workspace) % 256 != 0) return fail(TESS_E_WORKSPACE, "workspace must be 256-byte aligned");
  // processes from the most gluons down: the longest tiles are handed out first
  int order[tess::kPersistMaxProc];
  for (int i = 0; i < n_proc; ++i) order[i] = i;
  std::stable_sort(order, order + n_proc, [&](int a, int b) { return procs[a].n_gluons > procs[b].n_gluons; });
  tess::PersistParams Q;
  memset(&Q, 0, sizeof Q);
  tess::PersistFold F;
  memset(&F, 0, sizeof F);
  Q.counter = (int *)workspace;
  int items = 0, nmax = 4, max_bins = 0;
  for (int j = 0; j < n_proc; ++j) {
    const int i = order[j];
    const tess_outputs *out = &outs[i];
    if (!out->acc) return fail(TESS_E_INVALID, "outputs[%d].acc must not be NULL", i);
    if (procs[i].hist_bins > 0 && !out->hist) return fail(TESS_E_INVALID, "process %d: hist_bins > 0 needs hist", i);
    if (n_events[i] > (UINT64_MAX - first_events[i])) return fail(TESS_E_INVALID, "event range overflows 64 bits");
    if ((rc = check_device_ptr(out->acc, ctx->device, "acc"))) return rc;
    if ((rc = check_device_ptr(out->hist, ctx->device, "hist"))) return rc;
    tess_outputs o = *out;
    void *dev = nullptr;
    if ((rc = output_ptr(out->weight, ctx->device, "weight", &dev))) return rc;
    o.weight = (double *)dev;
    if ((rc = output_ptr(out->me2, ctx->device, "me2", &dev))) return rc;
    o.me2 = (double *)dev;
    if ((rc = output_ptr(out->pass, ctx->device, "pass", &dev))) return rc;
    o.pass = (uint8_t *)dev;
    if ((rc = output_ptr(out->ht, ctx->device, "ht", &dev))) return rc;
    o.ht = (double *)dev;
    if ((rc = output_ptr(out->ptlead, ctx->device, "ptlead", &dev))) return rc;
    o.ptlead = (double *)dev;
    if ((rc = output_ptr(out->rmin, ctx->device, "rmin", &dev))) return rc;
    o.rmin = (double *)dev;
    tess::PersistProc &pp = Q.proc[j];
    fill_params(&procs[i], seeds[i], first_events[i], n_events[i], &o, &pp.P);
    pp.n = procs[i].n_gluons;
    pp.tiles = (int)((n_events[i] + tess::kBlock - 1) / tess::kBlock);
    pp.first_item = items;
    pp.tile_sums = (double *)((char *)workspace + offs[i]);
    items += pp.tiles;
    nmax = std::max(nmax, pp.n);
    max_bins = std::max(max_bins, procs[i].hist_bins);
    F.tile_sums[j] = pp.tile_sums;
    F.acc[j] = out->acc;
    F.hist[j] = out->hist;
    F.tiles[j] = pp.tiles;
    F.hist_bins[j] = procs[i].hist_bins;
    F.n_events[j] = n_events[i];
  }
  Q.nproc = n_proc;
  Q.items = items;
  if (items == 0) return ok();
  const cudaError_t e =
      tess::persist_launch(Q, F, nmax, max_bins, ctx->sm_count, (cudaStream_t)stream, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "persistent launch");
  return ok();
}

extern "C" int tess_peak_flops(tess_ctx *ctx, int kind, int reps, double *tflops, void *stream) {
  if (!ctx || !tflops) return fail(TESS_E_INVALID, "ctx and tflops must not be NULL");
  if (kind != TESS_PEAK_FP32 && kind != TESS_PEAK_FP32X2 && kind != TESS_PEAK_FP64)
    return fail(TESS_E_INVALID, "kind = %d is not a TESS_PEAK_* value", kind);
  if (reps < 1 || reps > 1000) return fail(TESS_E_INVALID, "reps = %d outside 1..1000", reps);
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  float ms = 0.f;
  double flop = 0.0;
  const cudaError_t e = tess::peak_probe(kind, ctx->sm_count, reps, (cudaStream_t)stream, &ms, &flop);
  if (e != cudaSuccess) return cuda_fail(e, "peak probe");
  *tflops = flop / (ms * 1e-3) / 1e12;
  return ok();
}

// ===========================================================================
// Allocation-free generation (tess_generate_noalloc).
//
// Callers that cannot call cudaMalloc or hand the library a workspace -- for
// example a host program whose memory manager reserves the whole device at
// start-up and forbids any other allocation, or a latency-critical loop that
// cannot afford an allocation's implicit device synchronisation -- use this
// variant.  It runs the fused event kernel with its per-block partial sums
// in the fixed file-scope array below instead of a caller workspace.
// The array (TESS_NOALLOC_SCRATCH_BYTES) lives on every GPU that loads this
// library until the process exits.  In host code its name is only a host-side
// stand-in, so its device address is looked up once per device (with that
// device current) on the first call and cached.
// ===========================================================================
static __device__ __align__(256) double g_noalloc_partials[TESS_NOALLOC_SCRATCH_BYTES / sizeof(double)];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of g_noalloc_partials on `device`, which must be current.
int noalloc_scratch(int device, double **out) {
  if (device < 0 || device >= kNoallocMaxDevices) return fail(TESS_E_INVALID, "device index %d too large", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_ptr[device] = (double *)p;
  }
  *out = g_noalloc_ptr[device];
  return TESS_OK;
}

}  // namespace

extern "C" int tess_generate_noalloc(tess_ctx *ctx, const tess_process *proc, uint64_t seed, uint64_t first_event,
                                     uint64_t n_events, const tess_outputs *out, void *stream) {
  if (!ctx) return fail(TESS_E_INVALID, "ctx is NULL");
  int rc = check_process(proc);
  if (rc) return rc;
  if (proc->helicity_mode == TESS_POL_RANDOM || proc->flags != 0)
    return fail(TESS_E_UNSUPPORTED,
                "tess_generate_noalloc is built for TESS_HEL_SUM and TESS_HEL_SAMPLE without TESS_FLAG_CUT_FIRST");
  // Sampled events at the FP32 precisions run tess_generate's chunked
  // two-kernel pipeline (FP32 / double-float kinematics), whose chunk buffer
  // needs a workspace; the fused event kernel used here has FP64 kinematics,
  // so it would not reproduce those results.  Only FP64 is offered there.
  if (proc->helicity_mode == TESS_HEL_SAMPLE && proc->precision != TESS_FP64)
    return fail(TESS_E_UNSUPPORTED,
                "tess_generate_noalloc: sampled helicities are built for TESS_FP64 only (the FP32 forms need "
                "tess_generate's workspace)");
  if (proc->hist_bins > TESS_NOALLOC_MAX_BINS)
    return fail(TESS_E_INVALID, "tess_generate_noalloc supports at most %d histogram bins (%d requested)",
                TESS_NOALLOC_MAX_BINS, proc->hist_bins);
  if (!out || !out->acc) return fail(TESS_E_INVALID, "outputs and outputs->acc must not be NULL");
  if (proc->hist_bins > 0 && !out->hist) return fail(TESS_E_INVALID, "hist_bins > 0 needs outputs->hist");
  if (n_events > (UINT64_MAX - first_event)) return fail(TESS_E_INVALID, "event range overflows 64 bits");
  if (n_events == 0) return ok();
  DeviceGuard g(ctx->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  if ((rc = check_device_ptr(out->acc, ctx->device, "acc"))) return rc;
  if ((rc = check_device_ptr(out->hist, ctx->device, "hist"))) return rc;
  // per-event arrays: device memory or mapped pinned host memory, as tess_generate
  tess_outputs o = *out;
  void *dev = nullptr;
  if ((rc = output_ptr(out->weight, ctx->device, "weight", &dev))) return rc;
  o.weight = (double *)dev;
  if ((rc = output_ptr(out->me2, ctx->device, "me2", &dev))) return rc;
  o.me2 = (double *)dev;
  if ((rc = output_ptr(out->pass, ctx->device, "pass", &dev))) return rc;
  o.pass = (uint8_t *)dev;
  if ((rc = output_ptr(out->ht, ctx->device, "ht", &dev))) return rc;
  o.ht = (double *)dev;
  if ((rc = output_ptr(out->ptlead, ctx->device, "ptlead", &dev))) return rc;
  o.ptlead = (double *)dev;
  if ((rc = output_ptr(out->rmin, ctx->device, "rmin", &dev))) return rc;
  o.rmin = (double *)dev;
  double *partials = nullptr;
  if ((rc = noalloc_scratch(ctx->device, &partials))) return rc;

  // Rows of partial sums that fit in the fixed array; every row the finalize
  // step reads is written by this call's event kernel, so nothing in the
  // array needs clearing between calls.
  const int stride = tess::partial_stride(proc->hist_bins);
  const int max_rows = (int)(TESS_NOALLOC_SCRATCH_BYTES / sizeof(double)) / stride;
  int grid = grid_for(ctx, proc, n_events);
  if (grid > max_rows) grid = max_rows;

  const int n = proc->n_gluons;
  const bool sum = proc->helicity_mode == TESS_HEL_SUM;
  tess::EventParams P;
  fill_params(proc, seed, first_event, n_events, &o, &P);

  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = proc->precision == TESS_FP64 ? tess::launch_generate_f64(n, sum, P, partials, grid, s)
                                               : tess::launch_generate_f32(n, sum, P, partials, grid, s);
  if (e != cudaSuccess) return cuda_fail(e, "event kernel launch");
  tess::finalize_kernel<<<1, 256, 0, s>>>(partials, grid, proc->hist_bins, n_events, out->acc, out->hist);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel launch");
  return ok();
}
