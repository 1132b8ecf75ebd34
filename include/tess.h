/*
 * tess.h -- C ABI of the GB300 (sm_103a) leading-order, leading-colour
 * multi-gluon event generator ("TESS": Giele, Stavenga, Winter,
 * "Thread-Scalable Evaluation of Multi-Jet Observables", arXiv:1002.3446).
 *
 * Every step of an event runs in this library's CUDA kernels: counter-based
 * random numbers -> Rambo phase space -> parton luminosity, alpha_s, jet cuts
 * and observables -> helicity polarisation vectors -> Berends-Giele
 * colour-ordered amplitude -> event weight -> cross-section and histogram
 * accumulation (Sec. 3 of the paper, Fig. 1 stages).
 *
 * Conventions for every entry point
 *   - Return value: TESS_OK (0) on success, a negative TESS_E_* code on
 *     failure; tess_last_error() then returns a message (thread-local).
 *   - Memory: the library allocates no device memory in tess_generate,
 *     tess_me2, tess_generate_batched or tess_autotune.  The caller owns every buffer; device
 *     pointers are plain CUDA device addresses (e.g. from cudaMalloc or a
 *     torch tensor) on the context's device.  Host pointers are marked "host".
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Generating calls are asynchronous on that stream;
 *     calls that return host data synchronise it.
 *   - Inputs are never retained after a call returns.
 *   - n is the TOTAL number of gluons (the paper's n): gg -> (n-2) g.
 */
#ifndef TESS_H
#define TESS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TESS_OK 0
#define TESS_E_INVALID (-1)     /* bad argument (size, pointer, value)          */
#define TESS_E_UNSUPPORTED (-2) /* n or mode combination not built              */
#define TESS_E_CUDA (-3)        /* a CUDA runtime call or launch failed         */
#define TESS_E_WORKSPACE (-4)   /* workspace missing or too small               */
#define TESS_E_NUMERICAL (-5)   /* non-finite weights were produced             */

#define TESS_MIN_N 4
#define TESS_MAX_N 12
#define TESS_MAX_BINS 1024
#define TESS_ACC_LEN 8

/* precision */
#define TESS_FP64 0          /* every step in FP64                                 */
#define TESS_FP32_CURRENTS 1 /* Berends-Giele currents, vertex contractions, Rambo
                                seeds, cuts and observables in FP32; Rambo's boost
                                and rescale, the polarisation Gram products and
                                the accumulation in native FP64                   */
#define TESS_FP32_DS 2       /* as TESS_FP32_CURRENTS, but the Rambo boost/rescale
                                in double-float (two-float, ~44-bit) arithmetic
                                on the FP32 pipe instead of native FP64, which
                                runs at 1/64 of the FP32 rate on GB300, and the
                                polarisation basis in FP32 from the rounded
                                momenta; weights and accumulation stay FP64     */
/* helicity_mode */
#define TESS_HEL_SUM 0    /* exact sum over 2^n helicities and (n-1)! orderings (n <= 5) */
#define TESS_HEL_SAMPLE 1 /* one helicity configuration and colour ordering per event,
                             sampled uniformly; estimator 2^n (n-1)! |A|^2          */
#define TESS_POL_RANDOM 2 /* the paper's choice (Sec. 3): every polarisation vector a
                             random unit vector orthogonal to the gluon momentum,
                             eps = cos(phi) e1 + sin(phi) e2 with phi = 2 pi u from n
                             more draws per event (after the colour-ordering draws),
                             so the currents are real; one sampled colour ordering;
                             estimator 2^n (n-1)! |A|^2 (unbiased for the helicity
                             sum).  Not for tess_gradients or tess_generate_noalloc. */
/* flags */
#define TESS_FLAG_CUT_FIRST 1 /* cut-first generation (FP32 forms, sampled modes): the kinematics
                                 kernel compacts the events that pass the cuts, and the amplitude
                                 kernel evaluates only those (Sec. 3 notes that events failing the
                                 cuts need no matrix element).  Failing events get weight 0 and
                                 me2 0 (not evaluated); every other output is as without the flag.
                                 Not for TESS_FP64, TESS_HEL_SUM, tess_gradients or
                                 tess_generate_noalloc. */
#define TESS_FLAG_PDF_GRID 2 /* the paper's tabulated PDF and alpha_s (Sec. 3): x g(x) on 1025 nodes uniform
                                in the x draw u (ln x = u ln x_min) and alpha_s on 513 nodes uniform in
                                ln mu^2 over [2 ln(mu_r_factor m pT_min), 2 ln(mu_r_factor sqrt(S))], each
                                node the function rounded to FP32, read by linear interpolation in FP32
                                (s = position in node units, i = min(floor(s), last segment), t = s - i,
                                value = fma(t, g[i+1] - g[i], g[i])).  Tables built per call in the
                                workspace.  FP32 forms with sampled events only. */
/* hist_observable */
#define TESS_OBS_PTLEAD 0
#define TESS_OBS_HT 1
#define TESS_OBS_RMIN 2

/* Process and run parameters (Sec. 4 workload: sqrt(S) = 14 TeV, jet cuts
 * pT > pt_min, |eta| < eta_max, Delta R > dr_min).  Units: GeV. */
typedef struct tess_process {
  int32_t n_gluons;        /* total gluons, TESS_MIN_N..TESS_MAX_N            */
  int32_t precision;       /* TESS_FP64, TESS_FP32_CURRENTS or TESS_FP32_DS   */
  int32_t helicity_mode;   /* TESS_HEL_SUM, TESS_HEL_SAMPLE or TESS_POL_RANDOM */
  int32_t hist_observable; /* TESS_OBS_*                                      */
  int32_t hist_bins;       /* 0 = no histogram, else 1..TESS_MAX_BINS         */
  int32_t nf;              /* flavours in the one-loop running of alpha_s     */
  double sqrt_s;           /* hadronic centre-of-mass energy (> 0)            */
  double pt_min;           /* > 0                                             */
  double eta_max;          /* > 0                                             */
  double dr_min;           /* >= 0                                            */
  double alphas_mz;        /* alpha_s(M_Z) (> 0)                              */
  double mz;               /* M_Z (> 0)                                       */
  double mu_r_factor;      /* mu_R = mu_r_factor * H_T (> 0)                  */
  double hist_lo, hist_hi; /* histogram range [lo, hi), uniform bins          */
  int32_t flags;           /* 0 or TESS_FLAG_CUT_FIRST | TESS_FLAG_PDF_GRID  */
  int32_t reserved;        /* 0                                               */
} tess_process;

/* Per-call outputs (caller-owned; NULL = not requested, except acc).
 * Per-event arrays have n_events entries, indexed by event - first_event.
 *   weight  event weight in pb (0 for events failing the cuts)
 *   me2     helicity/colour estimator E of sum |A|^2 in GeV^(8-2n) (before
 *           couplings, luminosity and phase space), computed for every event
 *   pass    1 if the event passes the cuts (events are flagged, not dropped)
 *   ht, ptlead, rmin   observables (H_T, leading-jet pT, min Delta R)
 * In tess_generate and tess_generate_batched the per-event arrays may be
 * device memory or pinned host memory mapped into the device's address
 * space (cudaHostAlloc, cudaHostRegister): the kernels then store into host
 * memory directly (NVLink-C2C on Grace-Blackwell), with no separate copy;
 * other host memory is rejected with TESS_E_INVALID.  acc, hist and the
 * workspace are always device memory.
 * acc  [TESS_ACC_LEN] doubles, ACCUMULATED into (zero it before the first
 *      call): {sum w, sum w^2, n_pass, n_generated, compensation of sum w,
 *      compensation of sum w^2, n_nonfinite, n_stalled}; n_stalled counts
 *      amplitude blocks that gave up waiting (after about a second) for a
 *      staged input copy, whose remaining events are missing from the sums
 *      (tess_result then fails with TESS_E_CUDA).  Repeated calls over
 *      disjoint event ranges give the run total (checkpoint = copy of acc).
 * hist [4 * (hist_bins + 2)] doubles, accumulated into: sum w per bin, then
 *      sum w^2 per bin, then their two compensation terms.  Bin 0 is the
 *      underflow, 1..hist_bins the uniform bins, hist_bins+1 the overflow.
 *      Only events that pass the cuts are filled.                         */
typedef struct tess_outputs {
  double *weight;
  double *me2;
  uint8_t *pass;
  double *ht;
  double *ptlead;
  double *rmin;
  double *acc;
  double *hist;
} tess_outputs;

typedef struct tess_ctx tess_ctx;

/* Library version string, e.g. "tess-gb300 0.1".  (Library plumbing: no
 * counterpart in the paper.) */
const char *tess_version(void);

/* Thread-local message for the last failing call on this thread ("" if none).
 * (Library plumbing: no counterpart in the paper.) */
const char *tess_last_error(void);

/* Create a context on CUDA device `device` (reads its properties; allocates
 * no device memory).  Paper: the initialization phase of Sec. 3 (start-up
 * before the Fig. 1 stages), done once here instead of per sweep.  *ctx receives the handle; free it with tess_destroy.
 * A context holds the tuned variant table, the cached graph of
 * tess_generate_batched, the stage timers and the streams of the overlapped
 * schedules: calls on one context from several host threads must be
 * serialised by the caller (contexts are independent of each other; one per
 * thread or per device is the simple rule). */
int tess_init(int device, tess_ctx **ctx);
void tess_destroy(tess_ctx *ctx);

/* Bytes of device workspace tess_generate needs for this process and event
 * count: per-block partial sums of the accumulation and, for sampled
 * helicities, one chunk of per-event amplitude inputs (tess_set_chunk_bytes;
 * two under the overlapped schedules).  0 is never
 * returned for a valid process.  Paper: the events in flight of one sweep
 * (Sec. 2, the number of events per multiprocessor and Table 2); here a
 * chunk plays the sweep's role.  Host-only, no
 * errors beyond TESS_E_INVALID / TESS_E_UNSUPPORTED for a bad process. */
int tess_workspace_size(const tess_ctx *ctx, const tess_process *proc, uint64_t n_events, size_t *bytes);

/* Number of kernel launches one tess_generate call with these arguments
 * makes (for launch accounting and graph sizing).  Paper: the kernel
 * start-up cost of Sec. 3's initialization phase, which matters when the
 * kernel time is small (n = 4). */
int tess_kernel_launches(const tess_ctx *ctx, const tess_process *proc, uint64_t n_events, int *launches);

/* Generate events [first_event, first_event + n_events) of the counter-based
 * stream `seed` (Sec. 3 stages: phase space, phase-space weight, matrix-
 * element weight, epilogue; cross-section formula at the end of Sec. 3).
 * Writes the requested per-event outputs and accumulates acc/hist.
 * workspace: device buffer of at least tess_workspace_size() bytes, 256-byte
 * aligned, not shared with a concurrent call.  n_events may be 0 (no-op).
 * Errors: TESS_E_INVALID (bad process/pointers), TESS_E_UNSUPPORTED (n out of
 * range, HEL_SUM with n > 5), TESS_E_WORKSPACE, TESS_E_CUDA (launch).     */
int tess_generate(tess_ctx *ctx, const tess_process *proc, uint64_t seed, uint64_t first_event,
                  uint64_t n_events, const tess_outputs *out, void *workspace, size_t workspace_bytes,
                  void *stream);

/* ---- Stage timing ----------------------------------------------------------------
 * Paper: the per-stage time split of Sec. 3 (Fig. 1: Rambo, phase-space
 * weight, matrix-element weight, epilogue).  With timing enabled, tess_generate records a CUDA event pair on its stream
 * around every launch it makes; tess_stage_times synchronises on them and
 * returns the summed device time (ms) and launch count per stage since the
 * previous read: [0] kinematics kernel, [1] amplitude kernel, [2] finalize,
 * [3] fused event kernel (exact-sum mode).  Events only; no device memory. */
int tess_stage_timing(tess_ctx *ctx, int enable);
int tess_stage_times(tess_ctx *ctx, double *ms /* [4] */, int *launches /* [4] */);

/* ---- Batched mixed multiplicities -------------------------------------------
 * Paper: Sec. 3's initialization phase (kernel start-up is a significant part
 * of the time when the kernel is short, as at n = 4); one launch serves
 * several multiplicities.  n_proc (1..16) processes -- typically gg -> 2..10 gluons with different
 * event counts -- in one call.  Process i generates events
 * [first_events[i], first_events[i] + n_events[i]) of stream seeds[i] into
 * outs[i] (accumulating into its acc/hist, as tess_generate).  The per-process
 * pipelines are recorded one after another as a single chain of one CUDA
 * graph (nine concurrent branches measured slower than nine plain launches,
 * 3.6e9 against 4.2e9 events/s for gg -> 2..10 gluons), captured on an
 * internal stream the first time an argument set is seen and replayed on
 * `stream` after that, so a batch is a single graph launch with no launch
 * gaps.  Capture happens inside this call; do not call it while `stream`
 * is being captured.  workspace: tess_workspace_size_batched() bytes (the
 * per-process workspaces back to back).  Errors as tess_generate. */
int tess_workspace_size_batched(const tess_ctx *ctx, int n_proc, const tess_process *procs,
                                const uint64_t *n_events, size_t *bytes);
int tess_generate_batched(tess_ctx *ctx, int n_proc, const tess_process *procs, const uint64_t *seeds,
                          const uint64_t *first_events, const uint64_t *n_events, const tess_outputs *outs,
                          void *workspace, size_t workspace_bytes, void *stream);

/* ---- Batched mixed multiplicities, one persistent launch ----------------------
 * Paper: Sec. 3's initialization phase (kernel start-up matters when the
 * kernel is short, n = 4); here every multiplicity of a batch runs in one
 * kernel launch.  Same arguments and outputs as tess_generate_batched (n_proc
 * 1..16); each process must be TESS_FP32_DS with TESS_HEL_SAMPLE and no flags
 * (else TESS_E_UNSUPPORTED).  Work items are (process, tile of 128 events),
 * handed out by one atomic counter in the workspace to resident blocks (none
 * waits on another), from the process with the most gluons down; each block
 * runs the whole event path of its tile (double-float kinematics into a
 * shared-memory tile, the register-form amplitude up to n = 8, the loop form
 * above, the epilogue) and writes the tile's partial sums to the tile's own
 * row, which a second kernel folds per process in tile order, so the sums do
 * not depend on which block took which tile.  Three stream operations (a
 * 4-byte memset of the counter, the persistent kernel, the fold); no host
 * synchronisation, no allocation, so the call can be captured in a CUDA
 * graph by the caller.  Per-event values equal tess_generate's with the same
 * precision up to the FP32 summation order of the amplitude form.
 * workspace: tess_workspace_size_persistent() bytes, device, 256-byte aligned
 * (the counter and every tile's row of partial sums); calls that overlap on
 * the GPU must not share it.  Errors as tess_generate_batched. */
int tess_workspace_size_persistent(const tess_ctx *ctx, int n_proc, const tess_process *procs,
                                   const uint64_t *n_events, size_t *bytes);
int tess_generate_persistent(tess_ctx *ctx, int n_proc, const tess_process *procs, const uint64_t *seeds,
                             const uint64_t *first_events, const uint64_t *n_events, const tess_outputs *outs,
                             void *workspace, size_t workspace_bytes, void *stream);

/* ---- Amplitude-kernel autotuner ------------------------------------------------
 * Paper: Sec. 2 chooses the running configuration (threads and events per
 * multiprocessor, Table 1 / Table 2) by measurement before implementing the
 * algorithm; this does the same per (precision, n) on the GPU at hand.
 * Times every amplitude-kernel variant built for (precision, n) of proc on
 * probe_events sampled events (one warm-up, median of five timed runs, with
 * proc's histogram settings) and makes the fastest the context's choice for
 * later calls with that (precision, polarisation kind, n) -- the kinds being
 * helicity vectors (TESS_HEL_SAMPLE) and random real vectors
 * (TESS_POL_RANDOM); the choice ignores the histogram settings, so tune with
 * the ones the calls will use.  Choose
 * probe_events to span several chunks (a few million events) so that the
 * overlapped schedules can show their gain.  Variants (one thread per event
 * unless noted): TESS_K2_REG (current table in registers), TESS_K2_ROWS32 /
 * TESS_K2_ROWS64 (current row in registers, older rows in shared memory, 32 /
 * 64 threads per block), TESS_K2_LOOP (FP64 loop form), TESS_K2_REG_HI
 * (register form compiled for more resident blocks), TESS_K2_REG_TMA (inputs
 * staged in shared memory by bulk copies), TESS_K2_REG_TMA_HI (the same for
 * more resident blocks), TESS_K2_PAIR32 / TESS_K2_PAIR64 (two threads per
 * event sharing its current table in shared memory), TESS_K2_PAIR_W (the
 * O(n^3) tensor rewrite of the four-vertex sum, Sec. 3), and for
 * TESS_POL_RANDOM only TESS_K2_REAL / TESS_K2_REAL_HI / TESS_K2_ROWS_REAL
 * (real currents), the wavefront forms TESS_K2_WAVE* (two lanes of a warp
 * per event), the warp-lanes forms TESS_K2_LANES8/16/32 and the
 * warp-specialised one-kernel form TESS_K2_FUSED (TESS_FP32_DS, n <= 6) --
 * each under every chunk schedule
 * TESS_SCHED_* below.  acc_scratch: device, TESS_ACC_LEN doubles (not
 * written: the timed runs stop before folding their sums); workspace:
 * tess_workspace_size(proc, probe_events) bytes -- that size already covers
 * every variant and schedule.  *form_out receives the chosen TESS_K2_* (-1
 * for the exact-sum mode, which has one kernel); tess_plan_info reports the
 * chosen schedule.  Per-event outputs do not depend on the choice beyond FP32
 * summation order inside the amplitude (identical in FP64); the accumulated
 * sums can differ in the last bits, since the amplitude grid sets their
 * summation order.
 *
 * Chunk schedules (events are processed in chunks of tess_set_chunk_bytes,
 * each by a kinematics kernel and an amplitude kernel; TESS_K2_FUSED runs
 * one kernel per chunk and takes the serial ones):
 *   TESS_SCHED_SERIAL         both kernels of a chunk back to back on
 *                             `stream`; amplitude grid = resident blocks
 *   TESS_SCHED_OVERLAP        kinematics of chunk c+1 on `stream` while the
 *                             amplitude kernel of chunk c runs on a second
 *                             stream owned by the context (two chunk buffers;
 *                             needs more than one chunk, else serial)
 *   TESS_SCHED_OVERLAP_TILES  overlapped, one amplitude block per tile of
 *                             events (bounded so that the blocks' partial-sum
 *                             flushes stay small next to the chunk's traffic)
 *   TESS_SCHED_SERIAL_TILES   serial, one amplitude block per tile
 *   TESS_SCHED_SERIAL_HIST    serial; with a histogram, the amplitude kernel
 *                             keeps only the sums and a third kernel per
 *                             chunk fills the histogram from the events'
 *                             weights (8 more workspace bytes per chunk
 *                             event), so that the amplitude kernel's code
 *                             keeps the instruction cache to itself (not
 *                             with cut-first or TESS_K2_FUSED, and without
 *                             a histogram: TESS_SCHED_SERIAL) */
#define TESS_K2_REG 0
#define TESS_K2_ROWS32 1
#define TESS_K2_ROWS64 2
#define TESS_K2_LOOP 3
#define TESS_K2_REG_HI 4 /* register form compiled for 3-4 resident blocks per SM (FP32, n <= 7) */
#define TESS_K2_REG_TMA 5 /* register form, tile inputs staged in shared memory by bulk copies one
                             tile ahead (FP32, n <= 8) */
#define TESS_K2_REG_TMA_HI 6 /* the staged form compiled for 3 resident blocks per SM (FP32, n <= 7) */
#define TESS_K2_PAIR32 7     /* two threads per event, table in shared memory, 32 events per block (FP32) */
#define TESS_K2_PAIR64 8     /* the same with 64 events per block (FP32) */
#define TESS_K2_REAL 9       /* real currents in registers (FP32, TESS_POL_RANDOM only, n <= 9) */
#define TESS_K2_REAL_HI 10   /* the real form compiled for more resident blocks (FP32, TESS_POL_RANDOM, n <= 8) */
#define TESS_K2_ROWS_REAL 11 /* row form with real currents, 64 threads (FP32, TESS_POL_RANDOM, n >= 8) */
#define TESS_K2_PAIR_W 12    /* O(n^3) tensor rewrite of the four-vertex sum, two threads per event (FP32) */
#define TESS_K2_WAVE 13      /* row form with a runtime step loop, 64 events per block (FP32, n >= 6) */
#define TESS_K2_WAVE2 14     /* wavefront row form: two lanes of a warp per event build two rows of the
                                current table in step (Sec. 3's one thread per current of a length), 32 events
                                per block (FP32, n >= 6) */
#define TESS_K2_WAVE2U 15    /* TESS_K2_WAVE2 with the code of every step unrolled (FP32, n >= 6) */
#define TESS_K2_WAVE2P 16    /* TESS_K2_WAVE2 with the vertex algebra in packed FP32 pairs (f32x2: two lanes of
                                FP32 work per instruction; FP32, n >= 6) */
#define TESS_K2_WAVE2PU 17   /* TESS_K2_WAVE2P with the code of every step unrolled (FP32, n >= 6) */
#define TESS_K2_WAVE2L 18    /* TESS_K2_WAVE2 with only the row's currents in registers (momentum sums by
                                subtraction, split sums read back from the table), compiled for 12 resident
                                warps per SM where the tables leave room (FP32, n >= 6) */
#define TESS_K2_REG_HI4 19   /* register form compiled for 4 resident blocks of 128 per SM (128 registers, the
                                rest spilled; FP32, n <= 6) */
#define TESS_K2_REG_HI_PF 20 /* TESS_K2_REG_HI with the block's next tile of inputs prefetched into L2 before
                                each tile (FP32, n <= 7) */
#define TESS_K2_LANES8 21    /* 8 lanes of one warp per event sharing the currents of one length (Sec. 3's
                                one thread per current of a length), long sets split over lanes and their
                                partial sums added by warp shuffles; table in shared memory (FP32, n >= 6) */
#define TESS_K2_LANES16 22   /* the same with 16 lanes per event (FP32, n >= 6) */
#define TESS_K2_LANES32 23   /* the same with a whole warp per event (FP32, n >= 6) */
#define TESS_K2_FUSED 24     /* no separate kinematics kernel: one warp-specialised kernel per chunk, a
                                kinematics warpgroup handing tiles of 128 events to a register-form
                                amplitude warpgroup through shared memory; the events never leave the
                                chip (its plan needs no chunk buffer; tess_workspace_size still covers
                                every form) (TESS_FP32_DS with TESS_HEL_SAMPLE, no cut-first, n = 4..6) */
#define TESS_SCHED_SERIAL 0
#define TESS_SCHED_OVERLAP 1
#define TESS_SCHED_OVERLAP_TILES 2
#define TESS_SCHED_SERIAL_TILES 3
#define TESS_SCHED_SERIAL_HIST 4
int tess_autotune(tess_ctx *ctx, const tess_process *proc, uint64_t probe_events, double *acc_scratch,
                  void *workspace, size_t workspace_bytes, void *stream, int *form_out);

/* tess_autotune timed with the per-event outputs the later calls will write:
 * out is the tess_outputs of those calls (the per-event arrays it names, each
 * holding at least probe_events entries, device or mapped host memory, are
 * written with the probe's events; out->acc must be non-NULL and, like
 * out->hist, is not written, since the timed runs stop before the fold).
 * Variants differ in how their stores of the per-event arrays overlap the
 * arithmetic, so a choice tuned without them can lose a few per cent to the
 * runner-up when they are written.  Errors as tess_autotune, and
 * TESS_E_INVALID for a NULL out or out->acc. */
int tess_autotune_outputs(tess_ctx *ctx, const tess_process *proc, uint64_t probe_events,
                          const tess_outputs *out, void *workspace, size_t workspace_bytes, void *stream,
                          int *form_out);

/* Sets the variant for (precision, polarisation kind, n) of proc without
 * timing (Sec. 2 running configuration, chosen by the caller): form one of TESS_K2_* (-1: built-in default; a form not built for
 * (precision, n) or, for the real-current forms, for helicity vectors falls
 * back to the default), schedule one of TESS_SCHED_* (-1: default, serial).
 * Takes effect for later calls; TESS_E_INVALID for values out of range.  A
 * workspace sized by tess_workspace_size covers every choice. */
int tess_select_variant(tess_ctx *ctx, const tess_process *proc, int form, int schedule);

/* Bytes of per-event intermediate data (amplitude inputs and event factors)
 * per chunk of the sampled-event pipeline on this context, and per chunk
 * buffer of the FP32 gradient pipeline (tess_gradients); 0 restores the
 * defaults (4 GiB and 1 GiB).  Paper: the events in flight of one sweep (Sec. 2); here
 * the chunk is a trade between workspace and per-launch cost: every chunk
 * costs a kinematics and an amplitude launch, each with a ramp-up and a tail
 * of about one block's run time, so on GB300 fewer, larger chunks are faster
 * (measured at n = 6: 64 MB chunks 3.6e9 events/s, 1 GB 4.7e9, one 3.8 GB
 * chunk 4.9e9).  Takes effect for later calls (workspace sizes included:
 * tess_workspace_size and tess_gradients_workspace_size reflect it), and the
 * next tess_generate_batched call
 * recaptures its graph.  TESS_E_INVALID for a NULL ctx or a nonzero size
 * below 1 MiB.  Host-only. */
int tess_set_chunk_bytes(tess_ctx *ctx, size_t bytes);

/* What a call with (proc, n_events) would run (Sec. 2 running configuration):
 * info[0] amplitude variant
 * (TESS_K2_*, -1 for the exact-sum mode), info[1] the schedule in effect
 * (TESS_SCHED_*), info[2] number of chunks, info[3] amplitude-kernel grid
 * (blocks).  info: host, 4 ints.  Launches nothing. */
int tess_plan_info(const tess_ctx *ctx, const tess_process *proc, uint64_t n_events, int *info);

/* ---- Draws and gradients (no counterpart in the paper's method) --------------
 * tess_draws writes the generator's own random inputs of events (the
 * per-event random numbers whose generator Sec. 4 discusses with Fig. 2;
 * here Philox4x32-10, layout as in tess_generate)
 * [first_event, first_event + n_events) of stream `seed`:
 *   u      device [n_events][2 + 4(n-2)] doubles: u_x1, u_x2, then four Rambo
 *          uniforms per final-state gluon (layout of the counter-based draws)
 *   hel    device [n_events] uint32 helicity labels (bit i: leg i)
 *   order  device [n_events][n] uint8 colour orderings (order[0] = 0)
 * tess_gradients evaluates, for caller-given (u, hel, order) -- e.g. from
 * tess_draws, or uniforms transformed by a phase-space map -- the event weight
 * w (pb) of the sampled-mode estimator and its gradients:
 *   dw_du     [n_events][2 + 4(n-2)]  total derivative w.r.t. the uniforms
 *   dw_dk     [n_events][n][4]        w.r.t. the all-outgoing momenta at fixed
 *                                     x1, x2 (polarisation vectors and K sums
 *                                     follow k; beam-axis legs keep their basis)
 *   dw_dlnmu  [n_events]              w.r.t. ln mu_R (one-loop running)
 * all multiplied by dL_dw[e] when dL_dw is given (a vector-Jacobian product).
 * The cuts are a step function: events failing them have w = 0 and zero
 * gradients.  TESS_FP64: every step FP64, one kernel.  FP32 forms: the
 * kinematics of TESS_FP32_DS (FP32 seeds, cuts, observables, PDF, alpha_s,
 * polarisation basis; double-float boost/rescale rounded to FP32), an FP32
 * Berends-Giele forward pass and reverse sweep and an FP32 kinematics
 * adjoint (weights and the final scalings in FP64), run as three kernels per
 * chunk of events (kinematics -> amplitude inputs; 2 to 8 threads per event
 * for the recursion and its adjoint; kinematics again -> outputs, on a second
 * stream of the context beside the next chunk; the call is ordered on
 * `stream` as usual) through `workspace`:
 * tess_gradients_workspace_size(proc, n_events) bytes, device, 256-byte
 * aligned (0 bytes, NULL allowed, for TESS_FP64).  TESS_E_WORKSPACE if it is
 * missing or too small.  Any output pointer may be NULL. */
int tess_draws(tess_ctx *ctx, int n, uint64_t seed, uint64_t first_event, uint64_t n_events, double *u,
               uint32_t *hel, uint8_t *order, void *stream);
int tess_gradients_workspace_size(const tess_ctx *ctx, const tess_process *proc, uint64_t n_events, size_t *bytes);
int tess_gradients(tess_ctx *ctx, const tess_process *proc, uint64_t n_events, const double *u, const uint32_t *hel,
                   const uint8_t *order, const double *dL_dw, double *w, double *dw_du, double *dw_dk,
                   double *dw_dlnmu, void *workspace, size_t workspace_bytes, void *stream);

/* Colour-ordered matrix elements for caller-given kinematics (the
 * matrix-element stage alone, Eq. (BG-recursion) and the amplitude
 * equation of Sec. 3):  me2[e] = |A(order_e; hel_e)|^2 with
 * A = m / 2^((n-2)/2) in the Tr(T^a T^b) = delta^ab normalisation.
 *   k      device, [n_events][n][4] doubles: all-outgoing momenta
 *          (k_1 = -p_1, k_2 = -p_2 incoming; sum_i k_i = 0), (E, px, py, pz)
 *   order  device, [n_events][n] uint8: cyclic colour ordering, order[0] is
 *          the leg contracted last; each row a permutation of 0..n-1
 *   hel    device, [n_events] uint32: bit i = helicity label of leg i (0 ->
 *          eps_+ of the leg's physical direction, 1 -> eps_-)
 *   me2    device, [n_events] doubles (output)
 * precision: TESS_FP64, or TESS_FP32_CURRENTS / TESS_FP32_DS (FP32 currents). */
int tess_me2(tess_ctx *ctx, int n, int precision, uint64_t n_events, const double *k, const uint8_t *order,
             const uint32_t *hel, double *me2, void *stream);

/* Gauge check of Sec. 4 (a precision diagnostic), same arguments as tess_me2:
 * ratio[e] = |k^ . Num|^2 / |eps . Num|^2 for the leg order_e[0] contracted
 * last, Num the un-propagated current of the other legs and k^ that leg's
 * momentum divided by its energy.  Current conservation makes the
 * numerator vanish exactly, so the ratio measures the rounding of the
 * evaluation (FP32 currents vs FP64). */
int tess_gauge_ratio(tess_ctx *ctx, int n, int precision, uint64_t n_events, const double *k, const uint8_t *order,
                     const uint32_t *hel, double *ratio, void *stream);

/* Cross section from a device acc (synchronises the stream):
 * host out[4] = {sigma_pb, mc_error_pb, n_pass, n_generated}.
 * Paper: the Monte Carlo estimate of the cross-section formula at the end of
 * Sec. 3 (mean weight over all generated events) and its mean standard
 * deviation, from the compensated (Kahan-style) sums of Sec. 4 (Fig. 2
 * discussion): sigma = S1/N, error = sqrt((S2/N - sigma^2)/(N - 1)).
 * Returns TESS_E_CUDA (after filling out) if acc counts stalled blocks,
 * else TESS_E_NUMERICAL (after filling out) if non-finite weights were seen. */
int tess_result(tess_ctx *ctx, const double *acc, double *out, void *stream);

/* Copy per-event outputs to host buffers (synchronises the stream).  Any of
 * the host pointers may be NULL.  Paper: the last step of Sec. 3 returns the
 * results to the CPU for processing; events are flagged rather than dropped,
 * so the CPU can re-apply other cuts when histogramming (Sec. 3).
 * dev: device pointers as filled by tess_generate; errors TESS_E_INVALID
 * (NULL dev), TESS_E_CUDA (copy failed). */
int tess_weights(tess_ctx *ctx, const tess_outputs *dev, uint64_t n_events, double *host_weight,
                 uint8_t *host_pass, double *host_me2, void *stream);

/* Histogram from a device hist (synchronises): host sumw[hist_bins + 2] and
 * sumw2[hist_bins + 2], compensation folded in.  Paper: the differential
 * distributions of Sec. 4 (Fig. 3: H_T and Delta R_min), whose histogramming
 * the paper leaves to the CPU; here the bins are filled on the device and
 * only read back.  Errors TESS_E_INVALID (no histogram in proc), TESS_E_CUDA. */
int tess_histograms(tess_ctx *ctx, const tess_process *proc, const double *hist, double *host_sumw,
                    double *host_sumw2, void *stream);

/* ---- Arithmetic peaks (measurement; no counterpart in the paper) -------------
 * The paper reports times per event only; the rooflines of this library's
 * amplitude kernels divide by the GPU's own fused-multiply-add rate, measured
 * here: every thread of 4 x SMs blocks of 512 runs independent FMA chains
 * (inline PTX, so nothing is folded away) of kind
 *   TESS_PEAK_FP32    scalar fma.rn.f32
 *   TESS_PEAK_FP32X2  packed fma.rn.f32x2 (two FP32 lanes per instruction)
 *   TESS_PEAK_FP64    fma.rn.f64
 * *tflops = best of `reps` (>= 1) launches after one warm-up, FLOPs counted
 * as 2 per lane per FMA, timed with CUDA events on `stream` (synchronised).
 * Allocates no device memory.  The rate follows the SM clock of the moment:
 * sample the clock beside it.  Errors: TESS_E_INVALID (kind, reps),
 * TESS_E_CUDA. */
#define TESS_PEAK_FP32 0
#define TESS_PEAK_FP32X2 1
#define TESS_PEAK_FP64 2
int tess_peak_flops(tess_ctx *ctx, int kind, int reps, double *tflops, void *stream);

/* ---- Allocation-free generation (no counterpart in the paper) ----------------
 * Some callers cannot call cudaMalloc or give the library a workspace: for
 * example a host program whose memory manager reserves the whole device at
 * start-up and forbids other allocations, or a latency-critical loop that
 * cannot afford an allocation's implicit device synchronisation.  For them,
 * tess_generate_noalloc generates the same events as tess_generate (the
 * same per-event outputs, device memory or mapped pinned host memory, and
 * the same accumulation into acc / hist, which the caller still provides)
 * but keeps its scratch -- the per-block partial sums -- in a fixed device
 * array of TESS_NOALLOC_SCRATCH_BYTES that is part of the library.  It runs
 * the fused one-kernel-per-event form: for the exact sum (TESS_HEL_SUM) that
 * is tess_generate's own kernel; for sampled helicities it is offered at
 * TESS_FP64 only (FP64 in every step, equal to tess_generate to 1e-10
 * relative, but thread-per-event with no chunk pipeline, so several times
 * slower than tess_generate at large n), and the FP32 precisions with
 * sampled helicities return TESS_E_UNSUPPORTED.  Every GPU that
 * loads the library holds that array until the process exits.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine.
 *   - The first call on each device looks up the array's device address (a
 *     one-time set-up with that device current); make that first call before
 *     any stream capture.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and must be serialised by the caller.
 *     Nothing in it needs clearing: each call writes every partial row that it
 *     reads back.
 *   - At most TESS_NOALLOC_MAX_BINS histogram bins; more is TESS_E_INVALID.
 *     Other errors as tess_generate (no workspace errors).                  */
#define TESS_NOALLOC_SCRATCH_BYTES (1u << 20)
#define TESS_NOALLOC_MAX_BINS 254
int tess_generate_noalloc(tess_ctx *ctx, const tess_process *proc, uint64_t seed, uint64_t first_event,
                          uint64_t n_events, const tess_outputs *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TESS_H */
