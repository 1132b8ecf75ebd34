// Host side of the two-kernel pipeline: plan (workspace layout, chunk size,
// K2 grid) and the launch sequence of one tess_generate call.
#pragma once
#include <algorithm>

#include <cudaTypedefs.h>

#include "tess_pair.cuh"
#include "tess_pair_w.cuh"
#include "tess_pipeline.cuh"
#include "tess_wave.cuh"
#include "tess_wavep.cuh"
#include "tess_lanes.cuh"
#include "tess_fused.cuh"

namespace tess {

struct PipePlan {
  int form = 0;      // K2 variant (K2Form)
  int per_sm = 1;    // K2 blocks resident per SM
  int grid = 1;      // K2 blocks = partial rows
  int block = 128;   // events per K2 tile (= threads per block except the lane-pair forms)
  size_t smem = 0;   // K2 dynamic shared memory
  int cap = 128;     // events per chunk
  size_t chunk_target = 0;  // input to planning: bytes per chunk (0 = kChunkTargetBytes)
  int chunks = 1;
  size_t off_in = 0, off_efac = 0, off_wfac = 0, off_hval = 0, off_pass = 0;
  size_t off_col = 0, off_orig = 0, off_tcount = 0, off_toff = 0, off_dcount = 0;  // cut-first only
  size_t off_tables = 0;  // grid mode only: PDF and alpha_s tables (before the chunk buffers)
  size_t off_wev = 0;     // deferred histogram only: event weights of the chunk
  bool defer_hist = false;  // SCHED_SERIAL_HIST with a histogram: filled by its own kernel
  size_t kin_smem = 0;   // K1 dynamic shared memory (FP32 forms: the output tile)
  size_t buf_bytes = 0;  // one chunk buffer
  int sched = 0;         // Schedule
  bool overlap = false;  // double-buffered, K1 and K2 on two streams
  size_t bytes = 0;      // workspace bytes
};

// How the chunks are launched.
//   SCHED_SERIAL         K1 then K2 per chunk on the caller's stream; K2 grid
//                        = resident blocks (persistent, loops over tiles)
//   SCHED_OVERLAP        K1 of chunk c+1 on the caller's stream while K2 of
//                        chunk c runs on a second stream; two chunk buffers
//   SCHED_OVERLAP_TILES  as SCHED_OVERLAP with one K2 block per tile, so that
//                        K1 blocks are scheduled as K2 blocks retire
//   SCHED_SERIAL_TILES   serial with one K2 block per tile
//   SCHED_SERIAL_HIST    serial; with a histogram, K2 keeps only the sums
//                        and leaves each event's weight in the chunk buffer,
//                        and a third kernel per chunk (hist_chunk_kernel)
//                        fills the histogram (no cut-first, not the fused
//                        form; without a histogram it is SCHED_SERIAL)
// The per-tile grid is bounded so that the blocks' partial-row flushes stay
// under 1/50 of the chunk's own traffic (large histograms keep the
// persistent grid).
enum Schedule {
  SCHED_SERIAL = 0,
  SCHED_OVERLAP = 1,
  SCHED_OVERLAP_TILES = 2,
  SCHED_SERIAL_TILES = 3,
  SCHED_SERIAL_HIST = 4,
  SCHED_N = 5
};

// Streams and events of the overlapped pipeline (owned by the context).
struct OverlapRes {
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t k1done[2] = {nullptr, nullptr}, k2done[2] = {nullptr, nullptr};
};

// Default bytes of per-event intermediate data (amplitude inputs and event
// factors) per chunk.  Measured on GB300 at n = 6 (2^24 events, serial
// schedule): 64 MB chunks 3.57e9 events/s, 256 MB 4.28e9, 1 GB 4.69e9, one
// 3.8 GB chunk 4.86e9.  Each launch pays a ramp-up and a tail of about one
// block's run time (~30 us for the kinematics kernel), which small chunks
// multiply; an L2-sized chunk does not stay in L2 between the two kernels
// anyway (live L2 hit rate of the amplitude kernel's reads 26-35 % even at
// 16 MB), and streaming it through HBM costs the ALU-bound kernels nothing
// measurable.  4 GB bounds the workspace (two such buffers under an
// overlapped schedule) and keeps the per-chunk cost near 1 %.
#ifndef TESS_CHUNK_TARGET_MB
#define TESS_CHUNK_TARGET_MB 4096
#endif
constexpr size_t kChunkTargetBytes = (size_t)TESS_CHUNK_TARGET_MB << 20;

// plan_pipeline_t result: 0, a cudaError_t of a failed attribute / occupancy
// call, or this code when no block of the variant fits on an SM
constexpr int kPlanNoResidentBlock = -2;


// Optional host hook around each launch (stage timing); kinds below.
enum StageKind { STAGE_KIN = 0, STAGE_AMP = 1, STAGE_FINAL = 2, STAGE_FUSED = 3, STAGE_NKINDS = 4 };
struct StageHook {
  void (*mark)(void *self, int kind, bool begin, cudaStream_t s);
  void *self;
  void operator()(int kind, bool begin, cudaStream_t s) const {
    if (mark) mark(self, kind, begin, s);
  }
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Tensor map of a chunk buffer's amplitude inputs for the staged forms: a
// 2-D float tensor of `rows` rows of `cap` events (row stride cap * 4 bytes,
// a multiple of 512), box {32 events, all rows}.  cuTensorMapEncodeTiled is
// reached through the runtime's driver entry point (no driver library link).
inline cudaError_t encode_rows_map(CUtensorMap *map, const float *base, int rows, int cap) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cap, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cap * sizeof(float)};
  const cuuint32_t box[2] = {32u, (cuuint32_t)rows};
  const cuuint32_t elem[2] = {1u, 1u};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box, elem,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Amplitude-kernel (K2) variants.  All are one thread per event; they differ
// in where the current table lives and in the block shape:
//   K2_REG     table in registers (fully unrolled), 128 threads   FP32, n <= 8
//   K2_ROWS32  current row in registers, older rows in the thread's
//              shared-memory column, 32 threads per block         FP32, n >= 6
//   K2_ROWS64  the same with 64 threads per block                 FP32, n >= 6
//   K2_LOOP    loop form, table in local memory, 128 threads      FP64
//   K2_REG_HI  register form compiled for more resident blocks (3 per SM
//              for n >= 6, 4 below: fewer registers, a few spilled) FP32, n <= 7
//   K2_REG_TMA register form with the tile inputs staged in shared memory
//              by bulk copies one tile ahead, 128 threads         FP32, n <= 8
//   K2_REG_TMA_HI  the staged form compiled for 3 resident blocks   FP32, n <= 7
//   K2_PAIR32  two threads per event, table in shared memory, 32 events
//              per block (64 threads)                            FP32, any n
//   K2_PAIR64  the same with 64 events per block (128 threads)   FP32, any n
//   K2_REAL    register form with real currents, 128 threads; random real
//              polarisations only (TESS_POL_RANDOM)               FP32, n <= 9
//   K2_REAL_HI the real form compiled for more resident blocks   FP32, n <= 8
//   K2_ROWS_REAL  row form with real currents, 64 threads; random real
//              polarisations only                                 FP32, n >= 8
//   K2_PAIR_W  tensor form: the O(n^3) rewrite of the four-vertex sum
//              (antisymmetric tensors per set), lane-pair layout,
//              32 events per block                               FP32, any n
//   K2_WAVE    row form with a runtime step loop (one copy of the split
//              code serves every step), 64 events per block     FP32, n >= 6
//   K2_WAVE2   the same with two lanes of a warp per event building two
//              rows in step (tess_wave.cuh), 32 events per block (64
//              threads)                                          FP32, n >= 6
//   K2_WAVE2U  K2_WAVE2 with every step's code unrolled           FP32, n >= 6
//   K2_WAVE2P  K2_WAVE2 with the vertex algebra in packed FP32 pairs
//              (tess_wavep.cuh)                                  FP32, n >= 6
//   K2_WAVE2PU K2_WAVE2P with every step's code unrolled          FP32, n >= 6
//   K2_WAVE2L  K2_WAVE2 with only the row's currents in registers,
//              compiled for 12 resident warps per SM             FP32, n >= 6
//   K2_REG_HI4 register form compiled for 4 resident blocks (16 warps)
//              per SM: 128 registers, the rest spilled           FP32, n <= 6
//   K2_REG_HI_PF  K2_REG_HI with the block's next tile of inputs prefetched
//              into L2 before each tile                          FP32, n <= 7
//   K2_LANES8 / K2_LANES16 / K2_LANES32  8, 16 or 32 lanes of one warp per
//              event sharing the sets of one length, long sets split over
//              lanes and reduced by shuffles (tess_lanes.cuh), 128 threads
//                                                                FP32, n >= 6
//   K2_FUSED   no separate kinematics launch: one warp-specialised kernel
//              (tess_fused.cuh), a kinematics warpgroup feeding the
//              register form through shared memory, 256 threads, no
//              chunk buffer                  FP32 double-float, n = 4..6
enum K2Form {
  K2_REG = 0,
  K2_ROWS32 = 1,
  K2_ROWS64 = 2,
  K2_LOOP = 3,
  K2_REG_HI = 4,
  K2_REG_TMA = 5,
  K2_REG_TMA_HI = 6,
  K2_PAIR32 = 7,
  K2_PAIR64 = 8,
  K2_REAL = 9,
  K2_REAL_HI = 10,
  K2_ROWS_REAL = 11,
  K2_PAIR_W = 12,
  K2_WAVE = 13,
  K2_WAVE2 = 14,
  K2_WAVE2U = 15,
  K2_WAVE2P = 16,
  K2_WAVE2PU = 17,
  K2_WAVE2L = 18,
  K2_REG_HI4 = 19,
  K2_REG_HI_PF = 20,
  K2_LANES8 = 21,
  K2_LANES16 = 22,
  K2_LANES32 = 23,
  K2_FUSED = 24,
  K2_NFORMS = 25
};

// What a call offers the amplitude kernel: CAP_REAL_EPS, its polarisation
// vectors are real (random polarisations), which the real-current forms
// require; CAP_CUT_FIRST, its events are compacted (an index list), which the
// staged forms do not read; CAP_KIN_DS, its kinematics are the double-float
// form, the only one the fused kernel carries.
constexpr unsigned CAP_REAL_EPS = 1u, CAP_CUT_FIRST = 2u, CAP_PDF_GRID = 4u, CAP_KIN_DS = 8u;

template <int N, typename R>
constexpr bool k2_valid(int f, unsigned caps) {
  const bool real_eps = (caps & CAP_REAL_EPS) != 0, cut_first = (caps & CAP_CUT_FIRST) != 0;
  if constexpr (sizeof(R) == 8) {
    return f == K2_LOOP && !cut_first;
  } else {
    switch (f) {
      case K2_FUSED: return N >= 4 && N <= 6 && !real_eps && !cut_first && (caps & CAP_KIN_DS) != 0;
      case K2_REAL: return real_eps && N <= 9;
      case K2_REAL_HI: return real_eps && N <= 8;
      case K2_ROWS_REAL: return real_eps && N >= 8;
      case K2_PAIR_W: return true;
      case K2_REG_TMA: return N <= 8 && !cut_first;
      case K2_REG_TMA_HI: return N <= 7 && !cut_first;
      case K2_REG: return N <= 8;
      case K2_REG_HI:
      case K2_REG_HI_PF: return N <= 7;
      case K2_REG_HI4: return N <= 6;
      case K2_ROWS32:
      case K2_ROWS64:
      case K2_WAVE:
      case K2_WAVE2:
      case K2_WAVE2U:
      case K2_WAVE2P:
      case K2_WAVE2PU:
      case K2_WAVE2L:
      case K2_LANES8:
      case K2_LANES16:
      case K2_LANES32: return N >= 6;
      case K2_PAIR32:
      case K2_PAIR64: return true;
      default: return false;
    }
  }
}

template <int N, typename R>
constexpr int k2_default() {
  return sizeof(R) == 8 ? K2_LOOP : (N <= 7 ? K2_REG : K2_ROWS32);
}

template <int N, typename R, int F>
struct K2V {
  static constexpr int L = N - 1;
  static constexpr bool lanes = F == K2_LANES8 || F == K2_LANES16 || F == K2_LANES32;
  static constexpr bool fused = F == K2_FUSED;
  static constexpr int lanes_ln = F == K2_LANES8 ? 8 : (F == K2_LANES16 ? 16 : 32);
  static constexpr int block =
      lanes ? 128 / lanes_ln
            : ((F == K2_ROWS32 || F == K2_PAIR32 || F == K2_PAIR_W || F == K2_WAVE2 || F == K2_WAVE2U ||
                F == K2_WAVE2P || F == K2_WAVE2PU || F == K2_WAVE2L)
                   ? 32
                   : ((F == K2_ROWS64 || F == K2_PAIR64 || F == K2_ROWS_REAL || F == K2_WAVE) ? 64 : 128));
  static constexpr bool rows = F == K2_ROWS32 || F == K2_ROWS64;
  static constexpr bool pair = F == K2_PAIR32 || F == K2_PAIR64 || F == K2_PAIR_W;
  static constexpr int wave_g =
      (F == K2_WAVE2 || F == K2_WAVE2U || F == K2_WAVE2P || F == K2_WAVE2PU || F == K2_WAVE2L) ? 2 : 1;
  static constexpr bool wavep = F == K2_WAVE2P || F == K2_WAVE2PU;  // packed-pair arithmetic
  static constexpr bool wave_lean = F == K2_WAVE2L;
  static constexpr int wave_minb = wave_lean ? 6 : 1;
  static constexpr bool wave = F == K2_WAVE || F == K2_WAVE2 || F == K2_WAVE2U || wavep || wave_lean;
  static constexpr bool wave_unr = F == K2_WAVE2U || F == K2_WAVE2PU;
  static constexpr int threads =
      fused ? kFusedThreads
            : (lanes ? 128 : (pair ? 2 * block : (wave ? wave_g * block : block)));  // block = events per tile
  static constexpr int hi_blocks = N >= 6 ? 3 : 4;
  static constexpr int real_hi_blocks = N >= 8 ? 3 : 4;
  static void *fn() {
    if constexpr (fused)
      return (void *)fused_kernel<N>;
    else if constexpr (lanes)
      return (void *)bg_lanes_kernel<N, lanes_ln, 4>;
    else if constexpr (wavep)
      return (void *)bg_wavep_kernel<N, block, wave_g, wave_unr>;
    else if constexpr (wave)
      return (void *)bg_wave_kernel<N, block, wave_g, wave_unr, wave_lean, wave_minb>;
    else if constexpr (F == K2_PAIR_W)
      return (void *)bg_pair_w_kernel<N, block>;
    else if constexpr (F == K2_ROWS_REAL)
      return (void *)bg_rows_real_kernel<N, block>;
    else if constexpr (F == K2_REAL)
      return (void *)bg_real_kernel<N, 128>;
    else if constexpr (F == K2_REAL_HI)
      return (void *)bg_real_kernel<N, 128, real_hi_blocks>;
    else if constexpr (pair)
      return (void *)bg_pair_kernel<N, block>;
    else if constexpr (rows)
      return (void *)bg_rows_kernel<N, block>;
    else if constexpr (F == K2_REG_TMA)
      return (void *)bg_reg_tma_kernel<N, 128>;
    else if constexpr (F == K2_REG_TMA_HI)
      return (void *)bg_reg_tma_kernel<N, 128, 3>;
    else if constexpr (F == K2_REG)
      return (void *)bg_reg_kernel<N, float, 128>;
    else if constexpr (F == K2_REG_HI)
      return (void *)bg_reg_kernel<N, float, 128, hi_blocks>;
    else if constexpr (F == K2_REG_HI4)
      return (void *)bg_reg_kernel<N, float, 128, 4>;
    else if constexpr (F == K2_REG_HI_PF)
      return (void *)bg_reg_kernel<N, float, 128, hi_blocks, true>;
    else
      return (void *)bg_loop_kernel<N, 128>;
  }
  static size_t smem(int hist_bins) {
    if constexpr (fused)
      return FusedSmem<N>::bytes(hist_bins);
    else if constexpr (lanes)
      return lanes_smem_bytes<L, 4, lanes_ln>() + EpiSmem<threads>::bytes(hist_bins);
    else if constexpr (wave_lean)
      return wave_lean_smem_per_event<L>() * block + EpiSmem<threads>::bytes(hist_bins);
    else if constexpr (wave)
      return wave_smem_per_event<L>() * block + EpiSmem<threads>::bytes(hist_bins);
    else if constexpr (F == K2_PAIR_W)
      return PairWSmem<L, block>::bytes + EpiSmem<threads>::bytes(hist_bins);
    else if constexpr (F == K2_ROWS_REAL)
      return ((rows_real_smem_per_thread<L>() * block + 15) & ~(size_t)15) + EpiSmem<block>::bytes(hist_bins);
    else if constexpr (pair)
      return PairSmem<L, block>::bytes + EpiSmem<threads>::bytes(hist_bins);
    else if constexpr (rows)
      return rows_smem_per_thread<L>() * block + EpiSmem<block>::bytes(hist_bins);
    else if constexpr (F == K2_REG_TMA || F == K2_REG_TMA_HI)
      return RegStage<L, 128>::window + EpiSmem<128>::bytes(hist_bins);
    else
      return EpiSmem<128>::bytes(hist_bins);
  }
  static constexpr bool staged = F == K2_REG_TMA || F == K2_REG_TMA_HI;
  // map: tensor map of B.in (staged forms only)
  static cudaError_t launch(const ChunkParams &C, const ChunkBuf<R> &B, double *partials, int grid, size_t smem,
                            cudaStream_t s, const CUtensorMap *map) {
    if constexpr (fused)
      fused_kernel<N><<<grid, threads, smem, s>>>(C, partials);
    else if constexpr (lanes)
      bg_lanes_kernel<N, lanes_ln, 4><<<grid, threads, smem, s>>>(C, B, partials);
    else if constexpr (wavep)
      bg_wavep_kernel<N, block, wave_g, wave_unr><<<grid, threads, smem, s>>>(C, B, partials);
    else if constexpr (wave)
      bg_wave_kernel<N, block, wave_g, wave_unr, wave_lean, wave_minb><<<grid, threads, smem, s>>>(C, B, partials);
    else if constexpr (F == K2_PAIR_W)
      bg_pair_w_kernel<N, block><<<grid, threads, smem, s>>>(C, B, partials);
    else if constexpr (F == K2_ROWS_REAL)
      bg_rows_real_kernel<N, block><<<grid, block, smem, s>>>(C, B, partials);
    else if constexpr (F == K2_REAL)
      bg_real_kernel<N, 128><<<grid, 128, smem, s>>>(C, B, partials);
    else if constexpr (F == K2_REAL_HI)
      bg_real_kernel<N, 128, real_hi_blocks><<<grid, 128, smem, s>>>(C, B, partials);
    else if constexpr (pair)
      bg_pair_kernel<N, block><<<grid, threads, smem, s>>>(C, B, partials);
    else if constexpr (rows)
      bg_rows_kernel<N, block><<<grid, block, smem, s>>>(C, B, partials);
    else if constexpr (F == K2_REG_TMA)
      bg_reg_tma_kernel<N, 128><<<grid, 128, smem, s>>>(C, B, partials, *map);
    else if constexpr (F == K2_REG_TMA_HI)
      bg_reg_tma_kernel<N, 128, 3><<<grid, 128, smem, s>>>(C, B, partials, *map);
    else if constexpr (F == K2_REG)
      bg_reg_kernel<N, float, 128><<<grid, 128, smem, s>>>(C, B, partials);
    else if constexpr (F == K2_REG_HI)
      bg_reg_kernel<N, float, 128, hi_blocks><<<grid, 128, smem, s>>>(C, B, partials);
    else if constexpr (F == K2_REG_HI4)
      bg_reg_kernel<N, float, 128, 4><<<grid, 128, smem, s>>>(C, B, partials);
    else if constexpr (F == K2_REG_HI_PF)
      bg_reg_kernel<N, float, 128, hi_blocks, true><<<grid, 128, smem, s>>>(C, B, partials);
    else
      bg_loop_kernel<N, 128><<<grid, 128, smem, s>>>(C, B, partials);
    return cudaGetLastError();
  }
};

// Dispatch a runtime form to the compiled variants of (N, R).
template <int N, typename R, typename Fn>
auto with_form(int f, Fn &&fn) {
  if constexpr (sizeof(R) == 8) {
    return fn(K2V<N, R, K2_LOOP>{});
  } else {
    if (f == K2_PAIR32) return fn(K2V<N, R, K2_PAIR32>{});
    if (f == K2_PAIR64) return fn(K2V<N, R, K2_PAIR64>{});
    if (f == K2_PAIR_W) return fn(K2V<N, R, K2_PAIR_W>{});
    if constexpr (N <= 9) {
      if (f == K2_REAL) return fn(K2V<N, R, K2_REAL>{});
    }
    if constexpr (N <= 8) {
      if (f == K2_REAL_HI) return fn(K2V<N, R, K2_REAL_HI>{});
    }
    if constexpr (N <= 6) {
      if (f == K2_REG_HI4) return fn(K2V<N, R, K2_REG_HI4>{});
    }
    if constexpr (N >= 4 && N <= 6) {
      if (f == K2_FUSED) return fn(K2V<N, R, K2_FUSED>{});
    }
    if constexpr (N <= 7) {
      if (f == K2_REG_HI_PF) return fn(K2V<N, R, K2_REG_HI_PF>{});
      if (f == K2_REG_HI) return fn(K2V<N, R, K2_REG_HI>{});
      if (f == K2_REG_TMA_HI) return fn(K2V<N, R, K2_REG_TMA_HI>{});
    }
    if constexpr (N <= 8) {
      if (f == K2_REG) return fn(K2V<N, R, K2_REG>{});
      if (f == K2_REG_TMA) return fn(K2V<N, R, K2_REG_TMA>{});
    }
    if constexpr (N >= 8) {
      if (f == K2_ROWS_REAL) return fn(K2V<N, R, K2_ROWS_REAL>{});
    }
    if constexpr (N >= 6) {
      if (f == K2_WAVE) return fn(K2V<N, R, K2_WAVE>{});
      if (f == K2_WAVE2) return fn(K2V<N, R, K2_WAVE2>{});
      if (f == K2_WAVE2U) return fn(K2V<N, R, K2_WAVE2U>{});
      if (f == K2_WAVE2P) return fn(K2V<N, R, K2_WAVE2P>{});
      if (f == K2_WAVE2PU) return fn(K2V<N, R, K2_WAVE2PU>{});
      if (f == K2_WAVE2L) return fn(K2V<N, R, K2_WAVE2L>{});
      if (f == K2_LANES8) return fn(K2V<N, R, K2_LANES8>{});
      if (f == K2_LANES16) return fn(K2V<N, R, K2_LANES16>{});
      if (f == K2_LANES32) return fn(K2V<N, R, K2_LANES32>{});
      if (f == K2_ROWS64) return fn(K2V<N, R, K2_ROWS64>{});
      return fn(K2V<N, R, K2_ROWS32>{});
    } else {
      return fn(K2V<N, R, K2_REG>{});
    }
  }
}

template <int N, typename R>
int plan_pipeline_t(int sm_count, uint64_t n_events, int hist_bins, int form, int sched, unsigned caps,
                    PipePlan *pl) {
  constexpr int L = N - 1;
  if (!k2_valid<N, R>(form, caps)) form = k2_default<N, R>();
  if (form == K2_FUSED) {
    // its register split (setmaxnreg) assumes the launch's 128 registers a
    // thread; any other compiled count and the form is not offered
    cudaFuncAttributes fa;
    const cudaError_t e = with_form<N, R>(form, [&](auto K) { return cudaFuncGetAttributes(&fa, decltype(K)::fn()); });
    if (e != cudaSuccess) return (int)e;
    if (fa.numRegs != kFusedLaunchRegs) form = k2_default<N, R>();
  }
  pl->form = form;
  const bool fused = form == K2_FUSED;
  const int rc = with_form<N, R>(form, [&](auto K) {
    using KV = decltype(K);
    pl->block = KV::block;  // events per tile
    pl->smem = KV::smem(hist_bins);
    cudaError_t e = allow_max_smem(KV::fn());
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, KV::fn(), KV::threads, pl->smem)) != cudaSuccess)
      return (int)e;
    if (per_sm < 1) return kPlanNoResidentBlock;
    pl->per_sm = per_sm;
    return 0;
  });
  if (rc) return rc;
  if constexpr (sizeof(R) == 4) {
    pl->kin_smem = kin_tile_bytes<N>();
    const void *kin_fns[] = {
        (const void *)kin_ds_kernel<N, false, false>, (const void *)kin_ds_kernel<N, true, false>,
        (const void *)kin_ds_kernel<N, false, true>,  (const void *)kin_ds_kernel<N, true, true>,
        (const void *)kin_kernel<N, float, false, false>, (const void *)kin_kernel<N, float, true, false>,
        (const void *)kin_kernel<N, float, false, true>,  (const void *)kin_kernel<N, float, true, true>};
    cudaError_t e = cudaSuccess;
    for (const void *fn : kin_fns)
      if (e == cudaSuccess) e = allow_max_smem(fn);
    if (e != cudaSuccess) return (int)e;
  } else {
    pl->kin_smem = 0;
  }
  const int per_sm = pl->per_sm;
  const bool cut_first = (caps & CAP_CUT_FIRST) != 0;
  if (sched < 0 || sched >= SCHED_N) sched = SCHED_SERIAL;
  pl->defer_hist = sched == SCHED_SERIAL_HIST && hist_bins > 0 && !cut_first && !fused;
  const uint64_t per_event = (uint64_t)InRows<L>::rows * sizeof(R) + 3 * sizeof(double) + 1 +
                             (cut_first ? 2 * sizeof(int) : 0) + (pl->defer_hist ? sizeof(double) : 0);
  const uint64_t chunk_bytes = pl->chunk_target ? pl->chunk_target : kChunkTargetBytes;
  // events per chunk: a multiple of 128 below 2^31 (chunk columns are ints);
  // the fused kernel keeps its events on chip but takes the same chunks (one
  // launch per chunk)
  uint64_t target = std::min<uint64_t>(std::max<uint64_t>(128, (chunk_bytes / per_event) / 128 * 128),
                                       (uint64_t)INT32_MAX / 256 * 128);
  // A whole number of amplitude-grid waves per chunk: the chunk's tiles are
  // spread over the resident blocks, and a last wave with few tiles leaves
  // most SMs idle for one tile's time (measured at n = 6: 2330 tiles on 456
  // resident blocks ran as six waves, the sixth 2 % full, about 15 % of the
  // amplitude kernel's time).  Cut-first chunks have a data-dependent count.
  const uint64_t wave = (uint64_t)sm_count * (uint64_t)per_sm * (uint64_t)pl->block;
  if (!cut_first && target >= wave) target = std::max<uint64_t>(128, target / wave * wave / 128 * 128);
  const uint64_t want = (std::max<uint64_t>(n_events, 1) + 127) / 128 * 128;
  pl->cap = (int)std::min(target, want);
  pl->chunks = (int)((std::max<uint64_t>(n_events, 1) + pl->cap - 1) / pl->cap);
  const uint64_t tiles = ((uint64_t)pl->cap + pl->block - 1) / pl->block;
  pl->sched = sched;
  pl->overlap = (sched == SCHED_OVERLAP || sched == SCHED_OVERLAP_TILES) && pl->chunks > 1 && !fused;
  uint64_t resident = (uint64_t)sm_count * per_sm;
  if (sched == SCHED_OVERLAP_TILES || sched == SCHED_SERIAL_TILES) {
    const uint64_t flush_budget = (uint64_t)pl->cap * per_event / 50 / (partial_stride(hist_bins) * sizeof(double));
    resident = std::max(resident, flush_budget);
  }
  pl->grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, resident));
  size_t off = align256((size_t)pl->grid * partial_stride(hist_bins) * sizeof(double));
  pl->off_tables = 0;
  if (caps & CAP_PDF_GRID) {  // PDF and alpha_s tables of the grid mode
    pl->off_tables = off;
    off = align256(off + (size_t)(kPdfNodes + kAsNodes) * sizeof(float));
  }
  pl->off_in = off;
  if (fused) {  // partial rows (and grid tables) only
    pl->buf_bytes = 0;
    pl->bytes = off;
    return 0;
  }
  off = align256(off + (size_t)InRows<L>::rows * pl->cap * sizeof(R));
  pl->off_efac = off;
  off = align256(off + (size_t)pl->cap * sizeof(double));
  pl->off_wfac = off;
  off = align256(off + (size_t)pl->cap * sizeof(double));
  pl->off_hval = off;
  off = align256(off + (size_t)pl->cap * sizeof(double));
  pl->off_pass = off;
  off = align256(off + (size_t)pl->cap);
  if (pl->defer_hist) {
    const cudaError_t e = allow_max_smem((const void *)hist_chunk_kernel<kBlock>);  // up to 1024 bins: 68 KB
    if (e != cudaSuccess) return (int)e;
    pl->off_wev = off;
    off = align256(off + (size_t)pl->cap * sizeof(double));
  }
  if (cut_first) {  // compaction: column and source index per event, count per K1 tile, total
    pl->off_col = off;
    off = align256(off + (size_t)pl->cap * sizeof(int));
    pl->off_orig = off;
    off = align256(off + (size_t)pl->cap * sizeof(int));
    pl->off_tcount = off;
    off = align256(off + (size_t)(pl->cap / kBlock + 1) * sizeof(int));
    pl->off_toff = off;
    off = align256(off + (size_t)(pl->cap / kBlock + 1) * sizeof(int));
    pl->off_dcount = off;
    off = align256(off + sizeof(int));
  }
  pl->buf_bytes = off - pl->off_in;
  pl->bytes = pl->overlap ? off + pl->buf_bytes : off;  // second chunk buffer
  return 0;
}

template <int N, typename R>
cudaError_t run_pipeline_t(const EventParams &P, const PipePlan &pl, char *ws, cudaStream_t s,
                           const StageHook *hook, const OverlapRes *ov = nullptr) {
  double *partials = (double *)ws;
  cudaError_t e = cudaMemsetAsync(partials, 0, (size_t)pl.grid * partial_stride(P.hist_bins) * sizeof(double), s);
  if (e != cudaSuccess) return e;
  EventParams PG = P;
  if (P.pdf_grid) {  // tables for this call's process
    float *g = (float *)(ws + pl.off_tables);
    grid_fill_kernel<256><<<(kPdfNodes + kAsNodes + 255) / 256, 256, 0, s>>>(P, g);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    PG.grid_pdf = g;
    PG.grid_as = g + kPdfNodes;
  }
  ChunkBuf<R> BB[2];
  for (int b = 0; b < 2; ++b) {
    char *base = ws + (b ? pl.buf_bytes : 0);
    BB[b].in = (R *)(base + pl.off_in);
    BB[b].efac = (double *)(base + pl.off_efac);
    BB[b].wfac = (double *)(base + pl.off_wfac);
    BB[b].hval = (double *)(base + pl.off_hval);
    BB[b].pass = (uint8_t *)(base + pl.off_pass);
    BB[b].cap = pl.cap;
    if (P.cut_first) {
      BB[b].col = (int *)(base + pl.off_col);
      BB[b].orig = (int *)(base + pl.off_orig);
      BB[b].tcount = (int *)(base + pl.off_tcount);
      BB[b].toff = (int *)(base + pl.off_toff);
      BB[b].dcount = (int *)(base + pl.off_dcount);
    }
    if (pl.defer_hist) BB[b].wev = (double *)(base + pl.off_wev);
  }
  ChunkParams C;
  C.P = PG;
  CUtensorMap maps[2];
  const CUtensorMap *mp[2] = {nullptr, nullptr};
  if constexpr (sizeof(R) == 4) {
    const bool staged = with_form<N, R>(pl.form, [](auto K) { return decltype(K)::staged; });
    if (staged) {
      for (int b = 0; b < (pl.overlap ? 2 : 1); ++b) {
        if ((e = encode_rows_map(&maps[b], BB[b].in, InRows<N - 1>::rows, pl.cap)) != cudaSuccess) return e;
        mp[b] = &maps[b];
      }
    }
  }
  if (pl.overlap && ov) {
    // K1 of chunk c+1 (caller's stream) runs while K2 of chunk c (aux stream)
    // does; buffer c % 2 is reused only after K2 of chunk c-2 is done.
    cudaStream_t a = ov->aux;
    if ((e = cudaEventRecord(ov->fork, s)) != cudaSuccess || (e = cudaStreamWaitEvent(a, ov->fork, 0)) != cudaSuccess)
      return e;
    int c = 0;
    for (uint64_t off = 0; off < P.n_events; off += (uint64_t)pl.cap, ++c) {
      const int b = c & 1;
      C.chunk_first = off;
      C.count = (int)std::min<uint64_t>((uint64_t)pl.cap, P.n_events - off);
      if (c >= 2 && (e = cudaStreamWaitEvent(s, ov->k2done[b], 0)) != cudaSuccess) return e;
      if (hook) (*hook)(STAGE_KIN, true, s);
      if ((e = launch_kin<N, R>(C, BB[b], pl.kin_smem, s)) != cudaSuccess) return e;
      if (hook) (*hook)(STAGE_KIN, false, s);
      if ((e = cudaEventRecord(ov->k1done[b], s)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(a, ov->k1done[b], 0)) != cudaSuccess) return e;
      if (hook) (*hook)(STAGE_AMP, true, a);
      e = with_form<N, R>(pl.form,
                          [&](auto K) { return decltype(K)::launch(C, BB[b], partials, pl.grid, pl.smem, a, mp[b]); });
      if (e != cudaSuccess) return e;
      if (hook) (*hook)(STAGE_AMP, false, a);
      if ((e = cudaEventRecord(ov->k2done[b], a)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(ov->join, a)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(s, ov->join, 0);
  }
  if (pl.form == K2_FUSED) {  // one warp-specialised launch per chunk, no kinematics launch
    for (uint64_t off = 0; off < P.n_events; off += (uint64_t)pl.cap) {
      C.chunk_first = off;
      C.count = (int)std::min<uint64_t>((uint64_t)pl.cap, P.n_events - off);
      if (hook) (*hook)(STAGE_AMP, true, s);
      e = with_form<N, R>(pl.form,
                          [&](auto K) { return decltype(K)::launch(C, BB[0], partials, pl.grid, pl.smem, s, nullptr); });
      if (e != cudaSuccess) return e;
      if (hook) (*hook)(STAGE_AMP, false, s);
    }
    return cudaSuccess;
  }
  const ChunkBuf<R> &B = BB[0];
  // deferred histogram: the amplitude kernel adds only the sums to rows that
  // keep the histogram's columns (hist_bins < 0)
  ChunkParams CK = C;
  if (pl.defer_hist) CK.P.hist_bins = -P.hist_bins;
  for (uint64_t off = 0; off < P.n_events; off += (uint64_t)pl.cap) {
    C.chunk_first = CK.chunk_first = off;
    C.count = CK.count = (int)std::min<uint64_t>((uint64_t)pl.cap, P.n_events - off);
    if (hook) (*hook)(STAGE_KIN, true, s);
    if ((e = launch_kin<N, R>(C, B, pl.kin_smem, s)) != cudaSuccess) return e;
    if (hook) (*hook)(STAGE_KIN, false, s);
    if (hook) (*hook)(STAGE_AMP, true, s);  // the amplitude stage includes the deferred histogram
    e = with_form<N, R>(pl.form,
                        [&](auto K) { return decltype(K)::launch(CK, B, partials, pl.grid, pl.smem, s, mp[0]); });
    if (e != cudaSuccess) return e;
    if (pl.defer_hist) {
      hist_chunk_kernel<kBlock><<<pl.grid, kBlock, EpiSmem<kBlock>::bytes(P.hist_bins), s>>>(C, B.wev, B.hval, B.pass,
                                                                                            partials);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (hook) (*hook)(STAGE_AMP, false, s);
  }
  return cudaSuccess;
}

}  // namespace tess
