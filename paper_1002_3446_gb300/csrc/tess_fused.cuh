// Warp-specialised one-kernel event path (FP32 currents, double-float
// kinematics, sampled helicities, n = 4..6): each block runs a kinematics
// warpgroup (threads 0..127) and an amplitude warpgroup (threads 128..255)
// that pass tiles of 128 events through a two-stage ring in shared memory.
//
// The two-kernel pipeline writes every event's amplitude inputs and factors
// (225 B at n = 6) to a chunk buffer in HBM and reads them back in a second
// launch, and each kernel alone is bound by instruction issue with idle issue
// slots of its own kind (the kinematics kernel on instruction fetch and
// dependent-issue stalls, the amplitude kernel on the input loads).  Here both
// kinds of work are resident on every SM at once, the hand-over stays on the
// chip, and one launch covers the call.
//
// Stages (Sec. 3's per-event steps, in order): the kinematics warpgroup runs
// the double-float kinematics of its tile (Philox draws, Rambo, cuts and
// observables, weight factor, polarisation basis, colour ordering and
// helicities) into stage b of the ring; the amplitude warpgroup takes the
// tile, runs the Berends-Giele register form (the whole current table in
// registers, one thread per event) and the event epilogue (weight, outputs,
// block sums, histogram).  Hand-over with named barriers: FULL[b] (the
// kinematics warps arrive after writing stage b, the amplitude warps wait)
// and EMPTY[b] (the amplitude warps arrive after their last read of stage b,
// the kinematics warps wait before refilling it).  Both warpgroups walk the
// same tile sequence (tile blockIdx.x + k gridDim.x), and the amplitude warps
// arrive on EMPTY[b] exactly when a refill of stage b follows, so every
// barrier phase has its 256 arrivals: the wait ends by construction.
//
// Registers: 2 blocks of 256 threads per SM launched at 128 registers a
// thread; the kinematics warpgroup gives 48 of them back (setmaxnreg.dec to
// 80, what the kinematics need) and the amplitude warpgroup takes them (inc
// to 176, the register form's table without spills).  80 + 176 = 2 x 128, so
// the increase is always satisfied from the block's own pool.  The host
// checks that the compiled kernel is launched at exactly 128 registers a
// thread and refuses the form otherwise.
#pragma once
#include "tess_pipeline.cuh"

namespace tess {

constexpr int kFusedThreads = 2 * kBlock;  // kinematics warpgroup + amplitude warpgroup
constexpr int kFusedLaunchRegs = 128;      // per thread at launch: 2 blocks per SM
constexpr int kFusedKinRegs = 80;
constexpr int kFusedAmpRegs = 176;
static_assert(kFusedKinRegs + kFusedAmpRegs == 2 * kFusedLaunchRegs, "register split within the block's pool");
static_assert(kFusedKinRegs % 8 == 0 && kFusedAmpRegs % 8 == 0, "setmaxnreg takes multiples of 8");

// Named barriers (0 is __syncthreads).  Each warp reconverges before one
// (bar.sync / bar.arrive are warp-aligned), and an arrive orders the
// arriving threads' shared-memory writes before the waiting threads' reads.
constexpr int kBarFull = 1;      // + stage
constexpr int kBarEmpty = 3;     // + stage
constexpr int kBarAmpOnly = 5;   // the amplitude warpgroup alone

template <int ID, int COUNT>
__device__ __forceinline__ void nbar_sync() {
  __syncwarp();
  asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}
template <int ID, int COUNT>
__device__ __forceinline__ void nbar_arrive() {
  __syncwarp();
  asm volatile("bar.arrive %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}
// Barrier ID + b of a ring stage b (compile-time barrier numbers).
template <int ID>
__device__ __forceinline__ void nbar_sync_stage(int b) {
  if (b)
    nbar_sync<ID + 1, kFusedThreads>();
  else
    nbar_sync<ID, kFusedThreads>();
}
template <int ID>
__device__ __forceinline__ void nbar_arrive_stage(int b) {
  if (b)
    nbar_arrive<ID + 1, kFusedThreads>();
  else
    nbar_arrive<ID, kFusedThreads>();
}

// One stage of the ring: the tile of amplitude inputs (InRows<L> rows of
// kBlock floats, the layout the kinematics scatter writes) and the events'
// factors.
template <int L>
struct FusedStage {
  static constexpr size_t tile_bytes = (size_t)InRows<L>::rows * kBlock * sizeof(float);
  static constexpr size_t bytes = tile_bytes + 3 * kBlock * sizeof(double) + kBlock;
  static_assert(tile_bytes % 16 == 0 && bytes % 16 == 0, "16-byte aligned stages");
  __device__ static ChunkBuf<float> buf(char *st) {
    ChunkBuf<float> B;
    B.in = (float *)st;
    B.efac = (double *)(st + tile_bytes);
    B.wfac = B.efac + kBlock;
    B.hval = B.wfac + kBlock;
    B.pass = (uint8_t *)(B.hval + kBlock);
    B.cap = kBlock;
    return B;
  }
};

template <int N>
struct FusedSmem {
  static constexpr int L = N - 1;
  static size_t bytes(int hist_bins) {
    return 2 * FusedStage<L>::bytes + 4 * kBlock * sizeof(double) + EpiSmem<kFusedThreads>::bytes(hist_bins);
  }
};

// Register-form amplitude of the event in column `col` of a tile (rows of
// kBlock floats).
template <int N>
__device__ __forceinline__ Cx<float> tile_amplitude(const float *tile, int col) {
  constexpr int L = N - 1;
  const float *in = tile + col;
  RV4<float> k[L];
  CV4<float> ev[L], e0;
#pragma unroll
  for (int a = 0; a < L; ++a) {
    load_k(in + (size_t)InRows<L>::k(a) * kBlock, (size_t)kBlock, k[a]);
    load_eps(in + (size_t)InRows<L>::eps(a) * kBlock, (size_t)kBlock, ev[a]);
  }
  load_eps(in + (size_t)InRows<L>::eps0 * kBlock, (size_t)kBlock, e0);
  return bg_amplitude<float, L>(k, ev, e0);
}

// Block sums of the amplitude warpgroup (col = its thread's column) added to
// the block's partial row, as epi_flush does for a whole block.
__device__ __forceinline__ void fused_flush(const EpiSmem<kFusedThreads> &S, int nb2, const Accum<kFusedThreads> &A,
                                            double *red, double *partials, int hist_bins, int col) {
  red[0 * kBlock + col] = A.sw;
  red[1 * kBlock + col] = A.sw2;
  red[2 * kBlock + col] = (double)A.npass;
  red[3 * kBlock + col] = (double)A.nbad;
  nbar_sync<kBarAmpOnly, kBlock>();  // also orders every warp's last histogram adds before the sums below
  for (int s = kBlock / 2; s > 0; s >>= 1) {
    if (col < s) {
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q * kBlock + col] += red[q * kBlock + col + s];
    }
    nbar_sync<kBarAmpOnly, kBlock>();
  }
  double *row = partials + (size_t)blockIdx.x * partial_stride(hist_bins);
  if (col < 4) row[col] += red[col * kBlock];
  for (int i = col; i < 2 * nb2; i += kBlock) row[kPartialHead + i] += epi_hist_sum(S, nb2, i);
}

// The chunk's events [C.chunk_first, + C.count) of the call; partial row
// blockIdx.x receives the block's sums (chunks run in order on one stream).
template <int N>
__global__ void __launch_bounds__(kFusedThreads, 2) fused_kernel(const __grid_constant__ ChunkParams C,
                                                                 double *partials) {
  static_assert(N >= 4 && N <= 6, "register form within 176 registers");
  constexpr int L = N - 1;
  using St = FusedStage<L>;
  extern __shared__ __align__(128) char fused_smem[];
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  double *red = (double *)(fused_smem + 2 * St::bytes);  // [4][kBlock]
  const EpiSmem<kFusedThreads> ES(fused_smem + 2 * St::bytes + 4 * kBlock * sizeof(double), nb2);
  epi_init(ES, nb2);  // every warp zeroes its own copy (the kinematics warps' stay zero)
  __syncthreads();
  const int ntiles = (C.count + kBlock - 1) / kBlock;
  if (threadIdx.x < kBlock) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kFusedKinRegs));
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int b = it & 1;
      if (it >= 2) nbar_sync_stage<kBarEmpty>(b);  // the amplitude warps are done with stage b
      char *st = fused_smem + b * St::bytes;
      ChunkParams Ct = C;
      Ct.chunk_first = C.chunk_first + (uint64_t)t * kBlock;
      Ct.count = min(kBlock, C.count - t * kBlock);
      const ChunkBuf<float> B = St::buf(st);
      const int e = (int)threadIdx.x;
      if (e < Ct.count) kin_ds<N, false, false>(Ct, B, e, B.in, true);
      nbar_arrive_stage<kBarFull>(b);
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kFusedAmpRegs));
    const int col = (int)threadIdx.x - kBlock;
    Accum<kFusedThreads> A;
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int b = it & 1;
      char *st = fused_smem + b * St::bytes;
      nbar_sync_stage<kBarFull>(b);  // stage b holds tile t
      ChunkParams Ct = C;
      Ct.chunk_first = C.chunk_first + (uint64_t)t * kBlock;
      Ct.count = min(kBlock, C.count - t * kBlock);
      const ChunkBuf<float> B = St::buf(st);
      double w = 0.0;
      int bin = -1;
      if (col < Ct.count) {
        const Cx<float> amp = tile_amplitude<N>(B.in, col);
        finish_event<kFusedThreads, float>(Ct, B, col, amp2_of(amp), A, w, bin);
      }
      // stage b is refilled only if this block has a tile two steps on
      if (t + 2 * (int)gridDim.x < ntiles) nbar_arrive_stage<kBarEmpty>(b);
      epi_tile<kFusedThreads>(ES, nb2, w, bin);
    }
    fused_flush(ES, nb2, A, red, partials, C.P.hist_bins, col);
  }
}

}  // namespace tess
