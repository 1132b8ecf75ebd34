// Batched mixed multiplicities in one persistent launch.
//
// Work items are (process, tile of kBlock events); a resident block takes the
// next item from one atomic counter (no block ever waits on another), runs the
// whole event path of the tile -- double-float kinematics into a shared-memory
// tile of amplitude inputs, the Berends-Giele amplitude, the event epilogue --
// and writes the tile's sums to the tile's own row of partial sums, which a
// second kernel folds per process in tile order (so the sums do not depend on
// which block took which tile).  Items are numbered from the process with the
// most gluons down, so the longest tiles are handed out first and the short
// ones fill the tail (Sec. 3: kernel start-up is a significant part of the
// time when the kernel is short, as at n = 4; here one launch serves every
// multiplicity).
//
// Per n the amplitude uses the thread-per-event forms that need no shared
// table: the register form (the whole current table in registers) up to n = 8
// and the loop form (table in the thread's local memory) above.  One launch
// has one shape, so its shared memory and registers are those of the largest
// n it can meet (the input tile of that n, the register form of n = 8); the
// per-n pipelines, each launched with its own tuned shape, are the
// comparison this form is measured against.
#pragma once
#include "tess_pipeline.cuh"

namespace tess {

constexpr int kPersistMaxProc = 16;

struct PersistProc {
  EventParams P;       // launch constants of the process (its per-event outputs included)
  double *tile_sums;   // [tiles][partial_stride(P.hist_bins)]
  int n;               // total gluons
  int tiles;           // ceil(n_events / kBlock)
  int first_item;      // its items are [first_item, first_item + tiles)
};

struct PersistParams {
  PersistProc proc[kPersistMaxProc];
  int nproc;
  int items;     // total work items
  int *counter;  // next item (zeroed before the launch)
};

// Amplitude of the event in column `col` of the input tile (rows of kBlock).
template <int N>
__device__ __forceinline__ Cx<float> persist_amplitude(const float *tile, int col) {
  constexpr int L = N - 1;
  const float *in = tile + col;
  if constexpr (N <= 8) {
    RV4<float> k[L];
    CV4<float> ev[L], e0;
#pragma unroll
    for (int a = 0; a < L; ++a) {
      load_k(in + (size_t)InRows<L>::k(a) * kBlock, (size_t)kBlock, k[a]);
      load_eps(in + (size_t)InRows<L>::eps(a) * kBlock, (size_t)kBlock, ev[a]);
    }
    load_eps(in + (size_t)InRows<L>::eps0 * kBlock, (size_t)kBlock, e0);
    return bg_amplitude<float, L>(k, ev, e0);
  } else {
    BGLoop<float, L> bg;
    CV4<float> e0;
#pragma unroll 1
    for (int a = 0; a < L; ++a) {
      const int X = BGLoop<float, L>::tri(a, a);
      load_k(in + (size_t)InRows<L>::k(a) * kBlock, (size_t)kBlock, bg.K[X]);
      load_eps(in + (size_t)InRows<L>::eps(a) * kBlock, (size_t)kBlock, bg.J[X]);
    }
    load_eps(in + (size_t)InRows<L>::eps0 * kBlock, (size_t)kBlock, e0);
    return bg.run(e0);
  }
}

// Shared memory of the persistent kernel for processes up to n = nmax: the
// input tile of the largest, the tile's factors, and the epilogue scratch.
struct PersistSmem {
  float *tile;
  double *efac, *wfac, *hval, *red;
  uint8_t *pass;
  char *epi;
  __host__ __device__ static size_t tile_bytes(int tile_floats) {
    return ((size_t)tile_floats * sizeof(float) + 15) & ~(size_t)15;
  }
  __device__ PersistSmem(char *base, int tile_floats) {
    tile = (float *)base;
    efac = (double *)(base + tile_bytes(tile_floats));
    wfac = efac + kBlock;
    hval = wfac + kBlock;
    red = hval + kBlock;  // [4][kBlock] block reduction of the tile's sums
    pass = (uint8_t *)(red + 4 * kBlock);
    epi = (char *)(pass + kBlock);
  }
  static size_t bytes(int tile_floats, int max_hist_bins) {
    return tile_bytes(tile_floats) + 7 * kBlock * sizeof(double) + kBlock + EpiSmem<kBlock>::bytes(max_hist_bins);
  }
};

// One tile of process pp: kinematics, amplitudes, epilogue, and the tile's
// row of partial sums (written, not accumulated: every row belongs to one
// tile).
template <int N>
__device__ __forceinline__ void persist_tile(const PersistProc &pp, int t, const PersistSmem &S) {
  ChunkParams C;
  C.P = pp.P;
  C.chunk_first = (uint64_t)t * kBlock;
  C.count = (int)min((uint64_t)kBlock, pp.P.n_events - C.chunk_first);
  ChunkBuf<float> B;
  B.in = S.tile;
  B.cap = kBlock;
  B.efac = S.efac;
  B.wfac = S.wfac;
  B.hval = S.hval;
  B.pass = S.pass;
  const int e = (int)threadIdx.x;
  const bool live = e < C.count;
  if (live) kin_ds<N, false, false>(C, B, e, S.tile, true);
  __syncthreads();
  const int nb2 = C.P.hist_bins > 0 ? C.P.hist_bins + 2 : 0;
  EpiSmem<kBlock> ES(S.epi, nb2);
  epi_init(ES, nb2);
  Accum<kBlock> A;
  double w = 0.0;
  int bin = -1;
  if (live) {
    const Cx<float> amp = persist_amplitude<N>(S.tile, e);
    finish_event<kBlock, float>(C, B, e, amp2_of(amp), A, w, bin);
  }
  __syncthreads();  // hw zeroed before epi_tile adds (no barrier there without a histogram)
  epi_tile<kBlock>(ES, nb2, w, bin);
  __syncthreads();
  // the tile's row: block sums of (w, w^2, n_pass, n_nonfinite), stall count 0, then the bins
  double *red = S.red;
  red[0 * kBlock + threadIdx.x] = A.sw;
  red[1 * kBlock + threadIdx.x] = A.sw2;
  red[2 * kBlock + threadIdx.x] = (double)A.npass;
  red[3 * kBlock + threadIdx.x] = (double)A.nbad;
  __syncthreads();
  for (int s = kBlock / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q * kBlock + threadIdx.x] += red[q * kBlock + threadIdx.x + s];
    }
    __syncthreads();
  }
  double *row = pp.tile_sums + (size_t)t * partial_stride(C.P.hist_bins);
  if (threadIdx.x < 4) row[threadIdx.x] = red[threadIdx.x * kBlock];
  if (threadIdx.x == 4) row[4] = 0.0;
  for (int i = threadIdx.x; i < 2 * nb2; i += kBlock) row[kPartialHead + i] = epi_hist_sum(ES, nb2, i);
  __syncthreads();  // the tile and factors are reused by the next item
}

template <int NMAX, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) persist_kernel(const __grid_constant__ PersistParams Q,
                                                               int tile_floats) {
  extern __shared__ __align__(16) char persist_smem[];
  const PersistSmem S(persist_smem, tile_floats);
  __shared__ int item_s;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(Q.counter, 1);
    __syncthreads();
    const int item = item_s;
    __syncthreads();  // every thread has read item_s before thread 0 overwrites it
    if (item >= Q.items) break;
    int p = 0;
    while (p + 1 < Q.nproc && item >= Q.proc[p + 1].first_item) ++p;
    const PersistProc &pp = Q.proc[p];
    const int t = item - pp.first_item;
    switch (pp.n) {
      case 4: persist_tile<4>(pp, t, S); break;
      case 5: persist_tile<5>(pp, t, S); break;
      case 6: persist_tile<6>(pp, t, S); break;
      case 7: persist_tile<7>(pp, t, S); break;
      case 8: persist_tile<8>(pp, t, S); break;
      case 9: if constexpr (NMAX >= 9) persist_tile<9>(pp, t, S); break;
      case 10: if constexpr (NMAX >= 10) persist_tile<10>(pp, t, S); break;
      case 11: if constexpr (NMAX >= 11) persist_tile<11>(pp, t, S); break;
      case 12: if constexpr (NMAX >= 12) persist_tile<12>(pp, t, S); break;
      default: break;
    }
  }
}

// Fold of every process's tile rows, in tile order, into its acc / hist:
// block (q, p) sums column q of process p (as the per-call finalize does).
struct PersistFold {
  const double *tile_sums[kPersistMaxProc];
  double *acc[kPersistMaxProc];
  double *hist[kPersistMaxProc];
  int tiles[kPersistMaxProc];
  int hist_bins[kPersistMaxProc];
  uint64_t n_events[kPersistMaxProc];
};

}  // namespace tess
