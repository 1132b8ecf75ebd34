// Host side of the persistent batched form (tess_persist.cuh): shared-memory
// sizing, occupancy-sized grid, and the launch of the persistent kernel and
// the fold.
#include <algorithm>

#include "tess_persist.cuh"

namespace tess {

constexpr int kFoldThreads = 64;

// Block (q, p): column q of process p's tile rows, each thread over the rows
// t, t + kFoldThreads, ... with compensation, then a fixed-shape compensated
// tree (deterministic); folded into the caller's accumulators with their own
// compensation terms.
__device__ __forceinline__ void persist_comp_add(double &s, double &c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

__global__ void __launch_bounds__(kFoldThreads) persist_fold_kernel(const __grid_constant__ PersistFold F) {
  const int p = blockIdx.y, q = blockIdx.x, t = threadIdx.x;
  const int hb = F.hist_bins[p];
  const int nb2 = hb > 0 ? hb + 2 : 0;
  if (q >= kPartialHead + 2 * nb2) return;  // uniform per block
  const int stride = partial_stride(hb);
  double s = 0.0, c = 0.0;
  for (int r = t; r < F.tiles[p]; r += kFoldThreads) persist_comp_add(s, c, F.tile_sums[p][(size_t)r * stride + q]);
  __shared__ double ss[kFoldThreads], cc[kFoldThreads];
  ss[t] = s;
  cc[t] = c;
  __syncthreads();
  for (int w = kFoldThreads / 2; w > 0; w >>= 1) {
    if (t < w) {
      double a = ss[t], ac = cc[t];
      persist_comp_add(a, ac, ss[t + w]);
      ss[t] = a;
      cc[t] = ac + cc[t + w];
    }
    __syncthreads();
  }
  if (t != 0) return;
  const double tot = ss[0] + cc[0];
  double *acc = F.acc[p], *hist = F.hist[p];
  if (q == 0 || q == 1) {
    double hs = acc[q], hc = acc[4 + q];
    persist_comp_add(hs, hc, tot);
    acc[q] = hs;
    acc[4 + q] = hc;
    if (q == 0) acc[3] += (double)F.n_events[p];
  } else if (q == 2) {
    acc[2] += tot;
  } else if (q == 3) {
    acc[6] += tot;
  } else if (q == 4) {
    acc[7] += tot;
  } else {
    const int h = q - kPartialHead;
    double hs = hist[h], hc = hist[2 * nb2 + h];
    persist_comp_add(hs, hc, tot);
    hist[h] = hs;
    hist[2 * nb2 + h] = hc;
  }
}


// Floats of the input tile for processes up to nmax gluons.
int persist_tile_floats(int nmax) {
  switch (nmax) {
    case 4: return InRows<3>::rows * kBlock;
    case 5: return InRows<4>::rows * kBlock;
    case 6: return InRows<5>::rows * kBlock;
    case 7: return InRows<6>::rows * kBlock;
    case 8: return InRows<7>::rows * kBlock;
    case 9: return InRows<8>::rows * kBlock;
    case 10: return InRows<9>::rows * kBlock;
    case 11: return InRows<10>::rows * kBlock;
    default: return InRows<11>::rows * kBlock;
  }
}

template <int NMAX, int MINB>
static cudaError_t persist_run(const PersistParams &Q, const PersistFold &F, int tile_floats, int max_hist_bins,
                               int sm_count, cudaStream_t s, int *grid_out) {
  const size_t smem = PersistSmem::bytes(tile_floats, max_hist_bins);
  cudaError_t e = allow_max_smem((const void *)persist_kernel<NMAX, MINB>);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_kernel<NMAX, MINB>, kBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::max(1, std::min(Q.items, sm_count * per_sm));
  if (grid_out) *grid_out = grid;
  if ((e = cudaMemsetAsync(Q.counter, 0, sizeof(int), s)) != cudaSuccess) return e;
  persist_kernel<NMAX, MINB><<<grid, kBlock, smem, s>>>(Q, tile_floats);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int cols = 0;
  for (int p = 0; p < Q.nproc; ++p) cols = std::max(cols, partial_stride(F.hist_bins[p]));
  persist_fold_kernel<<<dim3(cols, Q.nproc), kFoldThreads, 0, s>>>(F);
  return cudaGetLastError();
}

// The persistent kernel is built for two ranges of n: up to 8 (register
// forms only, no local-memory tables) and up to 12.
cudaError_t persist_launch(const PersistParams &Q, const PersistFold &F, int nmax, int max_hist_bins, int sm_count,
                           cudaStream_t s, int *grid_out) {
  const int tile_floats = persist_tile_floats(nmax);
  // three resident blocks per SM (168 registers, some spilled in the larger
  // forms): measured best for the gg -> 2..10 g batch against two (255
  // registers) and four (128)
  if (nmax <= 8) return persist_run<8, 3>(Q, F, tile_floats, max_hist_bins, sm_count, s, grid_out);
  return persist_run<12, 3>(Q, F, tile_floats, max_hist_bins, sm_count, s, grid_out);
}

}  // namespace tess
