// Launch helpers shared by the per-precision instantiation units.
#pragma once
#include <algorithm>

#include "tess_kernels.cuh"

namespace tess {

inline size_t generate_smem(int hist_bins) {
  const int nb2 = hist_bins > 0 ? hist_bins + 2 : 0;
  return (size_t)(2 * nb2 + kBlock) * sizeof(double) + (size_t)kBlock * sizeof(int);
}

template <int N, typename R, bool SUM>
cudaError_t launch_event(const EventParams &P, double *partials, int grid, cudaStream_t s) {
  event_kernel<N, R, SUM><<<grid, kBlock, generate_smem(P.hist_bins), s>>>(P, partials);
  return cudaGetLastError();
}

// Grid of the fused kernel: enough blocks to fill every SM at the kernel's
// occupancy (a fixed function of the device and the kernel), capped by the
// number of tiles.
template <int N, typename R, bool SUM>
int event_grid(int sm_count, uint64_t n_events, int hist_bins) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, event_kernel<N, R, SUM>, kBlock,
                                                    generate_smem(hist_bins)) != cudaSuccess)
    per_sm = 1;
  per_sm = std::max(per_sm, 1);
  const uint64_t tiles = (n_events + kBlock - 1) / kBlock;
  const uint64_t full = (uint64_t)sm_count * (uint64_t)per_sm;
  return (int)std::max<uint64_t>(1, std::min(tiles, full));
}

template <int N, typename R>
cudaError_t launch_me2_t(uint64_t n_events, const double *k, const uint8_t *order, const uint32_t *hel,
                         double *me2, cudaStream_t s) {
  const uint64_t blocks = (n_events + kBlock - 1) / kBlock;
  me2_kernel<N, R><<<(unsigned)blocks, kBlock, 0, s>>>(n_events, k, order, hel, me2);
  return cudaGetLastError();
}

}  // namespace tess
