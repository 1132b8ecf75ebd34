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

// Gauge check of Sec. 4 for caller-given kinematics (tess_gauge_ratio):
// |m|^2 of the ordering with the last leg's polarisation replaced by its
// momentum over its energy (current conservation: zero up to rounding), and
// the same with the polarisation itself; same inputs and units as me2_kernel.
template <typename R, int N>
__device__ __forceinline__ void gauge_amp2(const double (&kk)[N][4], double inv_rs, const int (&perm)[N], uint32_t hel,
                                           double &num, double &den) {
  constexpr int L = N - 1;
  double kp[N][4];
  int legp[N];
  gather_positions<N>(kk, perm, kp, legp);
  CV4<R> e0, ek, ep, em;
  {
    const double sg = legp[0] < 2 ? -1.0 : 1.0;
    polarisations<R>(sg * kp[0][1], sg * kp[0][2], sg * kp[0][3], ep, em);
    e0 = ((hel >> legp[0]) & 1u) ? em : ep;
    const double ie = 1.0 / fabs(kp[0][0]);
#pragma unroll
    for (int m = 0; m < 4; ++m) ek.c[m] = cx<R>(R(kp[0][m] * ie), R(0));
  }
  BGLoop<R, L> bg;
#pragma unroll
  for (int a = 0; a < L; ++a) {
    const int X = BGLoop<R, L>::tri(a, a);
#pragma unroll
    for (int m = 0; m < 4; ++m) bg.K[X].v[m] = R(kp[a + 1][m] * inv_rs);
    const double sg = legp[a + 1] < 2 ? -1.0 : 1.0;
    polarisations<R>(sg * kp[a + 1][1], sg * kp[a + 1][2], sg * kp[a + 1][3], ep, em);
    bg.J[X] = ((hel >> legp[a + 1]) & 1u) ? em : ep;
  }
  const Cx<R> an = bg.run(ek);  // run() rebuilds every multi-leg entry from the single legs
  const Cx<R> ad = bg.run(e0);
  num = (double)an.re * (double)an.re + (double)an.im * (double)an.im;
  den = (double)ad.re * (double)ad.re + (double)ad.im * (double)ad.im;
}

template <int N, typename R>
__global__ void __launch_bounds__(kBlock) gauge_kernel(uint64_t n_events, const double *__restrict__ k,
                                                       const uint8_t *__restrict__ order,
                                                       const uint32_t *__restrict__ hel, double *__restrict__ ratio) {
  const uint64_t e = (uint64_t)blockIdx.x * kBlock + threadIdx.x;
  if (e >= n_events) return;
  double kk[N][4];
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int m = 0; m < 4; ++m) kk[i][m] = k[(e * N + i) * 4 + m];
  int perm[N];
#pragma unroll
  for (int i = 0; i < N; ++i) perm[i] = order[e * N + i];
  const double s = 2.0 * (kk[0][0] * kk[1][0] - kk[0][1] * kk[1][1] - kk[0][2] * kk[1][2] - kk[0][3] * kk[1][3]);
  const double inv_rs = pow2_unit_inv(sqrt(fabs(s)));
  double num, den;
  gauge_amp2<R, N>(kk, inv_rs, perm, hel[e], num, den);
  ratio[e] = num / den;
}

template <int N, typename R>
cudaError_t launch_me2_t(uint64_t n_events, const double *k, const uint8_t *order, const uint32_t *hel,
                         double *me2, cudaStream_t s, bool gauge = false) {
  const uint64_t blocks = (n_events + kBlock - 1) / kBlock;
  if (gauge)
    gauge_kernel<N, R><<<(unsigned)blocks, kBlock, 0, s>>>(n_events, k, order, hel, me2);
  else
    me2_kernel<N, R><<<(unsigned)blocks, kBlock, 0, s>>>(n_events, k, order, hel, me2);
  return cudaGetLastError();
}

}  // namespace tess
