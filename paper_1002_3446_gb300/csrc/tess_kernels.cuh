// Kernels of the generator and their host-side launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tess_event.cuh"

namespace tess {

constexpr int kBlock = 128;       // threads (= events) per tile
constexpr int kPartialHead = 5;   // sum w, sum w^2, n_pass, n_nonfinite, n_stalled

// Workspace layout: one row of partials per block,
//   [sum w, sum w^2, n_pass, n_nonfinite, n_stalled, hist w (nb2), hist w^2 (nb2)].
// n_stalled counts blocks that gave up waiting for a staged input copy.
// hist_bins < 0: an amplitude kernel whose histogram (-hist_bins bins) a
// separate kernel fills; its rows keep the histogram's columns.
__host__ __device__ inline int partial_stride(int hist_bins) {
  const int h = hist_bins < 0 ? -hist_bins : hist_bins;
  return kPartialHead + (h > 0 ? 2 * (h + 2) : 0);
}

__device__ __forceinline__ int hist_bin(double v, double lo, double inv_w, int nb) {
  if (!(v >= lo)) return 0;
  const double t = (v - lo) * inv_w;
  if (!(t < (double)nb)) return nb + 1;
  return 1 + (int)t;
}

// Fused event kernel.  Each block walks tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...; each thread keeps FP64 running sums of its own events; the
// histogram of a tile is filled deterministically (each bin's thread scans
// the tile's (bin, w) pairs in order); at the end a fixed-shape tree sum
// writes the block's partial row.  Results are bit-reproducible for a given
// grid size.
template <int N, typename R, bool SUM>
__global__ void __launch_bounds__(kBlock) event_kernel(EventParams P, double *__restrict__ partials) {
  extern __shared__ double smem[];
  const int nb = P.hist_bins;
  const int nb2 = nb > 0 ? nb + 2 : 0;
  double *hw = smem;                             // [nb2]
  double *hw2 = smem + nb2;                      // [nb2]
  double *stage_w = smem + 2 * nb2;              // [kBlock]
  int *stage_b = (int *)(stage_w + kBlock);      // [kBlock]
  __shared__ double red[4][kBlock];
  for (int i = threadIdx.x; i < 2 * nb2; i += kBlock) smem[i] = 0.0;
  double sw = 0.0, sw2 = 0.0, npass = 0.0, nbad = 0.0;
  const uint64_t ntiles = (P.n_events + kBlock - 1) / kBlock;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t idx = tile * kBlock + threadIdx.x;
    double w = 0.0;
    int bin = -1;
    if (idx < P.n_events) {
      EventResult r = event<N, R, SUM>(P, P.first_event + idx);
      if (!isfinite(r.w)) {
        nbad += 1.0;
        r.w = 0.0;
      }
      if (P.weight) P.weight[idx] = r.w;
      if (P.me2) P.me2[idx] = r.me2;
      if (P.pass) P.pass[idx] = (uint8_t)r.pass;
      if (P.ht) P.ht[idx] = r.ht;
      if (P.ptlead) P.ptlead[idx] = r.ptlead;
      if (P.rmin) P.rmin[idx] = r.rmin;
      sw += r.w;
      sw2 += r.w * r.w;
      npass += (double)r.pass;
      w = r.w;
      if (nb > 0 && r.pass) {
        const double v = P.hist_obs == 0 ? r.ptlead : (P.hist_obs == 1 ? r.ht : r.rmin);
        bin = hist_bin(v, P.hist_lo, P.hist_inv_width, nb);
      }
    }
    if (nb > 0) {
      __syncthreads();
      stage_w[threadIdx.x] = w;
      stage_b[threadIdx.x] = bin;
      __syncthreads();
      for (int b = threadIdx.x; b < nb2; b += kBlock) {
        double a = 0.0, a2 = 0.0;
        for (int t = 0; t < kBlock; ++t) {
          if (stage_b[t] == b) {
            const double x = stage_w[t];
            a += x;
            a2 += x * x;
          }
        }
        hw[b] += a;
        hw2[b] += a2;
      }
    }
  }
  red[0][threadIdx.x] = sw;
  red[1][threadIdx.x] = sw2;
  red[2][threadIdx.x] = npass;
  red[3][threadIdx.x] = nbad;
  __syncthreads();
  for (int s = kBlock / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    }
    __syncthreads();
  }
  double *row = partials + (size_t)blockIdx.x * partial_stride(nb);
  if (threadIdx.x < 4) row[threadIdx.x] = red[threadIdx.x][0];
  if (threadIdx.x == 4) row[4] = 0.0;
  for (int i = threadIdx.x; i < 2 * nb2; i += kBlock) row[kPartialHead + i] = smem[i];
}

// Matrix element only, for caller-given kinematics.
template <int N, typename R>
__global__ void __launch_bounds__(kBlock) me2_kernel(uint64_t n_events, const double *__restrict__ k,
                                                     const uint8_t *__restrict__ order,
                                                     const uint32_t *__restrict__ hel, double *__restrict__ me2) {
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
  // momentum unit: the power of two nearest sqrt(s), s = 2 k_1.k_2
  const double s = 2.0 * (kk[0][0] * kk[1][0] - kk[0][1] * kk[1][1] - kk[0][2] * kk[1][2] - kk[0][3] * kk[1][3]);
  const double inv_rs = pow2_unit_inv(sqrt(fabs(s)));
  double a2 = ordered_amp2<R, N>(kk, inv_rs, perm, hel[e]);
  const double u2 = inv_rs * inv_rs;
#pragma unroll
  for (int i = 0; i < N - 4; ++i) a2 *= u2;
  me2[e] = a2 / (double)(1u << (N - 2));
}

}  // namespace tess
