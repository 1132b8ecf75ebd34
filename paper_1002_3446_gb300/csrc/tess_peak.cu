// Arithmetic-peak probes: the denominators of the amplitude kernels'
// rooflines, measured on the GPU at hand (at whatever SM clock it runs)
// instead of taken from unit counts.
//
// Each thread runs a fixed number of independent fused multiply-add chains
// (enough in flight to cover the pipe latency at full occupancy): scalar FP32
// (fma.rn.f32), packed FP32 pairs (fma.rn.f32x2, two lanes of work per
// instruction) and FP64 (fma.rn.f64).  The chains are inline PTX so the
// compiler keeps every operation; the results feed a sink that is written
// only for an impossible value, so no memory is needed.  Loops are bounded.
#include <cstdint>
#include <cuda_runtime.h>

#include "tess.h"

namespace tess {

static __device__ float g_peak_sink;

constexpr int kPeakThreads = 512;
constexpr int kPeakBlocksPerSm = 4;  // 2048 threads per SM

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads) peak_kernel(int iters, float s) {
  float r = 0.f;
  if (KIND == TESS_PEAK_FP32) {
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = s + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 16; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(acc[i]) : "f"(s), "f"(s));
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) r += acc[i];
  } else if (KIND == TESS_PEAK_FP32X2) {
    uint64_t acc[8];
    const uint64_t x = ((uint64_t)__float_as_uint(0.5f * s) << 32) | __float_as_uint(s);
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = x + (uint64_t)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i) asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(acc[i]) : "l"(x));
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) r += __uint_as_float((uint32_t)acc[i]) + __uint_as_float((uint32_t)(acc[i] >> 32));
  } else {
    double acc[8];
    const double d = (double)s;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = d + (double)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 8; ++i) asm volatile("fma.rn.f64 %0, %0, %1, %1;" : "+d"(acc[i]) : "d"(d));
    }
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += acc[i];
    r = (float)t;
  }
  if (r == -1.2345e-37f) g_peak_sink = r;  // never taken for the inputs used; keeps the chains live
}

// Best of `reps` timed launches (after one warm-up) of probe `kind` on
// `sms` SMs' worth of blocks; *flop receives the FLOPs of one launch (an
// FMA counts 2 per lane: f32x2 does 2 lanes' worth per instruction).
cudaError_t peak_probe(int kind, int sms, int reps, cudaStream_t s, float *best_ms, double *flop) {
  const int blocks = sms * kPeakBlocksPerSm;
  const int iters = kind == TESS_PEAK_FP64 ? 256 : 8192;
  const double fma_per_iter = kind == TESS_PEAK_FP64 ? 8.0 : 16.0;
  *flop = 2.0 * fma_per_iter * iters * (double)blocks * kPeakThreads;
  auto launch = [&]() {
    if (kind == TESS_PEAK_FP32)
      peak_kernel<TESS_PEAK_FP32><<<blocks, kPeakThreads, 0, s>>>(iters, 1.0f);
    else if (kind == TESS_PEAK_FP32X2)
      peak_kernel<TESS_PEAK_FP32X2><<<blocks, kPeakThreads, 0, s>>>(iters, 1.0f);
    else
      peak_kernel<TESS_PEAK_FP64><<<blocks, kPeakThreads, 0, s>>>(iters, 1.0f);
    return cudaGetLastError();
  };
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = launch();
  float best = 1e30f;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(a, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  *best_ms = best;
  return e;
}

}  // namespace tess
