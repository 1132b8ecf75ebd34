// Instantiations of the gradient and draws kernels, n = 11..12.
#include "tess_grad_pair.cuh"

namespace tess {

cudaError_t launch_grad_c(int n, bool fp64, const GradParams &G, void *ws, cudaStream_t s,
                           const GradStreams &gs) {
  switch (n) {
    case 11: return launch_grad_n<11>(fp64, G, ws, s, gs);
    case 12: return launch_grad_n<12>(fp64, G, ws, s, gs);
    default: return cudaErrorInvalidValue;
  }
}

size_t grad_workspace_c(int n, uint64_t n_events, size_t chunk_bytes) {
  switch (n) {
    case 11: return grad_workspace_bytes<11>(n_events, chunk_bytes);
    case 12: return grad_workspace_bytes<12>(n_events, chunk_bytes);
    default: return 0;
  }
}

cudaError_t launch_draws_c(int n, const EventParams &P, double *u, uint32_t *hel, uint8_t *order,
                               cudaStream_t s) {
  const unsigned blocks = (unsigned)((P.n_events + kBlock - 1) / kBlock);
  switch (n) {
    case 11:
      draws_kernel<11><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    case 12:
      draws_kernel<12><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tess
