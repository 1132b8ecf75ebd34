// Instantiations of the gradient and draws kernels, n = 9..10.
#include "tess_grad_pair.cuh"

namespace tess {

cudaError_t launch_grad_b(int n, bool fp64, const GradParams &G, void *ws, cudaStream_t s,
                           const GradStreams &gs) {
  switch (n) {
    case 9: return launch_grad_n<9>(fp64, G, ws, s, gs);
    case 10: return launch_grad_n<10>(fp64, G, ws, s, gs);
    default: return cudaErrorInvalidValue;
  }
}

size_t grad_workspace_b(int n, uint64_t n_events, size_t chunk_bytes) {
  switch (n) {
    case 9: return grad_workspace_bytes<9>(n_events, chunk_bytes);
    case 10: return grad_workspace_bytes<10>(n_events, chunk_bytes);
    default: return 0;
  }
}

cudaError_t launch_draws_b(int n, const EventParams &P, double *u, uint32_t *hel, uint8_t *order,
                               cudaStream_t s) {
  const unsigned blocks = (unsigned)((P.n_events + kBlock - 1) / kBlock);
  switch (n) {
    case 9:
      draws_kernel<9><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    case 10:
      draws_kernel<10><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tess
