// Instantiations of the gradient and draws kernels, n = 4..8.
#include "tess_grad_pair.cuh"

namespace tess {

cudaError_t launch_grad_a(int n, bool fp64, const GradParams &G, void *ws, cudaStream_t s,
                           const GradStreams &gs) {
  switch (n) {
    case 4: return launch_grad_n<4>(fp64, G, ws, s, gs);
    case 5: return launch_grad_n<5>(fp64, G, ws, s, gs);
    case 6: return launch_grad_n<6>(fp64, G, ws, s, gs);
    case 7: return launch_grad_n<7>(fp64, G, ws, s, gs);
    case 8: return launch_grad_n<8>(fp64, G, ws, s, gs);
    default: return cudaErrorInvalidValue;
  }
}

size_t grad_workspace_a(int n, uint64_t n_events, size_t chunk_bytes) {
  switch (n) {
    case 4: return grad_workspace_bytes<4>(n_events, chunk_bytes);
    case 5: return grad_workspace_bytes<5>(n_events, chunk_bytes);
    case 6: return grad_workspace_bytes<6>(n_events, chunk_bytes);
    case 7: return grad_workspace_bytes<7>(n_events, chunk_bytes);
    case 8: return grad_workspace_bytes<8>(n_events, chunk_bytes);
    default: return 0;
  }
}

cudaError_t launch_draws_a(int n, const EventParams &P, double *u, uint32_t *hel, uint8_t *order,
                               cudaStream_t s) {
  const unsigned blocks = (unsigned)((P.n_events + kBlock - 1) / kBlock);
  switch (n) {
    case 4:
      draws_kernel<4><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    case 5:
      draws_kernel<5><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    case 6:
      draws_kernel<6><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    case 7:
      draws_kernel<7><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    case 8:
      draws_kernel<8><<<blocks, kBlock, 0, s>>>(P, u, hel, order);
      return cudaGetLastError();
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tess
