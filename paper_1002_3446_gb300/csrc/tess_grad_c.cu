// Instantiations of the gradient and draws kernels, n = 11..12.
#include "tess_grad.cuh"

namespace tess {

cudaError_t launch_grad_c(int n, bool fp64, const GradParams &G, cudaStream_t s) {
  const unsigned blocks = (unsigned)((G.n_events + kBlock - 1) / kBlock);
  switch (n) {
    case 11:
      if (fp64)
        grad_kernel<11, double><<<blocks, kBlock, 0, s>>>(G);
      else
        grad_kernel<11, float><<<blocks, kBlock, 0, s>>>(G);
      return cudaGetLastError();
    case 12:
      if (fp64)
        grad_kernel<12, double><<<blocks, kBlock, 0, s>>>(G);
      else
        grad_kernel<12, float><<<blocks, kBlock, 0, s>>>(G);
      return cudaGetLastError();
    default: return cudaErrorInvalidValue;
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
