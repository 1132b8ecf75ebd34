// Instantiations of the gradient and draws kernels, n = 4..8.
#include "tess_grad.cuh"

namespace tess {

cudaError_t launch_grad_a(int n, bool fp64, const GradParams &G, cudaStream_t s) {
  const unsigned blocks = (unsigned)((G.n_events + kBlock - 1) / kBlock);
  switch (n) {
    case 4:
      if (fp64)
        grad_kernel<4, double><<<blocks, kBlock, 0, s>>>(G);
      else
        grad_kernel<4, float><<<blocks, kBlock, 0, s>>>(G);
      return cudaGetLastError();
    case 5:
      if (fp64)
        grad_kernel<5, double><<<blocks, kBlock, 0, s>>>(G);
      else
        grad_kernel<5, float><<<blocks, kBlock, 0, s>>>(G);
      return cudaGetLastError();
    case 6:
      if (fp64)
        grad_kernel<6, double><<<blocks, kBlock, 0, s>>>(G);
      else
        grad_kernel<6, float><<<blocks, kBlock, 0, s>>>(G);
      return cudaGetLastError();
    case 7:
      if (fp64)
        grad_kernel<7, double><<<blocks, kBlock, 0, s>>>(G);
      else
        grad_kernel<7, float><<<blocks, kBlock, 0, s>>>(G);
      return cudaGetLastError();
    case 8:
      if (fp64)
        grad_kernel<8, double><<<blocks, kBlock, 0, s>>>(G);
      else
        grad_kernel<8, float><<<blocks, kBlock, 0, s>>>(G);
      return cudaGetLastError();
    default: return cudaErrorInvalidValue;
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
