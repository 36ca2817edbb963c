// Reverse-mode (adjoint) kernels, FP64 instantiation.
#include "lbcad_adjoint.cuh"
template struct lbcad::LaunchAdj<double, false>;

namespace lbcad {
static __global__ void k_adj_accum(const double* __restrict__ pgrad, int nblocks, double* __restrict__ total) {
  if (threadIdx.x < 2) {
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += pgrad[2 * b + threadIdx.x];
    total[threadIdx.x] += v;
  }
}
cudaError_t adj_accumulate(const double* pgrad, int nblocks, double* total, cudaStream_t s) {
  k_adj_accum<<<1, 32, 0, s>>>(pgrad, nblocks, total);
  return cudaGetLastError();
}
}  // namespace lbcad
