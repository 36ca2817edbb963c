// Reverse-mode (adjoint) kernels, FP64 instantiation.
#include "lbcad_adjoint.cuh"
template struct lbcad::LaunchAdj<double, false>;

namespace lbcad {
// The per-block partials of d/dzeta and d/dq0 of one reverse step, added to total[0..1]: thread
// t adds value t & 1 of the blocks t >> 1, t >> 1 + 256, ... (independent loads, a short chain),
// then a fixed pairing tree over the 256 partial sums of each value.  FP64 additions take about
// 60 cycles on this part, so a single chain over thousands of blocks took longer than the
// reverse step's own kernels.  The order is fixed: the result is deterministic.
constexpr int kAccumThreads = 512;
static __global__ void __launch_bounds__(kAccumThreads)
    k_adj_accum(const double* __restrict__ pgrad, int nblocks, double* __restrict__ total) {
  __shared__ double red[kAccumThreads];
  const int t = threadIdx.x, v = t & 1;
  double a = 0.0;
#pragma unroll 4
  for (int b = t >> 1; b < nblocks; b += kAccumThreads / 2) a += pgrad[2 * b + v];
  red[t] = a;
  __syncthreads();
  for (int h = kAccumThreads / 2; h >= 2; h >>= 1) {
    if (t < h) red[t] += red[t + h];
    __syncthreads();
  }
  if (t < 2) total[t] += red[t];
}
cudaError_t adj_accumulate(const double* pgrad, int nblocks, double* total, cudaStream_t s) {
  k_adj_accum<<<1, kAccumThreads, 0, s>>>(pgrad, nblocks, total);
  return cudaGetLastError();
}
}  // namespace lbcad
