// peaks.cu -- arithmetic-throughput probes for the roofline denominators of the bench
// (not part of the hybrid step).  Each thread runs eight independent FMA chains
// x <- x * a + b (a, b kernel arguments, so the chains cannot be folded), long enough that
// launch overhead is negligible, on a grid of resident blocks covering every SM; the result
// is written out so that no chain is dead code.  Throughput = 2 flops per FMA.
#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T a, T b, int iters, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(int device, int iters, double* tflops) {
  if (!tflops || iters < 1) return -1;
  if (cudaSetDevice(device) != cudaSuccess) return -3;
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -3;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, 256, 0) != cudaSuccess) return -3;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  T* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * 256 * sizeof(T)) != cudaSuccess) return -2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = T(0.999999), b = T(1e-6);
  k_fma_chains<T><<<blocks, 256>>>(a, b, iters / 8 + 1, out);  // warm-up
  float best = -1.f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, 256>>>(a, b, iters, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.f || ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || best <= 0.f) return -3;
  const double fmas = (double)blocks * 256.0 * (double)iters * 16.0 * 8.0;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return 0;
}

}  // namespace

// Best of five launches of the FMA-chain kernel in FP64 (DFMA) and FP32 (FFMA): dense
// arithmetic throughput in TFLOP/s on `device`.  Returns 0, or a negative code.
extern "C" int peak_fp64_tflops(int device, int iters, double* tflops) { return probe<double>(device, iters, tflops); }
extern "C" int peak_fp32_tflops(int device, int iters, double* tflops) { return probe<float>(device, iters, tflops); }

namespace {
// One thread runs a chain of dependent additions; cycles per addition from clock64.
template <typename T>
__global__ void k_add_chain(T a, int n, T* out, long long* cycles) {
  T x = a;
  const long long t0 = clock64();
  for (int i = 0; i < n; ++i) x = x + a;
  const long long t1 = clock64();
  *out = x;
  *cycles = t1 - t0;
}
template <typename T>
int latency(int device, double* cyc) {
  if (!cyc || cudaSetDevice(device) != cudaSuccess) return -3;
  T* out = nullptr;
  long long* c = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess || cudaMalloc(&c, sizeof(long long)) != cudaSuccess) return -2;
  long long h = 0;
  k_add_chain<T><<<1, 1>>>(T(1e-3), 4096, out, c);
  k_add_chain<T><<<1, 1>>>(T(1e-3), 4096, out, c);
  cudaError_t e = cudaMemcpy(&h, c, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(out);
  cudaFree(c);
  if (e != cudaSuccess) return -3;
  *cyc = (double)h / 4096.0;
  return 0;
}
}  // namespace

// Latency in SM clock cycles of one dependent FP64 (DADD) or FP32 (FADD) addition.
extern "C" int add_latency_fp64_cycles(int device, double* cycles) { return latency<double>(device, cycles); }
extern "C" int add_latency_fp32_cycles(int device, double* cycles) { return latency<float>(device, cycles); }
