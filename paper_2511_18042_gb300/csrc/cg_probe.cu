// Throughput probe of the FP64 and FP32 fused multiply-add pipes, the
// denominators of the arithmetic roofline the benchmark reports: every
// thread runs eight independent FMA chains (no dependence between them, so
// the pipe, not latency, bounds the rate) on every SM, timed with CUDA
// events.  One FMA counts as two floating-point operations.  Built as its own
// library (libcgprobe.so): measurement infrastructure, not part of the solver.
#include <cuda_runtime.h>

#define CGP_API extern "C" __attribute__((visibility("default")))

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T b, T c) {
  T a0 = T(threadIdx.x) * T(1e-6), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == T(-1.25e30)) out[blockIdx.x] = s;  // never true: keeps the chains live
}

template <typename T>
int probe(double* flops_per_s, double* best_ms, int* sms) {
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -2;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -2;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, 256, 0) != cudaSuccess) return -2;
  int blocks = nsm * per_sm;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return -3;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int iters = sizeof(T) == 8 ? 4096 : 32768;
  T b = T(0.9999999), c = T(1e-7);
  k_fma_chains<T><<<blocks, 256>>>(out, iters, b, c);  // warm-up (clocks up)
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, 256>>>(out, iters, b, c);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return -2;
  double fmas = (double)blocks * 256.0 * 8.0 * iters;
  *flops_per_s = 2.0 * fmas / (best * 1e-3);
  *best_ms = best;
  *sms = nsm;
  return 0;
}

}  // namespace

// fp64 = 1: DFMA; 0: FFMA.  Returns 0, or a negative code on a CUDA error.
CGP_API int cgp_fma_peak(int fp64, double* flops_per_s, double* best_ms, int* sms) {
  return fp64 ? probe<double>(flops_per_s, best_ms, sms) : probe<float>(flops_per_s, best_ms, sms);
}
