// dg_probe.cu -- measured FMA throughput of the GPU (the denominator of the FP64/FP32 rooflines).
// Independent FMA chains per thread, grid a multiple of the SM count, bounded iteration count.
#include <cuda_runtime.h>

#include "../../include/dg.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T *sink, int iters, T a, T b) {
  T x0 = (T)threadIdx.x * (T)1e-3, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
  T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == (T)-1234.5) sink[threadIdx.x] = s;  // keeps the chains live; practically never taken
}

template <typename T>
dg_status run(cudaStream_t st, int iters, double *flops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  T *sink = nullptr;
  if (cudaMalloc(&sink, 256 * sizeof(T)) != cudaSuccess) return DG_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8;
  k_fma_chains<T><<<blocks, 256, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, 256, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return DG_ERR_CUDA;
  *flops = 2.0 * 32.0 * (double)iters * blocks * 256.0 / (best * 1e-3);
  return DG_OK;
}

}  // namespace

extern "C" dg_status dg_probe_fma(int kind, void *cuda_stream, double *flops) {
  if (!flops || (kind != 0 && kind != 1)) return DG_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return kind == 0 ? run<double>(st, 256, flops) : run<float>(st, 8192, flops);
}
