// dg_noalloc.cu -- integral diagnostics without any memory allocation (dg_invariants_noalloc).
//
// Some callers cannot allocate device memory at the point where they want the diagnostics: a host
// framework whose caching allocator already holds nearly all of the device memory (a cudaMalloc
// there fails, or forces the pool to give memory back), or real-time and embedded callers whose
// rules forbid any allocation after start-up. This variant of the invariants reduction therefore keeps its per-chunk partial sums in
// a fixed, file-scope device array instead of context memory, and takes every input and output
// from the caller.
//
// The scratch array holds kMaxChunks rows of 8 partial sums (128 KiB); each chunk covers kChunk
// nodes, so at most kChunk * kMaxChunks = 33,554,432 nodes (n_elems * (N+1)^3) are accepted.
// Every GPU that loads the library keeps the array until the process exits. All calls share it:
// two calls whose kernels overlap on the GPU (e.g. on different streams) race on it. A call
// overwrites every row it later reads, so nothing has to start at zero; the array keeps the last
// call's partial sums.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_invariants_node.cuh"

#define DG_NOALLOC_CHUNK 16384LL   // nodes per chunk (one CTA)
#define DG_NOALLOC_MAX_CHUNKS 2048  // rows of the scratch array

// the scratch array: 2048 rows x 8 partial sums = 128 KiB on every device that loads the library
static __device__ __align__(256) double g_partials[DG_NOALLOC_MAX_CHUNKS * 8];

namespace {

constexpr long long kChunk = DG_NOALLOC_CHUNK;
constexpr int kMaxChunks = DG_NOALLOC_MAX_CHUNKS;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

std::mutex g_mutex;
double *g_scratch[kMaxDevices] = {nullptr};  // device address of g_partials, per device

struct Weights {
  double w[DG_NMAX + 1];
};

// One CTA per chunk of kChunk nodes: the 8 LGL-quadrature sums of the chunk into row `blockIdx.x`.
__global__ void __launch_bounds__(kThreads) k_invariants_chunks(int n, long long total, double gam, Weights wts,
                                                                const double *__restrict__ U,
                                                                const double *__restrict__ Ut,
                                                                const double *__restrict__ J,
                                                                double *__restrict__ scratch) {
  __shared__ double red[8][kThreads];
  const int nn = n * n, nnn = nn * n;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long begin = (long long)blockIdx.x * kChunk;
  const long long end = begin + kChunk < total ? begin + kChunk : total;
  for (long long t = begin + threadIdx.x; t < end; t += kThreads) {
    const long long e = t / nnn;
    const int node = (int)(t % nnn);
    const int i = node % n, j = (node / n) % n, k = node / nn;
    const double wq = wts.w[i] * wts.w[j] * wts.w[k] * J[t];
    const size_t b = (size_t)e * 5 * nnn + node;
    double Uv[5], Tv[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) { Uv[v] = U[b + (size_t)v * nnn]; Tv[v] = Ut[b + (size_t)v * nnn]; }
    invariants_node(gam, wq, Uv, Tv, acc);
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) red[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int st = kThreads / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
#pragma unroll
      for (int m = 0; m < 8; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 8) scratch[blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

// Sum the rows in chunk order (deterministic) into the caller's out[8].
__global__ void k_invariants_rows(const double *__restrict__ scratch, int rows, double *__restrict__ out) {
  const int c = threadIdx.x;
  if (c >= 8) return;
  double s = 0.0;
  for (int b = 0; b < rows; ++b) s += scratch[b * 8 + c];
  out[c] = s;
}

}  // namespace

extern "C" dg_status dg_invariants_noalloc(int N, int n_elems, double gamma, const double *U, const double *Ut,
                                           const double *J, double *out8, void *cuda_stream) {
  if (N < 1 || N > DG_NMAX || n_elems <= 0 || !U || !Ut || !J || !out8 || !(gamma > 1.0)) return DG_ERR_ARG;
  const long long n = N + 1;
  const long long total = (long long)n_elems * n * n * n;
  if (total > kChunk * kMaxChunks) return DG_ERR_UNSUPPORTED;  // beyond the fixed scratch array
  // an error left pending by earlier, unrelated work is its owner's to read: refuse without clearing it
  if (cudaPeekAtLastError() != cudaSuccess) return DG_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return DG_ERR_UNSUPPORTED;
  double *scratch = nullptr;
  {
    // once per device, with that device current: the device address of the scratch array
    std::lock_guard<std::mutex> lk(g_mutex);
    if (!g_scratch[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
        cudaGetLastError();
        return DG_ERR_CUDA;
      }
      g_scratch[dev] = static_cast<double *>(p);
    }
    scratch = g_scratch[dev];
  }
  DgTables t;  // LGL weights, built on the host stack
  if (dg_build_tables(N, &t) != 0) return DG_ERR_ARG;
  Weights wts;
  for (int i = 0; i <= DG_NMAX; ++i) wts.w[i] = i <= N ? t.w[i] : 0.0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int rows = (int)((total + kChunk - 1) / kChunk);
  // no error was pending above, so an error read here is one of these launches
  k_invariants_chunks<<<rows, kThreads, 0, st>>>((int)n, total, gamma, wts, U, Ut, J, scratch);
  if (cudaGetLastError() != cudaSuccess) return DG_ERR_CUDA;
  k_invariants_rows<<<1, 32, 0, st>>>(scratch, rows, out8);
  if (cudaGetLastError() != cudaSuccess) return DG_ERR_CUDA;
  return DG_OK;
}
