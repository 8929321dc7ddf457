// dg_wall.cu -- dg_wall_model: the wall model of Sec. 3 on a batch of wall points (one thread each).
#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "dg_wall.cuh"

namespace {

__global__ void __launch_bounds__(256) k_wall_model(int n, const double *__restrict__ U, const double *__restrict__ h,
                                                    const double *__restrict__ nu, double uinf, double b, int vd,
                                                    double *__restrict__ utau, int *__restrict__ iters) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int it = 0;
  utau[i] = wall_utau<double>(U[i], h[i], nu[i], uinf, b, vd, it);
  if (iters) iters[i] = it;
}

}  // namespace

extern "C" dg_status dg_wall_model(int n, const double *U, const double *h, const double *nu, double uinf,
                                   double mainf, double gamma, double Pr, int van_driest, double *utau, int *iters,
                                   void *cuda_stream) {
  if (n < 0 || (n > 0 && (!U || !h || !nu || !utau)) || !(gamma > 1.0) || !(Pr > 0.0) || !(mainf >= 0.0))
    return DG_ERR_ARG;
  if (n == 0) return DG_OK;
  const double b = van_driest_b(mainf, gamma, Pr);
  k_wall_model<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(n, U, h, nu, uinf, b,
                                                                                     van_driest != 0, utau, iters);
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}
