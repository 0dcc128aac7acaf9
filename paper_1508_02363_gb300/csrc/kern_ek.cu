// Per-slot factors of E_k (Sec. 5.1) for a batch of k values, built on the device.
#include <cuda_runtime.h>

#include "launch.cuh"

namespace dbar {

// E_k = exp(conj(kz) - kz) = exp(-2i (k2 x + k1 y)) = ex(x) ey(y) on the grid
// x_j = L(-pi + 2 pi j/N) for nb values k = k[2s] + i k[2s+1] (Sec. 5.1), FP64:
// ex[s][j] = e^{-2i k2 x_j}, ey[s][j] = e^{-2i k1 x_j}.
__global__ void k_fill_ek(const double* __restrict__ k, int nb, int N, double L, cx<double>* __restrict__ ex,
                          cx<double>* __restrict__ ey) {
  const long long total = (long long)nb * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / N), j = (int)(i - (long long)s * N);
    const double x = L * (-M_PI + 2.0 * M_PI * (double)j / (double)N);
    double sn, cs;
    sincos(2.0 * k[2 * s + 1] * x, &sn, &cs);
    ex[i] = mkc(cs, -sn);
    sincos(2.0 * k[2 * s] * x, &sn, &cs);
    ey[i] = mkc(cs, -sn);
  }
}
cudaError_t launch_fill_ek(const double* k, int nb, int N, double L, cx<double>* ex, cx<double>* ey, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  const long long total = (long long)nb * N;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  k_fill_ek<<<blocks, 256, 0, s>>>(k, nb, N, L, ex, ey);
  return cudaGetLastError();
}

}  // namespace dbar
