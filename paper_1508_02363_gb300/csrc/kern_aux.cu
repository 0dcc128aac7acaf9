// Small helper kernels outside the solve's sweeps: the per-slot factors of E_k
// (Sec. 5.1) for a batch of k values, and the FP64 read-out of double-float fields.
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

// float -> double by bit manipulation on the integer pipes (exact, like the conversion
// instruction, which on GB300 occupies the small FP64 pipe): sign, exponent rebiased by
// 1023 - 127, mantissa shifted into place; zeros, subnormals, infinities and NaNs take
// the conversion instruction.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)b);
}

__global__ void k_dd_to_fp64(const cx<dd>* __restrict__ in, cx<double>* __restrict__ out, long long n) {
  // four independent 16-byte loads in flight per thread before the conversions; both
  // buffers 16-byte aligned
  const float4* src = reinterpret_cast<const float4*>(in);
  double2* dst = reinterpret_cast<double2*>(out);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = i0 + u * stride;
      if (i < n) v[u] = __ldg(src + i);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long i = i0 + u * stride;
      if (i < n)
        dst[i] = make_double2(f2d_bits(v[u].x) + f2d_bits(v[u].y), f2d_bits(v[u].z) + f2d_bits(v[u].w));
    }
  }
}
cudaError_t launch_dd_to_fp64(const void* in, cx<double>* out, long long n, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_dd_to_fp64<<<blocks, 256, 0, s>>>(reinterpret_cast<const cx<dd>*>(in), out, n);
  return cudaGetLastError();
}

}  // namespace dbar
