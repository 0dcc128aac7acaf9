// Small helper kernels outside the solve's sweeps: the per-slot factors of E_k
// (Sec. 5.1) for a batch of k values, the FP64 read-out of double-float fields,
// and a check of the bounded mbarrier wait the bulk-copy sweeps rely on.
#include <cuda_runtime.h>

#include "krylov.cuh"
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

// hi + lo (two floats) rounded to double, to nearest with ties to even, in integer
// arithmetic: the same result as f2d_bits(hi) + f2d_bits(lo), without the FP64 pipe (on
// GB300 a warp's FP64 add holds that narrow pipe for many cycles).  Both significands
// are placed in a 64-bit integer (the larger at bit 63's side, the other shifted, its
// dropped bits kept as a sticky flag), added or subtracted, and the sum is rounded to 53
// bits.  Zeros, subnormals and non-finite values take the FP64 add.
__device__ __forceinline__ double dd_sum_rn(float hi, float lo) {
  unsigned int uh = __float_as_uint(hi), ul = __float_as_uint(lo);
  if ((ul & 0x7fffffffu) == 0u) {  // lo = +-0: hi, or a zero whose sign the FP64 add would give
    if ((uh & 0x7fffffffu) == 0u) return ((uh & ul) >> 31) ? -0.0 : 0.0;
    return f2d_bits(hi);
  }
  const unsigned int eh = (uh >> 23) & 0xffu, el = (ul >> 23) & 0xffu;
  if (eh == 0u || el == 0u || eh == 0xffu || el == 0xffu) return f2d_bits(hi) + f2d_bits(lo);
  unsigned long long mh = (uh & 0x7fffffu) | 0x800000u, ml = (ul & 0x7fffffu) | 0x800000u;
  int Eh = (int)eh - 150, El = (int)el - 150;  // value = m 2^E
  unsigned int nh = uh >> 31, nl = ul >> 31;
  if (El > Eh || (El == Eh && ml > mh)) {  // the larger magnitude first
    const unsigned long long tm = mh; mh = ml; ml = tm;
    const int te = Eh; Eh = El; El = te;
    const unsigned int tn = nh; nh = nl; nl = tn;
  }
  const int d = Eh - El;
  const unsigned long long A = mh << 39;
  unsigned long long B = 0ull;
  bool sticky = false;
  if (d <= 39) {
    B = ml << (39 - d);
  } else if (d < 64) {
    B = ml >> (d - 39);
    sticky = (ml & ((1ull << (d - 39)) - 1ull)) != 0ull;
  } else {
    sticky = true;
  }
  unsigned long long S;
  if (nh == nl) {
    S = A + B;
  } else {
    S = A - B;
    if (sticky) S -= 1ull;  // the dropped fraction borrows one unit; it stays sticky
  }
  if (S == 0ull) return 0.0;
  int sh = 11 - __clzll((long long)S);  // bits below the 53 kept
  unsigned long long q;
  if (sh > 0) {
    const unsigned long long rem = S & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    q = S >> sh;
    if (rem > half || (rem == half && (sticky || (q & 1ull)))) ++q;
    if (q == (1ull << 53)) {
      q >>= 1;
      ++sh;
    }
  } else {
    q = S << (-sh);
  }
  const unsigned long long ef = (unsigned long long)(Eh - 39 + sh + 52 + 1023);
  return __longlong_as_double((long long)(((unsigned long long)nh << 63) | (ef << 52) | (q & ((1ull << 52) - 1ull))));
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
        dst[i] = make_double2(dd_sum_rn(v[u].x, v[u].y), dd_sum_rn(v[u].z, v[u].w));
    }
  }
}
cudaError_t launch_dd_to_fp64(const void* in, cx<double>* out, long long n, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_dd_to_fp64<<<blocks, 256, 0, s>>>(reinterpret_cast<const cx<dd>*>(in), out, n);
  return cudaGetLastError();
}

// One mbarrier wait of the kind the bulk-copy block update uses (mbarrier
// try_wait rounds, at most `rounds` of them).  complete = 1: a 16-byte bulk copy
// of src delivers the bytes the phase announces; complete = 0: the phase
// announces 16 bytes that no copy delivers, so the wait runs out.  out[0] = 1 if
// the phase completed, out[1] = the copied word, out[2] = rounds taken.  With a
// copy issued, a wait that runs out waits once more (bounded) for that copy to
// land before the CTA exits.
__global__ void k_wait_check(int complete, int rounds, const int4* __restrict__ src, int* __restrict__ out) {
  __shared__ __align__(16) int4 buf;
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_fence_init();
  mbar_expect_tx(&bar, (uint32_t)sizeof(int4));
  if (complete) bulk_g2s(&buf, src, (uint32_t)sizeof(int4), &bar);
  const uint32_t addr = smem_u32(&bar);
  int done = 0, i = 0;
  for (; i < rounds && !done; ++i) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr)
        : "memory");
  }
  if (!done && complete) mbar_wait(&bar, 0);  // drain the copy in flight
  out[0] = done;
  out[1] = done ? buf.x : 0;
  out[2] = i;
}
int wait_limit_rounds() { return kWaitLimit; }
cudaError_t launch_wait_check(int complete, int rounds, const int4* src, int* out, cudaStream_t s) {
  k_wait_check<<<1, 32, 0, s>>>(complete, rounds, src, out);
  return cudaGetLastError();
}

}  // namespace dbar
