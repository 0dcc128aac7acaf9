// Convolution regularisation of F^{-1}(S/xi) (Sec. 4.2, remark after eq.
// fourreg5a): G = S e^{-|xi|^2}, so
//   F^{-1}(S/xi) = F^{-1}(S (1 - e^{-|xi|^2})/xi) + (1/2pi) int F^{-1}(S)(z') W_0(z - z') d^2z'
// with W_0(w) = (i/w)(1 - e^{-|w|^2/4}).  The first term is smooth (0 at
// xi = 0) and goes through the raw inverse transforms of the pass kernels; the
// second is summed directly over every pair of grid points (trapezoidal rule
// of the box, area h^2 per point, h = 2 pi L/N): N^4 complex multiply-adds per
// field, the paper's "object in four real dimensions".
//
// GB300 mapping: the sum is a dense FP64 contraction with no reuse structure
// the tensor cores could take (FP64 tensor rates are far below the FP32 ones
// on this part), so it runs on the FP64 pipe from shared memory: each block
// owns a 32 x 32 tile of outputs of one field, and for each 32 x 32 tile of
// inputs stages the input values and the 63 x 63 window of the kernel table
// they need; a warp's lanes read consecutive window columns (no bank
// conflicts), the input value is a broadcast.  Four outputs per thread keep
// 16 FP64 FMAs in flight per pair of shared loads, so the FP64 pipe, not
// shared memory, is the bound.
#include <cuda_runtime.h>

#include "launch.cuh"

namespace dbar {

namespace {

constexpr int CT = 32;              // output and input tile edge
constexpr int CW = 2 * CT - 1;      // kernel window edge
constexpr int CWP = 2 * CT;         // window row pitch (elements)
constexpr int CONV_THREADS = 256;   // 8 warps; warp w owns tile rows w, w+8, w+16, w+24
constexpr int CONV_ROWS = CT / (CONV_THREADS / 32);
constexpr size_t CONV_SMEM = (size_t)(CW * CWP + CT * CT) * sizeof(cx<double>);

// field 2s   = sigma_s (-1)^{p1+p2} S (1 - e^{-|xi|^2}) / (xi 2 pi L^2)   (Mu, 0 at xi = 0)
// field 2s+1 = sigma_s (-1)^{p1+p2} S / (2 pi L^2)
// so that the raw inverse 2-D DFT of each is F_d^{-1} of S (1 - e^{-|xi|^2})/xi and of S.
__global__ void k_conv_split(const cx<double>* __restrict__ S, long long s_ss, const double* __restrict__ scale,
                             int scale_ss, const int* __restrict__ run, const cx<double>* __restrict__ Mu,
                             double inv2piL2, int N, cx<double>* __restrict__ out) {
  const int slot = blockIdx.y;
  if (run && !run[slot]) return;
  const long long n = (long long)N * N;
  const double sig = scale ? scale[(size_t)slot * scale_ss] : 1.0;
  const cx<double>* src = S + (size_t)slot * s_ss;
  cx<double>* o = out + (size_t)slot * 2 * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int p2 = (int)(i / N), p1 = (int)(i - (long long)p2 * N);
    const cx<double> v = cscale(src[i], sig);
    o[i] = cmul(v, Mu[i]);
    o[n + i] = cscale(v, ((p1 + p2) & 1) ? -inv2piL2 : inv2piL2);
  }
}

// h = u + sum_{y', x'} s[y'][x'] Kt[y - y' + N-1][x - x' + N-1] on one 32 x 32 output
// tile of one slot (u = field 2s, s = field 2s+1 of f).  Kt already carries h^2/(2 pi).
// MODE 0: out = h.  MODE 1: out = (2 pi L^2/N^2) E_k Q conj(h), the field the
// operator's forward transform takes (E_k = ex[x] ey[y] per slot).
template <int MODE>
__global__ void __launch_bounds__(CONV_THREADS, 2)
    k_conv_sum(const cx<double>* __restrict__ f, const cx<double>* __restrict__ Kt, int N,
               const int* __restrict__ run, const cx<double>* __restrict__ Q, long long q_ss,
               const cx<double>* __restrict__ ex, const cx<double>* __restrict__ ey, double sw,
               cx<double>* __restrict__ out, long long o_ss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<double>* win = reinterpret_cast<cx<double>*>(smem_raw);  // [CW][CWP]
  cx<double>* stile = win + CW * CWP;                          // [CT][CT]
  const int slot = blockIdx.y;
  if (run && !run[slot]) return;
  const long long n = (long long)N * N;
  const int nt = N / CT;
  const int ty0 = (blockIdx.x / nt) * CT, tx0 = (blockIdx.x % nt) * CT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const cx<double>* u = f + (size_t)slot * 2 * n;
  const cx<double>* s = u + n;
  const int KP = 2 * N;  // table row pitch
  double ar[CONV_ROWS], ai[CONV_ROWS];
#pragma unroll
  for (int r = 0; r < CONV_ROWS; ++r) ar[r] = ai[r] = 0.0;

  for (int iy0 = 0; iy0 < N; iy0 += CT) {
    for (int ix0 = 0; ix0 < N; ix0 += CT) {
      __syncthreads();  // the previous tile's readers are done
      // window row wr, column wc <-> table row wy + wr, column wx + wc with
      // wy = ty0 - iy0 + N - CT in [0, 2N - 2 - (CW - 1)] (likewise wx)
      const int wy = ty0 - iy0 + N - CT, wx = tx0 - ix0 + N - CT;
      for (int e = threadIdx.x; e < CW * CW; e += CONV_THREADS) {
        const int r = e / CW, c = e - r * CW;
        win[r * CWP + c] = Kt[(size_t)(wy + r) * KP + wx + c];
      }
      for (int e = threadIdx.x; e < CT * CT; e += CONV_THREADS) {
        const int r = e / CT, c = e - r * CT;
        stile[e] = s[(size_t)(iy0 + r) * N + ix0 + c];
      }
      __syncthreads();
#pragma unroll 2
      for (int ri = 0; ri < CT; ++ri) {
        const cx<double>* wrow = win + (warp - ri + CT - 1) * CWP + lane + CT - 1;
        const cx<double>* srow = stile + ri * CT;
#pragma unroll 4
        for (int ci = 0; ci < CT; ++ci) {
          const cx<double> sv = srow[ci];  // broadcast
#pragma unroll
          for (int r = 0; r < CONV_ROWS; ++r) {
            // output row warp + 8 r, column lane: window row warp + 8r - ri + CT-1, column lane - ci + CT-1
            const cx<double> kv = wrow[r * (CONV_THREADS / 32) * CWP - ci];
            ar[r] = fma(sv.re, kv.re, ar[r]);
            ar[r] = fma(-sv.im, kv.im, ar[r]);
            ai[r] = fma(sv.re, kv.im, ai[r]);
            ai[r] = fma(sv.im, kv.re, ai[r]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < CONV_ROWS; ++r) {
    const int y = ty0 + warp + r * (CONV_THREADS / 32), x = tx0 + lane;
    const size_t idx = (size_t)y * N + x;
    const cx<double> h = mkc(u[idx].re + ar[r], u[idx].im + ai[r]);
    cx<double> v = h;
    if (MODE == 1) {
      const cx<double> e = cscale(cmul(ex[(size_t)slot * N + x], ey[(size_t)slot * N + y]), sw);
      v = cmulc(cmul(e, Q[(size_t)slot * q_ss + idx]), h);
    }
    out[(size_t)slot * o_ss + idx] = v;
  }
}

}  // namespace

cudaError_t launch_conv_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_conv_sum<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CONV_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_sum<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CONV_SMEM);
  return e;
}

cudaError_t launch_conv_split(const cx<double>* S, long long s_ss, const double* scale, int scale_ss, const int* run,
                              const cx<double>* Mu, double inv2piL2, int N, cx<double>* out, int nslots,
                              cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const long long n = (long long)N * N;
  const int bx = (int)((n + 255) / 256 < 256 ? (n + 255) / 256 : 256);
  k_conv_split<<<dim3(bx, nslots), 256, 0, s>>>(S, s_ss, scale, scale_ss, run, Mu, inv2piL2, N, out);
  return cudaGetLastError();
}

cudaError_t launch_conv_sum(const cx<double>* f, const cx<double>* Kt, int N, const int* run, const cx<double>* Q,
                            long long q_ss, const cx<double>* ex, const cx<double>* ey, double sw, int w_out,
                            cx<double>* out, long long o_ss, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  if (N < CT || N % CT) return cudaErrorInvalidValue;
  const dim3 grid((N / CT) * (N / CT), nslots);
  if (w_out)
    k_conv_sum<1><<<grid, CONV_THREADS, CONV_SMEM, s>>>(f, Kt, N, run, Q, q_ss, ex, ey, sw, out, o_ss);
  else
    k_conv_sum<0><<<grid, CONV_THREADS, CONV_SMEM, s>>>(f, Kt, N, run, Q, q_ss, ex, ey, sw, out, o_ss);
  return cudaGetLastError();
}

}  // namespace dbar
