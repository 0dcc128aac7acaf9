// Krylov kernels (both precisions), the per-slot scalar kernels and the small
// helper kernels used at plan and solve set-up.
#include "krylov.cuh"
#include "launch.cuh"
#include "passes.cuh"

// 1: the block update streams the basis through shared memory by bulk asynchronous copies
#ifndef DBAR_BUPD_BULK
#define DBAR_BUPD_BULK 1
#endif

namespace dbar {

template <typename T>
cudaError_t launch_dots(const KryArgs& a, const cx<T>* V, long long vss, const cx<T>* KS, long long kss, int j,
                        int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  k_dots<T><<<dim3(a.nchunk, nslots), KR_THREADS, 0, s>>>(a, V, vss, KS, kss, j);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_update(const KryArgs& a, cx<T>* V, long long vss, const cx<T>* KS, long long kss, int j,
                          int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  k_update<T><<<dim3(a.nchunk, nslots), KR_THREADS, 0, s>>>(a, V, vss, KS, kss, j);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_xupdate(long long n, int mp1, const int* nsteps, const double* ycoef, const cx<T>* V,
                           long long vss, void* X, int x_dd, long long xss, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const int nchunk = (int)((n + KR_CHUNK - 1) / KR_CHUNK);
  if constexpr (std::is_same<T, float>::value) {
    if (x_dd) {
      k_xupdate<T, dd><<<dim3(nchunk, nslots), KR_THREADS, 0, s>>>(n, mp1, nsteps, ycoef, V, vss,
                                                                   reinterpret_cast<cx<dd>*>(X), xss);
      return cudaGetLastError();
    }
  }
  k_xupdate<T, double><<<dim3(nchunk, nslots), KR_THREADS, 0, s>>>(n, mp1, nsteps, ycoef, V, vss,
                                                                   reinterpret_cast<cx<double>*>(X), xss);
  return cudaGetLastError();
}

#define KR_INST(T)                                                                                     \
  template cudaError_t launch_dots<T>(const KryArgs&, const cx<T>*, long long, const cx<T>*, long long, int, \
                                      int, cudaStream_t);                                                 \
  template cudaError_t launch_update<T>(const KryArgs&, cx<T>*, long long, const cx<T>*, long long, int, int, \
                                        cudaStream_t);                                                    \
  template cudaError_t launch_xupdate<T>(long long, int, const int*, const double*, const cx<T>*, long long, \
                                         void*, int, long long, int, cudaStream_t);
KR_INST(float)
KR_INST(double)

template <typename T, int S>
cudaError_t launch_bdots(const BlockArgs& a, const cx<T>* V, long long vss, int J, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const size_t sm = (size_t)(KR_THREADS / 32) * block_items(J, S) * sizeof(T);
  k_bdots<T, S><<<dim3(a.nchunk, nslots), KR_THREADS, sm, s>>>(a, V, vss, J);
  return cudaGetLastError();
}
template <int S>
cudaError_t launch_bscalar(const BlockArgs& a, const CycleState& c, double* Hraw, double* bcoef, int* upd, int J,
                           int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const size_t sm = (size_t)(block_items(J, S) + (J + S) * S + S * S + S + 1) * sizeof(double);
  k_bscalar<S><<<nslots, KR_THREADS, sm, s>>>(a, c, Hraw, bcoef, upd, J);
  return cudaGetLastError();
}
template <typename T, int S>
cudaError_t launch_bupdate(const BlockArgs& a, const int* upd, cx<T>* V, long long vss, int J, int nslots,
                           cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
#if DBAR_BUPD_BULK
  if (a.n % KB_CHUNK == 0) {  // whole chunks: the basis streamed by bulk asynchronous copies
    const size_t sm = (size_t)KBStages<T>::value * KB_CHUNK * sizeof(cx<T>);
    k_bupdate_bulk<T, S, false><<<dim3(a.nwork, nslots), KR_THREADS, sm, s>>>(a, upd, V, vss, J);
    k_bupdate_bulk<T, S, true><<<dim3(a.nwork, nslots), KR_THREADS, sm, s>>>(a, upd, V, vss, J);
    return cudaGetLastError();
  }
#endif
  k_bupdate<T, S, false><<<dim3(a.nwork, nslots), KR_THREADS, 0, s>>>(a, upd, V, vss, J);
  k_bupdate<T, S, true><<<dim3(a.nwork, nslots), KR_THREADS, 0, s>>>(a, upd, V, vss, J);
  return cudaGetLastError();
}
#define KB_INST(T, S)                                                                                          \
  template cudaError_t launch_bdots<T, S>(const BlockArgs&, const cx<T>*, long long, int, int, cudaStream_t);  \
  template cudaError_t launch_bupdate<T, S>(const BlockArgs&, const int*, cx<T>*, long long, int, int,        \
                                            cudaStream_t);
KB_INST(float, 2)
KB_INST(float, 4)
KB_INST(double, 2)
KB_INST(double, 4)
template cudaError_t launch_bscalar<2>(const BlockArgs&, const CycleState&, double*, double*, int*, int, int,
                                       cudaStream_t);
template cudaError_t launch_bscalar<4>(const BlockArgs&, const CycleState&, double*, double*, int*, int, int,
                                       cudaStream_t);

cudaError_t launch_finalize_h(const KryArgs& a, double* H, int j, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  constexpr int per = KR_THREADS / 32;
  k_finalize_h<<<(nslots + per - 1) / per, KR_THREADS, 0, s>>>(a, H, j, nslots);
  return cudaGetLastError();
}
cudaError_t launch_givens(const KryArgs& a, const CycleState& c, int j, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  constexpr int per = KR_THREADS / 32;
  k_givens<<<(nslots + per - 1) / per, KR_THREADS, 0, s>>>(a, c, j, nslots);
  return cudaGetLastError();
}
cudaError_t launch_solve_y(const CycleState& c, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  k_solve_y<<<(nslots + 63) / 64, 64, 0, s>>>(c, nslots);
  return cudaGetLastError();
}
cudaError_t launch_cycle_start(const CycleState& c, const double* part, int nblk, int first, int nslots,
                               cudaStream_t s, const int* mask) {
  if (nslots <= 0) return cudaSuccess;
  k_cycle_start<<<nslots, KR_THREADS, 0, s>>>(c, part, nblk, first, mask);
  return cudaGetLastError();
}

// Q in both precisions (physical layout [y][x]).
__global__ void k_load_q(const cx<double>* __restrict__ Q, cx<double>* __restrict__ Q64, cx<float>* __restrict__ Q32,
                         long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cx<double> v = Q[i];
    Q64[i] = v;
    Q32[i] = ccast<float>(v);
  }
}
cudaError_t launch_load_q(const cx<double>* Q, cx<double>* Q64, cx<float>* Q32, int N, cudaStream_t s) {
  const long long n = (long long)N * N;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_load_q<<<blocks, 256, 0, s>>>(Q, Q64, Q32, n);
  return cudaGetLastError();
}

// Delta_n = W_n - V_n in both precisions ([n][y][x]).
__global__ void k_delta_build(const cx<double>* __restrict__ V, const cx<double>* __restrict__ W,
                              cx<double>* __restrict__ D64, cx<float>* __restrict__ D32, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cx<double> v = W[i] - V[i];
    D64[i] = v;
    D32[i] = ccast<float>(v);
  }
}
cudaError_t launch_delta_build(const cx<double>* V, const cx<double>* W, cx<double>* D64, cx<float>* D32, int N,
                               int nfields, cudaStream_t s) {
  const long long n = (long long)N * N * nfields;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_delta_build<<<blocks, 256, 0, s>>>(V, W, D64, D32, n);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_add_fields(const cx<T>* __restrict__ S, const cx<T>* __restrict__ KS, cx<T>* __restrict__ AS,
                             long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    AS[i] = S[i] + KS[i];
}
cudaError_t launch_add_fields(const void* S, const void* KS, void* AS, long long n, int fp32, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (fp32)
    k_add_fields<float><<<blocks, 256, 0, s>>>((const cx<float>*)S, (const cx<float>*)KS, (cx<float>*)AS, n);
  else
    k_add_fields<double><<<blocks, 256, 0, s>>>((const cx<double>*)S, (const cx<double>*)KS, (cx<double>*)AS, n);
  return cudaGetLastError();
}

cudaError_t launch_coef(const cx<double>* partA, int part_fp32, int M, int N, const cx<double>* Da64,
                        const cx<float>* Da32, double fillscale, cx<double>* coefp, int* ticket, cx<double>* coef,
                        int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const int rows = coef_rows(N);
  const dim3 grid(nslots, N / rows);
  if (part_fp32)
    k_coef<float><<<grid, rows, 0, s>>>(reinterpret_cast<const cx<float>*>(partA), seg_count(N), M > 1 ? M : 1, M,
                                        N, Da64, Da32, fillscale, coefp, ticket, coef);
  else
    k_coef<double><<<grid, rows, 0, s>>>(partA, seg_count(N), M > 1 ? M : 1, M, N, Da64, Da32, fillscale, coefp,
                                         ticket, coef);
  return cudaGetLastError();
}

__global__ void k_cast_fields(const cx<double>* __restrict__ in, cx<float>* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = ccast<float>(in[i]);
}
// x -> -x over n floats / doubles (the potential's sign flip between the two
// equations of the reflection coefficient)
__global__ void k_negate_f32(float* __restrict__ p, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = -p[i];
}
__global__ void k_negate_f64(double* __restrict__ p, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = -p[i];
}
cudaError_t launch_negate(void* p, long long n, int fp64, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (fp64) k_negate_f64<<<blocks, 256, 0, s>>>(reinterpret_cast<double*>(p), n);
  else k_negate_f32<<<blocks, 256, 0, s>>>(reinterpret_cast<float*>(p), n);
  return cudaGetLastError();
}

// out[slot][p2][p1] = scale_slot * in[slot][(p2 + s2) mod N][(p1 + s1) mod N],
// (s1, s2) = shift[slot]: h~(eta) = h(eta + xi0) on the periodic grid (the
// shifted regularisation of Sec. 5).  scale may be NULL (1).
template <typename T>
__global__ void k_roll(const cx<T>* __restrict__ in, long long in_ss, const double* __restrict__ scale, int scale_ss,
                       const int* __restrict__ shift, const int* __restrict__ run, int N, cx<T>* __restrict__ out,
                       long long out_ss) {
  const int slot = blockIdx.y;
  if (run && !run[slot]) return;
  const long long n = (long long)N * N;
  const int s1 = shift[2 * slot], s2 = shift[2 * slot + 1];
  const T sc = scale ? (T)scale[(size_t)slot * scale_ss] : (T)1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int p2 = (int)(i / N), p1 = (int)(i - (long long)p2 * N);
    const cx<T> v = in[(size_t)slot * in_ss + (size_t)((p2 + s2) & (N - 1)) * N + ((p1 + s1) & (N - 1))];
    out[(size_t)slot * out_ss + i] = mkc(sc * v.re, sc * v.im);
  }
}
template <typename T>
cudaError_t launch_roll(const cx<T>* in, long long in_ss, const double* scale, int scale_ss, const int* shift,
                        const int* run, int N, cx<T>* out, long long out_ss, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const long long n = (long long)N * N;
  const int bx = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  k_roll<T><<<dim3(bx, nslots), 256, 0, s>>>(in, in_ss, scale, scale_ss, shift, run, N, out, out_ss);
  return cudaGetLastError();
}
template cudaError_t launch_roll<float>(const cx<float>*, long long, const double*, int, const int*, const int*, int,
                                        cx<float>*, long long, int, cudaStream_t);
template cudaError_t launch_roll<double>(const cx<double>*, long long, const double*, int, const int*, const int*, int,
                                         cx<double>*, long long, int, cudaStream_t);
template cudaError_t launch_roll<dd>(const cx<dd>*, long long, const double*, int, const int*, const int*, int,
                                     cx<dd>*, long long, int, cudaStream_t);

// out[p2][p1] = conj(r[p2][p1] e^{-i t (k^2 + conj(k)^2)/4}), k = x_{p1} + i y_{p2} on the
// grid x_j = L(-pi + 2 pi j/N): the potential of the D-bar problem in k at time t
// (eq. rt; k^2 + conj(k)^2 = 2 (x^2 - y^2)).  Once per call, FP64.
__global__ void k_ds2_kernel_potential(const cx<double>* __restrict__ r, int N, double L, double t,
                                       cx<double>* __restrict__ out) {
  const long long n = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int p2 = (int)(i / N), p1 = (int)(i - (long long)p2 * N);
    const double x = L * (-M_PI + 2.0 * M_PI * p1 / N), y = L * (-M_PI + 2.0 * M_PI * p2 / N);
    double sn, cs;
    sincos(-0.5 * t * (x * x - y * y), &sn, &cs);
    const cx<double> v = r[i];
    out[i] = mkc(v.re * cs - v.im * sn, -(v.re * sn + v.im * cs));
  }
}
cudaError_t launch_ds2_kernel_potential(const cx<double>* r, int N, double L, double t, cx<double>* out,
                                        cudaStream_t s) {
  const long long n = (long long)N * N;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_ds2_kernel_potential<<<blocks, 256, 0, s>>>(r, N, L, t, out);
  return cudaGetLastError();
}

// out[i] = x[i][0] (the value at xi = 0 of slot i's solution) in FP64
// (at = NULL) or at the per-slot element index at[i]
__global__ void k_gather_s0(const void* __restrict__ x, long long xss, int nb, int x_dd, const long long* __restrict__ at,
                            cx<double>* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const size_t e = (size_t)i * xss + (at ? (size_t)at[i] : 0);
  if (x_dd) {
    const cx<dd> v = reinterpret_cast<const cx<dd>*>(x)[e];
    out[i] = mkc((double)v.re, (double)v.im);
  } else {
    out[i] = reinterpret_cast<const cx<double>*>(x)[e];
  }
}
cudaError_t launch_gather_s0(const void* x, long long xss, int nb, int x_dd, const long long* at, cx<double>* out,
                             cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  k_gather_s0<<<(nb + 127) / 128, 128, 0, s>>>(x, xss, nb, x_dd, at, out);
  return cudaGetLastError();
}

cudaError_t launch_cast_fields(const cx<double>* in, cx<float>* out, long long n, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_cast_fields<<<blocks, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

// Support of an FP32 potential: colf[x] = 1 if some Q[y][x] != 0, rowf[y] = 1 if some
// Q[y][x] != 0 (flags zeroed beforehand; concurrent writes store the same 1).
__global__ void k_q_support(const cx<float>* __restrict__ Q, int N, int* colf, int* rowf) {
  const long long n = (long long)N * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cx<float> v = Q[i];
    if (v.re != 0.f || v.im != 0.f) {
      colf[i % N] = 1;
      rowf[i / N] = 1;
    }
  }
}
cudaError_t launch_q_support(const cx<float>* Q, int N, int* flags, cudaStream_t s) {
  const long long n = (long long)N * N;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_q_support<<<blocks, 256, 0, s>>>(Q, N, flags, flags + N);
  return cudaGetLastError();
}

__global__ void k_split_fields(const cx<double>* __restrict__ in, cx<dd>* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = ccast<dd>(in[i]);
}
cudaError_t launch_split_fields(const cx<double>* in, cx<dd>* out, long long n, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_split_fields<<<blocks, 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

__global__ void k_check_finite(const double* __restrict__ p, long long n, int* flag) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(p[i])) *flag = 1;
}
cudaError_t launch_check_finite(const double* p, long long n, int* flag, cudaStream_t s) {
  const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  k_check_finite<<<blocks, 256, 0, s>>>(p, n, flag);
  return cudaGetLastError();
}

}  // namespace dbar
