// Launcher bodies; included by one translation unit per precision.
#pragma once
#include "krylov.cuh"
#include "launch.cuh"
#include "passes.cuh"

namespace dbar {

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
cudaError_t launch_pass_a(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const size_t sm = smem_pass_a<T>(a.g, a.M);
  cudaError_t e = set_smem(k_pass_a<T>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.N / a.g.lines, nslots);
  k_pass_a<T><<<grid, a.g.lines * a.g.tpl, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_pass_b(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const size_t sm = smem_pass_b<T>(a.g, a.M);
  cudaError_t e = set_smem(k_pass_b<T, MODE>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.N / a.g.lines, nslots);
  k_pass_b<T, MODE><<<grid, a.g.lines * a.g.tpl, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, typename TO, int MODE>
cudaError_t launch_pass_c(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const size_t sm = smem_pass_c<T>(a.g);
  cudaError_t e = set_smem(k_pass_c<T, TO, MODE>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.N / a.g.lines, nslots);
  k_pass_c<T, TO, MODE><<<grid, a.g.lines * a.g.tpl, sm, s>>>(a);
  return cudaGetLastError();
}

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
                           long long vss, cx<double>* X, long long xss, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  const int nchunk = (int)((n + KR_CHUNK - 1) / KR_CHUNK);
  k_xupdate<T><<<dim3(nchunk, nslots), KR_THREADS, 0, s>>>(n, mp1, nsteps, ycoef, V, vss, X, xss);
  return cudaGetLastError();
}

#define DBAR_INSTANTIATE(T, TO)                                                                            \
  template cudaError_t launch_pass_a<T>(const PassArgs<T>&, int, cudaStream_t);                           \
  template cudaError_t launch_pass_b<T, PB_MATVEC>(const PassArgs<T>&, int, cudaStream_t);                \
  template cudaError_t launch_pass_b<T, PB_RHS>(const PassArgs<T>&, int, cudaStream_t);                   \
  template cudaError_t launch_pass_b<T, PB_HOUT>(const PassArgs<T>&, int, cudaStream_t);                  \
  template cudaError_t launch_pass_b<T, PB_FWD>(const PassArgs<T>&, int, cudaStream_t);                   \
  template cudaError_t launch_pass_b<T, PB_INV>(const PassArgs<T>&, int, cudaStream_t);                   \
  template cudaError_t launch_pass_c<T, T, PC_KS>(const PassArgs<T>&, int, cudaStream_t);                 \
  template cudaError_t launch_pass_c<T, T, PC_FWD>(const PassArgs<T>&, int, cudaStream_t);                \
  template cudaError_t launch_pass_c<T, T, PC_INV>(const PassArgs<T>&, int, cudaStream_t);                \
  template cudaError_t launch_dots<T>(const KryArgs&, const cx<T>*, long long, const cx<T>*, long long, int, \
                                      int, cudaStream_t);                                                 \
  template cudaError_t launch_update<T>(const KryArgs&, cx<T>*, long long, const cx<T>*, long long, int, int, \
                                        cudaStream_t);                                                    \
  template cudaError_t launch_xupdate<T>(long long, int, const int*, const double*, const cx<T>*, long long, \
                                         cx<double>*, long long, int, cudaStream_t);

}  // namespace dbar
