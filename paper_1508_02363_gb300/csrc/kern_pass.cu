// The three pass kernels for one precision (DBAR_T) and one grid size
// (N = 2^DBAR_LOGN).  The build compiles this file once per (precision, size)
// so that every FFT is fully unrolled at compile time and the translation
// units build in parallel.
#include "launch.cuh"
#include "passes.cuh"

#ifndef DBAR_T
#error "DBAR_T (float, double or dd) must be defined"
#endif
#ifndef DBAR_KIND
#error "DBAR_KIND (0 float, 1 double, 2 double-float) must be defined"
#endif
#ifndef DBAR_LOGN
#error "DBAR_LOGN must be defined"
#endif

namespace dbar {

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int LOGN, bool SH, int RV>
static cudaError_t launch_a_shape(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  using G = RowG<T, LOGN, RV>;
  const size_t sm = (size_t)G::LINES * G::P * sizeof(cx<T>);
  cudaError_t e = set_smem(k_pass_a<T, LOGN, SH, RV>, sm);
  if (e != cudaSuccess) return e;
  k_pass_a<T, LOGN, SH, RV><<<dim3(G::N / G::LINES, nslots), G::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t launch_pass_a_n(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if (a.dshift) return launch_a_shape<T, LOGN, true, 0>(a, nslots, s);  // shifted quotient (iterated equation)
  if constexpr (std::is_same<T, float>::value) {
    if (a.rowv == 1) return launch_a_shape<T, LOGN, false, 1>(a, nslots, s);
    if (a.rowv == 2) return launch_a_shape<T, LOGN, false, 2>(a, nslots, s);
    if (a.rowv == 3) return launch_a_shape<T, LOGN, false, 3>(a, nslots, s);
    if (a.rowv == 4) return launch_a_shape<T, LOGN, false, 4>(a, nslots, s);
  }
  return launch_a_shape<T, LOGN, false, 0>(a, nslots, s);
}

template <typename T, int LOGN, int MODE, int CV>
cudaError_t launch_pass_b_n(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if constexpr (CV == 2) {  // two slots per block (operator mode)
    using G = ColG<T, LOGN, 0>;
    const size_t sm = align16((size_t)2 * G::COLS * G::P * sizeof(cx<T>)) + (size_t)2 * (a.M + 2) * sizeof(cx<T>);
    cudaError_t e = set_smem(k_pass_b2<T, LOGN>, sm);
    if (e != cudaSuccess) return e;
    const int ntile = (a.sx1 - a.sx0) / G::COLS;  // column tiles of the potential's support
    if (ntile <= 0) return cudaSuccess;
    k_pass_b2<T, LOGN><<<dim3((nslots + 1) / 2, ntile), G::THREADS, sm, s>>>(a, nslots);
    return cudaGetLastError();
  }
  using G = ColG<T, LOGN, CV>;
  const size_t sm = align16((size_t)G::COLS * G::P * sizeof(cx<T>)) + (size_t)(a.M + 2) * sizeof(cx<T>);
  cudaError_t e = set_smem(k_pass_b<T, LOGN, MODE, CV>, sm);
  if (e != cudaSuccess) return e;
  const int ntile = (a.sx1 - a.sx0) / G::COLS;  // column tiles of the potential's support
  if (ntile <= 0) return cudaSuccess;
  k_pass_b<T, LOGN, MODE, CV><<<dim3(nslots, ntile), G::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int LOGN, int RV>
static cudaError_t launch_ca_shape(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  using G = RowG<T, LOGN, RV>;
  const size_t sm = (size_t)G::LINES * G::P * sizeof(cx<T>);
  cudaError_t e = set_smem(k_pass_ca<T, LOGN, RV>, sm);
  if (e != cudaSuccess) return e;
  k_pass_ca<T, LOGN, RV><<<dim3(G::N / G::LINES, nslots), G::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t launch_pass_ca_n(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (a.rowv == 1) return launch_ca_shape<T, LOGN, 1>(a, nslots, s);
    if (a.rowv == 2) return launch_ca_shape<T, LOGN, 2>(a, nslots, s);
    if (a.rowv == 3) return launch_ca_shape<T, LOGN, 3>(a, nslots, s);
    if (a.rowv == 4) return launch_ca_shape<T, LOGN, 4>(a, nslots, s);
  }
  return launch_ca_shape<T, LOGN, 0>(a, nslots, s);
}

template <typename T, typename TO, int LOGN, int MODE, int RV>
static cudaError_t launch_c_shape(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  using G = RowG<T, LOGN, RV>;
  const size_t sm = (size_t)G::LINES * G::P * sizeof(cx<T>);
  cudaError_t e = set_smem(k_pass_c<T, TO, LOGN, MODE, RV>, sm);
  if (e != cudaSuccess) return e;
  k_pass_c<T, TO, LOGN, MODE, RV><<<dim3(G::N / G::LINES, nslots), G::THREADS, sm, s>>>(a);
  return cudaGetLastError();
}

template <typename T, typename TO, int LOGN, int MODE>
cudaError_t launch_pass_c_n(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  // the operator's K S (no per-block partial sums): the autotuned shape
  if constexpr (std::is_same<T, float>::value && MODE == PC_KS) {
    if (a.rowv == 1) return launch_c_shape<T, TO, LOGN, MODE, 1>(a, nslots, s);
    if (a.rowv == 2) return launch_c_shape<T, TO, LOGN, MODE, 2>(a, nslots, s);
    if (a.rowv == 3) return launch_c_shape<T, TO, LOGN, MODE, 3>(a, nslots, s);
    if (a.rowv == 4) return launch_c_shape<T, TO, LOGN, MODE, 4>(a, nslots, s);
  }
  return launch_c_shape<T, TO, LOGN, MODE, 0>(a, nslots, s);
}

typedef DBAR_T TT;
#if DBAR_KIND == 2
// double-float: the right-hand side and the true residual of the refinement
template cudaError_t launch_pass_a_n<dd, DBAR_LOGN>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<dd, DBAR_LOGN, PB_MATVEC, 0>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<dd, DBAR_LOGN, PB_RHS, 0>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<dd, DBAR_LOGN, PB_WF, 0>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<dd, DBAR_LOGN, PB_FWD, 0>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<dd, float, DBAR_LOGN, PC_RHS>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<dd, float, DBAR_LOGN, PC_RES>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<dd, dd, DBAR_LOGN, PC_KS>(const PassArgs<dd>&, int, cudaStream_t);
#else
template cudaError_t launch_pass_a_n<TT, DBAR_LOGN>(const PassArgs<TT>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<TT, DBAR_LOGN, PB_MATVEC, 0>(const PassArgs<TT>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<TT, DBAR_LOGN, PB_RHS, 0>(const PassArgs<TT>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<TT, DBAR_LOGN, PB_HOUT, 0>(const PassArgs<TT>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<TT, DBAR_LOGN, PB_FWD, 0>(const PassArgs<TT>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<TT, DBAR_LOGN, PB_INV, 0>(const PassArgs<TT>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<TT, TT, DBAR_LOGN, PC_KS>(const PassArgs<TT>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<TT, TT, DBAR_LOGN, PC_FWD>(const PassArgs<TT>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<TT, TT, DBAR_LOGN, PC_INV>(const PassArgs<TT>&, int, cudaStream_t);
#if DBAR_KIND == 0
template cudaError_t launch_pass_b_n<float, DBAR_LOGN, PB_MATVEC, 1>(const PassArgs<float>&, int, cudaStream_t);
template cudaError_t launch_pass_b_n<float, DBAR_LOGN, PB_MATVEC, 2>(const PassArgs<float>&, int, cudaStream_t);
#endif
template cudaError_t launch_pass_ca_n<TT, DBAR_LOGN>(const PassArgs<TT>&, int, cudaStream_t);
#if DBAR_KIND == 1
template cudaError_t launch_pass_c_n<double, double, DBAR_LOGN, PC_RHS>(const PassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<double, float, DBAR_LOGN, PC_RHS>(const PassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<double, double, DBAR_LOGN, PC_RES>(const PassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pass_c_n<double, float, DBAR_LOGN, PC_RES>(const PassArgs<double>&, int, cudaStream_t);
#endif
#endif

}  // namespace dbar
