// Size dispatch: maps the run-time grid size onto the per-size launchers.
#include <type_traits>

#include "launch.cuh"

namespace dbar {

#define DBAR_SIZES(X) X(5) X(6) X(7) X(8) X(9) X(10) X(11)

template <typename T>
cudaError_t launch_pass_a(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  switch (a.g.logN) {
#define CASE(L) \
  case L: return launch_pass_a_n<T, L>(a, nslots, s);
    DBAR_SIZES(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_pass_ca(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  switch (a.g.logN) {
#define CASE(L) \
  case L: return launch_pass_ca_n<T, L>(a, nslots, s);
    DBAR_SIZES(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T, int MODE>
cudaError_t launch_pass_b(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  if constexpr (std::is_same<T, float>::value && MODE == PB_MATVEC) {
    if (a.colv == 1) {
      switch (a.g.logN) {
#define CASE(L) \
  case L: return launch_pass_b_n<T, L, MODE, 1>(a, nslots, s);
        DBAR_SIZES(CASE)
#undef CASE
      }
      return cudaErrorInvalidValue;
    }
    if (a.colv == 2) {
      switch (a.g.logN) {
#define CASE(L) \
  case L: return launch_pass_b_n<T, L, MODE, 2>(a, nslots, s);
        DBAR_SIZES(CASE)
#undef CASE
      }
      return cudaErrorInvalidValue;
    }
  }
  switch (a.g.logN) {
#define CASE(L) \
  case L: return launch_pass_b_n<T, L, MODE, 0>(a, nslots, s);
    DBAR_SIZES(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

template <typename T, typename TO, int MODE>
cudaError_t launch_pass_c(const PassArgs<T>& a, int nslots, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  switch (a.g.logN) {
#define CASE(L) \
  case L: return launch_pass_c_n<T, TO, L, MODE>(a, nslots, s);
    DBAR_SIZES(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

#define INST(T)                                                                         \
  template cudaError_t launch_pass_a<T>(const PassArgs<T>&, int, cudaStream_t);  \
  template cudaError_t launch_pass_ca<T>(const PassArgs<T>&, int, cudaStream_t);  \
  template cudaError_t launch_pass_b<T, PB_MATVEC>(const PassArgs<T>&, int, cudaStream_t); \
  template cudaError_t launch_pass_b<T, PB_RHS>(const PassArgs<T>&, int, cudaStream_t);    \
  template cudaError_t launch_pass_b<T, PB_HOUT>(const PassArgs<T>&, int, cudaStream_t);   \
  template cudaError_t launch_pass_b<T, PB_FWD>(const PassArgs<T>&, int, cudaStream_t);    \
  template cudaError_t launch_pass_b<T, PB_INV>(const PassArgs<T>&, int, cudaStream_t);    \
  template cudaError_t launch_pass_c<T, T, PC_KS>(const PassArgs<T>&, int, cudaStream_t);  \
  template cudaError_t launch_pass_c<T, T, PC_FWD>(const PassArgs<T>&, int, cudaStream_t); \
  template cudaError_t launch_pass_c<T, T, PC_INV>(const PassArgs<T>&, int, cudaStream_t);
INST(float)
INST(double)
template cudaError_t launch_pass_c<double, double, PC_RHS>(const PassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pass_c<double, float, PC_RHS>(const PassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pass_c<double, double, PC_RES>(const PassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pass_c<double, float, PC_RES>(const PassArgs<double>&, int, cudaStream_t);
template cudaError_t launch_pass_a<dd>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_b<dd, PB_MATVEC>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_b<dd, PB_RHS>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_b<dd, PB_WF>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_b<dd, PB_FWD>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_c<dd, float, PC_RHS>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_c<dd, float, PC_RES>(const PassArgs<dd>&, int, cudaStream_t);
template cudaError_t launch_pass_c<dd, dd, PC_KS>(const PassArgs<dd>&, int, cudaStream_t);

}  // namespace dbar
