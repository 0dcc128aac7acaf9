// Host-side launchers of the pass and Krylov kernels.  Each precision is
// instantiated in its own translation unit (kern_f32.cu, kern_f64.cu) so the
// two compile in parallel.
#pragma once
#include "types.cuh"

namespace dbar {

template <typename T>
struct Lines {
  // lines (rows or columns) per block: lines * N/16 threads, lines * N elements of shared memory
  static int get(int N) {
    const int cap = sizeof(T) == 4 ? 8192 : 4096;
    const int l = cap / N;
    return l < N ? l : N;
  }
};

template <typename T>
inline Geo make_geo(int N) {
  Geo g;
  g.N = N;
  g.logN = 0;
  while ((1 << g.logN) < N) ++g.logN;
  g.tpl = N / 16;
  g.lines = Lines<T>::get(N);
  g.P = line_pitch(N);
  return g;
}

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename T>
inline size_t smem_pass_a(const Geo& g, int M) {
  const int MA = M > 1 ? M : 1;
  const int nseg = g.tpl >= 32 ? g.tpl / 32 : 1;
  return align16((size_t)g.lines * g.P * sizeof(cx<T>)) + (size_t)g.lines * nseg * (MA + 1) * sizeof(cx<double>) +
         (size_t)g.lines * (M + 2) * sizeof(cx<double>);
}
template <typename T>
inline size_t smem_pass_b(const Geo& g, int M) {
  return align16((size_t)g.lines * g.P * sizeof(cx<T>)) + (size_t)(M + 2) * sizeof(cx<T>);
}
template <typename T>
inline size_t smem_pass_c(const Geo& g) {
  return (size_t)g.lines * g.P * sizeof(cx<T>);
}

template <typename T>
cudaError_t launch_pass_a(const PassArgs<T>& a, int nslots, cudaStream_t s);
template <typename T, int MODE>
cudaError_t launch_pass_b(const PassArgs<T>& a, int nslots, cudaStream_t s);
template <typename T, typename TO, int MODE>
cudaError_t launch_pass_c(const PassArgs<T>& a, int nslots, cudaStream_t s);

template <typename T>
cudaError_t launch_dots(const KryArgs& a, const cx<T>* V, long long vss, const cx<T>* KS, long long kss, int j,
                        int nslots, cudaStream_t s);
template <typename T>
cudaError_t launch_update(const KryArgs& a, cx<T>* V, long long vss, const cx<T>* KS, long long kss, int j,
                          int nslots, cudaStream_t s);
template <typename T>
cudaError_t launch_xupdate(long long n, int mp1, const int* nsteps, const double* ycoef, const cx<T>* V,
                           long long vss, cx<double>* X, long long xss, int nslots, cudaStream_t s);

cudaError_t launch_finalize_h(const KryArgs& a, double* H, int j, int nslots, cudaStream_t s);
cudaError_t launch_givens(const KryArgs& a, const CycleState& c, int j, int nslots, cudaStream_t s);
cudaError_t launch_solve_y(const CycleState& c, int nslots, cudaStream_t s);
cudaError_t launch_cycle_start(const CycleState& c, const double* part, int nblk, int first, int nslots,
                               cudaStream_t s);

// small helpers (kern_f64.cu)
cudaError_t launch_transpose_q(const cx<double>* Q, cx<double>* QT64, cx<float>* QT32, int N, cudaStream_t s);
cudaError_t launch_delta_build(const cx<double>* V, const cx<double>* W, cx<double>* DT64, cx<float>* DT32, int N,
                               int nfields, cudaStream_t s);
cudaError_t launch_add_fields(const void* S, const void* KS, void* AS, long long n, int fp32, cudaStream_t s);
cudaError_t launch_taylor_final(const cx<double>* partA, int nblkA, int M, int N, cx<double>* out, int nslots,
                                cudaStream_t s);
cudaError_t launch_cast_fields(const cx<double>* in, cx<float>* out, long long n, cudaStream_t s);
cudaError_t launch_check_finite(const double* p, long long n, int* flag, cudaStream_t s);

}  // namespace dbar
