// Host-side launchers of the pass and Krylov kernels.  The pass kernels are
// instantiated per precision and grid size in their own translation units
// (kern_pass.cu compiled once per pair) so they compile in parallel.
#pragma once
#include <string>

#include "../../include/dbar.h"
#include "types.cuh"

namespace dbar {}  // namespace dbar

// Records msg as the calling thread's last error (dbar_last_error) and returns st.
dbar_status dbar_internal_fail(dbar_status st, const std::string& msg);

namespace dbar {

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

inline int ilog2(int N) {
  int l = 0;
  while ((1 << l) < N) ++l;
  return l;
}
template <typename T>
inline Geo make_geo(int N) {
  Geo g;
  g.N = N;
  g.logN = ilog2(N);
  g.tpl = N / 16;
  g.lines = row_lines(g.logN);
  g.P = pitch_of(N);
  return g;
}
// blocks per slot of the row passes (A and C)
inline int row_blocks(int N) { return N / row_lines(ilog2(N)); }
// warp segments of one row line (N/16 threads, at most 32 per segment): the
// number of row-moment partials pass A writes per row and moment
inline int seg_count(int N) { return N / 16 >= 32 ? N / 512 : 1; }
// rows per block of k_coef (one row per thread): the whole row set for N <= 256 (one block
// per slot: no cross-block combination; small grids come in large batches), else N/8
inline int coef_rows(int N) { return N <= 256 ? N : N / 8; }

// per-size launchers (kern_pass.cu, one translation unit per precision and size)
template <typename T, int LOGN>
cudaError_t launch_pass_a_n(const PassArgs<T>& a, int nslots, cudaStream_t s);
template <typename T, int LOGN, int MODE, int CV>
cudaError_t launch_pass_b_n(const PassArgs<T>& a, int nslots, cudaStream_t s);
template <typename T, typename TO, int LOGN, int MODE>
cudaError_t launch_pass_c_n(const PassArgs<T>& a, int nslots, cudaStream_t s);
template <typename T, int LOGN>
cudaError_t launch_pass_ca_n(const PassArgs<T>& a, int nslots, cudaStream_t s);

// size dispatch (dispatch.cu)
template <typename T>
cudaError_t launch_pass_a(const PassArgs<T>& a, int nslots, cudaStream_t s);
// fused chain step rows: pass C of the column-pass output -> out (K p), then
// pass A of K p -> out2 (and the Taylor moment partials)
template <typename T>
cudaError_t launch_pass_ca(const PassArgs<T>& a, int nslots, cudaStream_t s);
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
                           long long vss, void* X, int x_dd, long long xss, int nslots, cudaStream_t s);
// FP64 copy of n double-float complex values
cudaError_t launch_dd_to_fp64(const void* in, cx<double>* out, long long n, cudaStream_t s);

template <typename T, int S>
cudaError_t launch_bdots(const BlockArgs& a, const cx<T>* V, long long vss, int J, int nslots, cudaStream_t s);
template <int S>
cudaError_t launch_bscalar(const BlockArgs& a, const CycleState& c, double* Hraw, double* bcoef, int* upd, int J,
                           int nslots, cudaStream_t s);
template <typename T, int S>
// two launches: slots continuing their cycle (upd 1), slots in their last
// block (upd 2, which also add V y to x)
cudaError_t launch_bupdate(const BlockArgs& a, const int* upd, cx<T>* V, long long vss, int J, int nslots,
                           cudaStream_t s);

cudaError_t launch_finalize_h(const KryArgs& a, double* H, int j, int nslots, cudaStream_t s);
cudaError_t launch_givens(const KryArgs& a, const CycleState& c, int j, int nslots, cudaStream_t s);
cudaError_t launch_solve_y(const CycleState& c, int nslots, cudaStream_t s);
cudaError_t launch_cycle_start(const CycleState& c, const double* part, int nblk, int first, int nslots,
                               cudaStream_t s, const int* mask = nullptr);

// small helpers (kern_f64.cu)
cudaError_t launch_load_q(const cx<double>* Q, cx<double>* Q64, cx<float>* Q32, int N, cudaStream_t s);
cudaError_t launch_delta_build(const cx<double>* V, const cx<double>* W, cx<double>* D64, cx<float>* D32, int N,
                               int nfields, cudaStream_t s);
cudaError_t launch_add_fields(const void* S, const void* KS, void* AS, long long n, int fp32, cudaStream_t s);
// part_fp32: partials written by the FP32 pass A (cx<float>), else cx<double>.
// coefp: [slots][N / coef_rows(N)][M+2] block partials; ticket: [slots] zeroed
// counters (re-armed by the kernel).
cudaError_t launch_coef(const cx<double>* partA, int part_fp32, int M, int N, const cx<double>* Da64,
                        const cx<float>* Da32, double fillscale, cx<double>* coefp, int* ticket, cx<double>* coef,
                        int nslots, cudaStream_t s);
cudaError_t launch_negate(void* p, long long n, int fp64, cudaStream_t s);
cudaError_t launch_ds2_kernel_potential(const cx<double>* r, int N, double L, double t, cx<double>* out,
                                        cudaStream_t s);
cudaError_t launch_gather_s0(const void* x, long long xss, int nb, int x_dd, const long long* at, cx<double>* out,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_roll(const cx<T>* in, long long in_ss, const double* scale, int scale_ss, const int* shift,
                        const int* run, int N, cx<T>* out, long long out_ss, int nslots, cudaStream_t s);
// convolution regularisation (conv.cu; Sec. 4.2, remark after eq. fourreg5a), FP64.
// Once per device before the first launch (shared-memory opt-in of the direct sum).
cudaError_t launch_conv_prepare();
// out[slot][0] = sigma S Mu, out[slot][1] = sigma (-1)^{p1+p2} S / (2 pi L^2)  ([slot][2][N*N])
cudaError_t launch_conv_split(const cx<double>* S, long long s_ss, const double* scale, int scale_ss, const int* run,
                              const cx<double>* Mu, double inv2piL2, int N, cx<double>* out, int nslots,
                              cudaStream_t s);
// h = f[slot][0] + direct sum of f[slot][1] against Kt ([2N-1][2N], h^2/(2 pi) W_0 at the
// grid differences); w_out = 0: out = h, 1: out = sw E_k Q conj(h).  N a multiple of 32.
cudaError_t launch_conv_sum(const cx<double>* f, const cx<double>* Kt, int N, const int* run, const cx<double>* Q,
                            long long q_ss, const cx<double>* ex, const cx<double>* ey, double sw, int w_out,
                            cx<double>* out, long long o_ss, int nslots, cudaStream_t s);
cudaError_t launch_cast_fields(const cx<double>* in, cx<float>* out, long long n, cudaStream_t s);
cudaError_t launch_split_fields(const cx<double>* in, cx<dd>* out, long long n, cudaStream_t s);
cudaError_t launch_check_finite(const double* p, long long n, int* flag, cudaStream_t s);
// flags[x] = 1 where column x of Q has a nonzero entry, flags[N + y] = 1 where row y has
// one ([2N], zeroed beforehand)
cudaError_t launch_q_support(const cx<float>* Q, int N, int* flags, cudaStream_t s);
// column-pass tiles of every variant at N are aligned to this many columns
inline int col_align(int N) {
  const int l = ilog2(N), c0 = col_cols(l, 8, 0), c1 = col_cols(l, 8, 1);
  return c0 > c1 ? c0 : c1;
}

}  // namespace dbar
