// Argument structures shared by the kernels and the host driver.
#pragma once
#include "cx.cuh"

namespace dbar {

struct Geo {
  int N, logN, tpl, lines, P;
};

template <typename T>
struct PassArgs {
  Geo g;
  int colv;  // column-pass tile variant (autotuned)
  int rowv;  // row-pass shape of the FP32 operator's row passes (autotuned; 0 elsewhere)
  int M;  // Taylor order
  // input field (T), per-slot stride in complex elements; optional per-slot scale
  const cx<T>* in;
  long long in_ss;
  const double* in_scale;
  int in_scale_ss;
  // outputs
  void* out;
  long long out_ss;
  void* out2;  // second output (pass C right-hand side / residual: Krylov start vector)
  long long out2_ss;
  // pass C residual inputs, stored in the residual's arithmetic (FP64 or
  // double-float: x and b of the mixed path never pass through FP64)
  const cx<T>* b;
  const cx<T>* x;
  long long f_ss;
  const int* run;  // per-slot flags (nullable)
  // tables
  const cx<T>* tw;       // [N]   e^{-2 pi i t/N}
  const cx<T>* Da;       // [MA+1][N]
  const cx<double>* Da64;
  const cx<T>* Delta;    // [M+1][N (y index)][N (x index)]  W_n - V_n
  const cx<T>* Q;        // [N (y index)][N (x index)], per slot at stride q_ss (0: shared)
  long long q_ss;
  const cx<T>* ex;       // [slot][N]  e^{-2 i k2 x_j}
  const cx<T>* ey;       // [slot][N]  e^{-2 i k1 y_j}
  double inv2piL;        // 1/(2 pi L)
  float inv2piL_f;       // the same, rounded once on the host (FP32 pass A)
  float hx_f;            // grid spacing 2 pi L / N, rounded once (FP32 fused row pass moments)
  double sw;             // 2 pi L^2 / N^2
  double fillscale;      // 1/(2 pi L^2), or 0 for the zero-fill reading
  cx<double>* partA;     // [slot][p2][nseg][MA+1] row-moment partials (pass A -> k_coef);
                         // stored as cx<float> by the FP32 pass A
  int nseg;              // warp segments per row: seg_count(N)
  const cx<double>* coef;  // [slot][M+2] c_0..c_M, d' (k_coef output, read by pass B)
  double* part;          // [slot][gridDim.x] squared-norm partials (pass C)
  const float* nscale;   // [slot] power-of-two ~1/||b|| (double-float residual norms)
  int neg;               // row pass C: the transform's output negated (K of the iterated equation)
  // pass A of the iterated equation's shifted quotient (eq. dbarinvShift): per slot the signed
  // grid offset (s1, s2) of xi0 by which the input was rolled, so that the divisor of rolled
  // element p is the unwrapped xi_{p + s} - xi0 (nullable: the plain divisor xi_p)
  const int* dshift;
  // support of the potential in the FP32 inner operator (and the double-float
  // residual): the columns [sx0, sx1) (a multiple of every column-pass tile width)
  // outside which Q is exactly zero, so that w = E_k Q conj(h) is exactly zero there:
  // pass A stores and pass C loads only those columns of the pass intermediates, and
  // pass B transforms only those columns.  Rows [sy0, sy1): pass B loads its tables
  // only there (the full range -- no per-row test -- unless the plan sets a band).
  int sx0, sx1, sy0, sy1;
};


constexpr int KR_THREADS = 256;
constexpr int KR_EPT = 8;  // complex elements per thread
constexpr int KR_CHUNK = KR_THREADS * KR_EPT;

struct KryArgs {
  long long n;       // complex elements per vector (N*N)
  int mp1;           // basis vectors per slot (restart + 1)
  int nchunk;        // blocks per slot
  const int* run;    // per-slot flags of the current cycle
  const double* sigma;  // [slot][mp1]
  double* coef;         // [slot][mp1] update coefficients
  double* part;         // [slot][mp1][nchunk]
  double* part2;        // [slot][nchunk]
};

// s-step (block) Arnoldi sweeps (krylov.cuh)
constexpr int KB_EPT = 4;                      // complex elements per thread (block sweeps)
constexpr int KB_CHUNK = KR_THREADS * KB_EPT;  // elements per block of a block sweep
constexpr double kBlockPivot = 1e-5;           // smallest accepted Cholesky pivot of the normalised Gram
constexpr int kBlockDotBlocks = 128;           // dot-sweep blocks per slot (fewer partials to fold in FP64)

struct BlockArgs {
  long long n;          // complex elements per vector
  int mp1;              // basis vectors per slot (restart + 1)
  int nwork;            // KB_CHUNK-element chunks per vector (update sweep: one block each)
  int nchunk;           // dot-sweep blocks per slot (each sums several chunks): partials per item
  int nitem;            // partial-sum items per slot (capacity): mp1 * S + S (S + 1) / 2
  const int* run;       // per-slot flags
  const double* sigma;  // [slot][mp1] scales of the stored basis vectors
  const double* bcoef;  // [slot][S*S + mp1*S]: R^{-1} / ||p|| (S x S), then -sigma_r (C R^{-1})_{r,i}
  double* part;         // [slot][nitem][nchunk]
  // solution update fused into a slot's last block: x += sum_i ycoef_i v~_i
  const double* ycoef;  // [slot][mp1] y_i sigma_i (written by the block's scalar step)
  void* X;              // [slot][n] at stride xss: cx<double>, or cx<dd> when x_dd
  long long xss;
  int x_dd;
  int* err;             // set to 1 when a bounded device wait runs out (nullable)
  int tx_extra;         // bytes the first bulk-copy stage announces beyond its copy (test hook; 0)
};

__host__ __device__ constexpr int block_items(int J, int S) { return J * S + S * (S + 1) / 2; }

struct CycleState {
  double* H;       // [slot][m][m+1]  column j holds rows 0..j+1
  double* cs;      // [slot][m]
  double* sn;      // [slot][m]
  double* g;       // [slot][m+1]
  double* sigma;   // [slot][m+1]
  double* ycoef;   // [slot][m+1]
  double* thr;     // [slot] stop threshold of the current cycle
  double* bnorm;   // [slot]
  float* nscale;   // [slot] 2^-e with 2^e ~ ||b|| (scales FP32 squared norms of residuals)
  double* resid;   // [slot] last true relative residual
  int* run;        // [slot]
  int* active;     // [slot]
  int* nsteps;     // [slot]
  int* itot;       // [slot] total inner iterations
  int* ncyc;       // [slot]
  int m;
  int max_iter;
  int max_outer;
  double tol;
  double inner_tol;  // > 0: mixed-precision inner criterion relative to beta
};

// pass B modes: operator, right-hand side, h only, raw column DFTs, and the
// operator's first half (column IDFT, h, w = E_k Q conj(h); no column DFT)
enum { PB_MATVEC = 0, PB_RHS = 1, PB_HOUT = 2, PB_FWD = 3, PB_INV = 4, PB_W = 5, PB_WF = 6 };
// pass C modes: K S, right-hand side, FP64 residual, raw row DFTs
enum { PC_KS = 0, PC_RHS = 1, PC_RES = 2, PC_FWD = 3, PC_INV = 4 };

}  // namespace dbar
