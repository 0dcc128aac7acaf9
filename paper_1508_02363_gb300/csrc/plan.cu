// Plan, solve driver and C ABI of the spectral D-bar CGO solver.
//
// The driver runs the Sec. 4.3 algorithm (with Q -> E_k Q, Sec. 5.1) for a
// batch of k values on one GPU: right-hand side b = -i F(E_k Q), then GMRES
// cycles on the stacked real system.  In DBAR_FP64 mode a cycle is a
// restarted FP64 GMRES cycle; in DBAR_MIXED mode a cycle is an FP32 GMRES
// correction solve A d = r followed by the FP64 update x += d and the FP64
// true residual r = b - A x (iterative refinement).  Both end each cycle with
// the true FP64 residual, so the reported residual is always the FP64 one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <array>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/dbar.h"
#include "launch.cuh"
#include "plan_internal.h"

using namespace dbar;
typedef std::complex<double> zd;

namespace dbar {
// kern_aux.cu: ex[s][j] = e^{-2i k2 x_j}, ey[s][j] = e^{-2i k1 x_j} for k (device, [nb][2]) on the grid of box L
cudaError_t launch_fill_ek(const double* k, int nb, int N, double L, cx<double>* ex, cx<double>* ey, cudaStream_t s);
// kern_aux.cu: one bounded mbarrier wait (out[0] completed, out[1] copied word, out[2] rounds)
cudaError_t launch_wait_check(int complete, int rounds, const int4* src, int* out, cudaStream_t s);
int wait_limit_rounds();
}  // namespace dbar

static thread_local std::string g_last_error;

static dbar_status fail(dbar_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

dbar_status dbar_internal_fail(dbar_status st, const std::string& msg) { return fail(st, msg); }

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(e_ == cudaErrorMemoryAllocation ? DBAR_ENOMEM : DBAR_ECUDA,                \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

// Taylor orders up to which the column pass also skips its table loads on the rows
// outside the potential's support
constexpr int kRowBandMaxM = 4;

// Kernel kinds for the event profiler (dbar_profile_*).
enum {
  K_PASS_A, K_PASS_B, K_PASS_C, K_DOTS, K_UPDATE, K_SCALAR, K_XUPDATE,
  K_RES_A, K_RES_B, K_RES_C, K_RHS, K_OTHER, K_PASS_CA, K_CONV, K_NKINDS
};
static const char* const kKindNames[K_NKINDS] = {
    "inner_pass_a_rows", "inner_pass_b_cols", "inner_pass_c_rows", "arnoldi_dots", "arnoldi_update",
    "krylov_scalar", "solution_update", "fp64_residual_pass_a", "fp64_residual_pass_b",
    "fp64_residual_pass_c", "rhs", "other", "inner_pass_ca_rows", "conv_direct_sum"};

// CUDA-event timing of every launch of the solve, grouped by kind, plus the
// algorithmic bytes of each kind (fields read and written once per use).
struct Profiler {
  bool on = false;
  struct Rec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> pending;
  double ms[K_NKINDS] = {0};
  long long launches[K_NKINDS] = {0};
  double bytes[K_NKINDS] = {0};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void reset() {
    harvest();
    for (int i = 0; i < K_NKINDS; ++i) ms[i] = bytes[i] = 0, launches[i] = 0;
  }
  // after a stream synchronisation: fold every recorded pair into the totals
  void harvest() {
    for (const Rec& r : pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.kind] += t;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
    cudaGetLastError();
  }
  ~Profiler() {
    for (const Rec& r : pending) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

// A Krylov cycle as CUDA graphs: one graph per chunk of kGraphChunk steps and
// one for the cycle's tail (solution update, true residual, next start).
constexpr int kGraphChunk = 8;
struct GraphPart {
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;                      // kernel nodes per replay
  std::vector<Profiler::Rec> recs;      // event-record pairs captured with the kernels
};
struct CycleGraph {
  int nb = -1;
  bool prof = false;
  std::vector<GraphPart> parts;         // chunks 0..nchunks-1, then the tail
  void clear() {
    for (GraphPart& g : parts) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (const Profiler::Rec& r : g.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
      }
    }
    parts.clear();
    nb = -1;
  }
};

struct dbar_plan {
  dbar_params p;
  Profiler prof;
  cudaStream_t cap_stream = nullptr;    // stream the cycle graphs are captured on
  bool capturing = false;
  GraphPart* cap = nullptr;             // graph part being captured
  std::vector<GraphPart*> graph_ran;    // parts replayed since the last profile harvest
  CycleGraph graphs[2];                 // one per batch size in use (full and ragged)
  int per_slot_q = 0;   // 1: every slot has its own potential (serving); 0: one Q for all
  int colv = 0;         // FP32 column-pass tile variant (autotuned)
  double tune_ms[DBAR_COLUMN_VARIANTS] = {0.0, 0.0, 0.0};
  int rowv = 0;         // row-pass shape of the FP32 fused chain pass (autotuned)
  double row_ms[DBAR_ROW_VARIANTS] = {0.0, 0.0, 0.0, 0.0, 0.0};
  int rowv_ac = 0;      // row-pass shape of the FP32 passes A and C (autotuned separately)
  double row_ms_ac[DBAR_ROW_VARIANTS] = {0.0, 0.0, 0.0, 0.0, 0.0};
  int* dmask = nullptr;  // [B] device copy of a slot mask
  int* hmask = nullptr;  // [B] pinned host staging of it
  long long nlaunch = 0;  // kernels launched by this plan
  int N = 0, logN = 0, M = 0, MA = 0, B = 0, m = 0;
  int Min = 0;          // Taylor order of the FP32 inner passes (params.inner_M, else M)
  bool mixed = false;
  int device = 0;
  long long n = 0;  // N*N
  size_t bytes = 0;
  std::vector<void*> allocs;

  // tables
  cx<double>* tw64 = nullptr;
  cx<float>* tw32 = nullptr;
  cx<double>* Da64 = nullptr;
  cx<float>* Da32 = nullptr;
  cx<double>* Delta64 = nullptr;  // Delta_n = W_n - V_n, [n][y][x]
  cx<float>* Delta32 = nullptr;
  cx<double>* Q64 = nullptr;
  cx<float>* Q32 = nullptr;
  cx<double>* Qdev = nullptr;  // staging for a host Q
  cx<double>* ex64 = nullptr;
  cx<double>* ey64 = nullptr;
  cx<float>* ex32 = nullptr;
  cx<float>* ey32 = nullptr;
  // double-float copies for the right-hand side and residual of the mixed path
  bool resid_dd = false;
  cx<dd>* tw_dd = nullptr;
  cx<dd>* Da_dd = nullptr;
  cx<dd>* Delta_dd = nullptr;
  cx<dd>* Q_dd = nullptr;
  cx<dd>* ex_dd = nullptr;
  cx<dd>* ey_dd = nullptr;
  // workspaces
  // x and b: FP64, or double-float pairs (cx<dd>, same size) when the mixed
  // path's residual runs in double-float (resid_dd) -- see solution_fp64()
  cx<double>* x64 = nullptr;
  cx<double>* b64 = nullptr;
  void* T1 = nullptr;
  void* T2 = nullptr;
  void* V = nullptr;
  void* KS = nullptr;
  cx<double>* partA = nullptr;
  double* part = nullptr;
  double* part2 = nullptr;
  double* coef = nullptr;
  cx<double>* tcoef = nullptr;  // [B][M+2] Taylor coefficients of the field in flight
  cx<double>* coefp = nullptr;  // [B][N / coef_rows(N)][M+2] k_coef block partials
  int* ticket = nullptr;        // [B] k_coef completion counters (zero between launches)
  cx<double>* s0buf = nullptr;  // [B] solutions at xi = 0 (reflection coefficient)
  // iterated equation of Sec. 5 (params.iterated)
  bool iter = false;
  int* rolls = nullptr;         // [B][2] grid offset of xi0 = 2i conj(k) per slot, mod N (device)
  int* h_rolls = nullptr;       // [B][2] host staging
  int* dshift = nullptr;        // [B][2] the same offsets signed, in (-N/2, N/2] (pass A's divisor)
  int* h_dshift = nullptr;      // [B][2] host staging
  int* h_err = nullptr;         // pinned copy of flag[1]: a bounded device wait ran out
  // support of the potential in FP32 (Q32 exactly zero outside): columns [sx0, sx1), aligned
  // to every column-pass tile width; used by the FP32 inner operator and the double-float residual
  bool sup = false;
  int sx0 = 0, sx1 = 0, sy0 = 0, sy1 = 0;
  int* supflag = nullptr;       // [2N] device: column, then row flags of the support scan
  const cx<double>* x0d = nullptr;  // FP64 initial guesses of the batch being started (device), or none
  int inject_tx = 0;            // test hook: extra bytes announced by the next block-update launch
  void* It1 = nullptr;          // [B][n] rolled field (FP64-sized)
  void* It2 = nullptr;          // [B][n] first operator application (FP64-sized)
  // convolution regularisation (params.regularisation = DBAR_REG_CONV), FP64
  bool conv = false;
  cx<double>* Kt = nullptr;     // [2N-1][2N] (h^2/2pi) W_0(h(dx + i dy)) at [dy + N-1][dx + N-1]
  cx<double>* Mu = nullptr;     // [N][N] (-1)^{p1+p2} (1 - e^{-|xi|^2})/(xi 2 pi L^2), 0 at xi = 0
  cx<double>* Cv1 = nullptr;    // [B][2][n] smooth part and F^{-1} S (two fields per slot)
  cx<double>* Cv2 = nullptr;    // [B][2][n] their row transforms
  long long* gat = nullptr;     // [B] per-slot element index for the S(0) / h(xi0) gather
  cx<double>* ones64 = nullptr;  // [B][N] ones (E = 1), in each arithmetic
  cx<float>* ones32 = nullptr;
  cx<dd>* ones_dd = nullptr;
  int* flag = nullptr;
  CycleState cs;
  // s-step blocks (sstep > 1)
  int sstep = 1;
  int nchunk_b = 0, nitem_b = 0;
  double* Hraw = nullptr;   // [B][m][m+1] unrotated Hessenberg columns
  double* bcoef = nullptr;  // [B][S*S + (m+1)*S] sweep coefficients
  double* bpart = nullptr;  // [B][nitem_b][min(nchunk_b, kBlockDotBlocks)] block dot partials
  int* upd = nullptr;       // [B] slots whose block needs the update sweep
  // host staging
  int* h_active = nullptr;
  int* h_run = nullptr;  // [B] page-locked copy of the run flags after a cycle part (server stepping)
  int* h_nsteps = nullptr;
  cx<double>* h_ek = nullptr;  // pinned [B][2N]
  double* h_k = nullptr;       // pinned [B][2] k values of the batch being loaded
  double* kdev = nullptr;      // [B][2] the same on the device (E_k tables built there)

  double inv2piL = 0, sw = 0, fillscale = 0;

  bool dry = false;  // alloc() only counts bytes (the footprint of a mem_budget check)
  template <typename X>
  cudaError_t alloc(X** ptr, size_t count) {
    if (dry) {
      bytes += count * sizeof(X);
      *ptr = nullptr;
      return cudaSuccess;
    }
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(X));
    if (e != cudaSuccess) return e;
    allocs.push_back(q);
    bytes += count * sizeof(X);
    *ptr = reinterpret_cast<X*>(q);
    return cudaSuccess;
  }
  ~dbar_plan() {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(device);
    for (CycleGraph& g : graphs) g.clear();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* q : allocs) cudaFree(q);
    if (h_active) cudaFreeHost(h_active);
    if (h_nsteps) cudaFreeHost(h_nsteps);
    if (h_rolls) cudaFreeHost(h_rolls);
    if (h_dshift) cudaFreeHost(h_dshift);
    if (h_err) cudaFreeHost(h_err);
    if (hmask) cudaFreeHost(hmask);
    if (h_ek) cudaFreeHost(h_ek);
    if (h_k) cudaFreeHost(h_k);
    if (h_run) cudaFreeHost(h_run);
    cudaSetDevice(cur);
  }
  size_t inner_elem() const { return mixed ? sizeof(cx<float>) : sizeof(cx<double>); }
};

extern "C" void dbar_params_init(dbar_params* p, int N, double L) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->N = N;
  p->L = L;
  p->M = 2;
  p->prec = DBAR_MIXED;
  p->restart = 32;
  p->max_iter = 4000;
  p->tol = 1e-12;
  p->zero_fill = 0;
  p->max_batch = 0;
  p->inner_tol = 1e-6;
  p->max_outer = 40;
  p->resid_mode = DBAR_RESID_DOUBLE_FLOAT;
  p->graphs = 1;
  p->autotune = 1;
  p->gauss_w = 1.0;
  p->mem_budget = 0;
  p->support_skip = 1;
}

extern "C" const char* dbar_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Host-side tables (FP64, plain libm).
// ---------------------------------------------------------------------------

// W_n(z) = F^{-1}(conj(xi)^n/xi e^{-|xi|^2}) (Sec. 4.2, eq. fourreg5): with a = |z|^2/4,
//   closed form  i(2i)^n n!/z^{n+1} (1 - e^{-a} sum_{k<=n} a^k/k!)        (a >= n+1)
//   series       i(2i)^n n! (conj z/4)^{n+1} e^{-a} sum_{j>=0} a^j/(j+n+1)! (a <  n+1),
// the series being the expansion of the same bracket without cancellation.
static zd W_host(int n, zd z) {
  const double a = std::norm(z) / 4.0;
  zd pref(0.0, 1.0);
  double fact = 1.0;
  for (int r = 1; r <= n; ++r) {
    pref *= zd(0.0, 2.0);
    fact *= r;
  }
  pref *= fact;
  if (a < n + 1) {
    double term = 1.0;
    for (int r = 2; r <= n + 1; ++r) term /= r;  // 1/(n+1)!
    double acc = 0.0;
    for (int j = 0; j < 400; ++j) {
      acc += term;
      term *= a / (double)(j + n + 2);
      if (term < 1e-18 * acc) break;
    }
    zd pw(1.0, 0.0);
    const zd zb4 = std::conj(z) / 4.0;
    for (int r = 0; r <= n; ++r) pw *= zb4;
    return pref * pw * (std::exp(-a) * acc);
  }
  double part = 0.0, term = 1.0;
  for (int r = 0; r <= n; ++r) {
    if (r > 0) term *= a / r;
    part += term;
  }
  zd zp(1.0, 0.0);
  for (int r = 0; r <= n; ++r) zp *= z;
  return pref / zp * (1.0 - std::exp(-a) * part);
}

static double xgrid(int j, int N, double L) { return L * (-M_PI + 2.0 * M_PI * (double)j / (double)N); }

// Launch through the profiler: counts the launch and, when profiling is on,
// brackets it with CUDA events on the launching stream.
// f launches nk kernels (counted in dbar_launch_count)
template <typename F>
static cudaError_t timed(dbar_plan* P, cudaStream_t st, int kind, F&& f, int nk = 1) {
  if (P->capturing) {  // recorded into the cycle graph: counted and timed at each replay
    P->cap->kernels += nk;
    if (!P->prof.on) return f();
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecordWithFlags(a, st, cudaEventRecordExternal);  // a node that records at each replay
    cudaError_t e = f();
    cudaEventRecordWithFlags(b, st, cudaEventRecordExternal);
    P->cap->recs.push_back({kind, a, b});
    return e;
  }
  P->nlaunch += nk;
  if (!P->prof.on) return f();
  cudaEvent_t a = P->prof.get(), b = P->prof.get();
  cudaEventRecord(a, st);
  cudaError_t e = f();
  cudaEventRecord(b, st);
  P->prof.pending.push_back({kind, a, b});
  P->prof.launches[kind] += 1;
  return e;
}

static void fill_ek(const dbar_plan* P, const double* k, int nb, cx<double>* dst /*[nb][2N]*/) {
  const int N = P->N;
  for (int s = 0; s < nb; ++s) {
    const double k1 = k[2 * s], k2 = k[2 * s + 1];
    for (int j = 0; j < N; ++j) {
      const double x = xgrid(j, N, P->p.L);
      // E_k = exp(conj(kz) - kz) = exp(-2i (k2 x + k1 y)) = ex(x) ey(y)
      dst[(size_t)s * 2 * N + j] = mkc(std::cos(2.0 * k2 * x), -std::sin(2.0 * k2 * x));
      dst[(size_t)s * 2 * N + N + j] = mkc(std::cos(2.0 * k1 * x), -std::sin(2.0 * k1 * x));
    }
  }
}

static dbar_status upload_ek(dbar_plan* P, const double* k, int nb, cudaStream_t st) {
  const int N = P->N;
  if (P->iter) {
    // Sec. 5.3: xi0 = 2i conj(k) = 2 k2 + 2i k1 must be a grid point, offset (2 k2 L, 2 k1 L)
    for (int s = 0; s < nb; ++s) {
      const double m1 = 2.0 * k[2 * s + 1] * P->p.L, m2 = 2.0 * k[2 * s] * P->p.L;
      const double r1 = std::nearbyint(m1), r2 = std::nearbyint(m2);
      if (std::fabs(m1 - r1) > 1e-9 || std::fabs(m2 - r2) > 1e-9)
        return fail(DBAR_EINVAL, "iterated plan: 2k must lie on the xi-grid (2 k L integer in both components)");
      if (std::fabs(r1) > N / 2 || std::fabs(r2) > N / 2)
        return fail(DBAR_EINVAL, "iterated plan: 2 k L must lie within the grid's wavenumbers [-N/2, N/2]");
      P->h_rolls[2 * s] = (int)(((long long)r1 % N + N) % N);
      P->h_rolls[2 * s + 1] = (int)(((long long)r2 % N + N) % N);
      // signed offsets in (-N/2, N/2]: -N/2 is the Nyquist point, held on the positive side
      P->h_dshift[2 * s] = P->h_rolls[2 * s] > N / 2 ? P->h_rolls[2 * s] - N : P->h_rolls[2 * s];
      P->h_dshift[2 * s + 1] = P->h_rolls[2 * s + 1] > N / 2 ? P->h_rolls[2 * s + 1] - N : P->h_rolls[2 * s + 1];
    }
    CK(cudaMemcpyAsync(P->rolls, P->h_rolls, 2 * nb * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(P->dshift, P->h_dshift, 2 * nb * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  // E_k tables of the batch built on the device from its k values (one copy of 16 bytes per k;
  // the previous batch's copy has completed: every cycle loop ends with a stream synchronisation)
  std::memcpy(P->h_k, k, 2 * (size_t)nb * sizeof(double));
  CK(cudaMemcpyAsync(P->kdev, P->h_k, 2 * (size_t)nb * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(timed(P, st, K_OTHER, [&] { return launch_fill_ek(P->kdev, nb, N, P->p.L, P->ex64, P->ey64, st); }));
  CK(timed(P, st, K_OTHER, [&] { return launch_cast_fields(P->ex64, P->ex32, (long long)nb * N, st); }));
  CK(timed(P, st, K_OTHER, [&] { return launch_cast_fields(P->ey64, P->ey32, (long long)nb * N, st); }));
  if (P->resid_dd) {
    CK(timed(P, st, K_OTHER, [&] { return launch_split_fields(P->ex64, P->ex_dd, (long long)nb * N, st); }));
    CK(timed(P, st, K_OTHER, [&] { return launch_split_fields(P->ey64, P->ey_dd, (long long)nb * N, st); }));
  }
  return DBAR_OK;
}

template <typename T>
static PassArgs<T> base_args(const dbar_plan* P);

template <>
PassArgs<double> base_args<double>(const dbar_plan* P) {
  PassArgs<double> a;
  std::memset(&a, 0, sizeof(a));
  a.g = make_geo<double>(P->N);
  a.sx1 = a.sy1 = P->N;
  a.M = P->M;
  a.tw = P->tw64;
  a.Da = P->Da64;
  a.Da64 = P->Da64;
  a.Delta = P->Delta64;
  a.Q = P->Q64;
  a.ex = P->ex64;
  a.ey = P->ey64;
  a.inv2piL = P->inv2piL;
  a.inv2piL_f = (float)P->inv2piL;
  a.hx_f = (float)(2.0 * M_PI * P->p.L / P->N);
  a.sw = P->sw;
  a.fillscale = P->fillscale;
  a.partA = P->partA;
  a.nseg = seg_count(P->N);
  a.coef = P->tcoef;
  a.q_ss = P->per_slot_q ? P->n : 0;
  a.part = P->part2;
  a.nscale = P->cs.nscale;
  return a;
}
template <>
PassArgs<float> base_args<float>(const dbar_plan* P) {
  PassArgs<float> a;
  std::memset(&a, 0, sizeof(a));
  a.colv = P->colv;
  a.rowv = P->rowv_ac;  // passes A and C; the fused chain pass sets its own (P->rowv)
  a.g = make_geo<float>(P->N);
  a.sx1 = a.sy1 = P->N;
  a.M = P->Min;
  a.tw = P->tw32;
  a.Da = P->Da32;
  a.Da64 = P->Da64;
  a.Delta = P->Delta32;
  a.Q = P->Q32;
  a.ex = P->ex32;
  a.ey = P->ey32;
  a.inv2piL = P->inv2piL;
  a.inv2piL_f = (float)P->inv2piL;
  a.hx_f = (float)(2.0 * M_PI * P->p.L / P->N);
  a.sw = P->sw;
  a.fillscale = P->fillscale;
  a.partA = P->partA;
  a.nseg = seg_count(P->N);
  a.coef = P->tcoef;
  a.q_ss = P->per_slot_q ? P->n : 0;
  a.part = P->part2;
  a.nscale = P->cs.nscale;
  return a;
}

template <>
PassArgs<dd> base_args<dd>(const dbar_plan* P) {
  PassArgs<dd> a;
  std::memset(&a, 0, sizeof(a));
  a.g = make_geo<dd>(P->N);
  a.sx1 = a.sy1 = P->N;
  a.M = P->M;
  a.tw = P->tw_dd;
  a.Da = P->Da_dd;
  a.Da64 = P->Da64;
  a.Delta = P->Delta_dd;
  a.Q = P->Q_dd;
  a.ex = P->ex_dd;
  a.ey = P->ey_dd;
  a.inv2piL = P->inv2piL;
  a.inv2piL_f = (float)P->inv2piL;
  a.hx_f = (float)(2.0 * M_PI * P->p.L / P->N);
  a.sw = P->sw;
  a.fillscale = P->fillscale;
  a.partA = P->partA;
  a.nseg = seg_count(P->N);
  a.coef = P->tcoef;
  a.q_ss = P->per_slot_q ? P->n : 0;
  a.part = P->part2;
  a.nscale = P->cs.nscale;
  return a;
}

// E = 1 in the column pass: per-slot rows of ones in place of the slot's E_k
// factors (K_0 of the iterated equation, its right-hand side); the same layout
// keeps the column pass's indexing unchanged
// The FP32 inner operator's passes skip the columns where the potential is exactly
// zero in FP32 (and its column pass the table loads on the rows where it is): there
// w = E_k Q conj(h) = 0, so the skipped work is exactly zero (the same values as the
// full passes).  The double-float copy of Q
// is a pair of floats, zero exactly where the FP32 copy is, so the double-float
// right-hand side and residual passes skip the same columns and rows.
template <typename T>
static void set_support(const dbar_plan* P, PassArgs<T>& a) {
  if constexpr (std::is_same<T, float>::value || std::is_same<T, dd>::value) {
    if (P->sup) {
      a.sx0 = P->sx0;
      a.sx1 = P->sx1;
      // the row band only for low Taylor orders: at larger ones the per-row test costs the
      // table loads' batching more than the skipped loads save
      if ((std::is_same<T, float>::value ? P->Min : P->M) <= kRowBandMaxM) {
        a.sy0 = P->sy0;
        a.sy1 = P->sy1;
      }
    }
  }
}

template <typename T>
static void set_unit_e(const dbar_plan* P, PassArgs<T>& a) {
  if constexpr (std::is_same<T, float>::value) a.ex = a.ey = P->ones32;
  else if constexpr (std::is_same<T, double>::value) a.ex = a.ey = P->ones64;
  else a.ex = a.ey = P->ones_dd;
}

// Taylor coefficients of the fields pass A just read (k_coef), for pass B.
template <typename T>
static cudaError_t launch_coef_for(dbar_plan* P, const PassArgs<T>& a, int nb, cudaStream_t st) {
  return launch_coef(P->partA, std::is_same<T, float>::value, a.M, P->N, P->Da64, P->Da32, P->fillscale,
                     P->coefp, P->ticket, P->tcoef, nb, st);
}

// Convolution regularisation (Sec. 4.2, remark after eq. fourreg5a), FP64:
// h(S) = F^{-1}(S (1 - e^{-|xi|^2})/xi) + (1/2pi) sum over the grid of F^{-1}(S)(z') W_0(z - z') h^2.
// Split S into the two fields, inverse-transform both (2 nb fields through the raw
// row and column transforms), then the direct sum: out = h (w_out = 0) or
// out = sw E_k Q conj(h) (w_out = 1, the field the operator's forward transform takes).
static dbar_status conv_h(dbar_plan* P, const cx<double>* S, long long s_ss, const double* scale, int scale_ss,
                          const int* run, int w_out, cx<double>* out, long long o_ss, int nb, cudaStream_t st) {
  const long long n = P->n;
  const double inv2piL2 = 1.0 / (2.0 * M_PI * P->p.L * P->p.L);
  CK(timed(P, st, K_OTHER, [&] {
    return launch_conv_split(S, s_ss, scale, scale_ss, run, P->Mu, inv2piL2, P->N, P->Cv1, nb, st);
  }));
  PassArgs<double> a = base_args<double>(P);
  a.in = P->Cv1;
  a.in_ss = n;
  a.out = P->Cv2;
  a.out_ss = n;
  CK(timed(P, st, K_OTHER, [&] { return launch_pass_c<double, double, PC_INV>(a, 2 * nb, st); }));
  a.in = P->Cv2;
  a.out = P->Cv1;
  CK(timed(P, st, K_OTHER, [&] { return launch_pass_b<double, PB_INV>(a, 2 * nb, st); }));
  CK(timed(P, st, K_CONV, [&] {
    return launch_conv_sum(P->Cv1, P->Kt, P->N, run, P->Q64, a.q_ss, P->ex64, P->ey64, P->sw, w_out, out, o_ss, nb,
                           st);
  }));
  return DBAR_OK;
}

// The convolution route up to the state the fused column pass leaves in T2:
// w = sw E_k Q conj(h(S)) in T1, then its column DFT -> T2.
static dbar_status conv_to_T2(dbar_plan* P, const cx<double>* S, long long s_ss, const double* scale, int scale_ss,
                              const int* run, int nb, cudaStream_t st) {
  dbar_status s = conv_h(P, S, s_ss, scale, scale_ss, run, 1, reinterpret_cast<cx<double>*>(P->T1), P->n, nb, st);
  if (s != DBAR_OK) return s;
  PassArgs<double> a = base_args<double>(P);
  a.run = run;
  a.in = reinterpret_cast<const cx<double>*>(P->T1);
  a.in_ss = P->n;
  a.out = P->T2;
  a.out_ss = P->n;
  CK(timed(P, st, K_OTHER, [&] { return launch_pass_b<double, PB_FWD>(a, nb, st); }));
  return DBAR_OK;
}

// One application of K (A S = S + K S) to nb fields: S (T) -> T1 -> T2 -> out (T).
template <typename T>
static dbar_status apply_K(dbar_plan* P, const cx<T>* S, long long s_ss, const double* scale, int scale_ss,
                           cx<T>* out, long long o_ss, const int* run, int nb, cudaStream_t st, int unitE = 0,
                           int neg = 0, const int* dshift = nullptr) {
  PassArgs<T> a = base_args<T>(P);
  a.run = run;
  a.dshift = dshift;
  if (unitE) set_unit_e(P, a);
  a.neg = neg;
  set_support(P, a);
  if constexpr (std::is_same<T, double>::value) {
    if (P->conv) {  // convolution regularisation: T2 from the direct-sum route, then pass C
      dbar_status s = conv_to_T2(P, S, s_ss, scale, scale_ss, run, nb, st);
      if (s != DBAR_OK) return s;
      a.in = reinterpret_cast<const cx<T>*>(P->T2);
      a.in_ss = P->n;
      a.out = out;
      a.out_ss = o_ss;
      CK(timed(P, st, K_PASS_C, [&] { return launch_pass_c<T, T, PC_KS>(a, nb, st); }));
      return DBAR_OK;
    }
  }
  a.in = S;
  a.in_ss = s_ss;
  a.in_scale = scale;
  a.in_scale_ss = scale_ss;
  a.out = P->T1;
  a.out_ss = P->n;
  CK(timed(P, st, K_PASS_A, [&] { return launch_pass_a<T>(a, nb, st); }));
  CK(timed(P, st, K_SCALAR, [&] { return launch_coef_for(P, a, nb, st); }));
  a.in = reinterpret_cast<const cx<T>*>(P->T1);
  a.in_ss = P->n;
  a.in_scale = nullptr;
  a.out = P->T2;
  CK(timed(P, st, K_PASS_B, [&] { return launch_pass_b<T, PB_MATVEC>(a, nb, st); }));
  a.in = reinterpret_cast<const cx<T>*>(P->T2);
  a.out = out;
  a.out_ss = o_ss;
  CK(timed(P, st, K_PASS_C, [&] { return launch_pass_c<T, T, PC_KS>(a, nb, st); }));
  return DBAR_OK;
}

// The operator's K on nb fields: A = I + K.  Sec. 4 method: K = apply_K with
// E_k.  Iterated equation of Sec. 5 (eq. eqh2): A h = h - K_0(H(h)) with
// H(h) = -i F(q conj(F^{-1}(h/(xi - xi0)))) and K_0(S) = -i F(q conj(F^{-1}(S/xi))).
// By the shifted regularisation (eq. dbarinvShift), F^{-1}(h/(xi - xi0)) =
// e^{i xi0.x} F^{-1}(h~/(xi - xi0)~) with h~ = h(. + xi0) (a circular shift, which
// moves the Taylor data at xi0 to the origin) and the divisor taken at the unshifted
// points (no periodic wrap of xi - xi0: pass A's dshift); e^{-i xi0.x} = E_k, so
// H(h) = -K_{E_k}(h~), K_0(S) = -K_1(S) and K_it(h) = -K_1(K_{E_k}(h~)):
// a circular shift, one application with E_k, one with E = 1 and the sign.
template <typename T>
static dbar_status apply_op(dbar_plan* P, const cx<T>* S, long long s_ss, const double* scale, int scale_ss,
                            cx<T>* out, long long o_ss, const int* run, int nb, cudaStream_t st) {
  if (!P->iter) return apply_K<T>(P, S, s_ss, scale, scale_ss, out, o_ss, run, nb, st);
  const long long n = P->n;
  cx<T>* R = reinterpret_cast<cx<T>*>(P->It1);
  cx<T>* H = reinterpret_cast<cx<T>*>(P->It2);
  CK(timed(P, st, K_OTHER, [&] { return launch_roll<T>(S, s_ss, scale, scale_ss, P->rolls, run, P->N, R, n, nb, st); }));
  dbar_status s = apply_K<T>(P, R, n, nullptr, 0, H, n, run, nb, st, 0, 0, P->dshift);
  if (s != DBAR_OK) return s;
  return apply_K<T>(P, H, n, nullptr, 0, out, o_ss, run, nb, st, 1, 1);
}

// h(S) for FP64 fields (m output): pass A then pass B without the forward transform.
static dbar_status h_of_S64(dbar_plan* P, const cx<double>* S, long long s_ss, cx<double>* out, long long o_ss,
                            int nb, cudaStream_t st) {
  if (P->conv) return conv_h(P, S, s_ss, nullptr, 0, nullptr, 0, out, o_ss, nb, st);
  PassArgs<double> a = base_args<double>(P);
  a.in = S;
  a.in_ss = s_ss;
  a.out = P->T1;
  a.out_ss = P->n;
  CK(timed(P, st, K_OTHER, [&] { return launch_pass_a<double>(a, nb, st); }));
  CK(timed(P, st, K_OTHER, [&] { return launch_coef_for(P, a, nb, st); }));
  a.in = reinterpret_cast<const cx<double>*>(P->T1);
  a.in_ss = P->n;
  a.out = out;
  a.out_ss = o_ss;
  CK(timed(P, st, K_OTHER, [&] { return launch_pass_b<double, PB_HOUT>(a, nb, st); }));
  return DBAR_OK;
}

// b = -i F(E_k Q) computed in TC (FP64 or double-float) -> b64 (FP64 storage),
// the Krylov start vector V[slot][0] (TI) and |b|^2 partials.
template <typename TC, typename TI>
static dbar_status build_rhs_t(dbar_plan* P, int nb, cudaStream_t st, const int* dmask) {
  PassArgs<TC> a = base_args<TC>(P);
  set_support(P, a);
  a.run = dmask;
  if (P->iter) set_unit_e(P, a);  // iterated equation: b = -i F(q)
  a.out = P->T2;
  a.out_ss = P->n;
  CK(timed(P, st, K_RHS, [&] { return launch_pass_b<TC, PB_RHS>(a, nb, st); }));
  a.in = reinterpret_cast<const cx<TC>*>(P->T2);
  a.in_ss = P->n;
  a.out = P->b64;
  a.out_ss = P->n;
  a.out2 = P->V;
  a.out2_ss = (long long)(P->m + 1) * P->n;
  CK(timed(P, st, K_RHS, [&] { return launch_pass_c<TC, TI, PC_RHS>(a, nb, st); }));
  return DBAR_OK;
}

// r = b - A x computed in TC from the FP64 x and b -> V[slot][0] (TI) and |r|^2
// partials; only active slots.
template <typename TC, typename TI>
static dbar_status true_residual_t(dbar_plan* P, int nb, cudaStream_t st) {
  const long long n = P->n;
  // pass A, Taylor coefficients and the column pass on `in` -> T2
  auto passes_ab = [&](const cx<TC>* in, int unitE, const int* dshift) -> dbar_status {
    if constexpr (std::is_same<TC, double>::value)
      if (P->conv) return conv_to_T2(P, in, n, nullptr, 0, P->cs.active, nb, st);
    PassArgs<TC> a = base_args<TC>(P);
    set_support(P, a);
    a.run = P->cs.active;
    a.dshift = dshift;
    if (unitE) set_unit_e(P, a);
    a.in = in;
    a.in_ss = n;
    a.out = P->T1;
    a.out_ss = n;
    CK(timed(P, st, K_RES_A, [&] { return launch_pass_a<TC>(a, nb, st); }));
    CK(timed(P, st, K_SCALAR, [&] { return launch_coef_for(P, a, nb, st); }));
    a.in = reinterpret_cast<const cx<TC>*>(P->T1);
    a.out = P->T2;
    if constexpr (std::is_same<TC, dd>::value) {
      // one launch whose two transforms share one copy of the code (PB_WF): two
      // inlined double-float transforms would not fit the instruction cache
      CK(timed(P, st, K_RES_B, [&] { return launch_pass_b<TC, PB_WF>(a, nb, st); }));
    } else {
      CK(timed(P, st, K_RES_B, [&] { return launch_pass_b<TC, PB_MATVEC>(a, nb, st); }));
    }
    return DBAR_OK;
  };
  const cx<TC>* x = reinterpret_cast<const cx<TC>*>(P->x64);  // x stored in TC (FP64 or double-float)
  dbar_status s;
  PassArgs<TC> c = base_args<TC>(P);
  set_support(P, c);
  c.run = P->cs.active;
  c.in_ss = n;
  if (P->iter) {
    // K_it x = -K_1(K_{E_k}(x~)): shift, one application with E_k (-> It2), then E = 1 and the sign
    cx<TC>* R = reinterpret_cast<cx<TC>*>(P->It1);
    cx<TC>* H = reinterpret_cast<cx<TC>*>(P->It2);
    CK(timed(P, st, K_OTHER, [&] {
      return launch_roll<TC>(x, n, nullptr, 0, P->rolls, P->cs.active, P->N, R, n, nb, st);
    }));
    if ((s = passes_ab(R, 0, P->dshift)) != DBAR_OK) return s;
    c.in = reinterpret_cast<const cx<TC>*>(P->T2);
    c.out = H;
    c.out_ss = n;
    CK(timed(P, st, K_RES_C, [&] { return launch_pass_c<TC, TC, PC_KS>(c, nb, st); }));
    if ((s = passes_ab(H, 1, nullptr)) != DBAR_OK) return s;
    c.neg = 1;
  } else {
    if ((s = passes_ab(x, 0, nullptr)) != DBAR_OK) return s;
  }
  c.in = reinterpret_cast<const cx<TC>*>(P->T2);
  c.out = nullptr;
  c.out2 = P->V;
  c.out2_ss = (long long)(P->m + 1) * n;
  c.b = reinterpret_cast<const cx<TC>*>(P->b64);
  c.x = x;
  c.f_ss = n;
  CK(timed(P, st, K_RES_C, [&] { return launch_pass_c<TC, TI, PC_RES>(c, nb, st); }));
  return DBAR_OK;
}

template <typename TI>
static dbar_status build_rhs(dbar_plan* P, int nb, cudaStream_t st, const int* dmask = nullptr) {
  if constexpr (std::is_same<TI, float>::value)
    if (P->resid_dd) return build_rhs_t<dd, TI>(P, nb, st, dmask);
  return build_rhs_t<double, TI>(P, nb, st, dmask);
}

template <typename TI>
static dbar_status true_residual(dbar_plan* P, int nb, cudaStream_t st) {
  if constexpr (std::is_same<TI, float>::value)
    if (P->resid_dd) return true_residual_t<dd, TI>(P, nb, st);
  return true_residual_t<double, TI>(P, nb, st);
}

// Algorithmic bytes of one finished cycle (profiling only): every field the
// method reads or writes counted once per use (the FP32 pass intermediates T1
// and T2 on the potential's support columns only), F = one inner-precision field,
// F64 = one FP64 field.  Per Krylov step j of a slot: pass A 2F (read v_j,
// write T1), pass B 2F (read T1, write T2), pass C 2F (read T2, write K v_j),
// dots (j+2)F (v_0..v_j and K v_j), update (j+3)F (the same, plus the new
// vector); per launch of pass B the shared tables Q and Delta_0..Delta_M,
// (M+2)F.  s-step blocks (J basis vectors, S chain steps): pass A 2F, S pass B
// 2F, S-1 fused row passes 3F (read T2, write K p_i and T1), one pass C 2F,
// block dots (J+S)F, block update (J+2S)F, plus x read and written (2 F64) by
// the last block's update sweep.  Per cycle and slot: solution update (one
// vector per sweep: ns F + 2 F64), residual passes 2 F64 + 2 F64 + (3 F64 + F), plus
// (M+2) F64 of tables per pass-B launch.
static void account_cycle(dbar_plan* P, const int* act, const int* ns, int nb, int launched_steps) {
  if (!P->prof.on) return;
  const double F = (double)P->n * P->inner_elem(), F64 = (double)P->n * sizeof(cx<double>);
  const double fx = P->sup ? (double)(P->sx1 - P->sx0) / P->N : 1.0;
  // table rows the column passes read (the support's rows at low Taylor orders)
  const double fy = (P->sup && (P->mixed ? P->Min : P->M) <= kRowBandMaxM) ? (double)(P->sy1 - P->sy0) / P->N : 1.0;
  // the double-float residual passes skip the same columns (FP64 ones do not)
  const double rx = P->resid_dd ? fx : 1.0;
  const double ry = (P->resid_dd && P->sup && P->M <= kRowBandMaxM) ? (double)(P->sy1 - P->sy0) / P->N : 1.0;
  double* by = P->prof.bytes;
  int nact = 0;
  for (int s = 0; s < nb; ++s) {
    if (!act[s]) continue;
    ++nact;
    const int k = ns[s];
    if (P->conv) {
      // direct sum: N^4 complex multiply-adds (8 N^4 flops) per field, for the
      // k Krylov steps and the cycle's true residual (this kind counts flops)
      const double NN = (double)P->n;
      by[K_CONV] += 8.0 * NN * NN * (k + 1);
      by[K_PASS_C] += 2.0 * F * k;
      by[K_DOTS] += F * (k * 2.0 + k * (k - 1) / 2.0);
      by[K_UPDATE] += F * (k * 3.0 + k * (k - 1) / 2.0);
      by[K_XUPDATE] += F * k + 2.0 * F64;
      by[K_RES_C] += 3.0 * F64 + F;
      continue;
    }
    // the pass intermediates T1, T2 hold only the support's columns (fraction fx)
    if (P->sstep > 1) {
      // per block at J = b S + 1: S applications of K, dots (J + S) F,
      // update (J + 2S) F; the last block of the cycle counts in full
      const int S = P->sstep, nblk = (k + S - 1) / S;
      for (int b = 0; b < nblk; ++b) {
        const int J = b * S + 1;
        by[K_PASS_A] += (1.0 + fx) * F;            // v_{J-1} -> T1
        by[K_PASS_B] += 2.0 * fx * F * S;
        by[K_PASS_CA] += (1.0 + 2.0 * fx) * F * (S - 1);  // T2 -> K p_i and T1
        by[K_PASS_C] += (1.0 + fx) * F;
        by[K_DOTS] += F * (J + S);
        by[K_UPDATE] += F * (J + 2 * S);
      }
      by[K_UPDATE] += 2.0 * F64;  // x read and written by the slot's last update sweep
    } else {
      by[K_PASS_A] += (1.0 + fx) * F * k;
      by[K_PASS_B] += 2.0 * fx * F * k;
      by[K_PASS_C] += (1.0 + fx) * F * k;
      by[K_DOTS] += F * (k * 2.0 + k * (k - 1) / 2.0);
      by[K_UPDATE] += F * (k * 3.0 + k * (k - 1) / 2.0);
    }
    if (P->sstep <= 1) by[K_XUPDATE] += F * k + 2.0 * F64;
    by[K_RES_A] += (1.0 + rx) * F64;
    by[K_RES_B] += 2.0 * rx * F64;
    by[K_RES_C] += (2.0 + rx) * F64 + F;
  }
  if (P->conv) return;
  // shared tables Q, Delta_n per launch, on the support's columns (and rows)
  by[K_PASS_B] += (double)launched_steps * ((P->mixed ? P->Min : P->M) + 2) * F * fx * fy;
  if (nact) by[K_RES_B] += (P->M + 2) * F64 * rx * ry;
}

// Starts slots: x = 0, b = -i F(E_k Q), first cycle state.  hmask == nullptr:
// all nb slots; else only the slots with hmask[slot] != 0 (the others keep
// running undisturbed).
template <typename TI>
static dbar_status begin_slots(dbar_plan* P, int nb, const int* hmask, cudaStream_t st) {
  const long long n = P->n;
  const int nblkC = row_blocks(P->N);
  const int* dmask = nullptr;
  int nnew = nb;
  if (hmask) {
    nnew = 0;
    for (int s = 0; s < nb; ++s) {
      P->hmask[s] = hmask[s] ? 1 : 0;
      nnew += P->hmask[s];
      if (hmask[s]) CK(cudaMemsetAsync(P->x64 + (size_t)s * n, 0, (size_t)n * sizeof(cx<double>), st));
    }
    CK(cudaMemcpyAsync(P->dmask, P->hmask, nb * sizeof(int), cudaMemcpyHostToDevice, st));
    dmask = P->dmask;
  } else if (P->x0d) {
    // the caller's initial guess (FP64 on the device) in x's storage format
    if (P->resid_dd)
      CK(timed(P, st, K_OTHER, [&] { return launch_split_fields(P->x0d, reinterpret_cast<cx<dd>*>(P->x64), (long long)nb * n, st); }));
    else
      CK(cudaMemcpyAsync(P->x64, P->x0d, (size_t)nb * n * sizeof(cx<double>), cudaMemcpyDeviceToDevice, st));
  } else {
    CK(cudaMemsetAsync(P->x64, 0, (size_t)nb * n * sizeof(cx<double>), st));
  }
  dbar_status s = build_rhs<TI>(P, nb, st, dmask);
  if (s != DBAR_OK) return s;
  CK(timed(P, st, K_SCALAR, [&] { return launch_cycle_start(P->cs, P->part2, nblkC, 1, nb, st, dmask); }));
  if (!hmask && P->x0d) {
    // start from the true residual b - A x0; ||b|| (set above) stays the reference
    s = true_residual<TI>(P, nb, st);
    if (s != DBAR_OK) return s;
    CK(timed(P, st, K_SCALAR, [&] { return launch_cycle_start(P->cs, P->part2, nblkC, 2, nb, st); }));
  }
  if (P->prof.on) {
    const double F = (double)n * P->inner_elem(), F64 = (double)n * sizeof(cx<double>);
    P->prof.bytes[K_RHS] += nnew * (4.0 * F64 + F) + (P->M + 2) * F64;
  }
  return DBAR_OK;
}

// s-step blocks covering Krylov steps j0 <= j < j1 (multiples of S): per block,
// S applications of K along the chain (written into basis slots J..J+S-1),
// one dot sweep, the per-slot FP64 step, one update sweep.
template <typename TI, int S>
static dbar_status block_steps(dbar_plan* P, int nb, int j0, int j1, cudaStream_t st) {
  const long long n = P->n;
  const int m = P->m;
  const long long vss = (long long)(m + 1) * n;
  cx<TI>* V = reinterpret_cast<cx<TI>*>(P->V);
  BlockArgs ba;
  ba.n = n;
  ba.mp1 = m + 1;
  ba.nwork = P->nchunk_b;
  ba.nchunk = std::min(P->nchunk_b, kBlockDotBlocks);
  ba.nitem = P->nitem_b;
  ba.run = P->cs.run;
  ba.sigma = P->cs.sigma;
  ba.bcoef = P->bcoef;
  ba.part = P->bpart;
  ba.ycoef = P->cs.ycoef;
  ba.X = P->x64;
  ba.xss = n;
  ba.x_dd = P->resid_dd ? 1 : 0;
  ba.err = P->flag + 1;
  ba.tx_extra = 0;
  for (int c0 = j0; c0 < j1; c0 += S) {
    const int J = c0 + 1;  // basis vectors v_0..v_{J-1} exist
    if (P->iter || P->conv) {
      // operators made of several applications (iterated equation, convolution
      // route): the chain p_{i+1} = K p_i one whole application at a time
      for (int i = 0; i < S; ++i) {
        const cx<TI>* pin = V + (size_t)(J - 1 + i) * n;
        dbar_status s = apply_op<TI>(P, pin, vss, i == 0 ? P->cs.sigma + (J - 1) : nullptr, i == 0 ? m + 1 : 0,
                                     V + (size_t)(J + i) * n, vss, P->cs.run, nb, st);
        if (s != DBAR_OK) return s;
      }
    } else {
    // the chain p_{i+1} = K p_i into basis slots J..J+S-1: pass A of v_{J-1};
    // per step the coefficients and pass B, then pass C fused with the next
    // step's pass A (the last step: pass C alone)
    PassArgs<TI> a = base_args<TI>(P);
    set_support(P, a);
    a.run = P->cs.run;
    a.in = V + (size_t)(J - 1) * n;
    a.in_ss = vss;
    a.in_scale = P->cs.sigma + (J - 1);
    a.in_scale_ss = m + 1;
    a.out = P->T1;
    a.out_ss = n;
    CK(timed(P, st, K_PASS_A, [&] { return launch_pass_a<TI>(a, nb, st); }));
    a.in_scale = nullptr;
    for (int i = 0; i < S; ++i) {
      CK(timed(P, st, K_SCALAR, [&] { return launch_coef_for(P, a, nb, st); }));
      a.in = reinterpret_cast<const cx<TI>*>(P->T1);
      a.in_ss = n;
      a.out = P->T2;
      a.out_ss = n;
      CK(timed(P, st, K_PASS_B, [&] { return launch_pass_b<TI, PB_MATVEC>(a, nb, st); }));
      a.in = reinterpret_cast<const cx<TI>*>(P->T2);
      a.out = V + (size_t)(J + i) * n;
      a.out_ss = vss;
      if (i + 1 < S) {
        a.out2 = P->T1;
        a.out2_ss = n;
        PassArgs<TI> ca = a;
        ca.rowv = P->rowv;  // the fused pass's own shape
        CK(timed(P, st, K_PASS_CA, [&] { return launch_pass_ca<TI>(ca, nb, st); }));
      } else {
        CK(timed(P, st, K_PASS_C, [&] { return launch_pass_c<TI, TI, PC_KS>(a, nb, st); }));
      }
    }
    }
    CK(timed(P, st, K_DOTS, [&] { return launch_bdots<TI, S>(ba, V, vss, J, nb, st); }));
    CK(timed(P, st, K_SCALAR, [&] { return launch_bscalar<S>(ba, P->cs, P->Hraw, P->bcoef, P->upd, J, nb, st); }));
    ba.tx_extra = P->inject_tx;  // the test hook fires on one launch
    P->inject_tx = 0;
    CK(timed(P, st, K_UPDATE, [&] { return launch_bupdate<TI, S>(ba, P->upd, V, vss, J, nb, st); }, 2));
    ba.tx_extra = 0;
  }
  return DBAR_OK;
}

// Krylov steps j0 <= j < j1 of the current cycle for every running slot.
template <typename TI>
static dbar_status cycle_steps(dbar_plan* P, int nb, int j0, int j1, cudaStream_t st) {
  if (P->sstep == 4) return block_steps<TI, 4>(P, nb, j0, j1, st);
  if (P->sstep == 2) return block_steps<TI, 2>(P, nb, j0, j1, st);
  const long long n = P->n;
  const int m = P->m;
  const long long vss = (long long)(m + 1) * n;
  cx<TI>* V = reinterpret_cast<cx<TI>*>(P->V);
  cx<TI>* KS = reinterpret_cast<cx<TI>*>(P->KS);
  KryArgs ka;
  ka.n = n;
  ka.mp1 = m + 1;
  ka.nchunk = (int)((n + KR_CHUNK - 1) / KR_CHUNK);
  ka.run = P->cs.run;
  ka.sigma = P->cs.sigma;
  ka.coef = P->coef;
  ka.part = P->part;
  ka.part2 = P->part2;
  for (int j = j0; j < j1; ++j) {
    dbar_status s = apply_op<TI>(P, V + (size_t)j * n, vss, P->cs.sigma + j, m + 1, KS, n, P->cs.run, nb, st);
    if (s != DBAR_OK) return s;
    CK(timed(P, st, K_DOTS, [&] { return launch_dots<TI>(ka, V, vss, KS, n, j, nb, st); }));
    CK(timed(P, st, K_SCALAR, [&] { return launch_finalize_h(ka, P->cs.H, j, nb, st); }));
    CK(timed(P, st, K_UPDATE, [&] { return launch_update<TI>(ka, V, vss, KS, n, j, nb, st); }));
    CK(timed(P, st, K_SCALAR, [&] { return launch_givens(ka, P->cs, j, nb, st); }));
  }
  return DBAR_OK;
}

// End of a cycle: y, x += V y, true residual, start of the next cycle.
template <typename TI>
static dbar_status cycle_tail(dbar_plan* P, int nb, cudaStream_t st) {
  const long long n = P->n;
  const int m = P->m;
  const long long vss = (long long)(m + 1) * n;
  cx<TI>* V = reinterpret_cast<cx<TI>*>(P->V);
  if (P->sstep > 1) {
    // s-step cycles: each slot's last block already solved for y and added V y to x
    CK(cudaMemcpyAsync(P->h_nsteps, P->cs.nsteps, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  } else {
    CK(timed(P, st, K_SCALAR, [&] { return launch_solve_y(P->cs, nb, st); }));
    CK(cudaMemcpyAsync(P->h_nsteps, P->cs.nsteps, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(timed(P, st, K_XUPDATE, [&] {
      return launch_xupdate<TI>(n, m + 1, P->cs.nsteps, P->cs.ycoef, V, vss, P->x64, P->resid_dd, n, nb, st);
    }));
  }
  dbar_status s = true_residual<TI>(P, nb, st);
  if (s != DBAR_OK) return s;
  CK(timed(P, st, K_SCALAR, [&] { return launch_cycle_start(P->cs, P->part2, row_blocks(P->N), 0, nb, st); }));
  return DBAR_OK;
}

// true when some slot's cycle is still running (synchronises the stream)
static bool any_running(dbar_plan* P, int nb, cudaStream_t st) {
  if (cudaMemcpyAsync(P->h_active, P->cs.run, nb * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return true;
  int any = 0;
  for (int i = 0; i < nb; ++i) any |= P->h_active[i];
  return any != 0;
}

// One cycle for every active slot (FP64: a restarted GMRES cycle; mixed: an FP32
// correction cycle, x += d, true residual), ending with the next cycle's start.
// Between chunks of kGraphChunk steps the host stops launching once every slot
// has finished its cycle.  *launched_steps receives the Krylov steps launched.
template <typename TI>
static dbar_status one_cycle(dbar_plan* P, int nb, cudaStream_t st, int* launched_steps, bool early_stop = true) {
  int j0 = 0;
  while (j0 < P->m) {
    const int j1 = std::min(P->m, j0 + kGraphChunk);
    dbar_status s = cycle_steps<TI>(P, nb, j0, j1, st);
    if (s != DBAR_OK) return s;
    j0 = j1;
    if (early_stop && j0 < P->m && !any_running(P, nb, st)) break;
  }
  *launched_steps = j0;
  return cycle_tail<TI>(P, nb, st);
}

// One cycle as CUDA graphs: each chunk of kGraphChunk Krylov steps and the
// cycle's tail are captured once per batch size (and profiling state) on the
// plan's capture stream, then replayed on the caller's stream, with the same
// host check between chunks as the direct launches.
template <typename TI, typename F>
static dbar_status capture_part(dbar_plan* P, GraphPart* g, F&& body) {
  if (!P->cap_stream) CK(cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeRelaxed));
  P->capturing = true;
  P->cap = g;
  dbar_status s = body(P->cap_stream);
  P->capturing = false;
  P->cap = nullptr;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(P->cap_stream, &graph);
  if (s != DBAR_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail(DBAR_ECUDA, std::string("cycle capture: ") + cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) return fail(DBAR_ECUDA, std::string("cycle graph: ") + cudaGetErrorString(e2));
  return DBAR_OK;
}

// The captured parts of a cycle for nb slots (captured on first use).
template <typename TI>
static dbar_status cycle_graph(dbar_plan* P, int nb, CycleGraph** out) {
  CycleGraph* g = nullptr;
  for (CycleGraph& c : P->graphs)
    if (!c.parts.empty() && c.nb == nb && c.prof == P->prof.on) g = &c;
  const int nchunks = (P->m + kGraphChunk - 1) / kGraphChunk;
  if (!g) {
    g = (P->graphs[0].nb == nb || P->graphs[0].parts.empty()) ? &P->graphs[0] : &P->graphs[1];
    g->clear();
    g->parts.resize(nchunks + 1);
    for (int c = 0; c <= nchunks; ++c) {
      dbar_status s = (c < nchunks)
          ? capture_part<TI>(P, &g->parts[c], [&](cudaStream_t cs) {
              return cycle_steps<TI>(P, nb, c * kGraphChunk, std::min(P->m, (c + 1) * kGraphChunk), cs);
            })
          : capture_part<TI>(P, &g->parts[c], [&](cudaStream_t cs) { return cycle_tail<TI>(P, nb, cs); });
      if (s != DBAR_OK) {
        g->clear();
        return s;
      }
    }
    g->nb = nb;
    g->prof = P->prof.on;
  }
  *out = g;
  return DBAR_OK;
}

template <typename TI>
static dbar_status graph_cycle(dbar_plan* P, int nb, cudaStream_t st, int* launched_steps, bool early_stop = true) {
  CycleGraph* g = nullptr;
  const dbar_status gs = cycle_graph<TI>(P, nb, &g);
  if (gs != DBAR_OK) return gs;
  const int nchunks = (P->m + kGraphChunk - 1) / kGraphChunk;
  int launched = 0;
  for (int c = 0; c < nchunks; ++c) {
    CK(cudaGraphLaunch(g->parts[c].exec, st));
    P->nlaunch += g->parts[c].kernels;
    launched = std::min(P->m, (c + 1) * kGraphChunk);
    if (P->prof.on) P->graph_ran.push_back(&g->parts[c]);
    if (early_stop && c + 1 < nchunks && !any_running(P, nb, st)) break;
  }
  CK(cudaGraphLaunch(g->parts[nchunks].exec, st));
  P->nlaunch += g->parts[nchunks].kernels;
  if (P->prof.on) P->graph_ran.push_back(&g->parts[nchunks]);
  *launched_steps = launched;
  return DBAR_OK;
}

// after the graph parts replayed since the last call have completed: fold their
// event pairs into the profile (a part's events are re-recorded at each replay,
// so they are read before the part runs again)
static void harvest_graph(dbar_plan* P) {
  for (GraphPart* g : P->graph_ran)
    for (const Profiler::Rec& r : g->recs) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) P->prof.ms[r.kind] += t;
      P->prof.launches[r.kind] += 1;
    }
  P->graph_ran.clear();
  cudaGetLastError();
}

template <typename TI>
static dbar_status run_cycles(dbar_plan* P, int nb, cudaStream_t st) {
  dbar_status s = begin_slots<TI>(P, nb, nullptr, st);
  if (s != DBAR_OK) return s;
  std::vector<int> prev_act(nb, 0);
  int prev_launched = 0;
  bool pending_account = false;
  for (int cyc = 0; cyc <= P->p.max_outer; ++cyc) {
    CK(cudaMemcpyAsync(P->h_active, P->cs.active, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(P->h_err, P->flag + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (*P->h_err) {
      cudaMemsetAsync(P->flag + 1, 0, sizeof(int), st);
      cudaStreamSynchronize(st);
      // cycle graphs captured around the launch that ran out are not replayed again
      for (CycleGraph& g : P->graphs) g.clear();
      P->inject_tx = 0;
      return fail(DBAR_ETIMEOUT, "a bounded device wait ran out (bulk copies of the block update)");
    }
    P->prof.harvest();
    if (pending_account) {
      if (P->p.graphs) harvest_graph(P);
      account_cycle(P, prev_act.data(), P->h_nsteps, nb, prev_launched);
    }
    pending_account = false;
    int any = 0;
    for (int i = 0; i < nb; ++i) any |= P->h_active[i];
    if (!any) break;
    std::copy(P->h_active, P->h_active + nb, prev_act.begin());
    s = P->p.graphs ? graph_cycle<TI>(P, nb, st, &prev_launched) : one_cycle<TI>(P, nb, st, &prev_launched);
    if (s != DBAR_OK) return s;
    pending_account = true;
  }
  return DBAR_OK;
}

// ---------------------------------------------------------------------------
// Plan creation.
// ---------------------------------------------------------------------------
static bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static dbar_status check_params(const dbar_params* p) {
  if (!p) return fail(DBAR_EINVAL, "params is NULL");
  if (!pow2(p->N) || p->N < 32 || p->N > 2048) return fail(DBAR_EINVAL, "N must be a power of two in [32, 2048]");
  if (!(p->L > 0.0) || !std::isfinite(p->L)) return fail(DBAR_EINVAL, "L must be finite and > 0");
  if (p->M < 0 || p->M > 16) return fail(DBAR_EINVAL, "M must be in [0, 16]");
  if (p->prec != DBAR_FP64 && p->prec != DBAR_MIXED) return fail(DBAR_EINVAL, "prec must be DBAR_FP64 or DBAR_MIXED");
  if (p->restart < 1 || p->restart > 128) return fail(DBAR_EINVAL, "restart must be in [1, 128]");
  if (p->max_iter < 1 || p->max_outer < 1) return fail(DBAR_EINVAL, "max_iter and max_outer must be >= 1");
  if (!(p->tol > 0.0) || !(p->tol < 1.0)) return fail(DBAR_EINVAL, "tol must be in (0, 1)");
  if (p->prec == DBAR_MIXED && !(p->inner_tol > 0.0 && p->inner_tol < 1.0))
    return fail(DBAR_EINVAL, "inner_tol must be in (0, 1)");
  if (p->max_batch < 0 || p->max_batch > 65535) return fail(DBAR_EINVAL, "max_batch must be in [0, 65535]");
  if (p->autotune < 0 || p->autotune > 3) return fail(DBAR_EINVAL, "autotune must be 0, 1, 2 or 3");
  if (p->resid_mode != DBAR_RESID_DOUBLE_FLOAT && p->resid_mode != DBAR_RESID_FP64)
    return fail(DBAR_EINVAL, "resid_mode must be DBAR_RESID_DOUBLE_FLOAT or DBAR_RESID_FP64");
  if (p->sstep != 0 && p->sstep != 1 && p->sstep != 2 && p->sstep != 4)
    return fail(DBAR_EINVAL, "sstep must be 0, 1, 2 or 4");
  if (p->sstep > 1 && p->restart % p->sstep != 0) return fail(DBAR_EINVAL, "restart must be a multiple of sstep");
  if (p->iterated != 0 && p->iterated != 1) return fail(DBAR_EINVAL, "iterated must be 0 or 1");
  if (p->inner_M < 0 || p->inner_M > p->M) return fail(DBAR_EINVAL, "inner_M must be in [0, M]");
  if (!(p->gauss_w > 0.0) || !std::isfinite(p->gauss_w)) return fail(DBAR_EINVAL, "gauss_w must be finite and > 0");
  if (p->support_skip != 0 && p->support_skip != 1) return fail(DBAR_EINVAL, "support_skip must be 0 or 1");
  if (p->row_shape < 0 || p->row_shape > DBAR_ROW_VARIANTS) return fail(DBAR_EINVAL, "row_shape must be in [0, 5]");
  if (p->row_shape_plain < 0 || p->row_shape_plain > DBAR_ROW_VARIANTS)
    return fail(DBAR_EINVAL, "row_shape_plain must be in [0, 5]");
  if (p->regularisation != DBAR_REG_TAYLOR && p->regularisation != DBAR_REG_CONV)
    return fail(DBAR_EINVAL, "regularisation must be DBAR_REG_TAYLOR or DBAR_REG_CONV");
  if (p->regularisation == DBAR_REG_CONV) {
    if (p->prec != DBAR_FP64) return fail(DBAR_EINVAL, "the convolution regularisation runs in FP64 only (DBAR_FP64)");
    if (p->N > 256) return fail(DBAR_EINVAL, "the convolution regularisation needs N <= 256 (its direct sum costs N^4)");
    if (p->iterated) return fail(DBAR_EINVAL, "the convolution regularisation is not combined with the iterated equation");
    if (p->max_batch > 4096) return fail(DBAR_EINVAL, "the convolution regularisation takes max_batch <= 4096");
  }
  return DBAR_OK;
}

static dbar_status plan_tables(dbar_plan* P) {
  const int N = P->N;
  const double L = P->p.L;
  cudaStream_t st = 0;
  // twiddles e^{-2 pi i t/N}
  std::vector<cx<double>> tw(N);
  std::vector<cx<float>> tw32(N);
  for (int t = 0; t < N; ++t) {
    const double ang = 2.0 * M_PI * (double)t / (double)N;
    tw[t] = mkc(std::cos(ang), -std::sin(ang));
    tw32[t] = mkc((float)tw[t].re, (float)tw[t].im);
  }
  CK(cudaMemcpy(P->tw64, tw.data(), N * sizeof(cx<double>), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P->tw32, tw32.data(), N * sizeof(cx<float>), cudaMemcpyHostToDevice));
  {
    const size_t cnt = (size_t)P->B * N;
    std::vector<cx<double>> o64(cnt, mkc(1.0, 0.0));
    std::vector<cx<float>> o32(cnt, mkc(1.0f, 0.0f));
    std::vector<cx<dd>> odd(cnt, mkc(dd(1.0f), dd(0.0f)));
    CK(cudaMemcpy(P->ones64, o64.data(), cnt * sizeof(cx<double>), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->ones32, o32.data(), cnt * sizeof(cx<float>), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->ones_dd, odd.data(), cnt * sizeof(cx<dd>), cudaMemcpyHostToDevice));
  }
  // D_a(p) = sum_j x_j^a e^{+2 pi i p j/N}
  const int MA = P->MA;
  std::vector<cx<double>> D((size_t)(MA + 1) * N);
  std::vector<cx<float>> D32((size_t)(MA + 1) * N);
  for (int aa = 0; aa <= MA; ++aa)
    for (int p = 0; p < N; ++p) {
      double re = 0.0, im = 0.0;
      for (int j = 0; j < N; ++j) {
        const double xa = std::pow(xgrid(j, N, L), aa);
        const cx<double> w = tw[(size_t)((long long)p * j % N)];  // conj gives e^{+...}
        re += xa * w.re;
        im -= xa * w.im;
      }
      D[(size_t)aa * N + p] = mkc(re, im);
      D32[(size_t)aa * N + p] = mkc((float)re, (float)im);
    }
  CK(cudaMemcpy(P->Da64, D.data(), D.size() * sizeof(cx<double>), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(P->Da32, D32.data(), D32.size() * sizeof(cx<float>), cudaMemcpyHostToDevice));
  if (P->resid_dd) {
    std::vector<cx<dd>> twd(N), Dd(D.size());
    for (int t = 0; t < N; ++t) twd[t] = mkc(dd(tw[t].re), dd(tw[t].im));
    for (size_t i = 0; i < D.size(); ++i) Dd[i] = mkc(dd(D[i].re), dd(D[i].im));
    CK(cudaMemcpy(P->tw_dd, twd.data(), N * sizeof(cx<dd>), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->Da_dd, Dd.data(), Dd.size() * sizeof(cx<dd>), cudaMemcpyHostToDevice));
  }

  if (P->conv) {
    // convolution regularisation: the direct-sum kernel table and the smooth multiplier
    // W_0 of the Gaussian of width gw: gw W_0(gw z)
    const double h = 2.0 * M_PI * L / N, w = h * h / (2.0 * M_PI), gw = P->p.gauss_w;
    std::vector<cx<double>> kt((size_t)(2 * N - 1) * 2 * N, mkc(0.0, 0.0));
    for (int dy = -(N - 1); dy <= N - 1; ++dy)
      for (int dx = -(N - 1); dx <= N - 1; ++dx) {
        const zd v = W_host(0, zd(gw * h * dx, gw * h * dy)) * (gw * w);
        kt[(size_t)(dy + N - 1) * 2 * N + dx + N - 1] = mkc(v.real(), v.imag());
      }
    std::vector<cx<double>> mu((size_t)N * N);
    for (int p2 = 0; p2 < N; ++p2) {
      const int m2 = p2 <= N / 2 ? p2 : p2 - N;
      for (int p1 = 0; p1 < N; ++p1) {
        const int m1 = p1 <= N / 2 ? p1 : p1 - N;
        const zd xi((double)m1 / L, (double)m2 / L);
        const double sg = ((p1 + p2) & 1) ? -1.0 : 1.0;
        zd f(0.0, 0.0);
        if (m1 != 0 || m2 != 0) f = -std::expm1(-std::norm(xi) / (gw * gw)) / xi * sg / (2.0 * M_PI * L * L);
        mu[(size_t)p2 * N + p1] = mkc(f.real(), f.imag());
      }
    }
    CK(cudaMemcpy(P->Kt, kt.data(), kt.size() * sizeof(cx<double>), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(P->Mu, mu.data(), mu.size() * sizeof(cx<double>), cudaMemcpyHostToDevice));
    CK(launch_conv_prepare());
  }

  // Delta_n = W_n - V_n, V_n = F_d^{-1}(e^{-|xi|^2} conj(xi)^n / xi, 0 at xi = 0)
  //         = (1/(2 pi L^2)) IDFT((-1)^{p1+p2} e^{-|xi|^2} conj(xi)^n / xi).
  // A Gaussian of width gw (e^{-|xi|^2/gw^2}) scales the closed form: gw^{n+1} W_n(gw z).
  const double gw = P->p.gauss_w;
  const int nf = P->M + 1;
  const size_t nn = (size_t)N * N;
  std::vector<cx<double>> hE(nf * nn), hW(nf * nn);
  for (int p2 = 0; p2 < N; ++p2) {
    const int m2 = p2 <= N / 2 ? p2 : p2 - N;
    for (int p1 = 0; p1 < N; ++p1) {
      const int m1 = p1 <= N / 2 ? p1 : p1 - N;
      const zd xi((double)m1 / L, (double)m2 / L);
      const double sg = ((p1 + p2) & 1) ? -1.0 : 1.0;
      zd f(0.0, 0.0);
      if (m1 != 0 || m2 != 0) f = std::exp(-std::norm(xi) / (gw * gw)) / xi * sg / (2.0 * M_PI * L * L);
      for (int nn_ = 0; nn_ < nf; ++nn_) {
        hE[nn_ * nn + (size_t)p2 * N + p1] = mkc(f.real(), f.imag());
        f *= std::conj(xi);
      }
    }
  }
  for (int j2 = 0; j2 < N; ++j2)
    for (int j1 = 0; j1 < N; ++j1) {
      const zd z(xgrid(j1, N, L), xgrid(j2, N, L));
      double sc = gw;  // gw^{n+1}
      for (int nn_ = 0; nn_ < nf; ++nn_, sc *= gw) {
        const zd w = W_host(nn_, gw * z) * sc;
        hW[nn_ * nn + (size_t)j2 * N + j1] = mkc(w.real(), w.imag());
      }
    }
  // device scratch for the inverse transforms: reuse the x and b workspaces when large
  // enough, else allocate temporarily
  cx<double>* dE = nullptr;
  cx<double>* dW = nullptr;
  CK(cudaMalloc(&dE, nf * nn * sizeof(cx<double>)));
  cudaError_t e = cudaMalloc(&dW, nf * nn * sizeof(cx<double>));
  if (e != cudaSuccess) {
    cudaFree(dE);
    return fail(DBAR_ENOMEM, "plan scratch allocation failed");
  }
  dbar_status s = DBAR_OK;
  do {
    if (cudaMemcpy(dE, hE.data(), nf * nn * sizeof(cx<double>), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dW, hW.data(), nf * nn * sizeof(cx<double>), cudaMemcpyHostToDevice) != cudaSuccess) {
      s = fail(DBAR_ECUDA, "table upload failed");
      break;
    }
    // inverse 2-D DFT of the nf fields, in place through T1: rows (pass C raw inverse), columns (pass B raw inverse)
    PassArgs<double> a = base_args<double>(P);
    for (int f0 = 0; f0 < nf; f0 += P->B) {
      const int cnt = std::min(P->B, nf - f0);
      a.in = dE + f0 * nn;
      a.in_ss = (long long)nn;
      a.out = P->T1;
      a.out_ss = (long long)nn;
      if (launch_pass_c<double, double, PC_INV>(a, cnt, st) != cudaSuccess) { s = fail(DBAR_ECUDA, "pass C"); break; }
      a.in = reinterpret_cast<const cx<double>*>(P->T1);
      a.out = dE + f0 * nn;
      if (launch_pass_b<double, PB_INV>(a, cnt, st) != cudaSuccess) { s = fail(DBAR_ECUDA, "pass B"); break; }
    }
    if (s != DBAR_OK) break;
    if (launch_delta_build(dE, dW, P->Delta64, P->Delta32, N, nf, st) != cudaSuccess) {
      s = fail(DBAR_ECUDA, "delta build");
      break;
    }
    if (P->resid_dd && launch_split_fields(P->Delta64, P->Delta_dd, (long long)nf * nn, st) != cudaSuccess) {
      s = fail(DBAR_ECUDA, "delta split");
      break;
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = fail(DBAR_ECUDA, std::string("plan tables: ") + cudaGetErrorString(e));
  } while (0);
  cudaFree(dE);
  cudaFree(dW);
  return s;
}

// Column-pass tile autotuner: times each compiled variant of the FP32 column
// pass on this plan's own workspaces and keeps the faster one.  Results are
// bit-identical across variants (same arithmetic per column), so the choice
// only affects speed; it is cached per (device, N, M) for the process.
static std::mutex g_tune_mu;
struct TuneResult {
  int colv, rowv, rowv_ac;
  std::array<double, DBAR_COLUMN_VARIANTS> col_ms;
  std::array<double, DBAR_ROW_VARIANTS> row_ms, row_ms_ac;
};
static std::map<std::tuple<int, int, int>, TuneResult> g_tune_cache;

static dbar_status autotune_columns(dbar_plan* P) {
  const auto key = std::make_tuple(P->device, P->N, P->Min);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      P->colv = it->second.colv;
      P->rowv = it->second.rowv;
      P->rowv_ac = it->second.rowv_ac;
      for (int v = 0; v < DBAR_COLUMN_VARIANTS; ++v) P->tune_ms[v] = it->second.col_ms[v];
      for (int v = 0; v < DBAR_ROW_VARIANTS; ++v) P->row_ms[v] = it->second.row_ms[v];
      for (int v = 0; v < DBAR_ROW_VARIANTS; ++v) P->row_ms_ac[v] = it->second.row_ms_ac[v];
      return DBAR_OK;
    }
  }
  cudaStream_t st = 0;
  const int nb = std::min(P->B, 16);
  const size_t n = (size_t)P->n;
  CK(cudaMemset(P->T1, 0, (size_t)nb * n * sizeof(cx<float>)));
  CK(cudaMemset(P->T2, 0, (size_t)nb * n * sizeof(cx<float>)));
  CK(cudaMemset(P->tcoef, 0, (size_t)nb * (P->M + 2) * sizeof(cx<double>)));
  CK(cudaMemset(P->Q32, 0, n * sizeof(cx<float>)));
  CK(cudaMemset(P->ex32, 0, (size_t)nb * P->N * sizeof(cx<float>)));
  CK(cudaMemset(P->ey32, 0, (size_t)nb * P->N * sizeof(cx<float>)));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  int choice = 0;
  for (int cv = 0; cv < DBAR_COLUMN_VARIANTS; ++cv) {
    PassArgs<float> a = base_args<float>(P);
    a.colv = cv;
    a.in = reinterpret_cast<const cx<float>*>(P->T1);
    a.in_ss = (long long)n;
    a.out = P->T2;
    a.out_ss = (long long)n;
    for (int w = 0; w < 2; ++w) CK((launch_pass_b<float, PB_MATVEC>(a, nb, st)));
    CK(cudaEventRecord(e0, st));
    const int reps = 5;
    for (int r = 0; r < reps; ++r) CK((launch_pass_b<float, PB_MATVEC>(a, nb, st)));
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    P->tune_ms[cv] = ms / reps;
    if (ms < best) {
      best = ms;
      choice = cv;
    }
  }
  P->colv = choice;
  // row-pass shapes, timed on the fused row pass (the inner operator's largest row pass)
  best = 1e300;
  int rchoice = 0;
  for (int rv = 0; rv < DBAR_ROW_VARIANTS; ++rv) {
    PassArgs<float> a = base_args<float>(P);
    a.rowv = rv;
    a.in = reinterpret_cast<const cx<float>*>(P->T2);
    a.in_ss = (long long)n;
    a.out = P->KS;
    a.out_ss = (long long)n;
    a.out2 = P->T1;
    a.out2_ss = (long long)n;
    for (int w = 0; w < 2; ++w) CK(launch_pass_ca<float>(a, nb, st));
    CK(cudaEventRecord(e0, st));
    const int reps = 5;
    for (int r = 0; r < reps; ++r) CK(launch_pass_ca<float>(a, nb, st));
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    P->row_ms[rv] = ms / reps;
    if (ms < best) {
      best = ms;
      rchoice = rv;
    }
  }
  P->rowv = rchoice;
  // shapes of the plain row passes, timed on a pass A (scaled input) and a pass C (K S) per rep
  best = 1e300;
  int acchoice = 0;
  for (int rv = 0; rv < DBAR_ROW_VARIANTS; ++rv) {
    PassArgs<float> a = base_args<float>(P);
    a.rowv = rv;
    a.in = reinterpret_cast<const cx<float>*>(P->T2);
    a.in_ss = (long long)n;
    PassArgs<float> c = a;
    a.out = P->T1;
    a.out_ss = (long long)n;
    c.out = P->KS;
    c.out_ss = (long long)n;
    auto once = [&]() -> cudaError_t {
      cudaError_t e = launch_pass_a<float>(a, nb, st);
      return e != cudaSuccess ? e : launch_pass_c<float, float, PC_KS>(c, nb, st);
    };
    for (int w = 0; w < 2; ++w) CK(once());
    CK(cudaEventRecord(e0, st));
    const int reps = 5;
    for (int r = 0; r < reps; ++r) CK(once());
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    P->row_ms_ac[rv] = ms / reps;
    if (ms < best) {
      best = ms;
      acchoice = rv;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->rowv_ac = acchoice;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  TuneResult t;
  t.colv = choice;
  t.rowv = rchoice;
  t.rowv_ac = acchoice;
  for (int v = 0; v < DBAR_COLUMN_VARIANTS; ++v) t.col_ms[v] = P->tune_ms[v];
  for (int v = 0; v < DBAR_ROW_VARIANTS; ++v) t.row_ms[v] = P->row_ms[v];
  for (int v = 0; v < DBAR_ROW_VARIANTS; ++v) t.row_ms_ac[v] = P->row_ms_ac[v];
  g_tune_cache[key] = t;
  return DBAR_OK;
}

size_t plan_slot_bytes(const dbar_params* p, int per_slot_q) {
  const size_t n = (size_t)p->N * p->N;
  const size_t F64 = n * sizeof(cx<double>);
  const size_t Fi = n * (p->prec == DBAR_MIXED ? sizeof(cx<float>) : sizeof(cx<double>));
  size_t b = 4 * F64 + (size_t)(p->restart + 2) * Fi;  // x, b, T1, T2; basis, K v
  const int S = p->sstep > 0 ? p->sstep : 4;  // upper bound for the automatic choice
  if (S > 1)  // s-step partials, coefficients, unrotated Hessenberg
    b += ((size_t)(p->restart + 1) * S + S * (S + 1) / 2) *
             std::min<size_t>((n + KB_CHUNK - 1) / KB_CHUNK, kBlockDotBlocks) * sizeof(double) +
         ((size_t)S * (S + p->restart + 1) + (size_t)p->restart * (p->restart + 1)) * sizeof(double);
  if (per_slot_q) b += F64 + n * sizeof(cx<float>) + (p->prec == DBAR_MIXED ? F64 : 0);
  if (p->iterated) b += 2 * F64;  // shifted field and first operator application
  if (p->regularisation == DBAR_REG_CONV) b += 4 * F64;  // two fields per slot, twice
  return b;
}

size_t plan_fixed_bytes(const dbar_params* p) {
  const size_t n = (size_t)p->N * p->N;
  size_t b = (size_t)(3 * (p->M + 1) + 4) * n * sizeof(cx<double>);
  if (p->regularisation == DBAR_REG_CONV) b += ((size_t)(2 * p->N - 1) * 2 * p->N + n) * sizeof(cx<double>);
  return b;
}

// Every device workspace of a plan of B slots.  With P->dry set nothing is
// allocated and only P->bytes grows (the exact size, for mem_budget).
static cudaError_t alloc_workspaces(dbar_plan* P, int B, const char** what) {
  cudaError_t e = cudaSuccess;
  const size_t Fi = (size_t)P->n * P->inner_elem();
  const int nchunk = (int)((P->n + KR_CHUNK - 1) / KR_CHUNK);
#define AL(ptr, cnt)                     \
  do {                                   \
    e = P->alloc(&(ptr), (cnt));         \
    if (e != cudaSuccess) {              \
      *what = #ptr;                      \
      return e;                          \
    }                                    \
  } while (0)
  const size_t n = (size_t)P->n;
  AL(P->tw64, P->N);
  AL(P->ones64, (size_t)B * P->N);
  AL(P->ones32, (size_t)B * P->N);
  AL(P->ones_dd, (size_t)B * P->N);
  AL(P->tw32, P->N);
  AL(P->Da64, (size_t)(P->MA + 1) * P->N);
  AL(P->Da32, (size_t)(P->MA + 1) * P->N);
  AL(P->Delta64, (size_t)(P->M + 1) * n);
  AL(P->Delta32, (size_t)(P->M + 1) * n);
  const size_t nq = (size_t)(P->per_slot_q ? B : 1) * n;
  AL(P->Q64, nq);
  AL(P->Q32, nq);
  AL(P->Qdev, n);
  AL(P->ex64, (size_t)B * P->N);
  AL(P->ey64, (size_t)B * P->N);
  AL(P->ex32, (size_t)B * P->N);
  AL(P->ey32, (size_t)B * P->N);
  if (P->resid_dd) {
    AL(P->tw_dd, P->N);
    AL(P->Da_dd, (size_t)(P->MA + 1) * P->N);
    AL(P->Delta_dd, (size_t)(P->M + 1) * n);
    AL(P->Q_dd, nq);
    AL(P->ex_dd, (size_t)B * P->N);
    AL(P->ey_dd, (size_t)B * P->N);
  }
  AL(P->x64, (size_t)B * n);
  AL(P->b64, (size_t)B * n);
  cx<double>* t1 = nullptr;
  cx<double>* t2 = nullptr;
  AL(t1, (size_t)B * n);
  AL(t2, (size_t)B * n);
  P->T1 = t1;
  P->T2 = t2;
  unsigned char* vb = nullptr;
  AL(vb, (size_t)B * (P->m + 1) * Fi);
  P->V = vb;
  unsigned char* kb = nullptr;
  AL(kb, (size_t)B * Fi);
  P->KS = kb;
  AL(P->partA, (size_t)B * P->N * seg_count(P->N) * (P->MA + 1));
  AL(P->part, (size_t)B * (P->m + 1) * nchunk);
  AL(P->part2, (size_t)B * std::max(std::max(nchunk, P->N), 2 * (P->M + 2)));
  AL(P->coef, (size_t)B * (P->m + 1));
  AL(P->tcoef, (size_t)B * (P->M + 2));
  AL(P->coefp, (size_t)B * (P->N / coef_rows(P->N)) * (P->M + 2));
  AL(P->ticket, B);
  AL(P->s0buf, B);
  AL(P->gat, B);
  if (P->iter) {
    AL(P->rolls, 2 * (size_t)B);
    AL(P->dshift, 2 * (size_t)B);
    cx<double>* i1 = nullptr;
    cx<double>* i2 = nullptr;
    AL(i1, (size_t)B * n);
    AL(i2, (size_t)B * n);
    P->It1 = i1;
    P->It2 = i2;
  }
  if (P->conv) {
    AL(P->Kt, (size_t)(2 * P->N - 1) * 2 * P->N);
    AL(P->Mu, n);
    AL(P->Cv1, (size_t)B * 2 * n);
    AL(P->Cv2, (size_t)B * 2 * n);
  }
  AL(P->flag, 4);
  AL(P->supflag, 2 * (size_t)P->N);
  AL(P->kdev, 2 * (size_t)B);
  CycleState& c = P->cs;
  const int m = P->m;
  AL(c.H, (size_t)B * m * (m + 1));
  AL(c.cs, (size_t)B * m);
  AL(c.sn, (size_t)B * m);
  AL(c.g, (size_t)B * (m + 1));
  AL(c.sigma, (size_t)B * (m + 1));
  AL(c.ycoef, (size_t)B * (m + 1));
  AL(c.thr, B);
  AL(c.bnorm, B);
  AL(c.nscale, B);
  AL(c.resid, B);
  AL(c.run, B);
  AL(c.active, B);
  AL(c.nsteps, B);
  AL(c.itot, B);
  AL(c.ncyc, B);
  AL(P->dmask, B);
  if (P->sstep > 1) {
    const int S = P->sstep;
    P->nchunk_b = (int)((n + KB_CHUNK - 1) / KB_CHUNK);
    P->nitem_b = block_items(m + 1, S);
    AL(P->Hraw, (size_t)B * m * (m + 1));
    AL(P->bcoef, (size_t)B * (S * S + (m + 1) * S));
    AL(P->bpart, (size_t)B * P->nitem_b * std::min(P->nchunk_b, kBlockDotBlocks));
    AL(P->upd, B);
  }
#undef AL
  return cudaSuccess;
}

dbar_status plan_create_ex(const dbar_params* p, int per_slot_q, dbar_plan** out) {
  if (!out) return fail(DBAR_EINVAL, "out is NULL");
  *out = nullptr;
  dbar_status s = check_params(p);
  if (s != DBAR_OK) return s;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(DBAR_ECUDA, "no CUDA device is available");
  }
  dbar_plan* P = new (std::nothrow) dbar_plan();
  if (!P) return fail(DBAR_ENOMEM, "host allocation failed");
  P->p = *p;
  P->per_slot_q = per_slot_q ? 1 : 0;
  P->N = p->N;
  P->logN = 0;
  while ((1 << P->logN) < P->N) ++P->logN;
  P->M = p->M;
  P->MA = std::max(1, p->M);
  P->Min = (p->prec == DBAR_MIXED && p->inner_M > 0) ? p->inner_M : p->M;
  P->m = p->restart;
  P->iter = p->iterated != 0;
  P->conv = p->regularisation == DBAR_REG_CONV;
  // automatic choice: blocks of 4 for the Sec. 4 operator; one vector per sweep for the
  // multi-application operators (their solves take few iterations, which blocks overshoot)
  P->sstep = ((P->conv || P->iter) && p->sstep == 0) ? 1 : (p->sstep > 0 ? p->sstep : (p->restart % 4 == 0 ? 4 : (p->restart % 2 == 0 ? 2 : 1)));
  P->mixed = (p->prec == DBAR_MIXED);
  P->resid_dd = P->mixed && p->resid_mode == DBAR_RESID_DOUBLE_FLOAT;
  P->n = (long long)P->N * P->N;
  cudaGetDevice(&P->device);
  const double L = p->L;
  P->inv2piL = 1.0 / (2.0 * M_PI * L);
  P->sw = 2.0 * M_PI * L * L / ((double)P->N * P->N);
  P->fillscale = p->zero_fill ? 0.0 : 1.0 / (2.0 * M_PI * L * L);

  const size_t F64 = (size_t)P->n * sizeof(cx<double>);
  const size_t per_slot = plan_slot_bytes(p, per_slot_q);
  int B = p->max_batch;
  if (B == 0) {
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    const size_t fixed = (size_t)(2 * (P->M + 1) + 3) * F64;
    size_t avail = freeb > fixed ? (freeb - fixed) / 2 : 0;
    B = (int)std::min<size_t>(256, std::max<size_t>(1, avail / per_slot));
  }
  if (P->conv) B = std::min(B, 4096);  // the raw transforms take 2 B fields per launch
  if (p->mem_budget > 0) {
    // the plan's exact footprint is affine in the batch size: bytes(1), bytes(2)
    const char* what = nullptr;
    P->dry = true;
    alloc_workspaces(P, 1, &what);
    const size_t b1 = P->bytes;
    P->bytes = 0;
    alloc_workspaces(P, 2, &what);
    const size_t b2 = P->bytes;
    P->bytes = 0;
    P->dry = false;
    const size_t per = b2 - b1, fixed = b1 - per;
    if (b1 > p->mem_budget) {
      delete P;
      return fail(DBAR_ENOMEM, "mem_budget " + std::to_string(p->mem_budget) + " bytes is below one slot's plan (" +
                                   std::to_string(b1) + " bytes)");
    }
    const size_t fit = (p->mem_budget - fixed) / per;
    if (p->max_batch == 0) {
      B = (int)std::min<size_t>((size_t)B, fit);
    } else if ((size_t)B > fit) {
      delete P;
      return fail(DBAR_ENOMEM, "max_batch " + std::to_string(B) + " needs " + std::to_string(fixed + per * B) +
                                   " bytes, above mem_budget " + std::to_string(p->mem_budget));
    }
  }
  P->B = B;
  const int m = P->m;
  CycleState& c = P->cs;
  {
    const char* what = "";
    const cudaError_t e = alloc_workspaces(P, B, &what);
    if (e != cudaSuccess) {
      delete P;
      return fail(e == cudaErrorMemoryAllocation ? DBAR_ENOMEM : DBAR_ECUDA,
                  std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e));
    }
  }
  if (cudaMemset(P->ticket, 0, (size_t)B * sizeof(int)) != cudaSuccess ||
      cudaMemset(P->flag, 0, 4 * sizeof(int)) != cudaSuccess) {
    delete P;
    return fail(DBAR_ECUDA, "workspace initialisation failed");
  }
  c.m = m;
  c.max_iter = p->max_iter;
  c.max_outer = p->max_outer;
  c.tol = p->tol;
  c.inner_tol = P->mixed ? p->inner_tol : 0.0;
  if (cudaMallocHost(&P->h_active, (size_t)B * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->h_run, (size_t)B * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->hmask, (size_t)B * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->h_nsteps, (size_t)B * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->h_rolls, 2 * (size_t)B * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->h_dshift, 2 * (size_t)B * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->h_err, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&P->h_ek, (size_t)B * 2 * P->N * sizeof(cx<double>)) != cudaSuccess ||
      cudaMallocHost(&P->h_k, (size_t)B * 2 * sizeof(double)) != cudaSuccess) {
    delete P;
    return fail(DBAR_ENOMEM, "pinned host allocation failed");
  }
  s = plan_tables(P);
  if (s == DBAR_OK && P->mixed && p->autotune == 1) s = autotune_columns(P);
  if (P->mixed && p->autotune == 2) P->colv = 1;  // fixed second variant (tests)
  if (P->mixed && p->autotune == 3) P->colv = 2;  // fixed third variant (tests)
  if (P->mixed && p->row_shape > 0) P->rowv = P->rowv_ac = p->row_shape - 1;  // fixed row-pass shape
  if (P->mixed && p->row_shape_plain > 0) P->rowv_ac = p->row_shape_plain - 1;  // plain passes A, C
  if (s != DBAR_OK) {
    delete P;
    return s;
  }
  *out = P;
  return DBAR_OK;
}

extern "C" dbar_status dbar_plan_create(const dbar_params* p, dbar_plan_t* out) {
  return plan_create_ex(p, 0, out);
}

extern "C" dbar_status dbar_plan_destroy(dbar_plan_t plan) {
  delete plan;
  return DBAR_OK;
}

extern "C" dbar_status dbar_check_bounded_wait(int complete, int rounds, double* seconds, void* stream) {
  if (rounds < 1 || rounds > wait_limit_rounds()) return fail(DBAR_EINVAL, "rounds must be in [1, the sweeps' limit]");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int magic = 0x5eed;
  const int h_src[4] = {magic, 1, 2, 3};
  int h_out[3] = {0, 0, 0};
  void* mem = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&] {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (mem) cudaFree(mem);
  };
  if (cudaMalloc(&mem, 32) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess ||
      cudaMemcpyAsync(mem, h_src, sizeof(h_src), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(static_cast<char*>(mem) + 16, 0, 16, st) != cudaSuccess ||
      cudaEventRecord(e0, st) != cudaSuccess ||
      launch_wait_check(complete, rounds, static_cast<const int4*>(mem), reinterpret_cast<int*>(static_cast<char*>(mem) + 16),
                        st) != cudaSuccess ||
      cudaEventRecord(e1, st) != cudaSuccess ||
      cudaMemcpyAsync(h_out, static_cast<char*>(mem) + 16, sizeof(h_out), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    cleanup();
    return fail(DBAR_ECUDA, std::string("bounded-wait check: ") + cudaGetErrorString(e));
  }
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cleanup();
  if (seconds) *seconds = ms / 1e3;
  if (!h_out[0]) return fail(DBAR_ETIMEOUT, "bounded-wait check: the wait ran out after " + std::to_string(h_out[2]) + " rounds");
  if (h_out[1] != magic) return fail(DBAR_ECUDA, "bounded-wait check: the copied word is wrong");
  return DBAR_OK;
}

extern "C" dbar_status dbar_plan_info(dbar_plan_t plan, size_t* device_bytes, int* max_batch) {
  if (!plan) return fail(DBAR_EINVAL, "plan is NULL");
  if (device_bytes) *device_bytes = plan->bytes;
  if (max_batch) *max_batch = plan->B;
  return DBAR_OK;
}

// ---------------------------------------------------------------------------
// Solve.
// ---------------------------------------------------------------------------
static dbar_status check_k(const double* k, int nk) {
  if (nk < 0) return fail(DBAR_EINVAL, "nk < 0");
  if (nk > 0 && !k) return fail(DBAR_EINVAL, "k is NULL");
  for (int i = 0; i < 2 * nk; ++i)
    if (!std::isfinite(k[i])) return fail(DBAR_EINVAL, "k has a non-finite entry");
  return DBAR_OK;
}

// Q (complex128, device) -> Q64 / Q32 (plan copies), with a finiteness check.
static dbar_status load_Q_device(dbar_plan* P, const cx<double>* Qd, cudaStream_t st) {
  CK(cudaMemsetAsync(P->flag, 0, sizeof(int), st));
  CK(timed(P, st, K_OTHER, [&] { return launch_check_finite(reinterpret_cast<const double*>(Qd), 2 * P->n, P->flag, st); }));
  CK(timed(P, st, K_OTHER, [&] { return launch_load_q(Qd, P->Q64, P->Q32, P->N, st); }));
  if (P->resid_dd) CK(timed(P, st, K_OTHER, [&] { return launch_split_fields(P->Q64, P->Q_dd, P->n, st); }));
  // support of the FP32 potential (the inner operator skips the columns where it is zero)
  const bool scan = P->mixed && !P->per_slot_q && !P->iter && !P->conv && P->p.support_skip;
  std::vector<int> fl(scan ? 2 * P->N : 0);
  if (scan) {
    CK(cudaMemsetAsync(P->supflag, 0, 2 * (size_t)P->N * sizeof(int), st));
    CK(timed(P, st, K_OTHER, [&] { return launch_q_support(P->Q32, P->N, P->supflag, st); }));
    CK(cudaMemcpyAsync(fl.data(), P->supflag, 2 * (size_t)P->N * sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, P->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) return fail(DBAR_EINVAL, "Q has a non-finite entry");
  P->sup = scan;
  if (scan) {
    const int N = P->N, A = col_align(N);
    int x0 = N, x1 = -1, y0 = N, y1 = -1;
    for (int i = 0; i < N; ++i) {
      if (fl[i]) x0 = std::min(x0, i), x1 = i;
      if (fl[N + i]) y0 = std::min(y0, i), y1 = i;
    }
    if (x1 < 0) {  // Q = 0 in FP32: the inner operator is zero
      P->sx0 = P->sx1 = P->sy0 = P->sy1 = 0;
    } else {
      P->sx0 = (x0 / A) * A;
      P->sx1 = std::min(N, ((x1 + A) / A) * A);
      P->sy0 = y0;
      P->sy1 = y1 + 1;
    }
  }
  return DBAR_OK;
}

// A host Q is copied as it is; the device-side check of load_Q_device rejects
// non-finite entries (the same DBAR_EINVAL as for a device Q).
static dbar_status load_Q(dbar_plan* P, const double* Q, int on_device, cudaStream_t st) {
  if (!Q) return fail(DBAR_EINVAL, "Q is NULL");
  if (on_device) return load_Q_device(P, reinterpret_cast<const cx<double>*>(Q), st);
  CK(cudaMemcpyAsync(P->Qdev, Q, P->n * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
  return load_Q_device(P, P->Qdev, st);
}

// Device address of a host buffer that kernels may write (page-locked and
// mapped into the device's address space, e.g. cudaHostAlloc memory), else
// nullptr (pageable memory: the solution goes out by cudaMemcpyAsync).
static cx<double>* mapped_host(void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the query's error state
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? reinterpret_cast<cx<double>*>(at.devicePointer) : nullptr;
}

// FP64 view of the solutions of slots [s0, s0 + nb): x itself, or, with
// double-float storage, an FP64 copy written over b (no longer needed once a
// slot's solve has finished).
static dbar_status solution_fp64(dbar_plan* P, int s0, int nb, cudaStream_t st, const cx<double>** out) {
  const long long n = P->n;
  if (!P->resid_dd) {
    *out = P->x64 + (size_t)s0 * n;
    return DBAR_OK;
  }
  cx<double>* dst = P->b64 + (size_t)s0 * n;
  CK(timed(P, st, K_OTHER, [&] { return launch_dd_to_fp64(P->x64 + (size_t)s0 * n, dst, (long long)nb * n, st); }));
  *out = dst;
  return DBAR_OK;
}

// The caller's initial guesses of slots [k0, k0 + nb) (host or device, any
// alignment) staged into T1, checked for non-finite entries; P->x0d points there.
static dbar_status load_x0(dbar_plan* P, const double* x0, int k0, int nb, int on_device, cudaStream_t st) {
  const size_t cnt = (size_t)nb * P->n;
  cx<double>* dst = reinterpret_cast<cx<double>*>(P->T1);
  CK(cudaMemcpyAsync(dst, x0 + (size_t)k0 * P->n * 2, cnt * sizeof(cx<double>),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(P->flag, 0, sizeof(int), st));
  CK(timed(P, st, K_OTHER, [&] { return launch_check_finite(reinterpret_cast<const double*>(dst), 2 * (long long)cnt, P->flag, st); }));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, P->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad) return fail(DBAR_EINVAL, "x0 has a non-finite entry");
  P->x0d = dst;
  return DBAR_OK;
}

extern "C" dbar_status dbar_solve_cgo(dbar_plan_t P, const double* Q, int nk, const double* k, const double* x0,
                                      double* S_out, double* m_out, int* iters, double* resid, int io_on_device,
                                      void* stream) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  dbar_status s = check_k(k, nk);
  if (s != DBAR_OK) return s;
  if (nk > 0 && !S_out) return fail(DBAR_EINVAL, "S_out is NULL");
  if (P->iter && m_out) return fail(DBAR_EINVAL, "an iterated plan returns h only (m_out must be NULL)");
  if (nk == 0) return DBAR_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = load_Q(P, Q, io_on_device, st);
  if (s != DBAR_OK) return s;
  const long long n = P->n;
  const cudaMemcpyKind d2o = io_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  // where the conversion kernel can write S itself: a device S_out, or a mapped
  // host S_out when m_out (computed from S on the device) is not requested;
  // 16-byte aligned for its vector stores
  cx<double>* direct = nullptr;
  if (P->resid_dd && nk > 0)
    direct = io_on_device ? reinterpret_cast<cx<double>*>(S_out) : (m_out ? nullptr : mapped_host(S_out));
  if (reinterpret_cast<uintptr_t>(direct) % 16 != 0) direct = nullptr;
  bool noconv = false;
  std::vector<int> it(2 * P->B), nc(P->B);
  std::vector<double> rs(P->B);
  for (int k0 = 0; k0 < nk; k0 += P->B) {
    const int nb = std::min(P->B, nk - k0);
    s = upload_ek(P, k + 2 * k0, nb, st);
    if (s != DBAR_OK) return s;
    if (x0 && (s = load_x0(P, x0, k0, nb, io_on_device, st)) != DBAR_OK) return s;
    s = P->mixed ? run_cycles<float>(P, nb, st) : run_cycles<double>(P, nb, st);
    P->x0d = nullptr;
    if (s != DBAR_OK) return s;
    const cx<double>* S64 = nullptr;
    if (direct) {
      // double-float solution converted straight into the caller's buffer (device
      // memory, or mapped host memory written over the host link by the kernel)
      cx<double>* dst = direct + (size_t)k0 * n;
      CK(timed(P, st, K_OTHER, [&] { return launch_dd_to_fp64(P->x64, dst, (long long)nb * n, st); }));
      S64 = dst;
    } else {
      s = solution_fp64(P, 0, nb, st, &S64);
      if (s != DBAR_OK) return s;
      CK(cudaMemcpyAsync(S_out + (size_t)k0 * n * 2, S64, (size_t)nb * n * sizeof(cx<double>), d2o, st));
    }
    if (m_out) {
      s = h_of_S64(P, S64, n, reinterpret_cast<cx<double>*>(P->T2), n, nb, st);
      if (s != DBAR_OK) return s;
      CK(cudaMemcpyAsync(m_out + (size_t)k0 * n * 2, P->T2, (size_t)nb * n * sizeof(cx<double>), d2o, st));
    }
    CK(cudaMemcpyAsync(it.data(), P->cs.itot, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(nc.data(), P->cs.ncyc, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(rs.data(), P->cs.resid, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int i = 0; i < nb; ++i) {
      if (iters) {
        iters[2 * (k0 + i)] = it[i];
        iters[2 * (k0 + i) + 1] = nc[i];
      }
      if (resid) resid[k0 + i] = rs[i];
      if (!(rs[i] <= P->p.tol)) noconv = true;
    }
  }
  if (noconv) return fail(DBAR_ENOCONV, "some k did not reach tol");
  return DBAR_OK;
}

// DS II reflection coefficient over a list of k (Sec. 6.1): per k the CGO
// problem at k/2 with +Q and with -Q, r = (i/2)(S_+(0) - S_-(0)) times the
// time factor of eq. rt.  Per batch of slots the two solves run one after the
// other with the plan's Q copies negated in between; only S(0) leaves the GPU.
// (m^(1)_+ - m^(1)_-)/2 for each k, Sec. 6's convention (the CGO problems at k/2
// with the plan's potential +Q and -Q, m^(1) = i S(0)), times the time factor
// of eq. rt at t; the plan's potential is loaded.  The DS II reflection
// coefficient (eq. rviah) and, with the roles of z and k exchanged, the
// reconstructed potential (eq. qRec) are both this quantity.
static dbar_status m1_half_difference(dbar_plan* P, int nk, const double* k, double t, double* r_out, int* iters,
                                      double* resid, cudaStream_t st) {
  dbar_status s = DBAR_OK;
  const long long n = P->n;
  std::vector<double> khalf(2 * (size_t)nk);
  for (int i = 0; i < 2 * nk; ++i) khalf[i] = 0.5 * k[i];
  auto negate_q = [&]() -> dbar_status {
    CK(timed(P, st, K_OTHER, [&] { return launch_negate(P->Q64, 2 * n, 1, st); }));
    CK(timed(P, st, K_OTHER, [&] { return launch_negate(P->Q32, 2 * n, 0, st); }));
    if (P->resid_dd) CK(timed(P, st, K_OTHER, [&] { return launch_negate(P->Q_dd, 4 * n, 0, st); }));
    return DBAR_OK;
  };
  bool noconv = false;
  std::vector<cx<double>> s0(2 * (size_t)P->B);
  std::vector<int> it(P->B), nc(P->B);
  std::vector<double> rs(P->B);
  if (P->iter) {
    // Sec. 5.3 route: one solve of eq. eqh2 per k (at k/2), r = i h(i conj k),
    // the value of h at the grid offset of xi0 = i conj(k)
    std::vector<long long> at(P->B);
    for (int k0 = 0; k0 < nk; k0 += P->B) {
      const int nb = std::min(P->B, nk - k0);
      s = upload_ek(P, khalf.data() + 2 * k0, nb, st);
      if (s != DBAR_OK) return s;
      for (int i = 0; i < nb; ++i) at[i] = (long long)P->h_rolls[2 * i + 1] * P->N + P->h_rolls[2 * i];
      CK(cudaMemcpyAsync(P->gat, at.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, st));
      s = P->mixed ? run_cycles<float>(P, nb, st) : run_cycles<double>(P, nb, st);
      if (s != DBAR_OK) return s;
      CK(timed(P, st, K_OTHER, [&] { return launch_gather_s0(P->x64, n, nb, P->resid_dd ? 1 : 0, P->gat, P->s0buf, st); }));
      CK(cudaMemcpyAsync(s0.data(), P->s0buf, nb * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(it.data(), P->cs.itot, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(nc.data(), P->cs.ncyc, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(rs.data(), P->cs.resid, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i < nb; ++i) {
        if (iters) {
          iters[2 * (size_t)(k0 + i)] = it[i];
          iters[2 * (size_t)(k0 + i) + 1] = nc[i];
        }
        if (resid) resid[k0 + i] = rs[i];
        if (!(rs[i] <= P->p.tol)) noconv = true;
        const std::complex<double> h0(s0[i].re, s0[i].im);
        const std::complex<double> kk(k[2 * (k0 + i)], k[2 * (k0 + i) + 1]);
        std::complex<double> r = std::complex<double>(0.0, 1.0) * h0;
        r *= std::exp(std::complex<double>(0.0, -t / 4.0) * (kk * kk + std::conj(kk) * std::conj(kk)));
        r_out[2 * (size_t)(k0 + i)] = r.real();
        r_out[2 * (size_t)(k0 + i) + 1] = r.imag();
      }
    }
    if (noconv) return fail(DBAR_ENOCONV, "some k did not reach tol");
    return DBAR_OK;
  }
  for (int k0 = 0; k0 < nk; k0 += P->B) {
    const int nb = std::min(P->B, nk - k0);
    s = upload_ek(P, khalf.data() + 2 * k0, nb, st);
    if (s != DBAR_OK) return s;
    for (int pm = 0; pm < 2; ++pm) {  // pm = 0: S_+ (potential Q), 1: S_- (potential -Q)
      if (pm == 1) {
        s = negate_q();
        if (s != DBAR_OK) return s;
      }
      s = P->mixed ? run_cycles<float>(P, nb, st) : run_cycles<double>(P, nb, st);
      if (s != DBAR_OK) return s;
      CK(timed(P, st, K_OTHER, [&] { return launch_gather_s0(P->x64, n, nb, P->resid_dd ? 1 : 0, nullptr, P->s0buf, st); }));
      CK(cudaMemcpyAsync(s0.data() + (size_t)pm * P->B, P->s0buf, nb * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(it.data(), P->cs.itot, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(nc.data(), P->cs.ncyc, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(rs.data(), P->cs.resid, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int i = 0; i < nb; ++i) {
        if (iters) {
          int* o = iters + 2 * (size_t)(k0 + i);
          o[0] = (pm ? o[0] : 0) + it[i];
          o[1] = pm ? std::max(o[1], nc[i]) : nc[i];
        }
        if (resid) resid[k0 + i] = pm ? std::max(resid[k0 + i], rs[i]) : rs[i];
        if (!(rs[i] <= P->p.tol)) noconv = true;
      }
      if (pm == 1) {
        s = negate_q();  // the plan's potential back to +Q for the next batch
        if (s != DBAR_OK) return s;
      }
    }
    for (int i = 0; i < nb; ++i) {
      const std::complex<double> sp(s0[i].re, s0[i].im), sm(s0[(size_t)P->B + i].re, s0[(size_t)P->B + i].im);
      const std::complex<double> kk(k[2 * (k0 + i)], k[2 * (k0 + i) + 1]);
      std::complex<double> r = std::complex<double>(0.0, 0.5) * (sp - sm);
      r *= std::exp(std::complex<double>(0.0, -t / 4.0) * (kk * kk + std::conj(kk) * std::conj(kk)));
      r_out[2 * (size_t)(k0 + i)] = r.real();
      r_out[2 * (size_t)(k0 + i) + 1] = r.imag();
    }
  }
  if (noconv) return fail(DBAR_ENOCONV, "some k did not reach tol");
  return DBAR_OK;
}

extern "C" dbar_status dbar_reflection(dbar_plan_t P, const double* Q, int nk, const double* k, double t,
                                       double* r_out, int* iters, double* resid, int q_on_device, void* stream) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  if (P->per_slot_q) return fail(DBAR_EINVAL, "dbar_reflection needs a plan with one shared potential");
  dbar_status s = check_k(k, nk);
  if (s != DBAR_OK) return s;
  if (!std::isfinite(t)) return fail(DBAR_EINVAL, "t is not finite");
  if (nk > 0 && !r_out) return fail(DBAR_EINVAL, "r_out is NULL");
  if (nk == 0) return DBAR_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = load_Q(P, Q, q_on_device, st);
  if (s != DBAR_OK) return s;
  return m1_half_difference(P, nk, k, t, r_out, iters, resid, st);
}

// DS II potential from the reflection coefficient (Sec. 1 eq. dbarrecA/B, qRec;
// time dependence eq. rt; Sec. 6.2): with Sec. 6's k/2 convention the D-bar
// problem in k is the CGO problem in the variable k with the potential
// conj(r(k, t)) and the parameter z/2, and q(z, t) = (m~^(1)_+ - m~^(1)_-)/2.
extern "C" dbar_status dbar_ds2_potential(dbar_plan_t P, const double* r, double t, int nz, const double* z,
                                          double* q_out, int* iters, double* resid, int r_on_device, void* stream) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  if (P->per_slot_q) return fail(DBAR_EINVAL, "dbar_ds2_potential needs a plan with one shared potential");
  dbar_status s = check_k(z, nz);
  if (s != DBAR_OK) return s;
  if (!std::isfinite(t)) return fail(DBAR_EINVAL, "t is not finite");
  if (!r) return fail(DBAR_EINVAL, "r is NULL");
  if (nz > 0 && !q_out) return fail(DBAR_EINVAL, "q_out is NULL");
  if (nz == 0) return DBAR_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const long long n = P->n;
  const cx<double>* rd = reinterpret_cast<const cx<double>*>(r);
  if (!r_on_device) {
    for (long long i = 0; i < 2 * n; ++i)
      if (!std::isfinite(r[i])) return fail(DBAR_EINVAL, "r has a non-finite entry");
    CK(cudaMemcpyAsync(P->T1, r, n * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
    rd = reinterpret_cast<const cx<double>*>(P->T1);
  }
  // potential of the problem in k: conj(r(k) e^{-i t (k^2 + conj(k)^2)/4}) on the plan's grid
  CK(timed(P, st, K_OTHER, [&] { return launch_ds2_kernel_potential(rd, P->N, P->p.L, t, P->Qdev, st); }));
  s = load_Q_device(P, P->Qdev, st);
  if (s != DBAR_OK) return s;
  return m1_half_difference(P, nz, z, 0.0, q_out, iters, resid, st);
}

// ---------------------------------------------------------------------------
// Stage entry points.
// ---------------------------------------------------------------------------
static dbar_status check_stage(dbar_plan* P, int nk) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  if (nk < 0 || nk > P->B) return fail(DBAR_EINVAL, "nk must be in [0, max_batch]");
  return DBAR_OK;
}

extern "C" dbar_status dbar_apply(dbar_plan_t P, const void* Q, int nk, const double* k, const void* S, void* AS,
                                  int fp32, void* stream) {
  dbar_status s = check_stage(P, nk);
  if (s != DBAR_OK) return s;
  s = check_k(k, nk);
  if (s != DBAR_OK) return s;
  if (nk == 0) return DBAR_OK;
  if (!Q || !S || !AS) return fail(DBAR_EINVAL, "NULL pointer");
  if (fp32 && P->conv) return fail(DBAR_EINVAL, "the convolution regularisation has FP64 kernels only");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = load_Q_device(P, reinterpret_cast<const cx<double>*>(Q), st);
  if (s != DBAR_OK) return s;
  s = upload_ek(P, k, nk, st);
  if (s != DBAR_OK) return s;
  const long long n = P->n;
  if (fp32)
    s = apply_op<float>(P, reinterpret_cast<const cx<float>*>(S), n, nullptr, 0, reinterpret_cast<cx<float>*>(P->KS),
                        n, nullptr, nk, st);
  else
    s = apply_op<double>(P, reinterpret_cast<const cx<double>*>(S), n, nullptr, 0,
                         reinterpret_cast<cx<double>*>(P->b64), n, nullptr, nk, st);
  if (s != DBAR_OK) return s;
  CK(launch_add_fields(S, fp32 ? P->KS : (void*)P->b64, AS, (long long)nk * n, fp32, st));
  CK(cudaStreamSynchronize(st));
  return DBAR_OK;
}

extern "C" dbar_status dbar_rhs(dbar_plan_t P, const double* Q, int nk, const double* k, double* b, void* stream) {
  dbar_status s = check_stage(P, nk);
  if (s != DBAR_OK) return s;
  s = check_k(k, nk);
  if (s != DBAR_OK) return s;
  if (nk == 0) return DBAR_OK;
  if (!Q || !b) return fail(DBAR_EINVAL, "NULL pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = load_Q_device(P, reinterpret_cast<const cx<double>*>(Q), st);
  if (s != DBAR_OK) return s;
  s = upload_ek(P, k, nk, st);
  if (s != DBAR_OK) return s;
  s = P->mixed ? build_rhs<float>(P, nk, st) : build_rhs<double>(P, nk, st);
  if (s != DBAR_OK) return s;
  const cx<double>* b64 = P->b64;
  if (P->resid_dd) {  // b is held as double-float pairs
    cx<double>* t2 = reinterpret_cast<cx<double>*>(P->T2);
    CK(launch_dd_to_fp64(P->b64, t2, (long long)nk * P->n, st));
    b64 = t2;
  }
  CK(cudaMemcpyAsync(b, b64, (size_t)nk * P->n * sizeof(cx<double>), cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return DBAR_OK;
}

extern "C" dbar_status dbar_m_from_S(dbar_plan_t P, int nk, const double* S, double* m, void* stream) {
  dbar_status s = check_stage(P, nk);
  if (s != DBAR_OK) return s;
  if (nk == 0) return DBAR_OK;
  if (!S || !m) return fail(DBAR_EINVAL, "NULL pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  s = h_of_S64(P, reinterpret_cast<const cx<double>*>(S), P->n, reinterpret_cast<cx<double>*>(m), P->n, nk, st);
  if (s != DBAR_OK) return s;
  CK(cudaStreamSynchronize(st));
  return DBAR_OK;
}

extern "C" dbar_status dbar_taylor(dbar_plan_t P, int nk, const void* S, double* coef, int fp32, void* stream) {
  dbar_status s = check_stage(P, nk);
  if (s != DBAR_OK) return s;
  if (nk == 0) return DBAR_OK;
  if (!S || !coef) return fail(DBAR_EINVAL, "NULL pointer");
  if (P->conv) return fail(DBAR_EINVAL, "the convolution regularisation has no Taylor coefficients");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (fp32) {
    PassArgs<float> a = base_args<float>(P);
    a.M = P->M;  // the plan's order, whatever the inner solve uses
    a.in = reinterpret_cast<const cx<float>*>(S);
    a.in_ss = P->n;
    a.out = P->T1;
    a.out_ss = P->n;
    CK(launch_pass_a<float>(a, nk, st));
  } else {
    PassArgs<double> a = base_args<double>(P);
    a.in = reinterpret_cast<const cx<double>*>(S);
    a.in_ss = P->n;
    a.out = P->T1;
    a.out_ss = P->n;
    CK(launch_pass_a<double>(a, nk, st));
  }
  cx<double>* dc = P->tcoef;
  CK(launch_coef(P->partA, fp32, P->M, P->N, P->Da64, P->Da32, 1.0, P->coefp, P->ticket, dc, nk, st));
  CK(cudaMemcpyAsync(coef, dc, (size_t)nk * (P->M + 2) * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return DBAR_OK;
}

extern "C" dbar_status dbar_fft2(dbar_plan_t P, int nk, const void* in, void* out, int sign, int fp32, void* stream) {
  dbar_status s = check_stage(P, nk);
  if (s != DBAR_OK) return s;
  if (nk == 0) return DBAR_OK;
  if (!in || !out) return fail(DBAR_EINVAL, "NULL pointer");
  if (sign != 1 && sign != -1) return fail(DBAR_EINVAL, "sign must be +1 or -1");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (fp32) {
    PassArgs<float> a = base_args<float>(P);
    a.in = reinterpret_cast<const cx<float>*>(in);
    a.in_ss = P->n;
    a.out = P->T1;
    a.out_ss = P->n;
    CK(sign < 0 ? (launch_pass_c<float, float, PC_FWD>(a, nk, st)) : (launch_pass_c<float, float, PC_INV>(a, nk, st)));
    a.in = reinterpret_cast<const cx<float>*>(P->T1);
    a.out = out;
    CK(sign < 0 ? (launch_pass_b<float, PB_FWD>(a, nk, st)) : (launch_pass_b<float, PB_INV>(a, nk, st)));
  } else {
    PassArgs<double> a = base_args<double>(P);
    a.in = reinterpret_cast<const cx<double>*>(in);
    a.in_ss = P->n;
    a.out = P->T1;
    a.out_ss = P->n;
    CK(sign < 0 ? (launch_pass_c<double, double, PC_FWD>(a, nk, st))
                : (launch_pass_c<double, double, PC_INV>(a, nk, st)));
    a.in = reinterpret_cast<const cx<double>*>(P->T1);
    a.out = out;
    CK(sign < 0 ? (launch_pass_b<double, PB_FWD>(a, nk, st)) : (launch_pass_b<double, PB_INV>(a, nk, st)));
  }
  CK(cudaStreamSynchronize(st));
  return DBAR_OK;
}

// ---------------------------------------------------------------------------
// Slot-level interface (serving).
// ---------------------------------------------------------------------------
int plan_batch(const dbar_plan* P) { return P->B; }
size_t plan_device_bytes(const dbar_plan* P) { return P->bytes; }

dbar_status plan_load_slot(dbar_plan* P, int slot, const double* Q, double k1, double k2, cudaStream_t st) {
  if (!P || slot < 0 || slot >= P->B || !Q) return fail(DBAR_EINVAL, "plan_load_slot: bad argument");
  if (!P->per_slot_q) return fail(DBAR_EINVAL, "plan_load_slot: the plan has one shared potential");
  const long long n = P->n;
  const int N = P->N;
  CK(cudaMemcpyAsync(P->Qdev, Q, n * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
  CK(timed(P, st, K_OTHER, [&] { return launch_load_q(P->Qdev, P->Q64 + slot * n, P->Q32 + slot * n, N, st); }));
  if (P->resid_dd)
    CK(timed(P, st, K_OTHER, [&] { return launch_split_fields(P->Q64 + slot * n, P->Q_dd + slot * n, n, st); }));
  const double k[2] = {k1, k2};
  cx<double>* h = P->h_ek + (size_t)slot * 2 * N;
  fill_ek(P, k, 1, h);
  CK(cudaMemcpyAsync(P->ex64 + (size_t)slot * N, h, N * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(P->ey64 + (size_t)slot * N, h + N, N * sizeof(cx<double>), cudaMemcpyHostToDevice, st));
  CK(launch_cast_fields(P->ex64 + (size_t)slot * N, P->ex32 + (size_t)slot * N, N, st));
  CK(launch_cast_fields(P->ey64 + (size_t)slot * N, P->ey32 + (size_t)slot * N, N, st));
  if (P->resid_dd) {
    CK(launch_split_fields(P->ex64 + (size_t)slot * N, P->ex_dd + (size_t)slot * N, N, st));
    CK(launch_split_fields(P->ey64 + (size_t)slot * N, P->ey_dd + (size_t)slot * N, N, st));
  }
  return DBAR_OK;
}

dbar_status plan_begin(dbar_plan* P, int nb, const int* hmask, cudaStream_t st) {
  if (!P || nb < 0 || nb > P->B) return fail(DBAR_EINVAL, "plan_begin: bad argument");
  return P->mixed ? begin_slots<float>(P, nb, hmask, st) : begin_slots<double>(P, nb, hmask, st);
}

dbar_status plan_active(dbar_plan* P, int nb, int* active, cudaStream_t st) {
  if (!P || nb < 0 || nb > P->B || !active) return fail(DBAR_EINVAL, "plan_active: bad argument");
  CK(cudaMemcpyAsync(P->h_active, P->cs.active, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  P->prof.harvest();
  std::copy(P->h_active, P->h_active + nb, active);
  return DBAR_OK;
}

// One part of a cycle: part c < plan_cycle_parts launches Krylov steps
// [c kGraphChunk, (c + 1) kGraphChunk) and queues a copy of the run flags to page-locked
// memory (plan_parts_running reads it once the stream has passed this point);
// part == plan_cycle_parts launches the cycle's tail.  No host synchronisation.
template <typename TI>
static dbar_status cycle_part(dbar_plan* P, int nb, int c, cudaStream_t st) {
  const int nchunks = (P->m + kGraphChunk - 1) / kGraphChunk;
  if (P->p.graphs) {
    CycleGraph* g = nullptr;
    const dbar_status gs = cycle_graph<TI>(P, nb, &g);
    if (gs != DBAR_OK) return gs;
    CK(cudaGraphLaunch(g->parts[c].exec, st));
    P->nlaunch += g->parts[c].kernels;
    if (P->prof.on) P->graph_ran.push_back(&g->parts[c]);
  } else {
    const dbar_status s = c < nchunks ? cycle_steps<TI>(P, nb, c * kGraphChunk, std::min(P->m, (c + 1) * kGraphChunk), st)
                                      : cycle_tail<TI>(P, nb, st);
    if (s != DBAR_OK) return s;
  }
  if (c < nchunks) CK(cudaMemcpyAsync(P->h_run, P->cs.run, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  return DBAR_OK;
}

int plan_cycle_parts(const dbar_plan* P) { return (P->m + kGraphChunk - 1) / kGraphChunk; }

dbar_status plan_step_part(dbar_plan* P, int nb, int part, cudaStream_t st) {
  if (!P || nb < 0 || nb > P->B || part < 0 || part > plan_cycle_parts(P))
    return fail(DBAR_EINVAL, "plan_step_part: bad argument");
  return P->mixed ? cycle_part<float>(P, nb, part, st) : cycle_part<double>(P, nb, part, st);
}

bool plan_parts_running(const dbar_plan* P, int nb) {
  int any = 0;
  for (int i = 0; i < nb; ++i) any |= P->h_run[i];
  return any != 0;
}

dbar_status plan_read_slot(dbar_plan* P, int slot, double* S, double* m, int* itot, int* ncyc, double* resid,
                           cudaStream_t st) {
  if (!P || slot < 0 || slot >= P->B || !S) return fail(DBAR_EINVAL, "plan_read_slot: bad argument");
  const long long n = P->n;
  const cx<double>* S64 = nullptr;
  dbar_status s0 = solution_fp64(P, slot, 1, st, &S64);
  if (s0 != DBAR_OK) return s0;
  CK(cudaMemcpyAsync(S, S64, n * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
  if (m) {
    dbar_status s = h_of_S64(P, S64, n, reinterpret_cast<cx<double>*>(P->T2), n, 1, st);
    if (s != DBAR_OK) return s;
    CK(cudaMemcpyAsync(m, P->T2, n * sizeof(cx<double>), cudaMemcpyDeviceToHost, st));
  }
  int it = 0, nc = 0;
  double rs = 0.0;
  CK(cudaMemcpyAsync(&it, P->cs.itot + slot, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&nc, P->cs.ncyc + slot, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&rs, P->cs.resid + slot, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (itot) *itot = it;
  if (ncyc) *ncyc = nc;
  if (resid) *resid = rs;
  return DBAR_OK;
}

// ---------------------------------------------------------------------------
// Profiling.
// ---------------------------------------------------------------------------
extern "C" int dbar_profile_nkinds(void) { return K_NKINDS; }

extern "C" const char* dbar_profile_kind_name(int kind) {
  return (kind >= 0 && kind < K_NKINDS) ? kKindNames[kind] : "";
}

extern "C" dbar_status dbar_profile(dbar_plan_t P, int enable) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  P->prof.reset();
  P->prof.on = enable != 0;
  return DBAR_OK;
}

extern "C" dbar_status dbar_profile_read(dbar_plan_t P, int kind, double* ms, long long* launches, double* bytes) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  if (kind < 0 || kind >= K_NKINDS) return fail(DBAR_EINVAL, "kind out of range");
  P->prof.harvest();
  if (ms) *ms = P->prof.ms[kind];
  if (launches) *launches = P->prof.launches[kind];
  if (bytes) *bytes = P->prof.bytes[kind];
  return DBAR_OK;
}

extern "C" dbar_status dbar_plan_tuning(dbar_plan_t P, int* column_variant, double* ms_per_variant,
                                        int* row_shape, double* ms_per_row_shape) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  if (column_variant) *column_variant = P->colv;
  if (ms_per_variant)
    for (int v = 0; v < DBAR_COLUMN_VARIANTS; ++v) ms_per_variant[v] = P->tune_ms[v];
  if (row_shape) *row_shape = P->rowv;
  if (ms_per_row_shape)
    for (int v = 0; v < DBAR_ROW_VARIANTS; ++v) ms_per_row_shape[v] = P->row_ms[v];
  return DBAR_OK;
}

extern "C" dbar_status dbar_plan_row_tuning(dbar_plan_t P, int* row_shape, double* ms_per_row_shape) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  if (row_shape) *row_shape = P->rowv_ac;
  if (ms_per_row_shape)
    for (int v = 0; v < DBAR_ROW_VARIANTS; ++v) ms_per_row_shape[v] = P->row_ms_ac[v];
  return DBAR_OK;
}

extern "C" dbar_status dbar_plan_inject_wait_timeout(dbar_plan_t P) {
  if (!P) return fail(DBAR_EINVAL, "plan is NULL");
  if (P->sstep <= 1 || P->iter || P->conv)
    return fail(DBAR_EINVAL, "the plan has no block-update sweeps (sstep > 1, Sec. 4 equation)");
  P->inject_tx = 16;
  for (CycleGraph& g : P->graphs) g.clear();  // the next cycle is captured with the hook in place
  return DBAR_OK;
}

extern "C" dbar_status dbar_launch_count(dbar_plan_t P, long long* count) {
  if (!P || !count) return fail(DBAR_EINVAL, "NULL argument");
  *count = P->nlaunch;
  return DBAR_OK;
}
