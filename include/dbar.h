/*
 * dbar.h -- C ABI of the GB300 spectral D-bar CGO solver.
 *
 * Method: C. Klein, K. McLaughlin, "Spectral approach to D-bar problems".
 * A CGO solution m of  dbar m = 1/2 E_k Q (conj(m) + 1),  E_k = e^{conj(kz)-kz}
 * (Sec. 1, eq:038/eq:039) is found through S = xi m^ (eq:042), which solves
 * the real-linear system (eq:MainEQa, Sec. 5.1 eq:MainEQDS)
 *     A S := S + i F(E_k Q conj(F^{-1}(S/xi))) = b := -i F(E_k Q),
 * with F^{-1}(S/xi) regularised as in Sec. 4.2 (eq. Sreg, Gchoice, fourreeg4,
 * fourreg5): a Taylor-Gaussian G of order M is removed before the division by
 * xi and its inverse transform sum_n c_n W_n is added back in closed form.
 * The system is solved by GMRES on the stacked real and imaginary parts
 * (Sec. 4.1, Sec. 4.3).
 *
 * Discretisation (Sec. 4.1, eq. domain / xidomain): x_j = L(-pi + 2 pi j/N),
 * j = 0..N-1, the same in y; xi_m = m/L, m in [-N/2+1, N/2].
 *
 * Layouts (all arrays row-major, complex numbers interleaved re,im):
 *   physical fields  [y index j2][x index j1]           (Q, m)
 *   Fourier fields   [p2][p1], p = m mod N (natural DFT order; m = p for
 *                    p <= N/2, else p - N)                (S, b, A S)
 *   batched fields   [k][...] with stride N*N complex.
 *
 * Conventions: every entry point returns a dbar_status; no C++ exception
 * crosses the ABI.  On failure the message of the calling thread's last error
 * is available from dbar_last_error().  Host pointers are ordinary pageable
 * or pinned memory; "device" pointers are CUDA global memory on the device
 * the plan was created on.  The caller owns every buffer it passes; the plan
 * owns its own device tables and workspaces.  Calls are ordered on the given
 * CUDA stream (NULL = legacy default stream) and return after the stream has
 * drained, unless stated otherwise.
 */
#ifndef DBAR_H
#define DBAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DBAR_OK = 0,
  DBAR_EINVAL = 1,   /* bad argument: N not a power of two in [32, 2048], L <= 0,
                        NaN/Inf in Q or k, null pointer where one is required  */
  DBAR_ENOMEM = 2,   /* a device allocation failed                              */
  DBAR_ENOCONV = 3,  /* some k missed tol within max_iter / max_outer; outputs
                        are still written (best iterate and its residual)       */
  DBAR_ETIMEOUT = 4, /* a bounded device wait ran out (kernel-side limit)     */
  DBAR_ECUDA = 5,    /* a CUDA call failed; see dbar_last_error()               */
  DBAR_EBUSY = 6     /* reserved for asynchronous interfaces                    */
} dbar_status;

typedef enum {
  DBAR_FP64 = 0,     /* GMRES entirely in FP64 (restarted on the true residual) */
  DBAR_MIXED = 1     /* FP32 inner GMRES, FP64 true residual and update
                        (iterative refinement)                                  */
} dbar_prec;

typedef enum {
  DBAR_RESID_DOUBLE_FLOAT = 0, /* float pairs (hi + lo, ~48-bit significand) on the
                                  FP32 pipes; default                          */
  DBAR_RESID_FP64 = 1          /* native FP64                                   */
} dbar_resid_mode;

/* How F^{-1}(S/xi) is regularised at xi = 0 (eq. Sreg: S/xi = (S - G)/xi + G/xi). */
typedef enum {
  DBAR_REG_TAYLOR = 0, /* G = e^{-|xi|^2} sum_{n<=M} c_n conj(xi)^n (Sec. 4.2, eq.
                          Gchoice), F^{-1}(G/xi) = sum c_n W_n in closed form;
                          the method of the paper (default)                    */
  DBAR_REG_CONV = 1    /* G = S e^{-|xi|^2} (Sec. 4.2, remark after eq.
                          fourreg5a): (S - G)/xi = S (1 - e^{-|xi|^2})/xi is
                          smooth and goes through the FFT, and
                          F^{-1}(G/xi) = (1/2pi) int F^{-1}(S)(z') W_0(z - z') d^2z'
                          is summed directly over every pair of grid points
                          (N^4 complex multiply-adds per field).  The paper
                          keeps it as an independent test of the Taylor code.
                          FP64 only (prec = DBAR_FP64), N <= 256, not with
                          iterated, sstep 0 means 1 here; M is unused and
                          dbar_taylor returns DBAR_EINVAL                     */
} dbar_regularisation;

typedef struct {
  int N;             /* grid points per axis: power of two, 32 <= N <= 2048    */
  double L;          /* box [-pi L, pi L]^2 (Sec. 4.1, eq. domain), L > 0        */
  int M;             /* Taylor order of G (Sec. 4.2, eq. Gchoice), 0 <= M <= 16 */
  int prec;          /* dbar_prec                                               */
  int restart;       /* Krylov vectors per cycle, 1..128                        */
  int max_iter;      /* cap on the total inner iterations of one k              */
  double tol;        /* target ||b - A S||_2 / ||b||_2 (stacked real 2-norm)    */
  int zero_fill;     /* value of (S-G)/xi at xi = 0: 0 = analytic limit
                        dS/dxi(0) (default), 1 = zero                          */
  int max_batch;     /* k values solved concurrently; 0 = chosen from memory    */
  double inner_tol;  /* DBAR_MIXED: relative residual reduction per FP32 cycle  */
  int max_outer;     /* cap on cycles (restarts / refinement steps)             */
  int resid_mode;    /* DBAR_MIXED: arithmetic of the right-hand side and of the
                        true residual b - A x (dbar_resid_mode)                 */
  int graphs;        /* 1: each Krylov cycle is captured once as a CUDA graph
                        and replayed (default); 0: kernels launched one by one  */
  int autotune;      /* 1 (default): at plan creation, time the compiled tile
                        shapes of the FP32 column pass on the plan's own
                        workspaces and keep the faster (results are identical
                        across shapes); cached per (device, N, M).
                        0: first shape; 2: second; 3: third (for checks)       */
  int sstep;         /* Krylov vectors formed per sweep of the stored basis.
                        2 or 4: s-step blocks -- the chain p, Kp, ..., of
                        K = A - I is orthogonalised against the basis in one
                        pass (block Gram-Schmidt + Cholesky QR), which cuts
                        the basis traffic per Krylov vector about S-fold; the
                        Krylov space and the minimisation are those of GMRES,
                        convergence is checked at block ends; restart must be
                        a multiple of sstep.  1: one vector per sweep
                        (classical Gram-Schmidt per step).  0 (default): 4
                        if restart is a multiple of 4, else 2 if even, else 1;
                        1 for iterated and convolution plans               */
  int iterated;      /* 1: the plan solves the iterated integral equation of
                        Sec. 5.2-5.3 (eq. eqh2, shifted regularisation eq.
                        dbarinvShift) for h instead of the Sec. 4 equation for
                        S: h - K_0(H(h)) = -i F(Q), supported near the origin
                        for every k; 2k must lie on the xi-grid (2 k L integer
                        in both components, within [-N/2, N/2]).  sstep 0
                        means 1 here (solves of a few iterations, which
                        blocks overshoot); sstep 2 or 4 chain whole
                        applications of its operator in a block;
                        dbar_solve_cgo returns h in S_out and takes no m_out.
                        0 (default): the Sec. 4 equation                      */
  int regularisation; /* dbar_regularisation; 0 (DBAR_REG_TAYLOR) by default */
  int inner_M;       /* DBAR_MIXED: Taylor order of the FP32 inner operator,
                        0 <= inner_M <= M; 0 (default) means M.  The right-hand
                        side and the true residual always use M, so the result
                        is the M solution; a smaller inner order only changes
                        the correction solves (the M = 2 and M = 11 operators
                        differ by ~1e-8 relative, below FP32 rounding) and
                        saves their table reads and moments                  */
  double gauss_w;    /* width w of the Gaussian of G (Sec. 4.2, eq. Gchoice with
                        e^{-|xi|^2} read as e^{-|xi|^2/w^2}); w > 0, 1 (default)
                        is the paper's choice.  The Taylor data c_n and the fill
                        value do not depend on w; the closed-form part becomes
                        F^{-1}(G/xi) = sum_n c_n w^{n+1} W_n(w z) (eq. fourreg5
                        at w z).  With DBAR_REG_CONV: G = S e^{-|xi|^2/w^2}    */
  size_t mem_budget; /* device bytes the plan may hold once created; 0 (default)
                        = no limit.  With max_batch = 0 the batch is the largest
                        that fits (at most 256); a plan that cannot fit
                        max_batch slots (or one slot) fails with DBAR_ENOMEM.
                        Plan creation briefly takes 2(M+1) FP64 fields more
                        for building its tables                               */
  int support_skip;  /* DBAR_MIXED, one potential per plan, Sec. 4 equation: 1
                        (default): the FP32 inner operator and the double-float
                        residual skip the grid columns on which Q is exactly
                        zero in FP32 (and in its double-float copy, a pair of
                        floats), where w = E_k Q conj(h) is exactly zero --
                        the same values, less work and traffic for a potential
                        concentrated near the origin; 0: every column         */
  int row_shape;     /* DBAR_MIXED: lines per block of the FP32 operator's row
                        passes.  0 (default): timed at plan creation with
                        autotune = 1 (else the first shape); 1..5: the first
                        (256 threads at N = 1024), second (half as many lines)
                        or third shape (twice as many), and the first two with
                        a larger register budget per thread (three quarters
                        of the threads resident per SM).  The arithmetic per
                        line is the same in every shape.  Pins the fused chain
                        row pass, and the plain row passes A and C unless
                        row_shape_plain is set                                */
  int row_shape_plain; /* DBAR_MIXED: 1..5 pins the shape of the plain row
                        passes A and C alone (tuned apart from the fused chain
                        pass, whose best shape differs); 0: row_shape's rule   */
} dbar_params;

typedef struct dbar_plan* dbar_plan_t;

/* Defaults for a grid: M = 2, DBAR_MIXED, restart 32, tol 1e-12,
 * inner_tol 1e-6, max_outer 40, max_iter 4000, analytic fill,
 * DBAR_RESID_DOUBLE_FLOAT, graphs on, autotune on, sstep 0 (automatic),
 * gauss_w 1, no memory budget, support_skip 1. */
void dbar_params_init(dbar_params* p, int N, double L);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* dbar_last_error(void);

/* Builds the grid tables on the current CUDA device: twiddles, the per-axis
 * moment tables D_a(p) = sum_j x_j^a e^{2 pi i p j/N} used for the Taylor
 * coefficients (Sec. 4.3 step 4a, eq. fourreeg4), and the correction fields
 * W_n - F_d^{-1}(e^{-|xi|^2} conj(xi)^n/xi) that carry the closed-form part of
 * the regularisation (Sec. 4.2, eq. fourreg5).  Workspaces for max_batch k
 * values are allocated here.  *out receives the plan; on failure *out = NULL.
 * Errors: DBAR_EINVAL, DBAR_ENOMEM, DBAR_ECUDA. */
dbar_status dbar_plan_create(const dbar_params* p, dbar_plan_t* out);

/* Frees every device resource of the plan (NULL is accepted). */
dbar_status dbar_plan_destroy(dbar_plan_t plan);

/* Check of the bounded device-side wait (no plan needed): one CTA on the
 * current device runs an mbarrier wait of the kind the bulk-copy block update
 * uses, at most `rounds` try_wait rounds (1 <= rounds <= the sweeps' own limit,
 * 2^18, about a second).  complete = 1: a 16-byte bulk copy completes the awaited phase and the
 * call returns DBAR_OK; complete = 0: nothing completes it, the wait runs out
 * and the call returns DBAR_ETIMEOUT with the context still usable.  seconds
 * (may be NULL) receives the kernel's duration.  Synchronous on stream.
 * Errors: DBAR_EINVAL (rounds), DBAR_ETIMEOUT, DBAR_ECUDA. */
dbar_status dbar_check_bounded_wait(int complete, int rounds, double* seconds, void* stream);

/* Bytes of device memory the plan holds, and the batch size it uses. */
dbar_status dbar_plan_info(dbar_plan_t plan, size_t* device_bytes, int* max_batch);

/* CGO solve for nk values of k with one potential Q (Sec. 4.3 algorithm with
 * Q -> E_k Q, Sec. 5.1).
 *   Q        N*N complex (2*N*N doubles), physical layout; host or device
 *   nk       number of k values (0 is accepted and does nothing)
 *   k        2*nk doubles (Re k, Im k), host memory
 *   x0       NULL, or nk*N*N complex: initial guess of S per k (Fourier grid;
 *            host or device like S_out).  GMRES (Sec. 4.1) leaves the start
 *            vector open; NULL starts from S = 0.  With x0 the first cycle
 *            starts from the true residual b - A x0 (FP64, or double-float on
 *            a mixed plan), tol stays relative to ||b||, and the iteration and
 *            cycle counts restart from 0.  Resuming an interrupted batch: pass
 *            the S_out of a call that returned DBAR_ENOCONV (e.g. capped by
 *            max_outer) as x0.  Non-finite entries give DBAR_EINVAL.  x0 may
 *            be the same buffer as S_out
 *   S_out    nk*N*N complex: S = xi m^ on the Fourier grid; host or device.
 *            A page-locked host S_out (cudaHostAlloc / cudaHostRegister, mapped
 *            into the device's address space) of a mixed plan is written by
 *            the device directly when m_out is NULL (no device staging copy)
 *   m_out    nk*N*N complex: m on the x-grid (Sec. 4.3, eq. S0Taylor: m = h);
 *            may be NULL
 *   iters    2*nk ints, host, may be NULL: (total inner iterations, cycles)
 *   resid    nk doubles, host, may be NULL: final ||b - A S||/||b|| in FP64
 *   io_on_device  1: Q, x0, S_out, m_out are device pointers; 0: host pointers
 *   stream   cudaStream_t or NULL
 * m^(1) = i S(0) (the 1/z coefficient, Sec. 6 eq:m1def) is S_out[k][0][0]*i.
 * Returns DBAR_ENOCONV when some k missed tol (outputs still written). */
dbar_status dbar_solve_cgo(dbar_plan_t plan, const double* Q, int nk, const double* k,
                           const double* x0, double* S_out, double* m_out, int* iters,
                           double* resid, int io_on_device, void* stream);

/* Uneven batches: many CGO solves (Sec. 4.3 with Q -> E_k Q, Sec. 5.1) on
 * grids of different sizes or with different potentials, one plan per grid.
 * Each batch is one dbar_solve_cgo call (same arguments, same results); the
 * batches of different plans run at the same time, one host thread and one
 * CUDA stream per plan, so that the launches of different grids overlap on
 * the GPU; batches of the same plan run in list order.  Work queued on
 * `stream` before the call finishes first; the call returns when every batch
 * is done.  Each batch's own status is written to its `status`; the call
 * returns the first failure in list order, else DBAR_ENOCONV if a batch missed
 * tol, else DBAR_OK.  A plan must not be used by another thread meanwhile. */
typedef struct {
  dbar_plan_t plan;   /* the grid (and settings) of this batch                     */
  const double* Q;    /* as dbar_solve_cgo                                          */
  int nk;
  const double* k;
  const double* x0;
  double* S_out;
  double* m_out;
  int* iters;
  double* resid;
  int io_on_device;
  dbar_status status; /* out: this batch's result                                   */
} dbar_batch;
dbar_status dbar_solve_batches(dbar_batch* batches, int nbatch, void* stream);

/* DS II reflection coefficient (Sec. 6.1, eq. MainEQDSpm, hpmdef, rviah,
 * m1def; time dependence eq. rt).  Sec. 6 replaces k by k/2, so for each k the
 * plan solves the CGO problem of dbar_solve_cgo at the parameter k/2 twice,
 * with the potential +Q (S_+) and -Q (S_-), and returns
 *     r(k, t) = (i/2) (S_+(0) - S_-(0)) exp(-i t (k^2 + conj(k)^2) / 4)
 * (eq. rviah: r = i h(i conj k) = (m^(1)_+ - m^(1)_-)/2, m^(1) = i S(0)).
 *   Q        N*N complex (interleaved doubles, row-major [y][x]); host, or
 *            device when q_on_device != 0
 *   k        2*nk doubles (Re, Im), host
 *   t        time of eq. rt (0: r(k, 0))
 *   r_out    host, 2*nk doubles (Re, Im of r(k, t))
 *   iters    host or NULL, nk*2 ints: inner iterations of both solves summed,
 *            and the larger outer-cycle count
 *   resid    host or NULL, nk doubles: the larger final relative residual
 * Only S(0) of each solve is copied off the GPU.  Plans made for serving are
 * rejected (DBAR_EINVAL).  Returns DBAR_ENOCONV when a solve missed tol
 * (r_out still written). */
dbar_status dbar_reflection(dbar_plan_t plan, const double* Q, int nk, const double* k, double t,
                            double* r_out, int* iters, double* resid, int q_on_device, void* stream);

/* DS II potential q(x, y, t) from the reflection coefficient (Sec. 1 eq.
 * dbarrecA/B and qRec with the time dependence eq. rt; Sec. 6.2).  The
 * D-bar problem in k is a CGO problem in the variable k: the plan's grid is
 * the k-grid (with Sec. 6's convention the reflection coefficient computed on
 * a plan of box L lives on the points m/L, i.e. on the grid of a plan with
 * box L' = N/(2 pi L)), its potential is conj(r(k) e^{-i t (k^2 + conj(k)^2)/4})
 * and its parameter is z/2, so that
 *     q(z, t) = (m~^(1)_+ - m~^(1)_-)/2,
 * the quantity dbar_reflection returns with the roles of z and k exchanged.
 *   r        N*N complex r(k, 0) on the plan's grid, row-major [k2][k1];
 *            host, or device when r_on_device != 0
 *   z        2*nz doubles (x, y) of the points where q is wanted, host; an
 *            iterated plan needs z L' integer in both components (the x-grid
 *            of the box L)
 *   q_out    host, 2*nz doubles (Re, Im of q(z, t))
 *   iters, resid as in dbar_reflection.  Returns DBAR_ENOCONV when a solve
 *   missed tol (q_out still written). */
dbar_status dbar_ds2_potential(dbar_plan_t plan, const double* r, double t, int nz, const double* z,
                               double* q_out, int* iters, double* resid, int r_on_device, void* stream);

/* --- stage entry points (device pointers; used for parity checks) -------- */

/* A S for nk fields (Sec. 4.3 step 4):  AS[i] = S[i] + i F(E_{k_i} Q conj(h(S[i]))).
 * fp32 = 0: S, AS, Q are complex128 (double pairs); fp32 = 1: complex64 (float
 * pairs), computed by the FP32 kernels of the inner solve.  nk <= max_batch. */
dbar_status dbar_apply(dbar_plan_t plan, const void* Q, int nk, const double* k,
                       const void* S, void* AS, int fp32, void* stream);

/* b = -i F(E_k Q) (Sec. 4.3 step 3), complex128, nk <= max_batch. */
dbar_status dbar_rhs(dbar_plan_t plan, const double* Q, int nk, const double* k,
                     double* b, void* stream);

/* m = h(S) = F^{-1}((S-G)/xi) + sum_n c_n W_n (eq. S0Taylor), complex128. */
dbar_status dbar_m_from_S(dbar_plan_t plan, int nk, const double* S, double* m, void* stream);

/* Taylor data of S (Sec. 4.3 step 4a, eq. fourreeg4): c[i][n], n = 0..M, with
 * n! c_n = (-i/2)^n F(z^n F^{-1} S)(0), then the fill value d = dS/dxi(0)
 * = (-i/2) F(conj(z) F^{-1} S)(0).  coef: host, nk*(M+2) complex (doubles).
 * fp32 selects the complex64 kernels as in dbar_apply. */
dbar_status dbar_taylor(dbar_plan_t plan, int nk, const void* S, double* coef, int fp32,
                        void* stream);

/* Unnormalised 2-D DFT over [y][x] (sign -1: forward e^{-2 pi i p.j/N}, +1:
 * inverse e^{+...}), nk fields, complex128 or complex64 (fp32 = 1). */
dbar_status dbar_fft2(dbar_plan_t plan, int nk, const void* in, void* out, int sign, int fp32,
                      void* stream);

/* Allocation-free variant of dbar_fft2, for callers that cannot allocate
 * device memory when they need a transform: plugins whose host runtime owns
 * all device memory through its own pool (a cudaMalloc would bypass its
 * accounting or fail against its reservation), and latency-critical loops
 * that forbid allocator calls (cudaMalloc/cudaFree may synchronise the device).
 * (The paper has no counterpart: this is an interface for such callers.)
 * It needs no plan.  Its intermediate field and twiddle tables live in the
 * library's own global arrays: every GPU that loads the library keeps 32 MiB
 * of scratch plus ~100 KiB of tables until the process exits.  Limit:
 * nk*N*N*sizeof(element) <= 32 MiB (2M complex128 or 4M complex64 values per
 * call: one 2048^2 complex64 field, two 1024^2 complex128 fields); larger
 * calls return DBAR_EINVAL.  N is a power of two in [32, 2048].
 * All calls share the scratch, so calls that overlap on the GPU race.  The
 * first call on a device uploads the twiddle tables and looks up the arrays'
 * device addresses with that device current.  in and out are
 * device pointers ([nk][N][N], complex128, or complex64 when fp32 = 1) and may
 * be equal; sign as in dbar_fft2.  Returns after the stream has drained
 * (the call ends with a synchronisation of `stream`).
 * Errors: DBAR_EINVAL (N, nk, sign, NULL pointers, size beyond the scratch),
 * DBAR_ECUDA. */
dbar_status dbar_fft2_noalloc(int N, int nk, const void* in, void* out, int sign, int fp32, void* stream);

/* --- serving: continuous batching ------------------------------------- */

/* Many CGO solves are needed per potential and across potentials (Sec. 1;
 * Sec. 7 outlook).  A server solves requests submitted from any host thread
 * on one GPU.  Requests of one grid class (N, L) share a batch ("lane") whose
 * slots each hold one request with its own Q and k; at every GMRES cycle
 * boundary a lane retires finished slots and admits waiting requests into the
 * free ones, so new work joins while older work is still iterating.  A
 * result does not depend on the requests it was batched with.  Device memory
 * is admitted by mem_budget (bytes): a lane gets the slots the budget leaves
 * room for; idle lanes are dropped when another grid class needs the memory.
 * The solver settings (M, prec, restart, tol, ...) come from `defaults`
 * (its N and L are ignored; max_batch > 0 caps the slots of a lane). */
typedef struct dbar_server* dbar_server_t;

typedef struct {
  int N;             /* grid of this request (power of two in [32, 2048])       */
  double L;          /* box [-pi L, pi L]^2                                      */
  const double* Q;   /* host, N*N complex128, physical layout; copied at submit  */
  double k_re, k_im; /* spectral parameter k                                     */
  int want_m;        /* 1: also return m = h(S) on the x-grid                    */
} dbar_request;

typedef struct {
  dbar_status status; /* DBAR_OK, DBAR_ENOCONV (tol missed), or the failure     */
  int iters;          /* total inner Krylov iterations                          */
  int cycles;         /* cycles (restarts / refinement steps)                   */
  double resid;       /* final ||b - A S|| / ||b||                              */
  double latency_ms;  /* submit -> done                                         */
  double queue_ms;    /* submit -> admitted into a slot                         */
  double run_ms;      /* admitted -> done                                       */
  const double* S;    /* N*N complex128 (Fourier grid); owned by the server     */
  const double* m;    /* N*N complex128 or NULL; owned by the server            */
} dbar_result;

dbar_status dbar_serve_create(const dbar_params* defaults, size_t mem_budget, dbar_server_t* out);
/* Errors: DBAR_EINVAL (bad N, L, NaN/Inf in Q or k), DBAR_ENOMEM (one slot of
 * this grid cannot fit the budget). */
dbar_status dbar_serve_submit(dbar_server_t srv, const dbar_request* rq, uint64_t* ticket);
/* DBAR_EBUSY while the request is pending; DBAR_OK with *out filled when done. */
dbar_status dbar_serve_poll(dbar_server_t srv, uint64_t ticket, dbar_result* out);
/* Blocks until done (timeout_s < 0: no limit); DBAR_ETIMEOUT when it runs out. */
dbar_status dbar_serve_wait(dbar_server_t srv, uint64_t ticket, double timeout_s, dbar_result* out);
/* Frees a finished request's buffers (its S and m pointers become invalid). */
dbar_status dbar_serve_release(dbar_server_t srv, uint64_t ticket);
/* Latency percentiles over finished requests, throughput since the first
 * submit, finished and pending counts (any pointer may be NULL). */
dbar_status dbar_serve_stats(dbar_server_t srv, double* p50_ms, double* p99_ms, double* solves_per_s,
                             uint64_t* completed, uint64_t* pending);
/* Host-side fault injection for tests: the next lane cycle reports a failure;
 * its in-flight requests are re-queued once and the lane's plan is rebuilt. */
dbar_status dbar_serve_inject_fault(dbar_server_t srv);
/* Stops the worker (pending requests are abandoned) and frees everything. */
dbar_status dbar_serve_destroy(dbar_server_t srv);

/* --- tracing ------------------------------------------------------------ */

/* Number of kernel kinds the profiler distinguishes, and the name of one. */
int dbar_profile_nkinds(void);
const char* dbar_profile_kind_name(int kind);

/* Turns CUDA-event timing of every kernel launch of dbar_solve_cgo on (1) or
 * off (0) and clears the counters.  With timing on, each launch is bracketed
 * by two events on the solve's stream; the totals are folded in at the
 * solve's host synchronisation points. */
dbar_status dbar_profile(dbar_plan_t plan, int enable);

/* Totals of one kind since dbar_profile(plan, 1): summed event time in ms,
 * launches, and the algorithmic bytes of those launches (every field the
 * method reads or writes counted once per use).  For the kind
 * "conv_direct_sum" (the direct sum of DBAR_REG_CONV, bound by FP64
 * arithmetic) the last value counts floating-point operations instead:
 * 8 N^4 per field and operator application.  Any pointer may be NULL. */
dbar_status dbar_profile_read(dbar_plan_t plan, int kind, double* ms, long long* launches, double* bytes);

/* Tile variants of the FP32 operator column pass: 0: 64-byte row segments,
 * 512 threads per block (N = 1024); 1: 32-byte segments, 256 threads; 2: the
 * shape of 0 with two k values per block (shared table tiles, the two slots'
 * transforms in lockstep). */
#define DBAR_COLUMN_VARIANTS 3

/* Row-pass shapes of the FP32 operator (row_shape). */
#define DBAR_ROW_VARIANTS 5

/* The autotuner's choices: column-pass tile variant in use and the measured ms
 * per launch of each variant in ms_per_variant[DBAR_COLUMN_VARIANTS]; row-pass
 * shape in use (0-based) and the ms per fused row-pass launch of each shape in
 * ms_per_row_shape[DBAR_ROW_VARIANTS] (0 when not tuned).  The FFT radix
 * schedule is fixed per N (radix 16 stages, then the remainder): a different
 * split would change the rounding, and so the results, from one tuning to
 * the next.  Any pointer may be NULL. */
dbar_status dbar_plan_tuning(dbar_plan_t plan, int* column_variant, double* ms_per_variant, int* row_shape,
                             double* ms_per_row_shape);

/* The row-pass shape of the FP32 operator's plain row passes (pass A of each
 * block's first vector, pass C of the last), tuned apart from the fused chain
 * pass that dbar_plan_tuning reports (their best shapes differ): the shape in
 * use (0-based) and the ms per pass A + pass C pair of each shape in
 * ms_per_row_shape[DBAR_ROW_VARIANTS] (0 when not tuned).  A fixed row_shape
 * parameter sets both.  Either pointer may be NULL; DBAR_EINVAL for a NULL plan. */
dbar_status dbar_plan_row_tuning(dbar_plan_t plan, int* row_shape, double* ms_per_row_shape);

/* Test hook for the device-side bounded waits (no counterpart in the paper):
 * the next block-update launch of this plan announces 16 bytes more on its
 * first bulk-copy stage than the copy delivers, so that stage's mbarrier phase
 * cannot complete and every wait on it runs out (2^18 try_wait rounds, about
 * a second, then as long again while the block drains its copies).  The solve
 * in progress returns DBAR_ETIMEOUT at its next cycle boundary; the plan drops
 * its captured cycle graphs and solves normally afterwards.  Nothing faults or
 * hangs.  Plans with s-step blocks only (sstep > 1, Sec. 4 equation); else
 * DBAR_EINVAL. */
dbar_status dbar_plan_inject_wait_timeout(dbar_plan_t plan);

/* Kernels launched by this plan since its creation (profiling on or off). */
dbar_status dbar_launch_count(dbar_plan_t plan, long long* count);

#ifdef __cplusplus
}
#endif

#endif /* DBAR_H */
