// Batched GMRES on the stacked real and imaginary parts (Sec. 4.1, Sec. 4.3:
// "Call GMRES with b = -iFQ").  The operator is only real-linear (it contains
// a complex conjugation), so the unknown is x = [Re S; Im S] in R^{2 N^2} and
// every inner product is <a, b> = Re sum conj(a) b; all Krylov coefficients
// are real.
//
// Each slot (one value of k) runs its own Arnoldi process; all slots advance
// in lock step and a per-slot flag masks slots whose cycle has finished.
// Orthogonalisation is classical Gram-Schmidt: one pass of dot products
// against all basis vectors, one update pass.  Basis vectors are stored
// unnormalised (v~_i) with a per-slot scale sigma_i = 1/||v~_i|| applied by
// every reader, which saves a normalisation pass.
//
// Reductions are two-level with a fixed order (per-block partials in FP64,
// then a single block per slot), so a slot's result does not depend on which
// other slots share the launch.
#pragma once
#include "types.cuh"

namespace dbar {

// Block sum of per-thread partials: within each warp in the partials' own
// precision (FP32 for the inner solve: GB300's FP64 pipe cannot keep up with
// one FP64 operation per element at HBM speed), across warps in FP64.
template <typename T>
__device__ __forceinline__ double block_sum_256(T v, double* sh) {
  v = warp_sum_t(v, 32);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;  // valid in thread 0
}

// part[slot][i][chunk] = <v~_i, w>, w = sigma_j v~_j + KS, i = 0..j
template <typename T>
__global__ void __launch_bounds__(KR_THREADS) k_dots(const KryArgs a, const cx<T>* __restrict__ V,
                                                      long long vss, const cx<T>* __restrict__ KS,
                                                      long long kss, int j) {
  __shared__ double red[KR_THREADS / 32][129];
  const int slot = blockIdx.y;
  if (!a.run[slot]) return;
  const long long base = (long long)blockIdx.x * KR_CHUNK + threadIdx.x;
  const cx<T>* Vs = V + (size_t)slot * vss;
  const T sj = (T)a.sigma[(size_t)slot * a.mp1 + j];
  cx<T> w[KR_EPT];
#pragma unroll
  for (int e = 0; e < KR_EPT; ++e) {
    const long long idx = base + (long long)e * KR_THREADS;
    if (idx < a.n) {
      const cx<T> vj = ldg(Vs + (size_t)j * a.n + idx);
      const cx<T> ks = ldg(KS + (size_t)slot * kss + idx);
      w[e] = mkc(sj * vj.re + ks.re, sj * vj.im + ks.im);
    } else {
      w[e] = mkc((T)0, (T)0);
    }
  }
  const int wid = threadIdx.x >> 5;
  for (int i = 0; i <= j; ++i) {
    T s = 0;
#pragma unroll
    for (int e = 0; e < KR_EPT; ++e) {
      const long long idx = base + (long long)e * KR_THREADS;
      if (idx < a.n) {
        const cx<T> vi = ldg(Vs + (size_t)i * a.n + idx);
        s += vi.re * w[e].re + vi.im * w[e].im;
      }
    }
    const T d = warp_sum_t(s, 32);
    if ((threadIdx.x & 31) == 0) red[wid][i] = (double)d;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double s = 0.0;
    for (int w2 = 0; w2 < KR_THREADS / 32; ++w2) s += red[w2][i];
    a.part[((size_t)slot * a.mp1 + i) * a.nchunk + blockIdx.x] = s;
  }
}

// H[slot][j][i] = h_i = sigma_i sum_chunks part;  coef[slot][i] = h_i sigma_i
// One warp per slot (KR_THREADS / 32 slots per block): the j + 1 reductions are
// warp shuffles, not block barriers, and thousands of small slots share blocks.
static __global__ void __launch_bounds__(KR_THREADS) k_finalize_h(const KryArgs a, double* H, int j, int nslots) {
  const int slot = blockIdx.x * (KR_THREADS / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (slot >= nslots || !a.run[slot]) return;
  for (int i = 0; i <= j; ++i) {
    double s = 0.0;
    const double* p = a.part + ((size_t)slot * a.mp1 + i) * a.nchunk;
    for (int c = lane; c < a.nchunk; c += 32) s += p[c];
    s = warp_sum(s, 32);
    if (lane == 0) {
      const double sg = a.sigma[(size_t)slot * a.mp1 + i];
      const double h = s * sg;
      H[((size_t)slot * (a.mp1 - 1) + j) * a.mp1 + i] = h;
      a.coef[(size_t)slot * a.mp1 + i] = h * sg;
    }
  }
}

// v~_{j+1} = sigma_j v~_j + KS - sum_i coef_i v~_i ; part2 = ||v~_{j+1}||^2 partials
template <typename T>
__global__ void __launch_bounds__(KR_THREADS) k_update(const KryArgs a, cx<T>* __restrict__ V, long long vss,
                                                        const cx<T>* __restrict__ KS, long long kss, int j) {
  __shared__ double sh[KR_THREADS / 32];
  const int slot = blockIdx.y;
  if (!a.run[slot]) return;
  const long long base = (long long)blockIdx.x * KR_CHUNK + threadIdx.x;
  cx<T>* Vs = V + (size_t)slot * vss;
  const T sj = (T)a.sigma[(size_t)slot * a.mp1 + j];
  cx<T> w[KR_EPT];
#pragma unroll
  for (int e = 0; e < KR_EPT; ++e) {
    const long long idx = base + (long long)e * KR_THREADS;
    if (idx < a.n) {
      const cx<T> vj = ldg(Vs + (size_t)j * a.n + idx);
      const cx<T> ks = ldg(KS + (size_t)slot * kss + idx);
      w[e] = mkc(sj * vj.re + ks.re, sj * vj.im + ks.im);
    } else {
      w[e] = mkc((T)0, (T)0);
    }
  }
  for (int i = 0; i <= j; ++i) {
    const T c = (T)a.coef[(size_t)slot * a.mp1 + i];
#pragma unroll
    for (int e = 0; e < KR_EPT; ++e) {
      const long long idx = base + (long long)e * KR_THREADS;
      if (idx < a.n) {
        const cx<T> vi = ldg(Vs + (size_t)i * a.n + idx);
        w[e] = mkc(w[e].re - c * vi.re, w[e].im - c * vi.im);
      }
    }
  }
  T s = 0;
#pragma unroll
  for (int e = 0; e < KR_EPT; ++e) {
    const long long idx = base + (long long)e * KR_THREADS;
    if (idx < a.n) {
      Vs[(size_t)(j + 1) * a.n + idx] = w[e];
      s += w[e].re * w[e].re + w[e].im * w[e].im;
    }
  }
  const double tot = block_sum_256(s, sh);
  if (threadIdx.x == 0) a.part2[(size_t)slot * a.nchunk + blockIdx.x] = tot;
}


// Givens step for Hessenberg column j of a slot whose rows 0..j+1 are in Hc:
// applies the earlier rotations, forms rotation j, updates g and the step
// counters; returns true when the slot's cycle stops after this column
// (residual estimate below the threshold, cycle full, iteration cap, or a
// zero subdiagonal: the Krylov space is invariant).
__device__ inline bool givens_column(const CycleState& c, int slot, int j, double* Hc) {
  const int m = c.m;
  const double sub = Hc[j + 1];
  double* cs = c.cs + (size_t)slot * m;
  double* sn = c.sn + (size_t)slot * m;
  double* g = c.g + (size_t)slot * (m + 1);
  for (int i = 0; i < j; ++i) {
    const double t0 = cs[i] * Hc[i] + sn[i] * Hc[i + 1];
    Hc[i + 1] = -sn[i] * Hc[i] + cs[i] * Hc[i + 1];
    Hc[i] = t0;
  }
  const double rho = hypot(Hc[j], Hc[j + 1]);
  double cj = 1.0, sj = 0.0;
  if (rho > 0.0) {
    cj = Hc[j] / rho;
    sj = Hc[j + 1] / rho;
  }
  cs[j] = cj;
  sn[j] = sj;
  Hc[j] = rho;
  Hc[j + 1] = 0.0;
  g[j + 1] = -sj * g[j];
  g[j] = cj * g[j];
  c.nsteps[slot] = j + 1;
  c.itot[slot] += 1;
  return fabs(g[j + 1]) <= c.thr[slot] || j + 1 >= m || sub == 0.0 || c.itot[slot] >= c.max_iter;
}

// Norm of the new vector, Givens rotation of column j, residual estimate.
// One warp per slot, as k_finalize_h.
static __global__ void __launch_bounds__(KR_THREADS) k_givens(const KryArgs a, CycleState c, int j, int nslots) {
  const int slot = blockIdx.x * (KR_THREADS / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (slot >= nslots || !c.run[slot]) return;
  double s = 0.0;
  for (int q = lane; q < a.nchunk; q += 32) s += a.part2[(size_t)slot * a.nchunk + q];
  s = warp_sum(s, 32);
  if (lane != 0) return;
  const int m = c.m;
  const double nrm = sqrt(s);
  double* Hc = c.H + ((size_t)slot * m + j) * (m + 1);
  Hc[j + 1] = nrm;
  c.sigma[(size_t)slot * (m + 1) + j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
  if (givens_column(c, slot, j, Hc)) c.run[slot] = 0;
}

// y = R^{-1} g (back substitution), ycoef_i = y_i sigma_i.
static __global__ void k_solve_y(CycleState c, int nslots) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= nslots) return;
  const int ns = c.active[slot] ? c.nsteps[slot] : 0;
  const int m = c.m;
  double* y = c.ycoef + (size_t)slot * (m + 1);
  const double* g = c.g + (size_t)slot * (m + 1);
  for (int i = ns - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < ns; ++l) s -= c.H[((size_t)slot * m + l) * (m + 1) + i] * y[l];
    const double d = c.H[((size_t)slot * m + i) * (m + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
  for (int i = 0; i < ns; ++i) y[i] *= c.sigma[(size_t)slot * (m + 1) + i];
  c.nsteps[slot] = ns;
}

// x += sum_i ycoef_i v~_i   (basis in T; x stored as XS: FP64, or double-float
// pairs for the mixed path's double-float residual).  The correction is
// accumulated in T (it carries the precision of the basis) and added to x once.
__device__ __forceinline__ cx<double> xadd(cx<double> x, cx<double> d) { return x + d; }
__device__ __forceinline__ cx<double> xadd(cx<double> x, cx<float> d) { return x + ccast<double>(d); }
__device__ __forceinline__ cx<dd> xadd(cx<dd> x, cx<float> d) { return mkc(x.re + dd(d.re), x.im + dd(d.im)); }
template <typename T, typename XS>
__global__ void __launch_bounds__(KR_THREADS) k_xupdate(long long n, int mp1, const int* __restrict__ nsteps,
                                                         const double* __restrict__ ycoef,
                                                         const cx<T>* __restrict__ V, long long vss,
                                                         cx<XS>* __restrict__ X, long long xss) {
  const int slot = blockIdx.y;
  const int ns = nsteps[slot];
  if (ns == 0) return;
  const long long base = (long long)blockIdx.x * KR_CHUNK + threadIdx.x;
  const cx<T>* Vs = V + (size_t)slot * vss;
  cx<T> acc[KR_EPT];
#pragma unroll
  for (int e = 0; e < KR_EPT; ++e) acc[e] = mkc((T)0, (T)0);
  for (int i = 0; i < ns; ++i) {
    const T cf = (T)ycoef[(size_t)slot * mp1 + i];
#pragma unroll
    for (int e = 0; e < KR_EPT; ++e) {
      const long long idx = base + (long long)e * KR_THREADS;
      if (idx < n) {
        const cx<T> vi = ldg(Vs + (size_t)i * n + idx);
        acc[e] = mkc(acc[e].re + cf * vi.re, acc[e].im + cf * vi.im);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < KR_EPT; ++e) {
    const long long idx = base + (long long)e * KR_THREADS;
    if (idx < n) {
      cx<XS>* xp = X + (size_t)slot * xss + idx;
      *xp = xadd(*xp, acc[e]);
    }
  }
}

// FP64 copy of double-float fields (solution read-out)
// Start of a cycle from a squared-norm partial sum over nblk blocks:
// beta = ||r||, sigma_0 = 1/beta, g = beta e_1, stop threshold, flags.
// first != 0: the vector is b itself (records ||b||).  mask (nullable): only the
// slots with mask[slot] != 0 (slots being started while others run).
// first = 1: a new solve from x = 0 (part holds |b|^2: sets ||b|| and the
// counters); 0: the next cycle of a running solve; 2: a new solve from a given
// x (after a first = 1 launch on b; part holds |b - A x|^2: the counters stay
// as that launch set them).
static __global__ void __launch_bounds__(KR_THREADS) k_cycle_start(CycleState c, const double* part, int nblk,
                                                             int first, const int* mask) {
  __shared__ double sh[KR_THREADS / 32];
  const int slot = blockIdx.x;
  if (mask && !mask[slot]) return;
  if (first != 1 && !c.active[slot]) return;
  double s = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) s += part[(size_t)slot * nblk + q];
  s = block_sum_256(s, sh);
  if (threadIdx.x != 0) return;
  const int m = c.m;
  const double beta = sqrt(s);
  if (first == 1) {
    c.bnorm[slot] = beta;
    c.nscale[slot] = beta > 0.0 ? (float)exp2(-(double)ilogb(beta)) : 1.f;
    c.itot[slot] = 0;
    c.ncyc[slot] = 0;
  }
  const double bn = c.bnorm[slot];
  const double rel = bn > 0.0 ? beta / bn : 0.0;
  c.resid[slot] = rel;
  const int act = (bn > 0.0) && (rel > c.tol) && (c.itot[slot] < c.max_iter) && (c.ncyc[slot] < c.max_outer);
  c.active[slot] = act;
  c.run[slot] = act;
  c.nsteps[slot] = 0;
  c.sigma[(size_t)slot * (m + 1)] = beta > 0.0 ? 1.0 / beta : 0.0;
  double* g = c.g + (size_t)slot * (m + 1);
  g[0] = beta;
  for (int i = 1; i <= m; ++i) g[i] = 0.0;
  double thr = 0.5 * c.tol * bn;
  if (c.inner_tol > 0.0) thr = fmax(thr, c.inner_tol * beta);
  c.thr[slot] = thr;
  if (act && first != 2) c.ncyc[slot] += 1;
  if (first == 2 && !act) c.ncyc[slot] = 0;  // x already meets tol: no cycle runs
}

// ---------------------------------------------------------------------------
// s-step (block) Arnoldi.  The Krylov space and the GMRES minimisation are the
// ones of the step-by-step process above; only the order of the work changes,
// so that each sweep over the stored basis serves S new directions instead of
// one (the basis sweeps are HBM-bound).  From the last basis vector
// v_{J-1} a block forms the monomial chain in K = A - I,
//     p_0 = v_{J-1},  p_{i+1} = K p_i   (i < S, stored raw in basis slots J+i),
// so A p_i = p_i + p_{i+1}.  One sweep then yields C = V^T p (J x S) and the
// Gram matrix p^T p (S x S); a per-slot FP64 step normalises the chain
// (p^_i = p_i / ||p_i||), forms G = p^T p - C^T C, its Cholesky factor R (the
// block's orthonormalisation, CholQR), and from A P^ = P^ B (B unit lower
// bidiagonal up to the normalisation) the S new columns of the Hessenberg
// matrix,  H_new = (T B - [H_prev Z; 0]) U^{-1},  where T holds the chain's
// coordinates in the new orthonormal basis, U its part on v_{J-1}..v_{J+S-2}
// and Z its part on v_0..v_{J-2}.  A second sweep writes the new basis vectors
// Q = (P^ - V C) R^{-1} over the chain.  A pivot of G below kBlockPivot ends
// the cycle after the columns it still supports (the outer refinement
// continues from the true residual).
// ---------------------------------------------------------------------------
// Warp reduce-scatter of S = 2 or 4 per-lane values: every lane returns the
// warp total of value lane / (32 / S).  Each halving step exchanges only the
// half of the values the partner keeps, so S values cost S - 1 + 5 - log2(S)
// shuffles instead of 5 S (fixed order: the result does not depend on timing).
template <int S, typename T>
__device__ __forceinline__ T warp_reduce_scatter(const T (&s)[S], int lane) {
  static_assert(S == 2 || S == 4, "S must be 2 or 4");
  const unsigned full = 0xffffffffu;
  T k;
  if constexpr (S == 4) {
    const bool h = lane & 16;
    T k0 = h ? s[2] : s[0], k1 = h ? s[3] : s[1];
    k0 += __shfl_xor_sync(full, h ? s[0] : s[2], 16);
    k1 += __shfl_xor_sync(full, h ? s[1] : s[3], 16);
    const bool g = lane & 8;
    k = g ? k1 : k0;
    k += __shfl_xor_sync(full, g ? k0 : k1, 8);
  } else {
    const bool h = lane & 16;
    k = h ? s[1] : s[0];
    k += __shfl_xor_sync(full, h ? s[0] : s[1], 16);
    k += __shfl_xor_sync(full, k, 8);
  }
  k += __shfl_xor_sync(full, k, 4);
  k += __shfl_xor_sync(full, k, 2);
  k += __shfl_xor_sync(full, k, 1);
  return k;
}

// part[slot][r*S+i][chunk] = <v~_r, p_{i+1}> (r < J); then <p_i, p_l>, i <= l.
template <typename T, int S>
__global__ void __launch_bounds__(KR_THREADS) k_bdots(const BlockArgs a, const cx<T>* __restrict__ V, long long vss,
                                                       int J) {
  // [KR_THREADS / 32][nit] warp totals in T (FP32 for the inner solve: no FP64 per warp)
  extern __shared__ __align__(16) unsigned char bd_smem[];
  T* redf = reinterpret_cast<T*>(bd_smem);
  const int slot = blockIdx.y;
  if (!a.run[slot]) return;
  const int nit = block_items(J, S);
  const cx<T>* Vs = V + (size_t)slot * vss;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // each warp accumulates its own row of red over the block's chunks
  for (int q = threadIdx.x; q < (KR_THREADS / 32) * nit; q += blockDim.x) redf[q] = 0;
  __syncthreads();
  for (int ch = blockIdx.x; ch < a.nwork; ch += gridDim.x) {
    const long long base = (long long)ch * KB_CHUNK + threadIdx.x;
    cx<T> w[S][KB_EPT];
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int e = 0; e < KB_EPT; ++e) {
        const long long idx = base + (long long)e * KR_THREADS;
        w[i][e] = idx < a.n ? ldg(Vs + (size_t)(J + i) * a.n + idx) : mkc((T)0, (T)0);
      }
    for (int r = 0; r < J; ++r) {
      T s[S];
#pragma unroll
      for (int i = 0; i < S; ++i) s[i] = 0;
#pragma unroll
      for (int e = 0; e < KB_EPT; ++e) {
        const long long idx = base + (long long)e * KR_THREADS;
        if (idx < a.n) {
          const cx<T> v = ldg(Vs + (size_t)r * a.n + idx);
#pragma unroll
          for (int i = 0; i < S; ++i) s[i] += v.re * w[i][e].re + v.im * w[i][e].im;
        }
      }
      const T d = warp_reduce_scatter<S>(s, lane);
      if ((lane & (32 / S - 1)) == 0) redf[wid * nit + r * S + lane / (32 / S)] += d;
    }
    int it = J * S;
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int l = i; l < S; ++l) {
        T s = 0;
#pragma unroll
        for (int e = 0; e < KB_EPT; ++e) s += w[i][e].re * w[l][e].re + w[i][e].im * w[l][e].im;
        const T d = warp_sum_t(s, 32);
        if (lane == 0) redf[wid * nit + it] += d;
        ++it;
      }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nit; q += blockDim.x) {
    T s = 0;
    for (int w2 = 0; w2 < KR_THREADS / 32; ++w2) s += redf[w2 * nit + q];
    a.part[((size_t)slot * a.nitem + q) * a.nchunk + blockIdx.x] = (double)s;
  }
}

// Per-slot FP64 step of a block (one CTA per slot; thread 0 does the small
// dense algebra, warp 0 the row-parallel parts: on GB300 a warp's FP64
// instruction holds the narrow FP64 pipe for many cycles whatever its active
// lanes, so the element-wise loops run one element per lane).  Writes the block's Hessenberg columns J-1.. (unrotated into
// Hraw, rotated into c.H with the Givens steps), the sweep coefficients, the
// scales of the new vectors, and upd[slot] = 1 for every slot that ran the
// block (its new vectors need the update sweep even when it stops here).
template <int S>
static __global__ void __launch_bounds__(KR_THREADS) k_bscalar(BlockArgs a, CycleState c, double* __restrict__ Hraw,
                                                               double* __restrict__ bcoef, int* __restrict__ upd,
                                                               int J) {
  extern __shared__ double sm[];  // val[nit], X[(J + S) * S], R[S][S], Sg[S + 1]
  const int slot = blockIdx.x;
  if (!c.run[slot]) {
    if (threadIdx.x == 0) upd[slot] = 0;
    return;
  }
  const int nit = block_items(J, S);
  double* val = sm;
  double* X = sm + nit;
  double(*R)[S] = reinterpret_cast<double(*)[S]>(X + (J + S) * S);
  double* Sg = X + (J + S) * S + S * S;
  for (int q = threadIdx.x; q < nit; q += blockDim.x) {
    const double* p = a.part + ((size_t)slot * a.nitem + q) * a.nchunk;
    double s = 0.0;
    for (int ch = 0; ch < a.nchunk; ++ch) s += p[ch];
    val[q] = s;
  }
  __syncthreads();
  const int m = c.m, rows = J + S;
  double* sg = c.sigma + (size_t)slot * (m + 1);
  // chain norms Sg[i] = ||p_i|| (Sg[0] = 1: v_{J-1} has unit norm); the diagonal items
  // of p^T p follow the J S items of V^T p
  if (threadIdx.x <= S) {
    const int i = threadIdx.x - 1;
    Sg[threadIdx.x] = threadIdx.x == 0 ? 1.0 : sqrt(fmax(val[J * S + i * S - i * (i - 1) / 2], 0.0));
  }
  __syncthreads();
  double G[S][S];
  {
    int it = J * S;
    for (int i = 0; i < S; ++i)
      for (int l = i; l < S; ++l, ++it) G[i][l] = val[it];
  }
  __syncthreads();  // the items of p^T p are read before C^ overwrites the V^T p items
  // C^ = coordinates of p^_{i+1} on v_r (in place in val), one item per thread
  for (int q = threadIdx.x; q < J * S; q += blockDim.x) {
    const int r = q / S, i = q - r * S;
    const double d = Sg[i + 1];
    val[q] = d > 0.0 ? val[q] * sg[r] / d : 0.0;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double Ri[S][S];
  // G = p^T p (normalised) - C^T C, Cholesky G = R^T R (lane 0; R shared with the warp)
  int nok = S;
  if (lane == 0) {
  for (int i = 0; i < S; ++i)
    for (int l = 0; l < S; ++l) R[i][l] = 0.0;
  for (int i = 0; i < S && nok == S; ++i) {
    for (int l = i; l < S; ++l) {
      const double dd = Sg[i + 1] * Sg[l + 1];
      double gv = dd > 0.0 ? G[i][l] / dd : 0.0;
      for (int r = 0; r < J; ++r) gv -= val[r * S + i] * val[r * S + l];
      for (int q = 0; q < i; ++q) gv -= R[q][i] * R[q][l];
      if (l == i) {
        if (!(gv > kBlockPivot) || Sg[i + 1] == 0.0) {
          nok = i;
          break;
        }
        R[i][i] = sqrt(gv);
      } else {
        R[i][l] = gv / R[i][i];
      }
    }
  }
  }
  nok = __shfl_sync(0xffffffffu, nok, 0);
  __syncwarp();
  const int ncols = nok > 0 ? nok : 1;  // nok = 0: p_1 lies in span(V), a happy breakdown column
  // R^{-1} on the accepted columns (zero elsewhere)
  for (int i = 0; i < S; ++i)
    for (int l = 0; l < S; ++l) Ri[i][l] = 0.0;
  for (int i = 0; i < nok; ++i) {
    Ri[i][i] = 1.0 / R[i][i];
    for (int q = i - 1; q >= 0; --q) {
      double s = 0.0;
      for (int l = q + 1; l <= i; ++l) s += R[q][l] * Ri[l][i];
      Ri[q][i] = -s / R[q][q];
    }
  }
  // T[r][k]: coordinates of p^_k on v_0..v_{J+S-1}
  auto T = [&](int r, int k) -> double {
    if (k == 0) return r == J - 1 ? 1.0 : 0.0;
    if (r < J) return val[r * S + k - 1];
    const int q = r - J;
    return q <= k - 1 ? R[q][k - 1] : 0.0;
  };
  // H_new = (T B - [H_prev Z; 0]) U^{-1}, column by column, one row per lane
  for (int i = 0; i < ncols; ++i) {
    const double bsub = Sg[i + 1] / Sg[i];
    for (int r = lane; r < rows; r += 32) {
      double v = T(r, i) + T(r, i + 1) * bsub;
      if (r < J && i > 0)
        for (int q = (r > 0 ? r - 1 : 0); q < J - 1; ++q)
          v -= Hraw[((size_t)slot * m + q) * (m + 1) + r] * val[q * S + i - 1];
      for (int l = 0; l < i; ++l) v -= X[r * S + l] * T(J - 1 + l, i);
      const double uii = i == 0 ? 1.0 : R[i - 1][i - 1];
      X[r * S + i] = r <= J + i ? v / uii : 0.0;
    }
    __syncwarp();
  }
  // sweep coefficients: Q = P^ R^{-1} - V C^ R^{-1}, on the raw stored vectors (one item per lane)
  double* bc = bcoef + (size_t)slot * (S * S + (m + 1) * S);
  for (int q = lane; q < S * S; q += 32) {
    const int k = q / S, i = q - k * S;
    bc[q] = Sg[k + 1] > 0.0 ? Ri[k][i] / Sg[k + 1] : 0.0;
  }
  for (int q = lane; q < J * S; q += 32) {
    const int r = q / S, i = q - r * S;
    double s = 0.0;
    for (int k = 0; k <= i; ++k) s += val[r * S + k] * Ri[k][i];
    bc[S * S + q] = -s * sg[r];
  }
  __syncwarp();
  if (lane != 0) return;
  // columns J-1+i: unrotated copy, then the Givens steps
  bool stop = false;
  for (int i = 0; i < ncols && !stop; ++i) {
    const int j = J - 1 + i;
    double* Hr = Hraw + ((size_t)slot * m + j) * (m + 1);
    double* Hc = c.H + ((size_t)slot * m + j) * (m + 1);
    for (int r = 0; r <= j + 1; ++r) Hr[r] = Hc[r] = X[r * S + i];
    stop = givens_column(c, slot, j, Hc);
  }
  if (ncols < S || J - 1 + 2 * S > m) stop = true;
  for (int i = 0; i < S; ++i) sg[J + i] = 1.0;
  upd[slot] = 1;
  if (stop) {
    // last block of this slot's cycle: y = R^{-1} g on the rotated columns, and
    // ycoef_i = y_i sigma_i, so that the update sweep also adds V y to x
    const int ns = c.nsteps[slot];
    double* y = c.ycoef + (size_t)slot * (m + 1);
    const double* g = c.g + (size_t)slot * (m + 1);
    for (int i = ns - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < ns; ++l) s -= c.H[((size_t)slot * m + l) * (m + 1) + i] * y[l];
      const double d = c.H[((size_t)slot * m + i) * (m + 1) + i];
      y[i] = d != 0.0 ? s / d : 0.0;
    }
    for (int i = 0; i < ns; ++i) y[i] *= sg[i];
    for (int i = ns; i <= m; ++i) y[i] = 0.0;
    upd[slot] = 2;
    c.run[slot] = 0;
  }
}

// Q_i = sum_k bcoef_ki p_{k+1} + sum_r bcoef'_ri v~_r, written over the chain
// (basis slots J..J+S-1); slots with upd[slot] != 0 only.  upd[slot] == 2 (the
// slot's last block of the cycle): also x += sum_r ycoef_r v~_r + sum_i
// ycoef_{J+i} Q_i, accumulated in T and added to x once (no separate pass
// over the basis).
template <typename T, int S, bool XU>
__global__ void __launch_bounds__(KR_THREADS) k_bupdate(const BlockArgs a, const int* __restrict__ upd,
                                                         cx<T>* __restrict__ V, long long vss, int J) {
  __shared__ T cf[S * S + 129 * S];
  __shared__ T yc[129 + S];
  const int slot = blockIdx.y;
  // XU: the launch for slots in their last block (upd == 2); the other launch
  // (upd == 1) keeps the lean register budget of the plain sweep
  const int u = upd[slot];
  if (u != (XU ? 2 : 1)) return;
  const double* bc = a.bcoef + (size_t)slot * (S * S + a.mp1 * S);
  for (int q = threadIdx.x; q < S * S + J * S; q += blockDim.x) cf[q] = (T)bc[q];
  if (XU)
    for (int q = threadIdx.x; q < J + S; q += blockDim.x) yc[q] = (T)a.ycoef[(size_t)slot * a.mp1 + q];
  __syncthreads();
  const long long base = (long long)blockIdx.x * KB_CHUNK + threadIdx.x;
  cx<T>* Vs = V + (size_t)slot * vss;
  cx<T> acc[S][KB_EPT];
  {
    cx<T> w[S][KB_EPT];
#pragma unroll
    for (int k = 0; k < S; ++k)
#pragma unroll
      for (int e = 0; e < KB_EPT; ++e) {
        const long long idx = base + (long long)e * KR_THREADS;
        w[k][e] = idx < a.n ? ldg(Vs + (size_t)(J + k) * a.n + idx) : mkc((T)0, (T)0);
      }
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int e = 0; e < KB_EPT; ++e) {
        cx<T> s = mkc((T)0, (T)0);
#pragma unroll
        for (int k = 0; k <= i; ++k) s = mkc(s.re + cf[k * S + i] * w[k][e].re, s.im + cf[k * S + i] * w[k][e].im);
        acc[i][e] = s;
      }
  }
  cx<T> dx[KB_EPT];
#pragma unroll
  for (int e = 0; e < KB_EPT; ++e) dx[e] = mkc((T)0, (T)0);
  for (int r = 0; r < J; ++r) {
    const T yr = XU ? yc[r] : (T)0;
#pragma unroll
    for (int e = 0; e < KB_EPT; ++e) {
      const long long idx = base + (long long)e * KR_THREADS;
      if (idx < a.n) {
        const cx<T> v = ldg(Vs + (size_t)r * a.n + idx);
#pragma unroll
        for (int i = 0; i < S; ++i) {
          const T c = cf[S * S + r * S + i];
          acc[i][e] = mkc(acc[i][e].re + c * v.re, acc[i][e].im + c * v.im);
        }
        if (XU) dx[e] = mkc(dx[e].re + yr * v.re, dx[e].im + yr * v.im);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int e = 0; e < KB_EPT; ++e) {
      const long long idx = base + (long long)e * KR_THREADS;
      if (idx < a.n) Vs[(size_t)(J + i) * a.n + idx] = acc[i][e];
    }
  if (XU) {
#pragma unroll
    for (int e = 0; e < KB_EPT; ++e) {
      const long long idx = base + (long long)e * KR_THREADS;
      if (idx >= a.n) continue;
      cx<T> d = dx[e];
#pragma unroll
      for (int i = 0; i < S; ++i) d = mkc(d.re + yc[J + i] * acc[i][e].re, d.im + yc[J + i] * acc[i][e].im);
      if constexpr (std::is_same<T, float>::value) {
        if (a.x_dd) {
          cx<dd>* xp = reinterpret_cast<cx<dd>*>(a.X) + (size_t)slot * a.xss + idx;
          *xp = xadd(*xp, d);
          continue;
        }
      }
      cx<double>* xp = reinterpret_cast<cx<double>*>(a.X) + (size_t)slot * a.xss + idx;
      *xp = xadd(*xp, d);
    }
  }
}


// ---------------------------------------------------------------------------
// Block update with the basis streamed through shared memory by bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier):
// KB_STAGES chunks of basis vectors are in flight per CTA while the threads
// work on an earlier one, so a CTA keeps ~KB_STAGES x 8 KB of reads
// outstanding with no registers held for them.  Same arithmetic, order and
// results as k_bupdate.  Every wait is bounded: when one runs out the CTA
// sets *a.err, stops computing, drains its own copies (bounded) and returns.
// Needs n to be a multiple of KB_CHUNK (chunks of whole 16-byte units).
// ---------------------------------------------------------------------------
// stages per CTA: 32 KB of shared memory for either element size
template <typename T>
struct KBStages {
  static constexpr int value = sizeof(cx<T>) == 8 ? 4 : 2;
};
constexpr int kWaitLimit = 1 << 18;  // try_wait rounds before a wait is declared lost (~1 s on GB300)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also announces the bytes the next copy will deliver
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// true once the barrier's phase with the given parity has completed; false after kWaitLimit rounds
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  for (int i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename T, int S, bool XU>
__global__ void __launch_bounds__(KR_THREADS) k_bupdate_bulk(const BlockArgs a, const int* __restrict__ upd,
                                                              cx<T>* __restrict__ V, long long vss, int J) {
  constexpr int KB_STAGES = KBStages<T>::value;
  extern __shared__ __align__(128) unsigned char kb_stage_raw[];
  cx<T>* stage = reinterpret_cast<cx<T>*>(kb_stage_raw);  // [KB_STAGES][KB_CHUNK]
  __shared__ __align__(8) uint64_t bar[KB_STAGES];
  __shared__ T cf[S * S + 129 * S];
  __shared__ T yc[129 + S];
  __shared__ int lost;
  const int slot = blockIdx.y;
  const int u = upd[slot];
  if (u != (XU ? 2 : 1)) return;
  constexpr uint32_t kBytes = KB_CHUNK * sizeof(cx<T>);
  cx<T>* Vs = V + (size_t)slot * vss;
  const long long c0 = (long long)blockIdx.x * KB_CHUNK;  // this CTA's chunk: elements c0 .. c0 + KB_CHUNK - 1
  if (threadIdx.x == 0) {
    lost = 0;
    for (int s = 0; s < KB_STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
    // the first KB_STAGES basis vectors of the sweep
    for (int r = 0; r < KB_STAGES && r < J; ++r) {
      // (a.tx_extra > 0 only under the test hook: that stage's phase cannot complete)
      mbar_expect_tx(&bar[r], kBytes + (r == 0 ? (uint32_t)a.tx_extra : 0u));
      bulk_g2s(stage + (size_t)r * KB_CHUNK, Vs + (size_t)r * a.n + c0, kBytes, &bar[r]);
    }
  }
  const double* bc = a.bcoef + (size_t)slot * (S * S + a.mp1 * S);
  for (int q = threadIdx.x; q < S * S + J * S; q += blockDim.x) cf[q] = (T)bc[q];
  if (XU)
    for (int q = threadIdx.x; q < J + S; q += blockDim.x) yc[q] = (T)a.ycoef[(size_t)slot * a.mp1 + q];
  __syncthreads();
  cx<T> acc[S][KB_EPT];
  {
    cx<T> w[S][KB_EPT];
#pragma unroll
    for (int k = 0; k < S; ++k)
#pragma unroll
      for (int e = 0; e < KB_EPT; ++e) w[k][e] = ldg(Vs + (size_t)(J + k) * a.n + c0 + threadIdx.x + e * KR_THREADS);
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int e = 0; e < KB_EPT; ++e) {
        cx<T> s = mkc((T)0, (T)0);
#pragma unroll
        for (int k = 0; k <= i; ++k) s = mkc(s.re + cf[k * S + i] * w[k][e].re, s.im + cf[k * S + i] * w[k][e].im);
        acc[i][e] = s;
      }
  }
  cx<T> dx[KB_EPT];
#pragma unroll
  for (int e = 0; e < KB_EPT; ++e) dx[e] = mkc((T)0, (T)0);
  int r = 0;
  for (; r < J; ++r) {
    const int st = r % KB_STAGES;
    if (!mbar_wait(&bar[st], (uint32_t)((r / KB_STAGES) & 1))) lost = 1;
    __syncthreads();  // every thread has waited (and sees `lost`)
    if (lost) break;
    const T yr = XU ? yc[r] : (T)0;
    const cx<T>* src = stage + (size_t)st * KB_CHUNK + threadIdx.x;
#pragma unroll
    for (int e = 0; e < KB_EPT; ++e) {
      const cx<T> v = src[e * KR_THREADS];
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const T c = cf[S * S + r * S + i];
        acc[i][e] = mkc(acc[i][e].re + c * v.re, acc[i][e].im + c * v.im);
      }
      if (XU) dx[e] = mkc(dx[e].re + yr * v.re, dx[e].im + yr * v.im);
    }
    __syncthreads();  // stage st has been read by every thread: refill it
    if (threadIdx.x == 0 && r + KB_STAGES < J) {
      mbar_expect_tx(&bar[st], kBytes);
      bulk_g2s(stage + (size_t)st * KB_CHUNK, Vs + (size_t)(r + KB_STAGES) * a.n + c0, kBytes, &bar[st]);
    }
  }
  if (r < J) {
    // a wait ran out: report it, drain this CTA's copies still in flight (bounded), return
    if (threadIdx.x == 0) {
      if (a.err) atomicExch(a.err, 1);
      const int issued = J < r + KB_STAGES ? J : r + KB_STAGES;
      for (int q = r; q < issued; ++q) mbar_wait(&bar[q % KB_STAGES], (uint32_t)((q / KB_STAGES) & 1));
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int e = 0; e < KB_EPT; ++e) Vs[(size_t)(J + i) * a.n + c0 + threadIdx.x + e * KR_THREADS] = acc[i][e];
  if (XU) {
#pragma unroll
    for (int e = 0; e < KB_EPT; ++e) {
      const long long idx = c0 + threadIdx.x + e * KR_THREADS;
      cx<T> d = dx[e];
#pragma unroll
      for (int i = 0; i < S; ++i) d = mkc(d.re + yc[J + i] * acc[i][e].re, d.im + yc[J + i] * acc[i][e].im);
      if constexpr (std::is_same<T, float>::value) {
        if (a.x_dd) {
          cx<dd>* xp = reinterpret_cast<cx<dd>*>(a.X) + (size_t)slot * a.xss + idx;
          *xp = xadd(*xp, d);
          continue;
        }
      }
      cx<double>* xp = reinterpret_cast<cx<double>*>(a.X) + (size_t)slot * a.xss + idx;
      *xp = xadd(*xp, d);
    }
  }
}

}  // namespace dbar
