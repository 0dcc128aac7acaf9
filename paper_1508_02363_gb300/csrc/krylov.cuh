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
static __global__ void __launch_bounds__(KR_THREADS) k_finalize_h(const KryArgs a, double* H, int j) {
  __shared__ double sh[KR_THREADS / 32];
  const int slot = blockIdx.x;
  if (!a.run[slot]) return;
  for (int i = 0; i <= j; ++i) {
    double s = 0.0;
    const double* p = a.part + ((size_t)slot * a.mp1 + i) * a.nchunk;
    for (int c = threadIdx.x; c < a.nchunk; c += blockDim.x) s += p[c];
    s = block_sum_256(s, sh);
    if (threadIdx.x == 0) {
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


// Norm of the new vector, Givens rotation of column j, residual estimate.
static __global__ void __launch_bounds__(KR_THREADS) k_givens(const KryArgs a, CycleState c, int j) {
  __shared__ double sh[KR_THREADS / 32];
  const int slot = blockIdx.x;
  if (!c.run[slot]) return;
  double s = 0.0;
  for (int q = threadIdx.x; q < a.nchunk; q += blockDim.x) s += a.part2[(size_t)slot * a.nchunk + q];
  s = block_sum_256(s, sh);
  if (threadIdx.x != 0) return;
  const int m = c.m;
  const double nrm = sqrt(s);
  double* Hc = c.H + ((size_t)slot * m + j) * (m + 1);
  Hc[j + 1] = nrm;
  c.sigma[(size_t)slot * (m + 1) + j + 1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
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
  if (fabs(g[j + 1]) <= c.thr[slot] || j + 1 >= m || nrm == 0.0 || c.itot[slot] >= c.max_iter)
    c.run[slot] = 0;
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

// x += sum_i ycoef_i v~_i   (x in FP64, basis in T).  The correction is
// accumulated in T (it carries the precision of the basis) and added to x once.
template <typename T>
__global__ void __launch_bounds__(KR_THREADS) k_xupdate(long long n, int mp1, const int* __restrict__ nsteps,
                                                         const double* __restrict__ ycoef,
                                                         const cx<T>* __restrict__ V, long long vss,
                                                         cx<double>* __restrict__ X, long long xss) {
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
      cx<double>* xp = X + (size_t)slot * xss + idx;
      *xp = *xp + ccast<double>(acc[e]);
    }
  }
}

// Start of a cycle from a squared-norm partial sum over nblk blocks:
// beta = ||r||, sigma_0 = 1/beta, g = beta e_1, stop threshold, flags.
// first != 0: the vector is b itself (records ||b||).  mask (nullable): only the
// slots with mask[slot] != 0 (slots being started while others run).
static __global__ void __launch_bounds__(KR_THREADS) k_cycle_start(CycleState c, const double* part, int nblk,
                                                             int first, const int* mask) {
  __shared__ double sh[KR_THREADS / 32];
  const int slot = blockIdx.x;
  if (mask && !mask[slot]) return;
  if (!first && !c.active[slot]) return;
  double s = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) s += part[(size_t)slot * nblk + q];
  s = block_sum_256(s, sh);
  if (threadIdx.x != 0) return;
  const int m = c.m;
  const double beta = sqrt(s);
  if (first) {
    c.bnorm[slot] = beta;
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
  if (act) c.ncyc[slot] += 1;
}

}  // namespace dbar
