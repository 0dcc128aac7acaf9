// The three memory passes of one application of the operator
//     A S = S + i F(E_k Q conj(h)),   h = F^{-1}(S/xi)  regularised   (Sec. 4.3)
// and the right-hand side b = -i F(E_k Q).
//
// The paper applies A with three 2-D FFTs (Sec. 4.3 remark): one inverse FFT
// for the Taylor coefficients c_n, one inverse FFT of (S-G)/xi and one forward
// FFT.  Here the same discrete operator is evaluated with two 2-D FFTs:
//
//  * Taylor data.  n! c_n = (-i/2)^n F_d(z^n F_d^{-1} S)(0) is a linear
//    functional of S.  Expanding z^n = sum_a C(n,a) x^a (iy)^{n-a} gives
//        c_n = (1/n!)(-i/2)^n N^{-2} sum_p (-1)^{p1+p2} S_p Z_n(p),
//        Z_n(p) = sum_a C(n,a) i^{n-a} D_a(p1) D_{n-a}(p2),
//        D_a(p) = sum_j x_j^a e^{2 pi i p j/N},
//    and the fill value d = (-i/2) N^{-2} sum_p (-1)^{p1+p2} S_p
//    (D_1(p1) D_0(p2) - i D_0(p1) D_1(p2)).  Pass A forms the row moments
//    R_a(p2) = sum_{p1} (-1)^{p1} S_p D_a(p1) while it reads S anyway.
//  * Singular part.  With S~ = S/xi (0 at xi = 0) and the fixed fields
//    V_n = F_d^{-1}(e^{-|xi|^2} conj(xi)^n / xi, 0 at xi = 0), linearity gives
//        h = F_d^{-1}((S - G)/xi | d at 0) + sum c_n W_n
//          = F_d^{-1}(S~) + sum_n c_n (W_n - V_n) + d/(2 pi L^2),
//    so G never has to be formed per point; Delta_n = W_n - V_n is built once
//    per plan (eq. fourreg5 for W_n).
//
// Pass A (rows):    read S row, moments, S~ (-1)^p /(2 pi L^2), row IDFT -> T1.
// Pass B (columns): column IDFT -> u; h = u + sum c_n Delta_n + d'; w =
//                   (2 pi L^2/N^2) E_k Q conj(h); column DFT -> T2.
// Pass C (rows):    row DFT; K S = i (-1)^p DFT(w) (= A S - S), or the
//                   right-hand side / residual epilogues.
#pragma once
#include "types.cuh"

namespace dbar {

__device__ __forceinline__ int wavenum(int p, int N) { return p <= (N >> 1) ? p : p - N; }

// From the summed row contributions to the coefficients:
//   n <= M:  c_n = (1/n!) (-i/2)^n N^-2 sum      (eq. fourreeg4, Sec. 4.3 step 4a)
//   n = M+1: d   = (-i/2) N^-2 sum * fillmul     (fill value dS/dxi(0), scaled)
__device__ __forceinline__ cx<double> taylor_coef(cx<double> s, int n, int M, int N, double fillmul) {
  const double invN2 = 1.0 / ((double)N * (double)N);
  s = mkc(s.re * invN2, s.im * invN2);
  if (n <= M) {
    for (int r = 0; r < n; ++r) s = cscale(mkc(s.im, -s.re), 0.5 / (double)(r + 1));
  } else {
    s = cscale(mkc(s.im, -s.re), 0.5 * fillmul);
  }
  return s;
}

// 1/(2 pi L (m1^2 + m2^2)) from c = 1/(2 pi L) already in T: exact division in
// FP64 and double-float; the fast reciprocal (a few ulp) in the FP32 inner solve.
template <typename T>
__device__ __forceinline__ T kappa_scale(T c, T den) {
  return c / den;
}
template <>
__device__ __forceinline__ float kappa_scale<float>(float c, float den) {
  return __fdividef(c, den);
}
// double-float: den is an exact integer in float (m1^2 + m2^2 < 2^24); its
// reciprocal y = rn(1/den) is corrected by one Newton step with the exact FMA
// residual e = 1 - den y (1/den = y (1 + e + ...), ~2^-48 relative), then c * (1/den).
template <>
__device__ __forceinline__ dd kappa_scale<dd>(dd c, dd den) {
  const float y = __frcp_rn(den.hi);
  const float e = __fmaf_rn(-den.hi, y, 1.0f);
  return c * dd_quick_two_sum(y, __fmul_rn(y, e));
}

// RV: row shape (row_lines_v); the blocks an SM keeps scale with 1/LINES so that the
// register budget per thread is the same for shapes 0-2; shapes 3 and 4 keep 3/4 as
// many threads per SM, which allows ~85 registers per thread instead of 64.
template <typename T, int LOGN, int RV = 0>
struct RowG {
  static constexpr int N = 1 << LOGN, TPL = N / 16, LINES = row_lines_v(LOGN, RV), THREADS = LINES * TPL;
  static constexpr int P = pitch_of(N);
#ifndef DBAR_ROW_MINB_F32
#define DBAR_ROW_MINB_F32 4
#endif
  static constexpr int MINB0 = sizeof(T) == 4 ? DBAR_ROW_MINB_F32 : 2;
  static constexpr int MINB1 = (RV >= 3 ? MINB0 * 3 / 4 : MINB0) > 0 ? (RV >= 3 ? MINB0 * 3 / 4 : MINB0) : 1;
  static constexpr int MINB = MINB1 * row_lines(LOGN) / LINES > 0 ? MINB1 * row_lines(LOGN) / LINES : 1;
};
template <typename T, int LOGN, int CV = 0>
struct ColG {
  static constexpr int N = 1 << LOGN, TPL = N / 16;
  static constexpr int CW = col_cw(LOGN, (int)sizeof(cx<T>), CV), TW = 32 / CW;
  static constexpr int COLS = col_cols(LOGN, (int)sizeof(cx<T>), CV), THREADS = COLS * TPL;
  static constexpr int WPG = TPL / TW;  // warps per group of CW columns
  static constexpr int P = pitch_of(N);
  static constexpr int MINB = 2;
};

// ---------------------------------------------------------------------------
// Pass A: rows of a Fourier field.  row_a() is the work on one row once its
// 16 values per thread are in registers (v[q] = S[p2][t + q TPL]): the
// Taylor row moments, S~ (-1)^p / (2 pi L^2), the row IDFT and the store to
// dst (this thread's first element of the row).  Used by k_pass_a and by the
// fused row pass k_pass_ca.
// ---------------------------------------------------------------------------
template <typename T, int LOGN, bool SH = false, bool MOM = true>
__device__ __forceinline__ void row_a(const PassArgs<T>& a, cx<T> (&v)[16], int slot, int p2, int t, cx<T>* sl,
                                      cx<T>* dst) {
  using G = RowG<T, LOGN>;
  constexpr int N = G::N, TPL = G::TPL;
  constexpr int SEGW = TPL >= 32 ? 32 : TPL, NSEG = TPL >= 32 ? TPL / 32 : 1;
  const int M = a.M, MA = M > 1 ? M : 1;
  // Row moments R_a(p2) = sum_p1 (-1)^p1 S D_a(p1), a = 0..MA, written as
  // per-warp-segment partials for k_coef, which combines them with D_b(p2)
  // in FP64: no block-wide tail here.  The FP32 pass writes FP32 partials (on
  // GB300 every FP64 conversion issued per warp occupies the small FP64 pipe
  // for tens of cycles).
  using PT = typename std::conditional<std::is_same<T, float>::value, float, double>::type;
  const int seg = TPL >= 32 ? t / 32 : 0;
  cx<PT>* part = reinterpret_cast<cx<PT>*>(a.partA) + ((size_t)slot * N + p2) * NSEG * (MA + 1);
  // a = 0: D_0(p) = N delta_{p,0}, so R_0 = N S(p1 = 0), held by the thread with t = 0
  if (t == 0) {
    const cx<T> s0 = v[0];
    part[0] = mkc((PT)s0.re * N, (PT)s0.im * N);
  }
  // (MOM false: the a >= 1 partials were written from the row's column-pass output, ca_moments)
  for (int aa = 1; MOM && aa <= MA; ++aa) {
    cx<T> acc = mkc((T)0, (T)0);
    const cx<T>* D = a.Da + (size_t)aa * N + t;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const cx<T> d = ldg(D + q * TPL);
      cx<T> s = v[q];
      if ((t + q * TPL) & 1) s = mkc(-s.re, -s.im);
      acc = acc + cmul(s, d);
    }
    // within a warp segment in T (16 x SEGW terms); segments are summed in k_coef
    const T re = warp_sum_t(acc.re, SEGW), im = warp_sum_t(acc.im, SEGW);
    if ((t & (SEGW - 1)) == 0) part[seg * (MA + 1) + aa] = mkc((PT)re, (PT)im);
  }

  // S~ (-1)^{p1+p2} / (2 pi L^2) with S~ = S/xi, xi = (m1 + i m2)/L, 0 at xi = 0.
  // The wavenumbers are formed in T from per-thread values (exact: |m| <= N/2,
  // m1^2 + m2^2 < 2^24), avoiding per-element int->float conversions, which
  // share GB300's small FP64/conversion pipe.
  T c2piL;
  if constexpr (std::is_same<T, float>::value) c2piL = a.inv2piL_f;
  else c2piL = (T)a.inv2piL;
  const T tf = (T)t;
  // Shifted quotient (iterated equation): the field was rolled by s, so element p holds the
  // value at p + s and its divisor is the unwrapped wavenumber m(p + s) - s, i.e. the
  // representative of p in [-N/2 + 1 - s, N/2 - s] (eq. dbarinvShift: no periodic wrap of
  // xi - xi0).  Exact in T: |m| <= N.
  auto scale_row = [&](int s1, int s2) {
    int m2 = wavenum(p2, N);
    if (m2 > (N >> 1) - s2) m2 -= N;
    else if (m2 < -(N >> 1) + 1 - s2) m2 += N;
    const T m2f = (T)m2;
    const T m2sq = m2f * m2f;
    const int hi1 = (N >> 1) - s1, lo1 = -(N >> 1) + 1 - s1;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p1 = t + q * TPL;
      const int m1 = wavenum(p1, N);
      T m1f = tf + (T)(q * TPL);
      if (p1 > (N >> 1)) m1f = m1f - (T)N;
      if (m1 > hi1) m1f = m1f - (T)N;
      else if (m1 < lo1) m1f = m1f + (T)N;
      const T den = m1f * m1f + m2sq;
      T f = (p1 == 0 && p2 == 0) ? (T)0 : kappa_scale<T>(c2piL, den);
      if ((p1 + p2) & 1) f = -f;
      v[q] = cmul(v[q], mkc(m1f * f, -(m2f * f)));
    }
  };
  if constexpr (SH) {
    scale_row(a.dshift[2 * slot], a.dshift[2 * slot + 1]);
  } else {
    const T m2f = (T)wavenum(p2, N);
    const T m2sq = m2f * m2f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p1 = t + q * TPL;
      T m1f = tf + (T)(q * TPL);
      if (p1 > (N >> 1)) m1f = m1f - (T)N;
      const T den = m1f * m1f + m2sq;
      T f = (p1 == 0 && p2 == 0) ? (T)0 : kappa_scale<T>(c2piL, den);
      if ((p1 + p2) & 1) f = -f;
      v[q] = cmul(v[q], mkc(m1f * f, -(m2f * f)));
    }
  }
  fft_line<T, LOGN, true, std::is_same<T, float>::value>(v, sl, t, a.tw);
  // only the columns the column pass reads (those where Q is not zero); the test is
  // skipped (a grid-uniform branch) when every column is read
  if (a.sx0 > 0 || a.sx1 < N) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = t + q * TPL;
      if (x >= a.sx0 && x < a.sx1) dst[q * TPL] = v[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) dst[q * TPL] = v[q];
  }
}

// SH: the shifted quotient of the iterated equation (a.dshift set)
template <typename T, int LOGN, bool SH, int RV = 0>
__global__ void __launch_bounds__(RowG<T, LOGN, RV>::THREADS, RowG<T, LOGN, RV>::MINB) k_pass_a(const PassArgs<T> a) {
  using G = RowG<T, LOGN, RV>;
  constexpr int N = G::N, TPL = G::TPL, LINES = G::LINES, P = G::P;
  extern __shared__ __align__(16) unsigned char smem[];
  const int slot = blockIdx.y;
  if (a.run && !a.run[slot]) return;
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  const int p2 = blockIdx.x * LINES + line;
  cx<T>* sl = reinterpret_cast<cx<T>*>(smem) + line * P;
  const T sc = a.in_scale ? (T)a.in_scale[(size_t)slot * a.in_scale_ss] : (T)1;
  cx<T> v[16];
  const cx<T>* src = a.in + (size_t)slot * a.in_ss + (size_t)p2 * N + t;
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = cscale(ldg(src + q * TPL), sc);
  row_a<T, LOGN, SH>(a, v, slot, p2, t, sl,
                     reinterpret_cast<cx<T>*>(a.out) + (size_t)slot * a.out_ss + (size_t)p2 * N + t);
}

// ---------------------------------------------------------------------------
// Row moments of the next chain vector S' = K p from the column-pass output T2
// of p, before the row DFT.  With S'(p1,p2) = i (-1)^{p1+p2} sum_x T2(x,p2)
// e^{-2 pi i p1 x/N} and D_a(p1) = sum_j x_j^a e^{+2 pi i p1 j/N}, the sum over
// p1 collapses (sum_p1 e^{2 pi i p1 (j - x)/N} = N delta_jx):
//     R_a(p2) = sum_p1 (-1)^p1 S'(p1,p2) D_a(p1) = i N (-1)^{p2} sum_x x_x^a T2(x,p2),
// a real-weighted sum with x_j = (2 pi L/N)(j - N/2) formed in registers: no
// table loads (the fused row pass is bound by its L1/shared-memory traffic).
// Written as row_a's per-warp-segment partials, a = 1..MA; row_a still writes
// the a = 0 moment.  FP32 only.
// ---------------------------------------------------------------------------
template <int LOGN>
__device__ __forceinline__ void ca_moments(const PassArgs<float>& a, const cx<float> (&v)[16], int slot, int p2,
                                           int t) {
  using G = RowG<float, LOGN>;
  constexpr int N = G::N, TPL = G::TPL;
  constexpr int SEGW = TPL >= 32 ? 32 : TPL, NSEG = TPL >= 32 ? TPL / 32 : 1;
  const int M = a.M, MA = M > 1 ? M : 1;
  const int seg = TPL >= 32 ? t / 32 : 0;
  cx<float>* part = reinterpret_cast<cx<float>*>(a.partA) + ((size_t)slot * N + p2) * NSEG * (MA + 1);
  const float tm = (float)(t - N / 2), hx = a.hx_f;
  const float sN = (p2 & 1) ? -(float)N : (float)N;  // N (-1)^{p2}
  float pw[16];  // x^a of this thread's columns
#pragma unroll
  for (int q = 0; q < 16; ++q) pw[q] = 1.f;
  for (int aa = 1; aa <= MA; ++aa) {
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      pw[q] *= hx * (tm + (float)(q * TPL));
      re = fmaf(pw[q], v[q].re, re);
      im = fmaf(pw[q], v[q].im, im);
    }
    re = warp_sum_t(re, SEGW);
    im = warp_sum_t(im, SEGW);
    if ((t & (SEGW - 1)) == 0) part[seg * (MA + 1) + aa] = mkc(-im * sN, re * sN);  // i N (-1)^p2 (re + i im)
  }
}

// ---------------------------------------------------------------------------
// Fused row pass of a Krylov chain step: pass C of K p_i (row DFT of the
// column pass output, K p_i = i (-1)^p DFT(w) -> out, the next chain vector)
// followed, on the same rows still in registers, by pass A of K p_i (-> out2).
// Saves the re-read of p_{i+1} and one launch per chain step.
// ---------------------------------------------------------------------------
template <typename T, int LOGN, int RV = 0>
__global__ void __launch_bounds__(RowG<T, LOGN, RV>::THREADS, RowG<T, LOGN, RV>::MINB) k_pass_ca(const PassArgs<T> a) {
  using G = RowG<T, LOGN, RV>;
  constexpr int N = G::N, TPL = G::TPL, LINES = G::LINES, P = G::P;
  extern __shared__ __align__(16) unsigned char smem[];
  const int slot = blockIdx.y;
  if (a.run && !a.run[slot]) return;
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  const int p2 = blockIdx.x * LINES + line;
  cx<T>* sl = reinterpret_cast<cx<T>*>(smem) + line * P;
  cx<T> v[16];
  const cx<T>* src = a.in + (size_t)slot * a.in_ss + (size_t)p2 * N + t;
  // columns outside the potential's support are exactly zero (not stored by the column pass)
  if (a.sx0 > 0 || a.sx1 < N) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = t + q * TPL;
      v[q] = (x >= a.sx0 && x < a.sx1) ? ldg(src + q * TPL) : mkc((T)0, (T)0);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = ldg(src + q * TPL);
  }
  constexpr bool F32 = std::is_same<T, float>::value;
  if constexpr (F32) ca_moments<LOGN>(a, v, slot, p2, t);  // moments of K p from T2 (FP32)
  fft_line<T, LOGN, false, F32>(v, sl, t, a.tw);
  cx<T>* kp = reinterpret_cast<cx<T>*>(a.out) + (size_t)slot * a.out_ss + (size_t)p2 * N + t;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    cx<T> y = v[q];
    if ((t + q * TPL + p2) & 1) y = mkc(-y.re, -y.im);
    y = cmuli(y);
    kp[q * TPL] = y;
    v[q] = y;
  }
  // (the inverse transform's first stage synchronises before it reuses the line buffer)
  row_a<T, LOGN, false, !F32>(a, v, slot, p2, t, sl,
                             reinterpret_cast<cx<T>*>(a.out2) + (size_t)slot * a.out2_ss + (size_t)p2 * N + t);
}

// ---------------------------------------------------------------------------
// Pass B: columns.  MODE PB_MATVEC operator, PB_RHS right-hand side, PB_HOUT h
// only (m output), PB_FWD / PB_INV raw column DFTs.  PB_WF: the operator with
// one copy of the transform's code for both transforms (the inverse as
// conj(DFT(conj(x))), the two in a loop), for the double-float pass whose two
// inlined transforms would not fit the instruction cache (measured 12 % faster
// than its first half, PB_W, followed by a separate PB_FWD launch, which moved
// the support columns through HBM once more).  A warp covers CW
// neighbouring columns x TW consecutive t, so the 16 loads and stores of each
// thread (rows t + q TPL of column j1) are coalesced row segments.
// ---------------------------------------------------------------------------
template <typename T, int LOGN, int MODE, int CV>
__global__ void __launch_bounds__(ColG<T, LOGN, CV>::THREADS, ColG<T, LOGN, CV>::MINB) k_pass_b(const PassArgs<T> a) {
  using G = ColG<T, LOGN, CV>;
  constexpr int N = G::N, TPL = G::TPL, P = G::P;
  extern __shared__ __align__(16) unsigned char smem[];
  // slot-major block order: the blocks resident together work on the same column
  // tiles of different slots and share the Q / Delta_n table tiles in L2 and L1
  const int slot = blockIdx.x;
  if (a.run && !a.run[slot]) return;
  const int M = a.M;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = (warp / G::WPG) * G::CW + lane % G::CW;
  const int t = (warp % G::WPG) * G::TW + lane / G::CW;
  const int j1 = a.sx0 + blockIdx.y * G::COLS + c;  // the column tiles of the potential's support
  cx<T>* sl = reinterpret_cast<cx<T>*>(smem) + c * P;
  constexpr size_t off = ((size_t)G::COLS * P * sizeof(cx<T>) + 15) & ~(size_t)15;
  cx<T>* coef = reinterpret_cast<cx<T>*>(smem + off);  // [M+1] c_n, then the fill d'

  constexpr bool WF = MODE == PB_WF;
  cx<T> v[16];
  if (MODE != PB_RHS) {
    const cx<T>* src = a.in + (size_t)slot * a.in_ss + (size_t)t * N + j1;
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = ldg(src + (size_t)q * TPL * N);
    // Taylor coefficients of this slot (k_coef), issued after the field loads
    if ((MODE == PB_MATVEC || MODE == PB_HOUT || MODE == PB_W || WF) && threadIdx.x < M + 2)
      coef[threadIdx.x] = ccast<T>(a.coef[(size_t)slot * (M + 2) + threadIdx.x]);
    if (MODE == PB_FWD) fft_line<T, LOGN, false, std::is_same<T, float>::value>(v, sl, t, a.tw);
    else if (!WF) fft_line<T, LOGN, true, std::is_same<T, float>::value>(v, sl, t, a.tw);
  }
#pragma unroll 1
  for (int ph = 0; ph < (WF ? 2 : 1); ++ph) {
  if constexpr (WF) {
    if (ph == 0) {
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q].im = -v[q].im;
    }
    fft_line_compact<T, LOGN, false>(v, sl, t, a.tw);
    if (ph == 1) break;
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q].im = -v[q].im;
  }
  if (MODE == PB_MATVEC || MODE == PB_HOUT || MODE == PB_W || WF) {
    __syncthreads();  // coefficients visible
    // h = u + sum_n c_n Delta_n + d'  (n outer, 16 independent loads per n)
    const cx<T> fill = coef[M + 1];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = v[q] + fill;
    // rows outside [sy0, sy1) (operator only, where the plan sets a band): Q = 0 there
    // and w = 0 below, so their table loads are skipped; a branch uniform over the grid
    const bool band = MODE != PB_HOUT && (a.sy0 > 0 || a.sy1 < N);  // (WF: as MATVEC)
    for (int n = 0; n <= M; ++n) {
      const cx<T> cn = coef[n];
      const cx<T>* D = a.Delta + ((size_t)n * N + t) * N + j1;
      if (band) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int y = t + q * TPL;
          if (y >= a.sy0 && y < a.sy1) v[q] = v[q] + cmul(cn, ldg(D + (size_t)q * TPL * N));
        }
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = v[q] + cmul(cn, ldg(D + (size_t)q * TPL * N));
      }
    }
  }
  if (MODE == PB_MATVEC || MODE == PB_RHS || MODE == PB_W || WF) {
    // w = (2 pi L^2/N^2) E_k Q conj(h)   (right-hand side: E_k Q)
    const cx<T> exv = cscale(ldg(a.ex + (size_t)slot * N + j1), (T)a.sw);
    const cx<T>* EY = a.ey + (size_t)slot * N + t;
    const cx<T>* QC = a.Q + (size_t)slot * a.q_ss + (size_t)t * N + j1;
    if (a.sy0 > 0 || a.sy1 < N) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int y = t + q * TPL;
        if (!(y >= a.sy0 && y < a.sy1)) {
          v[q] = mkc((T)0, (T)0);  // Q = 0 on this row: w = 0 exactly
          continue;
        }
        const cx<T> eq = cmul(cmul(exv, ldg(EY + q * TPL)), ldg(QC + (size_t)q * TPL * N));
        v[q] = (MODE == PB_RHS) ? eq : cmulc(eq, v[q]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const cx<T> eq = cmul(cmul(exv, ldg(EY + q * TPL)), ldg(QC + (size_t)q * TPL * N));
        v[q] = (MODE == PB_RHS) ? eq : cmulc(eq, v[q]);
      }
    }
    if (MODE != PB_W && !WF) fft_line<T, LOGN, false, std::is_same<T, float>::value>(v, sl, t, a.tw);
  }
  }
  cx<T>* dst = reinterpret_cast<cx<T>*>(a.out) + (size_t)slot * a.out_ss + (size_t)t * N + j1;
#pragma unroll
  for (int q = 0; q < 16; ++q) dst[(size_t)q * TPL * N] = v[q];
}

// ---------------------------------------------------------------------------
// Pass B, operator mode, two slots per block: slots 2b and 2b+1 on the same
// column tile (the Q / Delta_n tiles are read once for both), their transforms
// in lockstep.  Same arithmetic per element as k_pass_b<T, LOGN, PB_MATVEC, 0>.
// ---------------------------------------------------------------------------
template <typename T, int LOGN>
__global__ void __launch_bounds__(ColG<T, LOGN, 0>::THREADS, 1) k_pass_b2(const PassArgs<T> a, int nslots) {
  using G = ColG<T, LOGN, 0>;
  constexpr int N = G::N, TPL = G::TPL, P = G::P;
  constexpr bool TWM = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char smem[];
  const int s0 = 2 * blockIdx.x, s1 = s0 + 1 < nslots ? s0 + 1 : s0;
  const bool r0 = !a.run || a.run[s0];
  const bool r1 = s1 != s0 && (!a.run || a.run[s1]);
  if (!r0 && !r1) return;
  const int M = a.M;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = (warp / G::WPG) * G::CW + lane % G::CW;
  const int t = (warp % G::WPG) * G::TW + lane / G::CW;
  const int j1 = a.sx0 + blockIdx.y * G::COLS + c;  // the column tiles of the potential's support
  cx<T>* la = reinterpret_cast<cx<T>*>(smem) + c * P;
  cx<T>* lb = la + G::COLS * P;
  constexpr size_t off = ((size_t)2 * G::COLS * P * sizeof(cx<T>) + 15) & ~(size_t)15;
  cx<T>* coef = reinterpret_cast<cx<T>*>(smem + off);  // [2][M+2]

  cx<T> va[16], vb[16];
  {
    const cx<T>* sa = a.in + (size_t)s0 * a.in_ss + (size_t)t * N + j1;
    const cx<T>* sb = a.in + (size_t)s1 * a.in_ss + (size_t)t * N + j1;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      va[q] = ldg(sa + (size_t)q * TPL * N);
      vb[q] = ldg(sb + (size_t)q * TPL * N);
    }
  }
  if (threadIdx.x < 2 * (M + 2)) {
    const int h = threadIdx.x >= M + 2, i = threadIdx.x - h * (M + 2);
    coef[threadIdx.x] = ccast<T>(a.coef[(size_t)(h ? s1 : s0) * (M + 2) + i]);
  }
  fft_line2<T, LOGN, true, TWM>(va, vb, la, lb, t, a.tw);
  __syncthreads();  // coefficients visible
  {
    const cx<T> fa = coef[M + 1], fb = coef[2 * M + 3];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      va[q] = va[q] + fa;
      vb[q] = vb[q] + fb;
    }
  }
  const bool band = a.sy0 > 0 || a.sy1 < N;
  for (int n = 0; n <= M; ++n) {
    const cx<T> ca = coef[n], cb = coef[M + 2 + n];
    const cx<T>* D = a.Delta + ((size_t)n * N + t) * N + j1;
    if (band) {  // rows outside [sy0, sy1): Q = 0, w = 0 below; no table loads
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int y = t + q * TPL;
        if (y >= a.sy0 && y < a.sy1) {
          const cx<T> d = ldg(D + (size_t)q * TPL * N);
          va[q] = va[q] + cmul(ca, d);
          vb[q] = vb[q] + cmul(cb, d);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const cx<T> d = ldg(D + (size_t)q * TPL * N);
        va[q] = va[q] + cmul(ca, d);
        vb[q] = vb[q] + cmul(cb, d);
      }
    }
  }
  {
    const cx<T> xa = cscale(ldg(a.ex + (size_t)s0 * N + j1), (T)a.sw);
    const cx<T> xb = cscale(ldg(a.ex + (size_t)s1 * N + j1), (T)a.sw);
    const cx<T>* EA = a.ey + (size_t)s0 * N + t;
    const cx<T>* EB = a.ey + (size_t)s1 * N + t;
    const cx<T>* QA = a.Q + (size_t)s0 * a.q_ss + (size_t)t * N + j1;
    const cx<T>* QB = a.Q + (size_t)s1 * a.q_ss + (size_t)t * N + j1;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int y = t + q * TPL;
      if (band && !(y >= a.sy0 && y < a.sy1)) {  // Q = 0 on this row: w = 0 exactly
        va[q] = mkc((T)0, (T)0);
        vb[q] = mkc((T)0, (T)0);
        continue;
      }
      const cx<T> qa = ldg(QA + (size_t)q * TPL * N);
      const cx<T> qb = a.q_ss ? ldg(QB + (size_t)q * TPL * N) : qa;
      va[q] = cmulc(cmul(cmul(xa, ldg(EA + q * TPL)), qa), va[q]);
      vb[q] = cmulc(cmul(cmul(xb, ldg(EB + q * TPL)), qb), vb[q]);
    }
  }
  fft_line2<T, LOGN, false, TWM>(va, vb, la, lb, t, a.tw);
  cx<T>* da = reinterpret_cast<cx<T>*>(a.out) + (size_t)s0 * a.out_ss + (size_t)t * N + j1;
  cx<T>* db = reinterpret_cast<cx<T>*>(a.out) + (size_t)s1 * a.out_ss + (size_t)t * N + j1;
  if (r0) {
#pragma unroll
    for (int q = 0; q < 16; ++q) da[(size_t)q * TPL * N] = va[q];
  }
  if (r1) {
#pragma unroll
    for (int q = 0; q < 16; ++q) db[(size_t)q * TPL * N] = vb[q];
  }
}

// ---------------------------------------------------------------------------
// Taylor coefficients of each slot from pass A's row-moment partials, in a
// fixed order.  Row p2 contributes (-1)^{p2} times
//   n <= M:  sum_a C(n,a) i^{n-a} D_{n-a}(p2) R_a(p2)      (c_n, Sec. 4.3 step 4a)
//   n = M+1: R_1(p2) D_0(p2) - i R_0(p2) D_1(p2)          (fill value dS/dxi(0))
// and coef[slot] = c_0..c_M, then the fill d' = d * fillscale (taylor_coef).
// partA: [slot][p2][seg][a], the a = 0 moment in segment 0 only.
// Grid (slots, KC): block b sums rows [b, b+1) * blockDim.x (one row per
// thread; the FP64 work is spread over many SMs), writes its M+2 partial sums,
// and the last block of a slot to finish (atomic ticket) adds the KC partials
// in block order, scales them and re-arms the slot's ticket.
// ---------------------------------------------------------------------------
constexpr int KC_MAXM = 16;
template <typename PT>
static __global__ void __launch_bounds__(256) k_coef(const cx<PT>* __restrict__ partA, int nseg, int MA, int M,
                                              int N, const cx<double>* __restrict__ Da64,
                                              const cx<float>* __restrict__ Da32, double fillscale,
                                              cx<double>* __restrict__ coefp, int* __restrict__ ticket,
                                              cx<double>* __restrict__ coef) {
  // FP64 partials (FP64 and double-float passes): FP64 products and sums.
  // FP32 partials (the FP32 inner pass): FP32 products, double-float sums
  // over rows -- no FP64 per row on GB300's small FP64 pipe; the products
  // carry the FP32 precision the moments already have.
  constexpr bool F32 = std::is_same<PT, float>::value;
  using AT = typename std::conditional<F32, float, double>::type;  // product arithmetic
  using ST = typename std::conditional<F32, dd, double>::type;     // row-sum arithmetic
  __shared__ ST sre[256], sim[256];
  __shared__ bool last;
  const int slot = blockIdx.x, KC = gridDim.y;
  const int stride = nseg * (MA + 1);
  const int p2 = blockIdx.y * blockDim.x + threadIdx.x;
  const cx<PT>* R = partA + ((size_t)slot * N + p2) * stride;
  cx<AT> Rv[KC_MAXM + 1];  // R_a(p2), a = 0..MA (MA <= 16)
  for (int aa = 0; aa <= MA; ++aa) {
    cx<PT> s = R[aa];
    if (aa > 0)
      for (int sg = 1; sg < nseg; ++sg) s = s + R[sg * (MA + 1) + aa];
    Rv[aa] = ccast<AT>(s);
  }
  auto Dv = [&](int b) -> cx<AT> {
    if constexpr (F32) return Da32[(size_t)b * N + p2];
    else return Da64[(size_t)b * N + p2];
  };
  cx<double>* cp = coefp + ((size_t)slot * KC + blockIdx.y) * (M + 2);
  for (int n = 0; n < M + 2; ++n) {
    cx<AT> s = mkc((AT)0, (AT)0);
    if (n <= M) {
      int binom = 1;  // C(n, aa), exact for n <= 16
      for (int aa = 0; aa <= n; ++aa) {
        cx<AT> tmp = cmul(Dv(n - aa), Rv[aa]);
        const int e = (n - aa) & 3;
        if (e == 1) tmp = cmuli(tmp);
        else if (e == 2) tmp = mkc(-tmp.re, -tmp.im);
        else if (e == 3) tmp = mkc(tmp.im, -tmp.re);
        s = s + cscale(tmp, (AT)binom);
        binom = binom * (n - aa) / (aa + 1);
      }
    } else {
      const cx<AT> t1 = cmul(Rv[1], Dv(0));
      const cx<AT> t2 = cmul(Rv[0], Dv(1));
      s = mkc(t1.re + t2.im, t1.im - t2.re);
    }
    if (p2 & 1) s = mkc(-s.re, -s.im);
    // warp sums by shuffles, then the warps' sums (one barrier pair per coefficient)
    const ST wr = warp_sum_t(ST(s.re), 32), wi = warp_sum_t(ST(s.im), 32);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
      sre[wid] = wr;
      sim[wid] = wi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      ST tr = sre[0], ti = sim[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        tr = tr + sre[w];
        ti = ti + sim[w];
      }
      cp[n] = mkc((double)tr, (double)ti);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partials are visible before its ticket
    last = atomicAdd(ticket + slot, 1) == KC - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int n = threadIdx.x; n < M + 2; n += blockDim.x) {
    cx<double> s = mkc(0.0, 0.0);
    for (int b = 0; b < KC; ++b) {
      const double* q = reinterpret_cast<const double*>(coefp + ((size_t)slot * KC + b) * (M + 2) + n);
      s = s + mkc(__ldcg(q), __ldcg(q + 1));
    }
    coef[(size_t)slot * (M + 2) + n] = taylor_coef(s, n, M, N, fillscale);
  }
  if (threadIdx.x == 0) ticket[slot] = 0;
}

// ---------------------------------------------------------------------------
// Pass C: rows.  PC_KS: K S = i (-1)^p DFT(w) -> out (T).
// PC_RHS: b = -i (-1)^p DFT(w) -> out (FP64) and out2 (TO), |b|^2 partials.
// PC_RES: r = b - x - i (-1)^p DFT(w) -> out2 (TO), |r|^2 partials (T = FP64).
// PC_FWD / PC_INV: raw row DFTs -> out (T).
// ---------------------------------------------------------------------------
template <typename T, typename TO, int LOGN, int MODE, int RV = 0>
__global__ void __launch_bounds__(RowG<T, LOGN, RV>::THREADS, RowG<T, LOGN, RV>::MINB) k_pass_c(const PassArgs<T> a) {
  using G = RowG<T, LOGN, RV>;
  constexpr int N = G::N, TPL = G::TPL, LINES = G::LINES, P = G::P;
  extern __shared__ __align__(16) unsigned char smem[];
  const int slot = blockIdx.y;
  if (a.run && !a.run[slot]) return;
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  const int p2 = blockIdx.x * LINES + line;
  cx<T>* sl = reinterpret_cast<cx<T>*>(smem) + line * P;
  const cx<T>* src = a.in + (size_t)slot * a.in_ss + (size_t)p2 * N + t;
  cx<T> v[16];
  // columns outside the potential's support are exactly zero (not stored by the column pass)
  if (a.sx0 > 0 || a.sx1 < N) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int x = t + q * TPL;
      v[q] = (x >= a.sx0 && x < a.sx1) ? ldg(src + q * TPL) : mkc((T)0, (T)0);
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = ldg(src + q * TPL);
  }
  fft_line<T, LOGN, MODE == PC_INV, std::is_same<T, float>::value>(v, sl, t, a.tw);
  // squared-norm partials.  FP64 for FP64 fields and for the right-hand side
  // (once per solve); the double-float residual sums FP32 squares of r scaled
  // by the slot's power-of-two 1/||b|| (no FP64 per element on GB300's small
  // FP64 pipe, no underflow of small residuals), unscaled once per block.
  constexpr bool NF32 = !std::is_same<T, double>::value && MODE == PC_RES;
  using NT = typename std::conditional<NF32, float, double>::type;
  const float nsc = NF32 ? a.nscale[slot] : 1.f;
  NT nrm = 0;
  // double-float right-hand side (||b|| not known yet): FP32 squares scaled by
  // a power of two near 1 / (this thread's largest |value|), unscaled in FP64
  // once per thread
  constexpr bool RHS32 = !std::is_same<T, double>::value && MODE == PC_RHS;
  float rsc = 1.f, nrm32 = 0.f;
  if constexpr (RHS32) {
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < 16; ++q) mx = fmaxf(mx, fmaxf(fabsf((float)v[q].re), fabsf((float)v[q].im)));
    int e = (__float_as_int(mx) >> 23) & 0xff;  // biased exponent
    e = e < 1 ? 1 : (e > 253 ? 253 : e);
    rsc = __int_as_float((254 - e) << 23);  // 2^(127 - e)
  }
  const size_t rowoff = (size_t)p2 * N + t;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int p1 = t + q * TPL;
    const size_t idx = rowoff + q * TPL;
    cx<T> y = v[q];
    if (MODE == PC_KS || MODE == PC_RHS || MODE == PC_RES) {
      if (((p1 + p2) & 1) != (a.neg != 0)) y = mkc(-y.re, -y.im);
      y = (MODE == PC_RHS) ? mkc(y.im, -y.re) : cmuli(y);
    }
    if (MODE == PC_KS || MODE == PC_FWD || MODE == PC_INV) {
      reinterpret_cast<cx<T>*>(a.out)[(size_t)slot * a.out_ss + idx] = y;
    } else if (MODE == PC_RHS) {
      reinterpret_cast<cx<T>*>(a.out)[(size_t)slot * a.out_ss + idx] = y;
      reinterpret_cast<cx<TO>*>(a.out2)[(size_t)slot * a.out2_ss + idx] = ccast<TO>(y);
      if constexpr (RHS32) {
        const float yr = (float)y.re * rsc, yi = (float)y.im * rsc;
        nrm32 += yr * yr + yi * yi;
      } else {
        const double yr = (double)y.re, yi = (double)y.im;
        nrm += yr * yr + yi * yi;
      }
    } else {  // PC_RES
      const cx<T> bb = a.b[(size_t)slot * a.f_ss + idx];
      const cx<T> xx = a.x[(size_t)slot * a.f_ss + idx];
      const cx<T> r = mkc(bb.re - xx.re - y.re, bb.im - xx.im - y.im);
      reinterpret_cast<cx<TO>*>(a.out2)[(size_t)slot * a.out2_ss + idx] = ccast<TO>(r);
      if constexpr (NF32) {
        const float rr = (float)r.re * nsc, ri = (float)r.im * nsc;
        nrm += rr * rr + ri * ri;
      } else {
        const double rr = (double)r.re, ri = (double)r.im;
        nrm += rr * rr + ri * ri;
      }
    }
  }
  if constexpr (RHS32) {
    const double inv = (double)(1.0f / rsc);  // 2^(e - 127), exact
    nrm = (double)nrm32 * inv * inv;
  }
  if (MODE == PC_RHS || MODE == PC_RES) {
    __shared__ NT wred[32];
    nrm = warp_sum_t(nrm, 32);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
      NT s = 0;
      for (int w = 0; w < G::THREADS / 32; ++w) s += wred[w];
      a.part[(size_t)slot * gridDim.x + blockIdx.x] = NF32 ? (double)s / ((double)nsc * (double)nsc) : (double)s;
    }
  }
}

}  // namespace dbar
