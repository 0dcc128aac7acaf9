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

// ---------------------------------------------------------------------------
// Pass A: rows of a Fourier field.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(KMax<T>::threads) k_pass_a(const PassArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int slot = blockIdx.y;
  if (a.run && !a.run[slot]) return;
  const int N = a.g.N, TPL = a.g.tpl, P = a.g.P, lines = a.g.lines, M = a.M;
  const int MA = M > 1 ? M : 1;
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  const int p2 = blockIdx.x * lines + line;
  cx<T>* sl = reinterpret_cast<cx<T>*>(smem) + line * P;
  const T sc = a.in_scale ? (T)a.in_scale[(size_t)slot * a.in_scale_ss] : (T)1;
  const cx<T>* src = a.in + (size_t)slot * a.in_ss + (size_t)p2 * N;
  cx<T> v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = cscale(ldg(src + t + q * TPL), sc);

  // Row moments R_a(p2) = sum_p1 (-1)^p1 S D_a(p1), a = 0..MA.
  const int segw = TPL >= 32 ? 32 : TPL;
  const int nseg = TPL >= 32 ? TPL / 32 : 1;
  const int seg = TPL >= 32 ? t / 32 : 0;
  size_t off = ((size_t)lines * P * sizeof(cx<T>) + 15) & ~(size_t)15;
  cx<double>* red = reinterpret_cast<cx<double>*>(smem + off);
  cx<double>* lc = red + lines * nseg * (MA + 1);
  for (int aa = 0; aa <= MA; ++aa) {
    cx<T> acc = mkc((T)0, (T)0);
    const cx<T>* D = a.Da + (size_t)aa * N;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p1 = t + q * TPL;
      cx<T> s = v[q];
      if (p1 & 1) s = mkc(-s.re, -s.im);
      acc = acc + cmul(s, ldg(D + p1));
    }
    double re = warp_sum((double)acc.re, segw), im = warp_sum((double)acc.im, segw);
    if ((t & (segw - 1)) == 0) red[(line * nseg + seg) * (MA + 1) + aa] = mkc(re, im);
  }

  // S~ (-1)^{p1+p2} / (2 pi L^2) with S~ = S/xi, xi = (m1 + i m2)/L, 0 at xi = 0.
  const int m2 = wavenum(p2, N);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int p1 = t + q * TPL;
    const int m1 = wavenum(p1, N);
    const int den = m1 * m1 + m2 * m2;
    if (den == 0) {
      v[q] = mkc((T)0, (T)0);
    } else {
      T f = (T)a.inv2piL / (T)den;
      if ((p1 + p2) & 1) f = -f;
      v[q] = cmul(v[q], mkc((T)m1 * f, (T)(-m2) * f));
    }
  }
  fft_line<T, true>(v, sl, N, a.g.logN, t, TPL, a.tw);
  cx<T>* dst = reinterpret_cast<cx<T>*>(a.out) + (size_t)slot * a.out_ss + (size_t)p2 * N;
#pragma unroll
  for (int q = 0; q < 16; ++q) dst[t + q * TPL] = v[q];

  // Per-line combination with D_b(p2) (FP64), then the block partial sums.
  __syncthreads();
  if ((int)threadIdx.x < lines) {
    const int ln = threadIdx.x;
    const int pp2 = blockIdx.x * lines + ln;
    const double sg = (pp2 & 1) ? -1.0 : 1.0;
    cx<double> R[17];
    for (int aa = 0; aa <= MA; ++aa) {
      cx<double> s = mkc(0.0, 0.0);
      for (int sgi = 0; sgi < nseg; ++sgi) s = s + red[(ln * nseg + sgi) * (MA + 1) + aa];
      R[aa] = s;
    }
    for (int n = 0; n <= M; ++n) {
      cx<double> s = mkc(0.0, 0.0);
      double binom = 1.0;
      for (int aa = 0; aa <= n; ++aa) {
        // term C(n,a) i^{n-a} D_{n-a}(p2) R_a
        cx<double> tmp = cmul(a.Da64[(size_t)(n - aa) * N + pp2], R[aa]);
        const int e = (n - aa) & 3;
        if (e == 1) tmp = cmuli(tmp);
        else if (e == 2) tmp = mkc(-tmp.re, -tmp.im);
        else if (e == 3) tmp = mkc(tmp.im, -tmp.re);
        s = s + cscale(tmp, binom);
        binom = binom * (double)(n - aa) / (double)(aa + 1);
      }
      lc[ln * (M + 2) + n] = cscale(s, sg);
    }
    // fill value: R_1 D_0(p2) - i R_0 D_1(p2)
    cx<double> dv = cmul(R[1], a.Da64[pp2]);
    cx<double> t2 = cmul(R[0], a.Da64[(size_t)N + pp2]);
    dv = mkc(dv.re + t2.im, dv.im - t2.re);
    lc[ln * (M + 2) + M + 1] = cscale(dv, sg);
  }
  __syncthreads();
  for (int n = threadIdx.x; n < M + 2; n += blockDim.x) {
    cx<double> s = mkc(0.0, 0.0);
    for (int ln = 0; ln < lines; ++ln) s = s + lc[ln * (M + 2) + n];
    a.partA[((size_t)slot * gridDim.x + blockIdx.x) * (M + 2) + n] = s;
  }
}

// ---------------------------------------------------------------------------
// Pass B: columns.  MODE 0 operator, 1 right-hand side, 2 h only (m output),
// 3 raw forward column DFT, 4 raw inverse column DFT.
// ---------------------------------------------------------------------------

template <typename T, int MODE>
__global__ void __launch_bounds__(KMax<T>::threads) k_pass_b(const PassArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int slot = blockIdx.y;
  if (a.run && !a.run[slot]) return;
  const int N = a.g.N, TPL = a.g.tpl, P = a.g.P, cols = a.g.lines, M = a.M;
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  const int c0 = blockIdx.x * cols;
  const int j1 = c0 + line;
  cx<T>* tile = reinterpret_cast<cx<T>*>(smem);
  size_t off = ((size_t)cols * P * sizeof(cx<T>) + 15) & ~(size_t)15;
  cx<T>* coef = reinterpret_cast<cx<T>*>(smem + off);  // [M+1] c_n, then the fill d'

  if (MODE == PB_MATVEC || MODE == PB_HOUT) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const cx<double>* pa = a.partA + (size_t)slot * a.nblkA * (M + 2);
      for (int n = 0; n < M + 2; ++n) {
        double re = 0.0, im = 0.0;
        for (int b = lane; b < a.nblkA; b += 32) {
          const cx<double> x = pa[(size_t)b * (M + 2) + n];
          re += x.re;
          im += x.im;
        }
        re = warp_sum(re, 32);
        im = warp_sum(im, 32);
        if (lane == 0) coef[n] = ccast<T>(taylor_coef(mkc(re, im), n, M, N, a.fillscale));
      }
    }
  }
  if (MODE != PB_RHS) {
    const cx<T>* src = a.in + (size_t)slot * a.in_ss;
    for (int i = threadIdx.x; i < N * cols; i += blockDim.x) {
      const int row = i / cols, c = i - row * cols;
      tile[c * P + padi(row)] = ldg(src + (size_t)row * N + c0 + c);
    }
  }
  __syncthreads();
  cx<T>* sl = tile + line * P;
  cx<T> v[16];
  if (MODE != PB_RHS) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = sl[padi(t + q * TPL)];
    if (MODE == PB_FWD) fft_line<T, false>(v, sl, N, a.g.logN, t, TPL, a.tw);
    else fft_line<T, true>(v, sl, N, a.g.logN, t, TPL, a.tw);
  }
  if (MODE == PB_MATVEC || MODE == PB_RHS || MODE == PB_HOUT) {
    const cx<T> exv = ldg(a.ex + (size_t)slot * N + j1);
    const cx<T> fill = (MODE == PB_RHS) ? mkc((T)0, (T)0) : coef[M + 1];
    const T sw = (T)a.sw;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j2 = t + q * TPL;
      cx<T> h = mkc((T)0, (T)0);
      if (MODE != PB_RHS) {
        h = v[q] + fill;
        for (int n = 0; n <= M; ++n)
          h = h + cmul(coef[n], ldg(a.DeltaT + ((size_t)n * N + j1) * N + j2));
      }
      if (MODE == PB_HOUT) {
        v[q] = h;
      } else {
        const cx<T> eq = cscale(cmul(cmul(exv, ldg(a.ey + (size_t)slot * N + j2)),
                                     ldg(a.QT + (size_t)j1 * N + j2)), sw);
        v[q] = (MODE == PB_RHS) ? eq : cmulc(eq, h);
      }
    }
    if (MODE != PB_HOUT) fft_line<T, false>(v, sl, N, a.g.logN, t, TPL, a.tw);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) sl[padi(t + q * TPL)] = v[q];
  __syncthreads();
  cx<T>* dst = reinterpret_cast<cx<T>*>(a.out) + (size_t)slot * a.out_ss;
  for (int i = threadIdx.x; i < N * cols; i += blockDim.x) {
    const int row = i / cols, c = i - row * cols;
    dst[(size_t)row * N + c0 + c] = tile[c * P + padi(row)];
  }
}

// ---------------------------------------------------------------------------
// Pass C: rows.  MODE 0: K S = i (-1)^p DFT(w) -> out (T).
// MODE 1: b = -i (-1)^p DFT(w) -> out (FP64) and out2 (TO), |b|^2 partials.
// MODE 2: r = b - x - i (-1)^p DFT(w) -> out2 (TO), |r|^2 partials (T = FP64).
// MODE 3 / 4: raw forward / inverse row DFT -> out (T).
// ---------------------------------------------------------------------------

template <typename T, typename TO, int MODE>
__global__ void __launch_bounds__(KMax<T>::threads) k_pass_c(const PassArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int slot = blockIdx.y;
  if (a.run && !a.run[slot]) return;
  const int N = a.g.N, TPL = a.g.tpl, P = a.g.P, lines = a.g.lines;
  const int line = threadIdx.x / TPL, t = threadIdx.x - line * TPL;
  const int p2 = blockIdx.x * lines + line;
  cx<T>* sl = reinterpret_cast<cx<T>*>(smem) + line * P;
  const cx<T>* src = a.in + (size_t)slot * a.in_ss + (size_t)p2 * N;
  cx<T> v[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = ldg(src + t + q * TPL);
  fft_line<T, MODE == PC_INV>(v, sl, N, a.g.logN, t, TPL, a.tw);
  double nrm = 0.0;
  const size_t rowoff = (size_t)p2 * N;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int p1 = t + q * TPL;
    const size_t idx = rowoff + p1;
    cx<T> y = v[q];
    if (MODE == PC_KS || MODE == PC_RHS || MODE == PC_RES) {
      if ((p1 + p2) & 1) y = mkc(-y.re, -y.im);
      y = (MODE == PC_RHS) ? mkc(y.im, -y.re) : cmuli(y);
    }
    if (MODE == PC_KS || MODE == PC_FWD || MODE == PC_INV) {
      reinterpret_cast<cx<T>*>(a.out)[(size_t)slot * a.out_ss + idx] = y;
    } else if (MODE == PC_RHS) {
      reinterpret_cast<cx<double>*>(a.out)[(size_t)slot * a.out_ss + idx] = ccast<double>(y);
      reinterpret_cast<cx<TO>*>(a.out2)[(size_t)slot * a.out2_ss + idx] = ccast<TO>(y);
      nrm += (double)y.re * (double)y.re + (double)y.im * (double)y.im;
    } else {  // PC_RES
      const cx<double> bb = a.b[(size_t)slot * a.f_ss + idx];
      const cx<double> xx = a.x[(size_t)slot * a.f_ss + idx];
      const cx<double> r = mkc(bb.re - xx.re - (double)y.re, bb.im - xx.im - (double)y.im);
      reinterpret_cast<cx<TO>*>(a.out2)[(size_t)slot * a.out2_ss + idx] = ccast<TO>(r);
      nrm += r.re * r.re + r.im * r.im;
    }
  }
  if (MODE == PC_RHS || MODE == PC_RES) {
    __shared__ double wred[32];
    nrm = warp_sum(nrm, 32);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wred[w];
      a.part[(size_t)slot * gridDim.x + blockIdx.x] = s;
    }
  }
}

}  // namespace dbar
