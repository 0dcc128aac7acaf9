// Complex arithmetic and the in-shared-memory Stockham FFT used by every pass.
//
// The paper computes all transforms with 2-D FFTs (Sec. 4.1: "discrete
// Fourier series, computed via a Fast Fourier Transform"; Sec. 4.3 remark:
// the cost is "mainly in the FFT commands").  Here each 2-D transform is split
// into a row pass and a column pass; inside a pass every line (row or column)
// of length N is transformed by N/16 threads, each holding 16 elements in
// registers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace dbar {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mkc(T a, T b) {
  cx<T> r;
  r.re = a;
  r.im = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mkc(a.re + b.re, a.im + b.im); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mkc(a.re - b.re, a.im - b.im); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mkc(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return mkc(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mkc(a.re * s, a.im * s); }
template <typename T>
__device__ __forceinline__ cx<T> cconj(cx<T> a) { return mkc(a.re, -a.im); }
// i * a
template <typename T>
__device__ __forceinline__ cx<T> cmuli(cx<T> a) { return mkc(-a.im, a.re); }
template <typename T, typename U>
__device__ __forceinline__ cx<T> ccast(cx<U> a) { return mkc((T)a.re, (T)a.im); }

template <typename T>
__device__ __forceinline__ cx<T> ldg(const cx<T>* p) {
  return *reinterpret_cast<const cx<T>*>(p);
}
template <>
__device__ __forceinline__ cx<float> ldg(const cx<float>* p) {
  float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return mkc(v.x, v.y);
}
template <>
__device__ __forceinline__ cx<double> ldg(const cx<double>* p) {
  double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return mkc(v.x, v.y);
}

// Sum over groups of `width` lanes (a power of two <= 32); every lane gets its group's sum.
__device__ __forceinline__ double warp_sum(double v, int width) {
  for (int off = width >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// ---------------------------------------------------------------------------
// Double-float numbers: an unevaluated sum hi + lo of two floats (about 48
// significant bits).  Sums and products use the error-free transformations
// of Dekker (1971) and Knuth (TwoSum), as in the double-double arithmetic of
// Hida, Li and Bailey; every float operation is an explicitly rounded
// intrinsic so the compiler cannot fuse or reorder it.  On GB300 the FP32
// pipes are ~64x the FP64 pipe, so FP64-class transforms run several times
// faster in this form.
// ---------------------------------------------------------------------------
struct __align__(8) dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ dd(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr dd(float f) : hi(f), lo(0.f) {}
  // exact for |i| < 2^24 (grid indices and wavenumbers)
  __host__ __device__ constexpr dd(int i) : hi((float)i), lo(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ dd dd_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd(s, e);
}
__device__ __forceinline__ dd dd_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
  const dd s = dd_two_sum(a.hi, b.hi);
  return dd_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
// Product: p = rn(a.hi b.hi) and e = its exact error (FMA) + the cross terms.
// The pair is left unrenormalised (|e| stays within about one ulp of p):
// sums renormalise through TwoSum, and a product only ever multiplies e by
// a hi part, so the skipped QuickTwoSum changes nothing beyond ~2^-46.
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd(p, e);
}
__device__ __forceinline__ dd operator/(dd a, dd b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dd r = a - dd(q1) * b;
  return dd_quick_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) {
  a = a + b;
  return a;
}

// Complex double-float sums and products.  With DBAR_DD_CALLS they become
// out-of-line calls: the fully unrolled double-float transforms are large
// enough to miss in the instruction cache.
#ifdef DBAR_DD_CALLS
#define DBAR_DD_FN __noinline__
#else
#define DBAR_DD_FN __forceinline__
#endif
template <>
__device__ DBAR_DD_FN cx<dd> operator+(cx<dd> a, cx<dd> b) {
  return mkc(a.re + b.re, a.im + b.im);
}
template <>
__device__ DBAR_DD_FN cx<dd> operator-(cx<dd> a, cx<dd> b) {
  return mkc(a.re - b.re, a.im - b.im);
}
template <>
__device__ DBAR_DD_FN cx<dd> cmul(cx<dd> a, cx<dd> b) {
  return mkc(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}

template <>
__device__ __forceinline__ cx<dd> ldg(const cx<dd>* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return mkc(dd(v.x, v.y), dd(v.z, v.w));
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v, int width) {
  for (int off = width >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
template <>
__device__ __forceinline__ dd warp_sum_t<dd>(dd v, int width) {
  for (int off = width >> 1; off > 0; off >>= 1)
    v = v + dd(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
  return v;
}

// ---------------------------------------------------------------------------
// Register DFT of size R in {2,4,8,16}: radix-2 decimation in time after a
// bit-reversal permutation.  The butterfly twiddles exp(-+ i pi q/8) are the
// exact values cos(pi q/8), sin(pi q/8) written out.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double cos8(int q) {
  return q == 0 ? 1.0
       : q == 1 ? 0.92387953251128675613
       : q == 2 ? 0.70710678118654752440
       : q == 3 ? 0.38268343236508977173
       : q == 4 ? 0.0
       : q == 5 ? -0.38268343236508977173
       : q == 6 ? -0.70710678118654752440
                : -0.92387953251128675613;
}
__host__ __device__ constexpr double sin8(int q) {
  return q == 0 ? 0.0
       : q == 1 ? 0.38268343236508977173
       : q == 2 ? 0.70710678118654752440
       : q == 3 ? 0.92387953251128675613
       : q == 4 ? 1.0
       : q == 5 ? 0.92387953251128675613
       : q == 6 ? 0.70710678118654752440
                : 0.38268343236508977173;
}

// x * exp(s i pi q/8), s = +1 for the inverse transform, -1 for the forward one.
template <typename T, bool INV>
__device__ __forceinline__ cx<T> rot8(cx<T> x, int q) {
  if (q == 0) return x;
  if (q == 4) return INV ? mkc(-x.im, x.re) : mkc(x.im, -x.re);
  const T c = (T)cos8(q);
  const T s = INV ? (T)sin8(q) : (T)-sin8(q);
  return mkc(x.re * c - x.im * s, x.re * s + x.im * c);
}

__host__ __device__ constexpr int brev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
template <int R>
struct Log2 {
  static constexpr int v = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
};

template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_reg(cx<T>* v) {
  constexpr int LB = Log2<R>::v;
  cx<T> t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = v[brev(i, LB)];
#pragma unroll
  for (int m = 1; m < R; m *= 2) {
#pragma unroll
    for (int k = 0; k < m; ++k) {
#pragma unroll
      for (int b = 0; b < R; b += 2 * m) {
        const cx<T> a = t[b + k];
        const cx<T> c = rot8<T, INV>(t[b + k + m], (8 * k) / m);
        t[b + k] = a + c;
        t[b + k + m] = a - c;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = t[i];
}

// Padded shared-memory index: one spare slot every 16 elements keeps the
// stride-R writes of the first stage free of bank conflicts.  Lines (rows or
// columns) sit `pitch_of(N)` elements apart; the pitch is 2 mod 16, so the
// lanes of a warp that work on neighbouring lines hit distinct banks.
__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int pitch_of(int N) { return N + (N >> 4) + 2; }

// Register part of one Stockham stage (see fft_stage): twiddles, the R-point
// DFTs and, in the last stage, the reordering to v[q] = X[t + q TPL].
template <typename T, int N, int R, int NS, bool INV, bool LAST, bool TWM>
__device__ __forceinline__ void fft_stage_regs(cx<T> (&v)[16], int t, const cx<T>* __restrict__ tw) {
  constexpr int TPL = N / 16, B = 16 / R;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    if (NS > 1) {
      constexpr int STEP = N / (NS * R);
      const int k = (t + b * TPL) & (NS - 1);
      if constexpr (TWM) {
        // load w^r for r a power of two, form the rest as products (at most
        // three roundings deep): fewer L1 loads in the FP32 passes
        cx<T> wr[R];
#pragma unroll
        for (int r = 1; r < R; ++r) {
          if ((r & (r - 1)) == 0) {
            wr[r] = ldg(tw + r * k * STEP);
          } else {
            const int hb = 1 << (31 - __clz(r));
            wr[r] = cmul(wr[hb], wr[r - hb]);
          }
        }
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cx<T> w = wr[r];
          if (INV) w.im = -w.im;
          v[b * R + r] = cmul(v[b * R + r], w);
        }
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cx<T> w = ldg(tw + r * k * STEP);
          if (INV) w.im = -w.im;
          v[b * R + r] = cmul(v[b * R + r], w);
        }
      }
    }
    dft_reg<T, R, INV>(&v[b * R]);
  }
  if (LAST) {
    cx<T> u[16];
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) u[b + r * B] = v[b * R + r];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = u[i];
  }
}
// One Stockham stage of radix R on a line of length N held by TPL = N/16
// threads; each thread owns 16 elements, i.e. 16/R butterflies j = t + b TPL.
// Inputs x[j + r N/R] (already in registers in the first stage: v[r] =
// x[t + r TPL]), twiddle w^{r (j mod NS)} with w = e^{-+2 pi i/(NS R)} read
// from the table tw[s] = e^{-2 pi i s/N}, R-point DFT, outputs at
// ((j - j mod NS) R + j mod NS) + r NS.  The last stage (NS R = N) keeps its
// outputs in registers: v[q] = X[t + q TPL].
template <typename T, int N, int R, int NS, bool INV, bool FIRST, bool LAST, bool TWM>
__device__ __forceinline__ void fft_stage(cx<T> (&v)[16], cx<T>* line, int t, const cx<T>* __restrict__ tw) {
  constexpr int TPL = N / 16, B = 16 / R, NB = N / R;
  static_assert(!FIRST || R == 16, "the first stage is radix 16");
  static_assert(!LAST || NS * R == N, "the last stage completes the transform");
  if (!FIRST) {
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = line[padi(t + b * TPL + r * NB)];
  }
  fft_stage_regs<T, N, R, NS, INV, LAST, TWM>(v, t, tw);
  if (!LAST) {
    __syncthreads();  // every thread has read the inputs of this stage
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * TPL;
      const int k = j & (NS - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[padi(base + r * NS)] = v[b * R + r];
    }
    __syncthreads();
  }
}

// Full length-N transform, N = 2^LOGN in [32, 4096]: radix 16 first, then
// 16 and the remainder.  On entry v[q] = x[t + q TPL]; on exit v[q] = X[t + q TPL],
// X[p] = sum_j x[j] e^{-+2 pi i p j/N} (unnormalised; + for INV).  Every thread
// of the block calls this together (it synchronises the block).  TWM: stage
// twiddles w^r formed as products of loaded powers of two (fewer L1 loads;
// measured faster in every FP32 pass; FP32 only).
// The first two radix-16 stages of a transform with N >= 512 as one loop body (stage
// span NS = 1, then 16, at run time): the same operations as fft_stage, one copy of
// the code.  Used by the double-float column pass (fft_line_compact), whose two
// transforms of fully inlined stages would miss in the instruction cache.
template <typename T, int N, bool INV>
__device__ __forceinline__ void fft_stages16_looped(cx<T> (&v)[16], cx<T>* line, int t, const cx<T>* __restrict__ tw) {
  constexpr int R = 16, NB = N / R;
#pragma unroll 1
  for (int s = 0; s < 2; ++s) {
    const int NS = s == 0 ? 1 : 16;
    const int k = t & (NS - 1);
    if (s > 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = line[padi(t + r * NB)];
      const int STEP = N / (NS * R);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cx<T> w = ldg(tw + r * k * STEP);
        if (INV) w.im = -w.im;
        v[r] = cmul(v[r], w);
      }
    }
    dft_reg<T, R, INV>(v);
    __syncthreads();  // every thread has read the inputs of this stage
    const int base = (t - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) line[padi(base + r * NS)] = v[r];
    __syncthreads();
  }
}

template <typename T, int LOGN, bool INV, bool TWM = false>
__device__ __forceinline__ void fft_line(cx<T> (&v)[16], cx<T>* line, int t, const cx<T>* __restrict__ tw) {
  constexpr int N = 1 << LOGN;
  constexpr int L1 = LOGN - 4;
  static_assert(L1 >= 1 && L1 <= 8, "N must be in [32, 4096]");
  static_assert(!TWM || std::is_same<T, float>::value, "twiddle products are for FP32 transforms only");
  if constexpr (L1 <= 4) {
    fft_stage<T, N, 16, 1, INV, true, false, TWM>(v, line, t, tw);
    fft_stage<T, N, (1 << L1), 16, INV, false, true, TWM>(v, line, t, tw);
  } else {
    fft_stage<T, N, 16, 1, INV, true, false, TWM>(v, line, t, tw);
    fft_stage<T, N, 16, 16, INV, false, false, TWM>(v, line, t, tw);
    fft_stage<T, N, (1 << (L1 - 4)), 256, INV, false, true, TWM>(v, line, t, tw);
  }
}

// fft_line with the first two radix-16 stages looped (fft_stages16_looped) at N >= 512:
// the same results, less code.
template <typename T, int LOGN, bool INV>
__device__ __forceinline__ void fft_line_compact(cx<T> (&v)[16], cx<T>* line, int t, const cx<T>* __restrict__ tw) {
  constexpr int N = 1 << LOGN;
  constexpr int L1 = LOGN - 4;
  if constexpr (L1 > 4) {
    fft_stages16_looped<T, N, INV>(v, line, t, tw);
    fft_stage<T, N, (1 << (L1 - 4)), 256, INV, false, true, false>(v, line, t, tw);
  } else {
    fft_line<T, LOGN, INV, false>(v, line, t, tw);
  }
}

// One stage on two lines at once (same t, separate line buffers): one pair of
// barriers serves both, and each thread carries two independent butterfly chains.
template <typename T, int N, int R, int NS, bool INV, bool FIRST, bool LAST, bool TWM>
__device__ __forceinline__ void fft_stage2(cx<T> (&va)[16], cx<T> (&vb)[16], cx<T>* la, cx<T>* lb, int t,
                                           const cx<T>* __restrict__ tw) {
  constexpr int TPL = N / 16, B = 16 / R, NB = N / R;
  if (!FIRST) {
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        va[b * R + r] = la[padi(t + b * TPL + r * NB)];
        vb[b * R + r] = lb[padi(t + b * TPL + r * NB)];
      }
  }
  fft_stage_regs<T, N, R, NS, INV, LAST, TWM>(va, t, tw);
  fft_stage_regs<T, N, R, NS, INV, LAST, TWM>(vb, t, tw);
  if (!LAST) {
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * TPL;
      const int k = j & (NS - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        la[padi(base + r * NS)] = va[b * R + r];
        lb[padi(base + r * NS)] = vb[b * R + r];
      }
    }
    __syncthreads();
  }
}
// fft_line on two lines in lockstep.
template <typename T, int LOGN, bool INV, bool TWM = false>
__device__ __forceinline__ void fft_line2(cx<T> (&va)[16], cx<T> (&vb)[16], cx<T>* la, cx<T>* lb, int t,
                                          const cx<T>* __restrict__ tw) {
  constexpr int N = 1 << LOGN;
  constexpr int L1 = LOGN - 4;
  if constexpr (L1 <= 4) {
    fft_stage2<T, N, 16, 1, INV, true, false, TWM>(va, vb, la, lb, t, tw);
    fft_stage2<T, N, (1 << L1), 16, INV, false, true, TWM>(va, vb, la, lb, t, tw);
  } else {
    fft_stage2<T, N, 16, 1, INV, true, false, TWM>(va, vb, la, lb, t, tw);
    fft_stage2<T, N, 16, 16, INV, false, false, TWM>(va, vb, la, lb, t, tw);
    fft_stage2<T, N, (1 << (L1 - 4)), 256, INV, false, true, TWM>(va, vb, la, lb, t, tw);
  }
}

// Block shapes (shared by the kernels and the host launchers).
//  rows:    LINES lines of TPL = N/16 consecutive threads, 256 threads at most.
//  columns: COLS columns; a warp covers CW neighbouring columns x 32/CW
//           consecutive t, so each load of the 16 elements of a thread is a
//           set of 32*sizeof(cx)/CW-byte row segments (coalesced straight
//           from/to registers).
// Row-pass shapes of the FP32 inner passes (autotuned): lines per block of shape rv
// (0: row_lines, 1: half as many, 2: twice as many; within [1, N] and 1024 threads;
// 3 and 4: the lines of 0 and 1 with a larger register budget, see RowG).
__host__ __device__ constexpr int row_lines_v(int logN, int rv);
__host__ __device__ constexpr int row_lines(int logN) {
  return (256 / ((1 << logN) / 16)) < (1 << logN) ? (256 / ((1 << logN) / 16)) : (1 << logN);
}
__host__ __device__ constexpr int row_lines_v(int logN, int rv) {
  return (rv == 1 || rv == 4) ? (row_lines(logN) / 2 > 0 ? row_lines(logN) / 2 : 1)
       : rv == 2 ? ((row_lines(logN) * 2 <= (1 << logN) && row_lines(logN) * 2 * ((1 << logN) / 16) <= 1024)
                        ? row_lines(logN) * 2 : row_lines(logN))
                 : row_lines(logN);
}
// Column-pass tile shapes.  Variant 0: a warp reads DBAR_COL_SEG_BYTES-byte row
// segments, DBAR_COL_THREADS_F32 / _F64 threads per block.  Variant 1: 32-byte
// segments and 256 threads.  Plans pick one per grid size by timing (autotune).
#ifndef DBAR_COL_SEG_BYTES
#define DBAR_COL_SEG_BYTES 64
#endif
#ifndef DBAR_COL_THREADS_F32
#define DBAR_COL_THREADS_F32 512
#endif
#ifndef DBAR_COL_THREADS_F64
#define DBAR_COL_THREADS_F64 256
#endif
__host__ __device__ constexpr int col_threads(int esz, int cv = 0) {
  return cv ? 256 : (esz == 8 ? DBAR_COL_THREADS_F32 : DBAR_COL_THREADS_F64);
}
__host__ __device__ constexpr int col_cap(int logN, int esz, int cv = 0) {
  return col_threads(esz, cv) / ((1 << logN) / 16) > 0 ? col_threads(esz, cv) / ((1 << logN) / 16) : 1;
}
__host__ __device__ constexpr int col_cwd(int esz, int cv = 0) {
  return (cv ? 32 : DBAR_COL_SEG_BYTES) / esz > 0 ? (cv ? 32 : DBAR_COL_SEG_BYTES) / esz : 1;
}
__host__ __device__ constexpr int col_cw(int logN, int esz, int cv = 0) {
  // row segments of the variant's width when possible; small N: one warp spans all t of CW columns
  return ((1 << logN) / 16 >= 32 / col_cwd(esz, cv))
             ? (col_cwd(esz, cv) < col_cap(logN, esz, cv) ? col_cwd(esz, cv) : col_cap(logN, esz, cv))
             : 32 / ((1 << logN) / 16);
}
__host__ __device__ constexpr int col_cols(int logN, int esz, int cv = 0) {
  return (col_cap(logN, esz, cv) > col_cw(logN, esz, cv) ? col_cap(logN, esz, cv) : col_cw(logN, esz, cv)) <
                 (1 << logN)
             ? (col_cap(logN, esz, cv) > col_cw(logN, esz, cv) ? col_cap(logN, esz, cv) : col_cw(logN, esz, cv))
             : (1 << logN);
}

}  // namespace dbar
