// In-place mixed-radix FFTs of many lines held in shared memory.
//
// Two transforms are provided, each the transpose of the other:
//   * DIF (Gentleman-Sande): natural-order input, digit-reversed output.
//   * DIT: digit-reversed input, natural-order output.
// Reciprocal space is always in natural order (so sphere coefficients are
// scattered and gathered at h mod N), and real space is always in the
// digit-reversed order the DIF produces; the library never needs real-space
// points in natural order, so no reordering pass exists.  Position of natural
// index n for radices R_0, R_1, ...:  P_N(n) = (N/R_0)(n mod R_0) + P_{N/R_0}(n div R_0).
//
// Every butterfly reads and writes the same R positions, so a stage needs no
// second buffer; one block-wide barrier separates stages.  Threads are mapped
// line-fastest so that neighbouring threads touch neighbouring lines.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace wgw {

// Radix-R DFT of v[0..R-1] in registers, X_k = sum_j v_j exp(sign 2 pi i j k / R), natural order.
// P: packed FP32 sums (cadd / csub / cscl of common.cuh).
template <typename T, bool P = false>
WGW_HD void dft2(cplx<T>* v) {
  cplx<T> a = cadd<P>(v[0], v[1]), b = csub<P>(v[0], v[1]);
  v[0] = a; v[1] = b;
}

template <typename T, bool P = false>
WGW_HD void dft3(cplx<T>* v, int sign) {
  const T h = T(0.86602540378443864676);  // sin(2 pi / 3)
  cplx<T> t = cadd<P>(v[1], v[2]);
  cplx<T> u = csub<P>(v[0], cscl<P>(t, T(0.5)));
  cplx<T> w = mul_i(cscl<P>(csub<P>(v[1], v[2]), h), sign);
  v[0] = cadd<P>(v[0], t);
  v[1] = cadd<P>(u, w);
  v[2] = csub<P>(u, w);
}

template <typename T, bool P = false>
WGW_HD void dft4(cplx<T>* v, int sign) {
  cplx<T> a = cadd<P>(v[0], v[2]), b = csub<P>(v[0], v[2]);
  cplx<T> c = cadd<P>(v[1], v[3]), d = mul_i(csub<P>(v[1], v[3]), sign);
  v[0] = cadd<P>(a, c); v[2] = csub<P>(a, c);
  v[1] = cadd<P>(b, d); v[3] = csub<P>(b, d);
}

template <typename T, bool P = false>
WGW_HD void dft5(cplx<T>* v, int sign) {
  const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);  // cos(2pi/5), cos(4pi/5)
  const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);   // sin(2pi/5), sin(4pi/5)
  cplx<T> a1 = cadd<P>(v[1], v[4]), b1 = csub<P>(v[1], v[4]);
  cplx<T> a2 = cadd<P>(v[2], v[3]), b2 = csub<P>(v[2], v[3]);
  cplx<T> u1 = cadd<P>(cadd<P>(v[0], cscl<P>(a1, c1)), cscl<P>(a2, c2));
  cplx<T> u2 = cadd<P>(cadd<P>(v[0], cscl<P>(a1, c2)), cscl<P>(a2, c1));
  cplx<T> w1 = mul_i(cadd<P>(cscl<P>(b1, s1), cscl<P>(b2, s2)), sign);
  cplx<T> w2 = mul_i(csub<P>(cscl<P>(b1, s2), cscl<P>(b2, s1)), sign);
  v[0] = cadd<P>(cadd<P>(v[0], a1), a2);
  v[1] = cadd<P>(u1, w1); v[4] = csub<P>(u1, w1);
  v[2] = cadd<P>(u2, w2); v[3] = csub<P>(u2, w2);
}

template <typename T, bool P = false>
WGW_HD void dft8(cplx<T>* v, int sign) {
  const T r = T(0.70710678118654752440);  // 1/sqrt(2)
  cplx<T> a[4], b[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) { a[j] = cadd<P>(v[j], v[j + 4]); b[j] = csub<P>(v[j], v[j + 4]); }
  // b_j *= exp(sign i pi j / 4):  exp(sign i pi / 4) = (1 + sign i) r,  exp(sign 3 i pi / 4) = (-1 + sign i) r
  b[1] = cscl<P>(cadd<P>(b[1], mul_i(b[1], sign)), r);
  b[2] = mul_i(b[2], sign);
  b[3] = cscl<P>(csub<P>(mul_i(b[3], sign), b[3]), r);
  dft4<T, P>(a, sign);
  dft4<T, P>(b, sign);
#pragma unroll
  for (int k = 0; k < 4; ++k) { v[2 * k] = a[k]; v[2 * k + 1] = b[k]; }
}

template <typename T>
WGW_HD void dft_r(int R, cplx<T>* v, int sign) {
  switch (R) {
    case 2: dft2(v); break;
    case 3: dft3(v, sign); break;
    case 4: dft4(v, sign); break;
    case 5: dft5(v, sign); break;
    default: dft8(v, sign); break;
  }
}

// exp(sign 2 pi i k / N) from a table of exp(+2 pi i k / N), k in [0, N).
template <typename T>
WGW_HD cplx<T> twiddle(const cplx<T>* tw, int k, int sign) {
  cplx<T> w = tw[k];
  if (sign < 0) w.im = -w.im;
  return w;
}

// Map a line index to its offset when the lines are the rows 0..lo and
// N-hi..N-1 of a block (the footprint of a sphere of radius lo = hi = m).
WGW_HD int split_line(int li, int m, int n) { return li <= m ? li : li + n - 2 * m - 1; }

template <typename T, int R, bool P = false>
WGW_HD void dft_fixed(cplx<T>* v, int sign) {
  if constexpr (R == 2) dft2<T, P>(v);
  else if constexpr (R == 3) dft3<T, P>(v, sign);
  else if constexpr (R == 4) dft4<T, P>(v, sign);
  else if constexpr (R == 5) dft5<T, P>(v, sign);
  else dft8<T, P>(v, sign);
}

// One DIF stage of radix R over all lines (block size S, butterfly span M = S/R).
template <typename T, int R>
WGW_HD void dif_stage(cplx<T>* buf, int N, int S, const cplx<T>* tw, int sign, int nlines,
                      int line_stride, int elem_stride, int m_split, Thr th) {
  const int M = S / R, step = N / S, total = nlines * (N / R);
  for (int t = th.tid; t < total; t += th.nth) {
    const int li = t % nlines;
    const int rest = t / nlines;
    const int j2 = rest % M;
    const int blk = rest / M;
    const int line = m_split >= 0 ? split_line(li, m_split, N) : li;
    cplx<T>* base = buf + (size_t)line * line_stride + (size_t)(blk * S + j2) * elem_stride;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[(size_t)r * M * elem_stride];
    dft_fixed<T, R>(v, sign);
    base[0] = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cplx<T> x = v[r];
      if (j2) x = cmul(x, twiddle(tw, (step * j2 * r) % N, sign));
      base[(size_t)r * M * elem_stride] = x;
    }
  }
}

// One DIT stage of radix R (twiddles before the butterfly).
template <typename T, int R>
WGW_HD void dit_stage(cplx<T>* buf, int N, int S, const cplx<T>* tw, int sign, int nlines,
                      int line_stride, int elem_stride, int m_split, Thr th) {
  const int M = S / R, step = N / S, total = nlines * (N / R);
  for (int t = th.tid; t < total; t += th.nth) {
    const int li = t % nlines;
    const int rest = t / nlines;
    const int j2 = rest % M;
    const int blk = rest / M;
    const int line = m_split >= 0 ? split_line(li, m_split, N) : li;
    cplx<T>* base = buf + (size_t)line * line_stride + (size_t)(blk * S + j2) * elem_stride;
    cplx<T> v[R];
    v[0] = base[0];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cplx<T> x = base[(size_t)r * M * elem_stride];
      if (j2) x = cmul(x, twiddle(tw, (step * j2 * r) % N, sign));
      v[r] = x;
    }
    dft_fixed<T, R>(v, sign);
#pragma unroll
    for (int r = 0; r < R; ++r) base[(size_t)r * M * elem_stride] = v[r];
  }
}

#define WGW_RADIX_DISPATCH(FN, R, ...)                 \
  switch (R) {                                         \
    case 2: FN<T, 2>(__VA_ARGS__); break;              \
    case 3: FN<T, 3>(__VA_ARGS__); break;              \
    case 4: FN<T, 4>(__VA_ARGS__); break;              \
    case 5: FN<T, 5>(__VA_ARGS__); break;              \
    default: FN<T, 8>(__VA_ARGS__); break;             \
  }

// DIF over `nlines` lines: natural order in, digit-reversed order out.
// Line li starts at buf + off(li) * line_stride, element e at + e * elem_stride,
// with off(li) = li, or split_line(li, m_split, N) when m_split >= 0.
template <typename T>
WGW_HD void fft_dif(cplx<T>* buf, const FftPlan& p, const cplx<T>* tw, int sign, int nlines,
                    int line_stride, int elem_stride, int m_split, Thr th) {
  const int N = p.n;
  int S = N;
  for (int st = 0; st < p.nst; ++st) {
    WGW_RADIX_DISPATCH(dif_stage, p.radix[st], buf, N, S, tw, sign, nlines, line_stride, elem_stride,
                       m_split, th)
    WGW_SYNC();
    S /= p.radix[st];
  }
}

// DIT over `nlines` lines: digit-reversed order in, natural order out.
template <typename T>
WGW_HD void fft_dit(cplx<T>* buf, const FftPlan& p, const cplx<T>* tw, int sign, int nlines,
                    int line_stride, int elem_stride, int m_split, Thr th) {
  const int N = p.n;
  int sizes[6];
  {
    int S = N;
    for (int st = 0; st < p.nst; ++st) { sizes[st] = S; S /= p.radix[st]; }
  }
  for (int st = p.nst - 1; st >= 0; --st) {
    WGW_RADIX_DISPATCH(dit_stage, p.radix[st], buf, N, sizes[st], tw, sign, nlines, line_stride,
                       elem_stride, m_split, th)
    WGW_SYNC();
  }
}

// ---------------------------------------------------------------- compile-time sizes
// The same transforms with N known at compile time: the radix plan, strides and
// every index division fold to constants.  Butterflies are mapped fastest, lines
// slowest.  NC = 0 selects the runtime-N versions above.
struct CPlan {
  int nst;
  int radix[6];
  int size[6];   // block size S at each stage
};

constexpr CPlan cplan(int n) {
  CPlan p{0, {0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}};
  int r = n;
  int S = n;
  const int order[5] = {8, 4, 2, 3, 5};
  while (r > 1) {
    int f = 0;
    for (int i = 0; i < 5 && f == 0; ++i)
      if (r % order[i] == 0) f = order[i];
    if (f == 0 || p.nst >= 6) return CPlan{-1, {0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}};
    p.radix[p.nst] = f;
    p.size[p.nst] = S;
    ++p.nst;
    S /= f;
    r /= f;
  }
  return p;
}

template <typename T, int N, int S, int R, bool DIF>
WGW_HD void stage_c(cplx<T>* buf, const cplx<T>* tw, int sign, int nlines, int line_stride,
                    int elem_stride, int m_split, Thr th) {
  constexpr int M = S / R, step = N / S, NB = N / R;
  const int total = nlines * NB;
  for (int t = th.tid; t < total; t += th.nth) {
    const int b = t % NB, li = t / NB;
    const int j2 = b % M, blk = b / M;
    const int line = m_split >= 0 ? split_line(li, m_split, N) : li;
    cplx<T>* base = buf + (size_t)line * line_stride + (size_t)(blk * S + j2) * elem_stride;
    cplx<T> v[R];
    if constexpr (DIF) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = base[(size_t)r * M * elem_stride];
      dft_fixed<T, R>(v, sign);
      base[0] = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> x = v[r];
        if (M > 1 && j2) x = cmul(x, twiddle(tw, step * j2 * r, sign));
        base[(size_t)r * M * elem_stride] = x;
      }
    } else {
      v[0] = base[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cplx<T> x = base[(size_t)r * M * elem_stride];
        if (M > 1 && j2) x = cmul(x, twiddle(tw, step * j2 * r, sign));
        v[r] = x;
      }
      dft_fixed<T, R>(v, sign);
#pragma unroll
      for (int r = 0; r < R; ++r) base[(size_t)r * M * elem_stride] = v[r];
    }
  }
}

template <typename T, int N, int ST>
WGW_HD void dif_stages_c(cplx<T>* buf, const cplx<T>* tw, int sign, int nlines, int ls, int es,
                         int m_split, Thr th) {
  constexpr CPlan P = cplan(N);
  if constexpr (ST < P.nst) {
    stage_c<T, N, P.size[ST], P.radix[ST], true>(buf, tw, sign, nlines, ls, es, m_split, th);
    WGW_SYNC();
    dif_stages_c<T, N, ST + 1>(buf, tw, sign, nlines, ls, es, m_split, th);
  }
}

template <typename T, int N, int ST>
WGW_HD void dit_stages_c(cplx<T>* buf, const cplx<T>* tw, int sign, int nlines, int ls, int es,
                         int m_split, Thr th) {
  constexpr CPlan P = cplan(N);
  if constexpr (ST >= 0) {
    stage_c<T, N, P.size[ST], P.radix[ST], false>(buf, tw, sign, nlines, ls, es, m_split, th);
    WGW_SYNC();
    dit_stages_c<T, N, ST - 1>(buf, tw, sign, nlines, ls, es, m_split, th);
  }
}

// Dispatch: NC > 0 uses the compile-time transforms (p must describe N = NC).
template <typename T, int NC>
WGW_HD void fft_dif_n(cplx<T>* buf, const FftPlan& p, const cplx<T>* tw, int sign, int nlines,
                      int line_stride, int elem_stride, int m_split, Thr th) {
  if constexpr (NC > 0) {
    dif_stages_c<T, NC, 0>(buf, tw, sign, nlines, line_stride, elem_stride, m_split, th);
  } else {
    fft_dif<T>(buf, p, tw, sign, nlines, line_stride, elem_stride, m_split, th);
  }
}

template <typename T, int NC>
WGW_HD void fft_dit_n(cplx<T>* buf, const FftPlan& p, const cplx<T>* tw, int sign, int nlines,
                      int line_stride, int elem_stride, int m_split, Thr th) {
  if constexpr (NC > 0) {
    dit_stages_c<T, NC, cplan(NC).nst - 1>(buf, tw, sign, nlines, line_stride, elem_stride, m_split, th);
  } else {
    fft_dit<T>(buf, p, tw, sign, nlines, line_stride, elem_stride, m_split, th);
  }
}

// ---------------------------------------------------------------- register-resident lines
// One line of compile-time length N held by one thread (v[0..N-1], kept in registers once the
// loops are unrolled): the same stages as dif_stages_c / dit_stages_c, so the same
// digit-reversed positions, with every index and twiddle index a compile-time constant.
template <typename T, int N, int ST, int SIGN, bool PK = false>
WGW_HD void reg_dif(cplx<T>* v, const cplx<T>* tw) {
  constexpr CPlan P = cplan(N);
  if constexpr (ST < P.nst) {
    constexpr int S = P.size[ST], R = P.radix[ST], M = S / R, step = N / S;
#pragma unroll
    for (int blk = 0; blk < N / S; ++blk) {
#pragma unroll
      for (int j2 = 0; j2 < M; ++j2) {
        cplx<T> u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = v[blk * S + j2 + r * M];
        dft_fixed<T, R, PK>(u, SIGN);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          cplx<T> x = u[r];
          if (r > 0 && j2 > 0) x = cmul(x, twiddle(tw, step * j2 * r, SIGN));
          v[blk * S + j2 + r * M] = x;
        }
      }
    }
    reg_dif<T, N, ST + 1, SIGN, PK>(v, tw);
  }
}

template <typename T, int N, int ST, int SIGN, bool PK = false>
WGW_HD void reg_dit(cplx<T>* v, const cplx<T>* tw) {
  constexpr CPlan P = cplan(N);
  if constexpr (ST >= 0) {
    constexpr int S = P.size[ST], R = P.radix[ST], M = S / R, step = N / S;
#pragma unroll
    for (int blk = 0; blk < N / S; ++blk) {
#pragma unroll
      for (int j2 = 0; j2 < M; ++j2) {
        cplx<T> u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          cplx<T> x = v[blk * S + j2 + r * M];
          if (r > 0 && j2 > 0) x = cmul(x, twiddle(tw, step * j2 * r, SIGN));
          u[r] = x;
        }
        dft_fixed<T, R, PK>(u, SIGN);
#pragma unroll
        for (int r = 0; r < R; ++r) v[blk * S + j2 + r * M] = u[r];
      }
    }
    reg_dit<T, N, ST - 1, SIGN, PK>(v, tw);
  }
}

// Digit-reversed storage position of natural index n (host and device).
WGW_HD int fft_position(const FftPlan& p, int n) {
  int pos = 0, N = p.n;
  for (int st = 0; st < p.nst; ++st) {
    const int R = p.radix[st];
    N /= R;
    pos += N * (n % R);
    n /= R;
  }
  return pos;
}

}  // namespace wgw
