// Bodies of the pruned 3D FFT kernels (dual-space H application, Sec. 4.1).
//
// A "pair" packs two real-in-r functions a(r), b(r) into one complex grid
// z = a + i b (Gamma point).  In reciprocal space a function is held in the
// real plane-wave basis: element 0 = f(G=0) (real), elements 2j-1, 2j =
// sqrt2 Re f(G_j), sqrt2 Im f(G_j) for the j-th positive member G_j of the
// sphere (positive members numbered plane by plane in ascending (h, k, l)).
// With Z(G) = A(G) + i B(G):
//   Z(+G_j) = [(ar - bi) + i (ai + br)] / sqrt2,  Z(-G_j) = [(ar + bi) + i (br - ai)] / sqrt2,
//   A(G_j) = [Z(G_j) + Z(-G_j)^*] / 2,  B(G_j) = [Z(G_j) - Z(-G_j)^*] / (2i).
//
// The transform G -> r of a sphere of radius m (in every Miller index) runs
// along z on the 2m+1 rows |k| <= m of each plane h, then along y on the
// whole plane (plane kernel), then along x for each (y, z) on the 2m+1
// non-zero h (x-line kernel).  Between the kernels the data of one pair is
// T[h + m][y][z] (2m+1 planes of N x N complex, y and z in digit-reversed
// position).  Real-space arrays are [y][x][z] with all three coordinates in
// digit-reversed position (z fastest, so that threads that own consecutive
// x-lines (y, z) read and write consecutive addresses for every x).
//
// Every body has a storage type T (of the sphere vectors and real-space arrays
// in global memory) and a compute type C (of the butterflies, the twiddles,
// shared memory and the pair intermediate T[h][y][z]); C = T except for the
// float-float instances (T = double, C = ff).  Values cross between the two
// only where global T arrays are read or written.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "fft.cuh"

namespace wgw {

// Real-space arrays of the float-float passes hold float-float pairs in the 8-byte slots of their
// FP64 buffers (produced and consumed only by those passes), so that no element is converted on
// the FP64 pipe; every other pass stores T.
template <typename C, typename T>
WGW_HD C rs_ld(const T* p, size_t i) { return C(p[i]); }
template <>
WGW_HD ff rs_ld<ff, double>(const double* p, size_t i) { return reinterpret_cast<const ff*>(p)[i]; }
template <typename C, typename T>
WGW_HD void rs_st(T* p, size_t i, C v) { p[i] = T(v); }
template <>
WGW_HD void rs_st<ff, double>(double* p, size_t i, ff v) { reinterpret_cast<ff*>(p)[i] = v; }

// Strided batch of real-basis vectors: system s at base + s * ld.
template <typename T>
struct VecBatch {
  T* p;
  long ld;
  int n_sys;
};

// Per-system activity (null = all active).
WGW_HD bool is_active(const int* active, int s) { return active == nullptr || active[s] != 0; }

// Members of pair q: entries 2q and 2q+1 of a system list (null = identity) of n_list
// entries; the second member is -1 when 2q+1 >= n_list.  A list compacted on the device holds
// -1 past its count: s0 = -1 marks a pair the kernels skip.
WGW_HD void pair_members(const int* list, int n_list, int q, int& s0, int& s1) {
  s0 = list ? list[2 * q] : 2 * q;
  s1 = 2 * q + 1 < n_list ? (list ? list[2 * q + 1] : 2 * q + 1) : -1;
}

// Sphere points of a pair into shared memory, entries [e0, e1) of the plane tables: each thread
// takes kScatterBatch entries per round and issues all their global loads (table entry, then the
// four coefficients) before its first shared-memory store, so that the loads of a round are in
// flight together; a one-entry loop serialises a dependent load pair per entry, and that latency
// bounded the G -> r plane kernels.  Every entry lands in its own slot, so the result does not
// depend on the order.  put(e, en.x, z) stores value z of entry e.
// The float-float shared-memory kernels keep the one-entry loops: batching measured slower there
// (r -> G -12 %, G -> r -3 % on the 48^3 block; their time goes to float-float arithmetic).
template <typename C>
constexpr bool kBatchLoads = !std::is_same<C, ff>::value;
constexpr int kScatterBatch = 4;
template <typename T, typename C, typename PUT>
WGW_HD void scatter_pair(const SphereTab& sp, int e0, int e1, const T* x0, const T* x1, bool has1, PUT put,
                         Thr th) {
  const C s = C(kInvSqrt2);
  for (int base = e0 + th.tid; base < e1; base += kScatterBatch * th.nth) {
    int2 en[kScatterBatch];
    C ar[kScatterBatch], ai[kScatterBatch], br[kScatterBatch], bi[kScatterBatch];
#pragma unroll
    for (int q = 0; q < kScatterBatch; ++q) {
      const int e = base + q * th.nth;
      en[q] = e < e1 ? sp.ent[e] : int2{0, -1};
    }
#pragma unroll
    for (int q = 0; q < kScatterBatch; ++q) {
      const int j = en[q].y;
      const int i0 = j > 0 ? 2 * j - 1 : 0, i1 = j > 0 ? 2 * j : 0;
      ar[q] = ai[q] = br[q] = bi[q] = C(0);
      if (j >= 0) {
        ar[q] = C(x0[i0]);
        if (j > 0) ai[q] = C(x0[i1]);
        if (has1) {
          br[q] = C(x1[i0]);
          if (j > 0) bi[q] = C(x1[i1]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kScatterBatch; ++q) {
      const int j = en[q].y;
      if (j < 0) continue;
      const int neg = (en[q].x >> 16) & 1;
      cplx<C> z;
      if (j == 0) z = mk<C>(ar[q], br[q]);
      else z = neg ? mk<C>((ar[q] + bi[q]) * s, (br[q] - ai[q]) * s) : mk<C>((ar[q] - bi[q]) * s, (ai[q] + br[q]) * s);
      put(base + q * th.nth, en[q].x, z);
    }
  }
}

// G -> r along z then y for plane hi of one pair; writes T[hi] of that pair.
// smem: N * (N + 1) complex.
template <typename T, int NC = 0, typename C = T>
WGW_HD void plane_g2r_body(int pair, int hi, const SphereTab& sp, const FftPlan& pl,
                           const cplx<C>* tw, const T* X, long ldx, int n_list, const int* list,
                           cplx<C>* Tout, cplx<C>* B, Thr th) {
  const int N = NC > 0 ? NC : pl.n, LS = N + 1, m = sp.m;
  int s0, s1;
  pair_members(list, n_list, pair, s0, s1);
  const bool has1 = s1 >= 0;
  for (int i = th.tid; i < N * LS; i += th.nth) B[i] = mk<C>(C(0), C(0));
  WGW_SYNC();
  const T* x0 = X + (size_t)s0 * ldx;
  const T* x1 = X + (size_t)(has1 ? s1 : s0) * ldx;
  if constexpr (kBatchLoads<C>) {
    scatter_pair<T, C>(sp, sp.plane_off[hi], sp.plane_off[hi + 1], x0, x1, has1,
                       [&](int, int ex, cplx<C> z) { B[(ex & 0xff) * LS + ((ex >> 8) & 0xff)] = z; }, th);
  } else {
    const C s = C(kInvSqrt2);
    for (int e = sp.plane_off[hi] + th.tid; e < sp.plane_off[hi + 1]; e += th.nth) {
      const int2 en = sp.ent[e];
      const int kk = en.x & 0xff, ll = (en.x >> 8) & 0xff, neg = (en.x >> 16) & 1;
      const int j = en.y;
      cplx<C> z;
      if (j == 0) {
        z = mk<C>(C(x0[0]), has1 ? C(x1[0]) : C(0));
      } else {
        const C ar = C(x0[2 * j - 1]), ai = C(x0[2 * j]);
        const C br = has1 ? C(x1[2 * j - 1]) : C(0), bi = has1 ? C(x1[2 * j]) : C(0);
        z = neg ? mk<C>((ar + bi) * s, (br - ai) * s) : mk<C>((ar - bi) * s, (ai + br) * s);
      }
      B[kk * LS + ll] = z;
    }
  }
  WGW_SYNC();
  fft_dif_n<C, NC>(B, pl, tw, +1, 2 * m + 1, LS, 1, m, th);   // rows |k| <= m, along l -> z
  fft_dif_n<C, NC>(B, pl, tw, +1, N, 1, LS, -1, th);          // columns z, along k -> y
  cplx<C>* out = Tout + ((size_t)pair * (2 * m + 1) + hi) * N * N;
  for (int i = th.tid; i < N * N; i += th.nth) {
    const int y = i / N, z = i % N;
    out[i] = B[y * LS + z];
  }
}

// Register-resident form of plane_g2r_body (compile-time N) for planes hi0 .. hi0+np-1 of one
// pair: the rows |k| <= m of each plane are transformed along l -> z one row per thread,
// exchanged once through shared memory, then the N columns z of each plane along k -> y one
// column per thread, written straight to T[hi][y][z].  Several planes per block keep the
// threads busy in both phases (2m+1 rows, N columns per plane).
// smem B: np x (2m+1) x (N+1) complex, row kr = k + m of plane p at (p (2m+1) + kr) (N+1).

// PK: packed FP32 butterflies (cadd / csub / cscl of common.cuh) in the line transforms.
template <typename T, int N, typename C, bool PK = false>
WGW_HD void plane_g2r_reg_body(int pair, int hi0, int np, const SphereTab& sp, const cplx<C>* tw, const T* X,
                               long ldx, int n_list, const int* list, cplx<C>* Tout, cplx<C>* B, Thr th) {
  const int m = sp.m, NR = 2 * m + 1, LS = N + 1;
  int s0, s1;
  pair_members(list, n_list, pair, s0, s1);
  const bool has1 = s1 >= 0;
  for (int i = th.tid; i < np * NR * LS; i += th.nth) B[i] = mk<C>(C(0), C(0));
  WGW_SYNC();
  const T* x0 = X + (size_t)s0 * ldx;
  const T* x1 = X + (size_t)(has1 ? s1 : s0) * ldx;
  // The np planes' entries are contiguous in the tables: one scatter over all of them, the plane
  // of an entry found from the plane offsets.
  const int e_lo = sp.plane_off[hi0], e_hi = sp.plane_off[hi0 + np];
  scatter_pair<T, C>(sp, e_lo, e_hi, x0, x1, has1, [&](int e, int ex, cplx<C> z) {
    int p = 0;
    while (p + 1 < np && e >= sp.plane_off[hi0 + p + 1]) ++p;
    const int kk = ex & 0xff, ll = (ex >> 8) & 0xff;
    const int kr = kk <= m ? kk + m : kk - N + m;
    B[((size_t)p * NR + kr) * LS + ll] = z;
  }, th);
  WGW_SYNC();
  for (int t = th.tid; t < np * NR; t += th.nth) {   // rows: l -> z
    cplx<C>* row = B + (size_t)t * LS;
    cplx<C> v[N];
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = row[x];
    reg_dif<C, N, 0, +1, PK>(v, tw);
#pragma unroll
    for (int x = 0; x < N; ++x) row[x] = v[x];
  }
  WGW_SYNC();
  for (int t = th.tid; t < np * N; t += th.nth) {    // columns: k -> y
    const int p = t / N, zc = t % N;
    const cplx<C>* Bp = B + (size_t)p * NR * LS;
    cplx<C> v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) {
      const int kr = y <= m ? y + m : (y >= N - m ? y - N + m : -1);
      v[y] = kr >= 0 ? Bp[kr * LS + zc] : mk<C>(C(0), C(0));
    }
    reg_dif<C, N, 0, +1, PK>(v, tw);
    cplx<C>* out = Tout + ((size_t)pair * NR + hi0 + p) * N * N;
#pragma unroll
    for (int y = 0; y < N; ++y) out[(size_t)y * N + zc] = v[y];
  }
}

// x-line kernel modes.
enum XMode : int {
  XM_APPLY_V = 0,    // G->r along x, multiply by V(r), r->G along x (in place in T)
  XM_TO_REAL = 1,    // G->r along x, write Re / Im to real-space arrays R0 / R1
  XM_FROM_REAL = 2,  // read a0*b0 + i a1*b1 from real-space arrays, r->G along x into T
};

template <typename T>
struct XArgs {
  int mode;
  const T* V;              // APPLY_V: real-space potential [y][x][z]
  T* R0; T* R1;            // TO_REAL outputs (R1 may be null)
  long ldr;                // stride between real-space arrays of successive systems
  const T* A; const T* Bm; // FROM_REAL factors (Bm may be null = 1)
  long lda, ldb;           // per-system strides of A and Bm
  const int* a_index;      // FROM_REAL: index of the A array of system s (null = s)
  const int* b_index;      // FROM_REAL: index of the Bm array of system s (null = s)
  int n_sys;               // entries of the system list (pairs = (n_sys + 1) / 2)
  const int* list;         // system list (null = identity)
};

// One (pair, y) slab: S[z][x], N x (N + 1) complex.
template <typename T, int NC = 0, typename C = T>
WGW_HD void xline_body(int pair, int y, int m, const FftPlan& pl, const cplx<C>* tw,
                       cplx<C>* Tbuf, const XArgs<T>& a, cplx<C>* S, Thr th) {
  const int N = NC > 0 ? NC : pl.n, LS = N + 1, NP = 2 * m + 1;
  int s0, s1;
  pair_members(a.list, a.n_sys, pair, s0, s1);
  const bool has1 = s1 >= 0;
  cplx<C>* tp = Tbuf + (size_t)pair * NP * N * N + (size_t)y * N;   // T[hi][y][z] at tp[hi*N*N + z]
  const size_t slab = (size_t)y * N * N;                              // real-space [y][x][z] offset
  if (a.mode == XM_FROM_REAL) {
    const T* A0 = a.A + (size_t)(a.a_index ? a.a_index[s0] : s0) * a.lda + slab;
    const T* A1 = has1 ? a.A + (size_t)(a.a_index ? a.a_index[s1] : s1) * a.lda + slab : nullptr;
    const T* B0 = a.Bm ? a.Bm + (size_t)(a.b_index ? a.b_index[s0] : s0) * a.ldb + slab : nullptr;
    const T* B1 = (a.Bm && has1) ? a.Bm + (size_t)(a.b_index ? a.b_index[s1] : s1) * a.ldb + slab : nullptr;
    for (int i = th.tid; i < N * N; i += th.nth) {
      const int x = i / N, z = i % N;
      C re = rs_ld<C>(A0, i), im = A1 ? rs_ld<C>(A1, i) : C(0);
      if (B0) re = re * rs_ld<C>(B0, i);
      if (B1) im = im * rs_ld<C>(B1, i);
      S[z * LS + x] = mk<C>(re, im);
    }
    WGW_SYNC();
  } else {
    for (int i = th.tid; i < N * LS; i += th.nth) S[i] = mk<C>(C(0), C(0));
    WGW_SYNC();
    for (int i = th.tid; i < NP * N; i += th.nth) {
      const int hi = i / N, z = i % N;
      const int x = (hi - m + N) % N;
      S[z * LS + x] = tp[(size_t)hi * N * N + z];
    }
    WGW_SYNC();
    fft_dif_n<C, NC>(S, pl, tw, +1, N, LS, 1, -1, th);
  }
  if (a.mode == XM_TO_REAL) {
    T* r0 = a.R0 + (size_t)s0 * a.ldr + slab;
    T* r1 = (has1 && a.R1) ? a.R1 + (size_t)s1 * a.ldr + slab : nullptr;
    for (int i = th.tid; i < N * N; i += th.nth) {
      const int x = i / N, z = i % N;
      const cplx<C> v = S[z * LS + x];
      rs_st<C>(r0, i, v.re);
      if (r1) rs_st<C>(r1, i, v.im);
    }
    return;
  }
  if (a.mode == XM_APPLY_V) {
    const T* v = a.V + slab;
    for (int i = th.tid; i < N * N; i += th.nth) {
      const int x = i / N, z = i % N;
      S[z * LS + x] = cscale(S[z * LS + x], rs_ld<C>(v, i));
    }
    WGW_SYNC();
  }
  fft_dit_n<C, NC>(S, pl, tw, -1, N, LS, 1, -1, th);
  for (int i = th.tid; i < NP * N; i += th.nth) {
    const int hi = i / N, z = i % N;
    const int x = (hi - m + N) % N;
    tp[(size_t)hi * N * N + z] = S[z * LS + x];
  }
}

// The x-line pass with one line per thread held in registers (compile-time N): line l = y N + z
// of pair `pair`, same modes, layouts and positions as xline_body.  The pair intermediate is
// read and written at T[hi][l], so consecutive threads touch consecutive addresses.
template <typename T, int N, typename C, bool PK = false>
WGW_HD void xline_reg_body(int pair, int l, int m, const cplx<C>* tw, cplx<C>* Tbuf, const XArgs<T>& a) {
  const int NP = 2 * m + 1;
  int s0, s1;
  pair_members(a.list, a.n_sys, pair, s0, s1);
  const bool has1 = s1 >= 0;
  cplx<C>* tp = Tbuf + (size_t)pair * NP * N * N + l;   // T[hi][y][z] at tp[hi * N * N]
  const size_t line = (size_t)(l / N) * N * N + (l % N); // real-space [y][x][z]: element x at line + x N
  cplx<C> v[N];
  if (a.mode == XM_FROM_REAL) {
    const T* A0 = a.A + (size_t)(a.a_index ? a.a_index[s0] : s0) * a.lda + line;
    const T* A1 = has1 ? a.A + (size_t)(a.a_index ? a.a_index[s1] : s1) * a.lda + line : nullptr;
    const T* B0 = a.Bm ? a.Bm + (size_t)(a.b_index ? a.b_index[s0] : s0) * a.ldb + line : nullptr;
    const T* B1 = (a.Bm && has1) ? a.Bm + (size_t)(a.b_index ? a.b_index[s1] : s1) * a.ldb + line : nullptr;
#pragma unroll
    for (int x = 0; x < N; ++x) {
      C re = rs_ld<C>(A0, (size_t)x * N), im = A1 ? rs_ld<C>(A1, (size_t)x * N) : C(0);
      if (B0) re = re * rs_ld<C>(B0, (size_t)x * N);
      if (B1) im = im * rs_ld<C>(B1, (size_t)x * N);
      v[x] = mk<C>(re, im);
    }
  } else {
#pragma unroll
    for (int x = 0; x < N; ++x) {
      // natural index x <-> Miller h = x (x <= m) or x - N (x >= N - m); plane hi = h + m
      const bool in = x <= m || x >= N - m;
      const int hi = x <= m ? x + m : x - N + m;
      v[x] = in ? tp[(size_t)hi * N * N] : mk<C>(C(0), C(0));
    }
    reg_dif<C, N, 0, +1, PK>(v, tw);
  }
  if (a.mode == XM_TO_REAL) {
    T* r0 = a.R0 + (size_t)s0 * a.ldr + line;
    T* r1 = (has1 && a.R1) ? a.R1 + (size_t)s1 * a.ldr + line : nullptr;
#pragma unroll
    for (int x = 0; x < N; ++x) {
      rs_st<C>(r0, (size_t)x * N, v[x].re);
      if (r1) rs_st<C>(r1, (size_t)x * N, v[x].im);
    }
    return;
  }
  if (a.mode == XM_APPLY_V) {
    const T* vr = a.V + line;
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = cscale(v[x], rs_ld<C>(vr, (size_t)x * N));
  }
  reg_dit<C, N, cplan(N).nst - 1, -1, PK>(v, tw);
#pragma unroll
  for (int x = 0; x < N; ++x) {
    const bool in = x <= m || x >= N - m;
    const int hi = x <= m ? x + m : x - N + m;
    if (in) tp[(size_t)hi * N * N] = v[x];
  }
}

// Epilogue of the r -> G plane kernel, per real-basis element i of system s:
//   out[s][i] = vcoef * F[i] + (kin * g2[i] + shift[s]) * pin[s][i]   (pin may be null)
// where F is the transformed function (already scaled by 1/N^3).
template <typename T>
struct Epi {
  T* out; long ldo;
  const T* pin; long ldp;
  T vcoef;
  T kin;
  const T* shift;          // per system (null = 0)
  int n_sys;               // entries of the system list
  const int* active;
  const int* list;         // system list (null = identity)
};

// 0.5 |G|^2 of element i in compute type C (FP32 kernels read the FP32 copy).
template <typename C>
WGW_HD C g2_as(const SphereTab& sp, int i) { return C(sp.g2[i]); }
template <>
WGW_HD float g2_as<float>(const SphereTab& sp, int i) { return sp.g2f[i]; }

template <typename T, typename C>
WGW_HD void epi_store(const Epi<T>& e, const SphereTab& sp, int s, int i, C f) {
  C v = C(e.vcoef) * f;
  if (e.pin) {
    C c = C(e.kin) * g2_as<C>(sp, i);
    if (e.shift) c += C(e.shift[s]);
    v += c * C(e.pin[(size_t)s * e.ldp + i]);
  }
  e.out[(size_t)s * e.ldo + i] = T(v);
}

// Unpack one pair of values Z(G_j), Z(-G_j) into the two systems' real-basis elements.
template <typename T, typename C>
WGW_HD void unpack_store(const Epi<T>& ep, const SphereTab& sp, int s0, int s1, bool act0, bool act1,
                         int j, cplx<C> zp, cplx<C> zm, C scale) {
  const C a = zp.re, b = zp.im, c = zm.re, d = zm.im;
  // A(G_j) = ((a + c) + i (b - d)) / 2,  B(G_j) = ((b + d) - i (a - c)) / 2
  const C hs = C(0.5) * scale * C(kSqrt2);
  if (act0) {
    epi_store(ep, sp, s0, 2 * j - 1, (a + c) * hs);
    epi_store(ep, sp, s0, 2 * j, (b - d) * hs);
  }
  if (act1) {
    epi_store(ep, sp, s1, 2 * j - 1, (b + d) * hs);
    epi_store(ep, sp, s1, 2 * j, (c - a) * hs);
  }
}

// The epilogue inputs of one pair j (elements 2j-1, 2j of both systems): kin g2 + shift and pin,
// read before any output of the pair is written (the compiler cannot move a load of pin above a
// store to out, which may alias it, so epi_store's load-store sequence waits on every load).
template <typename C>
struct EpiIn {
  C c0[2], c1[2], p0[2], p1[2];
};

template <typename T, typename C>
WGW_HD EpiIn<C> epi_load(const Epi<T>& e, const SphereTab& sp, int s0, int s1, bool act0, bool act1, int j) {
  EpiIn<C> r;
#pragma unroll
  for (int q = 0; q < 2; ++q) r.c0[q] = r.c1[q] = r.p0[q] = r.p1[q] = C(0);
  if (!e.pin) return r;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int i = 2 * j - 1 + q;
    const C g = C(e.kin) * g2_as<C>(sp, i);
    r.c0[q] = r.c1[q] = g;
    if (act0) {
      if (e.shift) r.c0[q] += C(e.shift[s0]);
      r.p0[q] = C(e.pin[(size_t)s0 * e.ldp + i]);
    }
    if (act1) {
      if (e.shift) r.c1[q] += C(e.shift[s1]);
      r.p1[q] = C(e.pin[(size_t)s1 * e.ldp + i]);
    }
  }
  return r;
}

// epi_store with its inputs already loaded: the same arithmetic.
template <typename T, typename C>
WGW_HD void epi_store_in(const Epi<T>& e, int s, int i, C f, C c, C p) {
  C v = C(e.vcoef) * f;
  if (e.pin) v += c * p;
  e.out[(size_t)s * e.ldo + i] = T(v);
}

// unpack_store with loaded epilogue inputs.
template <typename T, typename C>
WGW_HD void unpack_store_in(const Epi<T>& ep, int s0, int s1, bool act0, bool act1, int j, cplx<C> zp,
                            cplx<C> zm, C scale, const EpiIn<C>& in) {
  const C a = zp.re, b = zp.im, c = zm.re, d = zm.im;
  const C hs = C(0.5) * scale * C(kSqrt2);
  if (act0) {
    epi_store_in(ep, s0, 2 * j - 1, (a + c) * hs, in.c0[0], in.p0[0]);
    epi_store_in(ep, s0, 2 * j, (b - d) * hs, in.c0[1], in.p0[1]);
  }
  if (act1) {
    epi_store_in(ep, s1, 2 * j - 1, (b + d) * hs, in.c1[0], in.p1[0]);
    epi_store_in(ep, s1, 2 * j, (c - a) * hs, in.c1[1], in.p1[1]);
  }
}

// Gather, unpack and epilogue of cnt sphere pairs: pair t has table entries ea(t) (the member G_j)
// and eb(t) (its mirror), values zp(t, ea), zm(t, eb).  Each thread takes kGatherBatch pairs per
// round: their table entries first, then their epilogue inputs, then the stores, so that the
// loads of a round are in flight together.
constexpr int kGatherBatch = 2;
template <typename T, typename C, typename EA, typename EB, typename ZP, typename ZM>
WGW_HD void gather_pairs(const Epi<T>& ep, const SphereTab& sp, int s0, int s1, bool act0, bool act1, int cnt,
                         C scale, EA ea, EB eb, ZP zp, ZM zm, Thr th) {
  for (int t0 = th.tid; t0 < cnt; t0 += kGatherBatch * th.nth) {
    int2 a[kGatherBatch], b[kGatherBatch];
#pragma unroll
    for (int q = 0; q < kGatherBatch; ++q) {
      const int t = t0 + q * th.nth;
      a[q] = b[q] = int2{0, -1};
      if (t < cnt) { a[q] = ea(t); b[q] = eb(t); }
    }
    EpiIn<C> in[kGatherBatch];
#pragma unroll
    for (int q = 0; q < kGatherBatch; ++q)
      if (a[q].y >= 0) in[q] = epi_load<T, C>(ep, sp, s0, s1, act0, act1, a[q].y);
#pragma unroll
    for (int q = 0; q < kGatherBatch; ++q) {
      const int t = t0 + q * th.nth;
      if (a[q].y >= 0)
        unpack_store_in(ep, s0, s1, act0, act1, a[q].y, zp(t, a[q]), zm(t, b[q]), scale, in[q]);
    }
  }
}

// r -> G along y then z for plane hi of one pair (in B), natural k, l afterwards.
template <typename C, int NC = 0>
WGW_HD void plane_r2g_load(int pair, int hi, const SphereTab& sp, const FftPlan& pl,
                           const cplx<C>* tw, const cplx<C>* Tin, cplx<C>* B, Thr th) {
  const int N = NC > 0 ? NC : pl.n, LS = N + 1, m = sp.m, NP = 2 * m + 1;
  const cplx<C>* in = Tin + ((size_t)pair * NP + hi) * N * N;
  for (int i = th.tid; i < N * N; i += th.nth) {
    const int y = i / N, z = i % N;
    B[y * LS + z] = in[i];
  }
  WGW_SYNC();
  fft_dit_n<C, NC>(B, pl, tw, -1, N, 1, LS, -1, th);          // columns z: y -> k (natural)
  fft_dit_n<C, NC>(B, pl, tw, -1, 2 * m + 1, LS, 1, m, th);   // rows |k| <= m: z -> l (natural)
}

WGW_HD int ent_pos(int2 en, int LS) { return (en.x & 0xff) * LS + ((en.x >> 8) & 0xff); }

// r -> G for planes +hp and -hp of one pair, gather the sphere, unpack, epilogue.
// smem: N * (N + 1) complex for the plane + npt_max complex (values of plane +hp).
template <typename T, int NC = 0, typename C = T>
WGW_HD void plane_r2g_body(int pair, int hp, const SphereTab& sp, const FftPlan& pl,
                           const cplx<C>* tw, const cplx<C>* Tin, const Epi<T>& ep,
                           cplx<C>* B, cplx<C>* Zp, Thr th) {
  const int N = NC > 0 ? NC : pl.n, LS = N + 1, m = sp.m;
  int s0, s1;
  pair_members(ep.list, ep.n_sys, pair, s0, s1);
  const bool has1 = s1 >= 0;
  const bool act0 = is_active(ep.active, s0), act1 = has1 && is_active(ep.active, s1);
  const C scale = C(1.0 / ((double)N * N * N));
  const int off_p = sp.plane_off[m + hp];
  const int cnt = sp.plane_off[m + hp + 1] - off_p;
  plane_r2g_load<C, NC>(pair, m + hp, sp, pl, tw, Tin, B, th);
  if (hp == 0) {
    // Plane 0 lists [G = 0, K positives, K mirrors].
    const int K = (cnt - 1) / 2;
    if constexpr (kBatchLoads<C>) {
      gather_pairs(ep, sp, s0, s1, act0, act1, K, scale, [&](int t) { return sp.ent[off_p + 1 + t]; },
                   [&](int t) { return sp.ent[off_p + 1 + K + t]; },
                   [&](int, int2 e) { return B[ent_pos(e, LS)]; }, [&](int, int2 e) { return B[ent_pos(e, LS)]; }, th);
    } else {
      for (int t = th.tid; t < K; t += th.nth) {
        const int2 ep_ = sp.ent[off_p + 1 + t];
        unpack_store(ep, sp, s0, s1, act0, act1, ep_.y, B[ent_pos(ep_, LS)],
                     B[ent_pos(sp.ent[off_p + 1 + K + t], LS)], scale);
      }
    }
    if (th.tid == 0) {
      const cplx<C> z0 = B[ent_pos(sp.ent[off_p], LS)];
      if (act0) epi_store(ep, sp, s0, 0, z0.re * scale);
      if (act1) epi_store(ep, sp, s1, 0, z0.im * scale);
    }
    return;
  }
  for (int t = th.tid; t < cnt; t += th.nth) Zp[t] = B[ent_pos(sp.ent[off_p + t], LS)];
  WGW_SYNC();
  const int off_m = sp.plane_off[m - hp];
  plane_r2g_load<C, NC>(pair, m - hp, sp, pl, tw, Tin, B, th);
  if constexpr (kBatchLoads<C>) {
    gather_pairs(ep, sp, s0, s1, act0, act1, cnt, scale, [&](int t) { return sp.ent[off_p + t]; },
                 [&](int t) { return sp.ent[off_m + t]; }, [&](int t, int2) { return Zp[t]; },
                 [&](int, int2 e) { return B[ent_pos(e, LS)]; }, th);
  } else {
    for (int t = th.tid; t < cnt; t += th.nth) {
      unpack_store(ep, sp, s0, s1, act0, act1, sp.ent[off_p + t].y, Zp[t],
                   B[ent_pos(sp.ent[off_m + t], LS)], scale);
    }
  }
}

// Register-resident r -> G of np planes hi[0..np) of one pair (compile-time N): the columns of
// every plane along y -> k one per thread straight from T[hi][y][z] (rows |k| <= m kept), one
// exchange through shared memory, then the rows along z -> l one per thread.  Leaves plane q in
// B + q (2m+1)(N+1) as B[k + m][l] (natural l).
template <typename C, int N, bool PK = false>
WGW_HD void plane_r2g_reg_load(int pair, const int* his, int np, int m, const cplx<C>* tw, const cplx<C>* Tin,
                               cplx<C>* B, Thr th) {
  const int NR = 2 * m + 1, LS = N + 1;
  for (int t = th.tid; t < np * N; t += th.nth) {
    const int q = t / N, zc = t % N;
    const cplx<C>* in = Tin + ((size_t)pair * NR + his[q]) * N * N;
    cplx<C>* Bq = B + (size_t)q * NR * LS;
    cplx<C> v[N];
#pragma unroll
    for (int y = 0; y < N; ++y) v[y] = in[(size_t)y * N + zc];
    reg_dit<C, N, cplan(N).nst - 1, -1, PK>(v, tw);
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (k <= m) Bq[(k + m) * LS + zc] = v[k];
      else if (k >= N - m) Bq[(k - N + m) * LS + zc] = v[k];
    }
  }
  WGW_SYNC();
  for (int t = th.tid; t < np * NR; t += th.nth) {
    cplx<C>* row = B + (size_t)t * LS;
    cplx<C> v[N];
#pragma unroll
    for (int x = 0; x < N; ++x) v[x] = row[x];
    reg_dit<C, N, cplan(N).nst - 1, -1, PK>(v, tw);
#pragma unroll
    for (int x = 0; x < N; ++x) row[x] = v[x];
  }
  WGW_SYNC();
}

template <int N>
WGW_HD int ent_pos_rows(int2 en, int m) {
  const int kk = en.x & 0xff;
  return (kk <= m ? kk + m : kk - N + m) * (N + 1) + ((en.x >> 8) & 0xff);
}

// plane_r2g_body with the register-resident load: planes +hp and -hp of one pair transformed
// together, then gathered, unpacked and passed through the epilogue.
// smem: 2 (2m+1)(N+1) complex.
template <typename T, int N, typename C, bool PK = false>
WGW_HD void plane_r2g_reg_body(int pair, int hp, const SphereTab& sp, const cplx<C>* tw, const cplx<C>* Tin,
                               const Epi<T>& ep, cplx<C>* B, Thr th) {
  const int m = sp.m, plane = (2 * m + 1) * (N + 1);
  int s0, s1;
  pair_members(ep.list, ep.n_sys, pair, s0, s1);
  const bool has1 = s1 >= 0;
  const bool act0 = is_active(ep.active, s0), act1 = has1 && is_active(ep.active, s1);
  const C scale = C(1.0 / ((double)N * N * N));
  const int off_p = sp.plane_off[m + hp];
  const int cnt = sp.plane_off[m + hp + 1] - off_p;
  const int his[2] = {m + hp, m - hp};
  plane_r2g_reg_load<C, N, PK>(pair, his, hp == 0 ? 1 : 2, m, tw, Tin, B, th);
  if (hp == 0) {
    const int K = (cnt - 1) / 2;
    gather_pairs(ep, sp, s0, s1, act0, act1, K, scale, [&](int t) { return sp.ent[off_p + 1 + t]; },
                 [&](int t) { return sp.ent[off_p + 1 + K + t]; },
                 [&](int, int2 e) { return B[ent_pos_rows<N>(e, m)]; },
                 [&](int, int2 e) { return B[ent_pos_rows<N>(e, m)]; }, th);
    if (th.tid == 0) {
      const cplx<C> z0 = B[ent_pos_rows<N>(sp.ent[off_p], m)];
      if (act0) epi_store(ep, sp, s0, 0, z0.re * scale);
      if (act1) epi_store(ep, sp, s1, 0, z0.im * scale);
    }
    return;
  }
  const int off_m = sp.plane_off[m - hp];
  gather_pairs(ep, sp, s0, s1, act0, act1, cnt, scale, [&](int t) { return sp.ent[off_p + t]; },
               [&](int t) { return sp.ent[off_m + t]; }, [&](int, int2 e) { return B[ent_pos_rows<N>(e, m)]; },
               [&](int, int2 e) { return B[plane + ent_pos_rows<N>(e, m)]; }, th);
}

// Density response of perturbation p on slab y (Eq. dfpt, one spin channel
// times f_s folded into coef):
//   D_p[y][x][z] = coef * sum_{v} psi_v(r) x_{(v,p)}(r),
// with systems ordered s = p * n_v + v and x_s(r) obtained from T by the
// G -> r pass along x.  The sum runs over v in a fixed order, so the result
// does not depend on how many perturbations share the launch.
// smem: N * (N + 1) complex + N * N real.
template <typename T, int NC = 0, typename C = T>
WGW_HD void drho_xline_body(int p, int y, int m, const FftPlan& pl, const cplx<C>* tw,
                            const cplx<C>* Tbuf, const T* psi_r, long ldpsi, int n_v, int n_sys,
                            T coef, T* D, long ldd, cplx<C>* S, C* acc, Thr th) {
  const int N = NC > 0 ? NC : pl.n, LS = N + 1, NP = 2 * m + 1;
  const size_t slab = (size_t)y * N * N;
  for (int i = th.tid; i < N * N; i += th.nth) acc[i] = C(0);
  const int s_lo = p * n_v, s_hi = (p + 1) * n_v;   // systems of p: [s_lo, s_hi)
  for (int q = s_lo / 2; 2 * q < s_hi; ++q) {
    for (int i = th.tid; i < N * LS; i += th.nth) S[i] = mk<C>(C(0), C(0));
    WGW_SYNC();
    const cplx<C>* tp = Tbuf + (size_t)q * NP * N * N + (size_t)y * N;
    for (int i = th.tid; i < NP * N; i += th.nth) {
      const int hi = i / N, z = i % N;
      S[z * LS + (hi - m + N) % N] = tp[(size_t)hi * N * N + z];
    }
    WGW_SYNC();
    fft_dif_n<C, NC>(S, pl, tw, +1, N, LS, 1, -1, th);
    const int sa = 2 * q, sb = 2 * q + 1;
    const bool ua = sa >= s_lo && sa < s_hi && sa < n_sys;
    const bool ub = sb >= s_lo && sb < s_hi && sb < n_sys;
    const T* pa = psi_r + (size_t)(sa - s_lo) * ldpsi + slab;
    const T* pb = psi_r + (size_t)(sb - s_lo) * ldpsi + slab;
    for (int i = th.tid; i < N * N; i += th.nth) {   // i = x N + z
      const cplx<C> v = S[(i % N) * LS + (i / N)];
      C a = acc[i];
      if (ua) a += rs_ld<C>(pa, i) * v.re;
      if (ub) a += rs_ld<C>(pb, i) * v.im;
      acc[i] = a;
    }
    WGW_SYNC();
  }
  T* d = D + (size_t)p * ldd + slab;
  for (int i = th.tid; i < N * N; i += th.nth) rs_st<C>(d, i, C(coef) * acc[i]);
}

}  // namespace wgw
