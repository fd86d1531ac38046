// Test-only host harness: steps the library's kernel bodies on the CPU (one
// "thread" per block, blocks in sequence) so that their index arithmetic can
// be checked against numpy and the oracle without a GPU.  It is built only by
// tests/test_emu_index.py and is not part of libwgw; the library itself has no
// host execution path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "fft_bodies.cuh"
#include "la_bodies.cuh"
#include "tables.h"

using namespace wgw;

namespace {

const Thr kOne = {0, 1};

struct Sph {
  SphereHostTables h;
  SphereTab tab() const {
    SphereTab t;
    t.m = h.m; t.n_pairs = h.n_pairs; t.plane_off = h.plane_off.data(); t.ent = h.ent.data();
    t.g2 = h.g2.data();
    t.g2f = h.g2f.data();
    return t;
  }
  RbMap map() const {
    RbMap r; r.n_pairs = h.n_pairs; r.i0 = &h.i0; r.pos = h.pos.data(); r.neg = h.neg.data();
    return r;
  }
};

template <typename T>
std::vector<cplx<T>> twiddles(int N) {
  std::vector<cplx<T>> tw(N);
  for (int k = 0; k < N; ++k) tw[k] = mk<T>((T)std::cos(2.0 * M_PI * k / N), (T)std::sin(2.0 * M_PI * k / N));
  return tw;
}

// When set, x-line passes at N = 24 go through the register-resident body.
bool g_reg = false;

template <typename T>
void run_xline(int q, int m, const FftPlan& pl, const std::vector<cplx<T>>& tw, cplx<T>* Tb, const XArgs<T>& a,
               cplx<T>* B) {
  const int N = pl.n;
  if (g_reg && N == 24) {
    for (int l = 0; l < N * N; ++l) xline_reg_body<T, 24, T>(q, l, m, tw.data(), Tb, a);
    return;
  }
  for (int y = 0; y < N; ++y) xline_body<T>(q, y, m, pl, tw.data(), Tb, a, B, kOne);
}

template <typename T>
void run_g2r(int q, int hi, const Sph& sp, const FftPlan& pl, const std::vector<cplx<T>>& tw, const T* X, long ldx,
             int n_sys, cplx<T>* Tb, cplx<T>* B) {
  if (g_reg && pl.n == 24) {
    // Blocks of three planes as on the device (the block starting at a multiple of 3 handles
    // planes hi0 .. hi0+2; called once per plane, it acts only at the block's first plane).
    if (hi % 3 == 0) {
      std::vector<cplx<T>> Bm((size_t)3 * (2 * sp.h.m + 1) * (pl.n + 1));
      plane_g2r_reg_body<T, 24, T>(q, hi, std::min(3, 2 * sp.h.m + 1 - hi), sp.tab(), tw.data(), X, ldx, n_sys,
                                   nullptr, Tb, Bm.data(), kOne);
    }
    return;
  }
  plane_g2r_body<T>(q, hi, sp.tab(), pl, tw.data(), X, ldx, n_sys, nullptr, Tb, B, kOne);
}

template <typename T>
void run_r2g(int q, int hp, const Sph& sp, const FftPlan& pl, const std::vector<cplx<T>>& tw, const cplx<T>* Tb,
             const Epi<T>& e, cplx<T>* B, cplx<T>* Zp) {
  if (g_reg && pl.n == 24) {
    std::vector<cplx<T>> B2((size_t)2 * (2 * sp.h.m + 1) * (pl.n + 1));
    plane_r2g_reg_body<T, 24, T>(q, hp, sp.tab(), tw.data(), Tb, e, B2.data(), kOne);
    return;
  }
  plane_r2g_body<T>(q, hp, sp.tab(), pl, tw.data(), Tb, e, B, Zp, kOne);
}

// G -> r of a batch of real-basis vectors (real-space arrays out[s], N^3 each).
template <typename T>
void to_real(const Sph& sp, const FftPlan& pl, const std::vector<cplx<T>>& tw, const T* X, long ldx,
             int n_sys, T* out) {
  const int N = pl.n, NP = 2 * sp.h.m + 1, pairs = (n_sys + 1) / 2;
  std::vector<cplx<T>> Tb((size_t)pairs * NP * N * N), B((size_t)N * (N + 1));
  for (int q = 0; q < pairs; ++q)
    for (int hi = 0; hi < NP; ++hi)
      run_g2r<T>(q, hi, sp, pl, tw, X, ldx, n_sys, Tb.data(), B.data());
  XArgs<T> a{};
  a.mode = XM_TO_REAL; a.R0 = out; a.R1 = out; a.ldr = (long)N * N * N; a.n_sys = n_sys;
  for (int q = 0; q < pairs; ++q) run_xline<T>(q, sp.h.m, pl, tw, Tb.data(), a, B.data());
}

template <typename T>
void sphere_to_rb_host(const Sph& sp, int n_sys, const double* c, long ldc, const double* scale, int part,
                       T* out, long ldo) {
  std::vector<double> tmp((size_t)n_sys * ldo, 0.0);
  for (int s = 0; s < n_sys; ++s)
    for (int i = 0; i < sp.h.nrb(); ++i) sphere_to_rb(s, c, ldc, scale, sp.map(), part, tmp.data(), ldo, i);
  for (size_t i = 0; i < tmp.size(); ++i) out[i] = (T)tmp[i];
}

// Storage type T, compute type C of the pipeline bodies (C = ff: float-float).
template <typename T, int NC = 0, typename C = T>
void apply_h_impl(double L, double ecut, int N, const double* vloc_c, int n_sys, const double* Xd,
                  const double* shift, double* outd, bool reg = false) {
  Sph w, r;
  build_sphere(L, ecut, N, w.h);
  build_sphere(L, 4 * ecut, N, r.h);
  FftPlan pl;
  make_plan(N, pl);
  auto tws = twiddles<T>(N);
  auto tw = twiddles<C>(N);
  const long N3 = (long)N * N * N;
  const int nw = w.h.nrb(), nr = r.h.nrb();
  std::vector<T> vrb(nr), vr(N3);
  sphere_to_rb_host<T>(r, 1, vloc_c, 2L * r.h.n, nullptr, 0, vrb.data(), nr);
  to_real<T>(r, pl, tws, vrb.data(), nr, 1, vr.data());
  if constexpr (std::is_same<C, ff>::value) {
    // float-float passes read real-space arrays as float-float pairs (in the FP64 slots)
    for (size_t i = 0; i < vr.size(); ++i) reinterpret_cast<ff*>(vr.data())[i] = ff(double(vr[i]));
  }
  std::vector<T> X((size_t)n_sys * nw), out((size_t)n_sys * nw), sh(n_sys);
  for (size_t i = 0; i < X.size(); ++i) X[i] = (T)Xd[i];
  for (int s = 0; s < n_sys; ++s) sh[s] = (T)shift[s];
  const int NP = 2 * w.h.m + 1, pairs = (n_sys + 1) / 2;
  std::vector<cplx<C>> Tb((size_t)pairs * NP * N * N), B((size_t)N * (N + 1)), Zp(w.h.npt_max + 1);
  std::vector<cplx<C>> Bm((size_t)3 * NP * (N + 1));
  for (int q = 0; q < pairs; ++q)
    for (int hi = 0; hi < NP; ++hi) {
      if constexpr (NC > 0) {
        if (reg) {
          if (hi % 3 == 0)
            plane_g2r_reg_body<T, NC, C>(q, hi, std::min(3, NP - hi), w.tab(), tw.data(), X.data(), nw, n_sys, nullptr,
                                         Tb.data(), Bm.data(), kOne);
          continue;
        }
      }
      plane_g2r_body<T, NC, C>(q, hi, w.tab(), pl, tw.data(), X.data(), nw, n_sys, nullptr, Tb.data(), B.data(), kOne);
    }
  XArgs<T> a{};
  a.mode = XM_APPLY_V; a.V = vr.data(); a.n_sys = n_sys;
  for (int q = 0; q < pairs; ++q) {
    if constexpr (NC > 0) {
      if (reg) {
        for (int l = 0; l < N * N; ++l) xline_reg_body<T, NC, C>(q, l, w.h.m, tw.data(), Tb.data(), a);
        continue;
      }
    }
    for (int y = 0; y < N; ++y) xline_body<T, NC, C>(q, y, w.h.m, pl, tw.data(), Tb.data(), a, B.data(), kOne);
  }
  Epi<T> e{};
  e.out = out.data(); e.ldo = nw; e.pin = X.data(); e.ldp = nw; e.vcoef = T(1); e.kin = T(1);
  e.shift = sh.data(); e.n_sys = n_sys;
  for (int q = 0; q < pairs; ++q)
    for (int hp = 0; hp <= w.h.m; ++hp) {
      if constexpr (NC > 0) {
        if (reg) {
          plane_r2g_reg_body<T, NC, C>(q, hp, w.tab(), tw.data(), Tb.data(), e, Bm.data(), kOne);
          continue;
        }
      }
      plane_r2g_body<T, NC, C>(q, hp, w.tab(), pl, tw.data(), Tb.data(), e, B.data(), Zp.data(), kOne);
    }
  for (size_t i = 0; i < out.size(); ++i) outd[i] = (double)out[i];
}

}  // namespace

extern "C" {

void emu_set_reg_xline(int on) { g_reg = on != 0; }

int emu_sphere_size(double L, double ecut, int N, int* n, int* n_pairs, int* m) {
  Sph s;
  build_sphere(L, ecut, N, s.h);
  *n = s.h.n; *n_pairs = s.h.n_pairs; *m = s.h.m;
  return 0;
}

int emu_sphere_maps(double L, double ecut, int N, int* miller, int* pos, int* neg) {
  Sph s;
  build_sphere(L, ecut, N, s.h);
  std::memcpy(miller, s.h.miller.data(), sizeof(int) * s.h.miller.size());
  std::memcpy(pos, s.h.pos.data(), sizeof(int) * s.h.pos.size());
  std::memcpy(neg, s.h.neg.data(), sizeof(int) * s.h.neg.size());
  return s.h.i0;
}

// One line: dir 0 = DIF, sign +1 (natural in, digit-reversed out); dir 1 = DIT, sign -1.
int emu_fft_line(int N, int dir, const double* in, double* out) {
  FftPlan pl;
  if (!make_plan(N, pl)) return 1;
  auto tw = twiddles<double>(N);
  std::vector<cplx<double>> b(N);
  for (int i = 0; i < N; ++i) b[i] = mk<double>(in[2 * i], in[2 * i + 1]);
  if (dir == 0) fft_dif<double>(b.data(), pl, tw.data(), +1, 1, N, 1, -1, kOne);
  else fft_dit<double>(b.data(), pl, tw.data(), -1, 1, N, 1, -1, kOne);
  for (int i = 0; i < N; ++i) { out[2 * i] = b[i].re; out[2 * i + 1] = b[i].im; }
  return 0;
}

// One line in float-float arithmetic (input rounded to float-float); dir as emu_fft_line.
int emu_fft_line_ff(int N, int dir, const double* in, double* out) {
  FftPlan pl;
  if (!make_plan(N, pl)) return 1;
  auto tw = twiddles<ff>(N);
  std::vector<cplx<ff>> b(N);
  for (int i = 0; i < N; ++i) b[i] = mk<ff>(ff(in[2 * i]), ff(in[2 * i + 1]));
  if (dir == 0) fft_dif<ff>(b.data(), pl, tw.data(), +1, 1, N, 1, -1, kOne);
  else fft_dit<ff>(b.data(), pl, tw.data(), -1, 1, N, 1, -1, kOne);
  for (int i = 0; i < N; ++i) { out[2 * i] = (double)b[i].re; out[2 * i + 1] = (double)b[i].im; }
  return 0;
}

// Float-float primitives on arrays: op 0 = a + b, 1 = a * b, 2 = a - b (inputs rounded to float-float).
int emu_ff_op(int op, int n, const double* a, const double* b, double* out) {
  for (int i = 0; i < n; ++i) {
    const ff x(a[i]), y(b[i]);
    const ff r = op == 0 ? x + y : op == 1 ? x * y : x - y;
    out[i] = (double)r;
  }
  return 0;
}

int emu_fft_position(int N, int n) {
  FftPlan pl;
  make_plan(N, pl);
  return fft_position(pl, n);
}

// (H - shift_s) applied to real-basis vectors X (n_sys x nrb) via the plane / x-line / plane bodies.
// flags bit 0: FP32; bit 1: the compile-time-N bodies (N = 24 only); bit 2: FP64 storage with
// float-float compute (compile-time N = 24 only).
int emu_apply_h(double L, double ecut, int N, const double* vloc_c, int n_sys, const double* X,
                const double* shift, double* out, int flags) {
  const bool fp32 = flags & 1, ct = flags & 2, ffc = flags & 4, reg = flags & 8, reg96 = flags & 16;
  if (reg96) {   // the 96-point register-resident FP32 bodies
    if (N != 96) return 1;
    apply_h_impl<float, 96>(L, ecut, N, vloc_c, n_sys, X, shift, out, true);
    return 0;
  }
  if ((ct || ffc || reg) && N != 24) return 1;
  if (ffc) {
    apply_h_impl<double, 24, ff>(L, ecut, N, vloc_c, n_sys, X, shift, out, reg);
  } else if (fp32) {
    if (ct || reg) apply_h_impl<float, 24>(L, ecut, N, vloc_c, n_sys, X, shift, out, reg);
    else apply_h_impl<float>(L, ecut, N, vloc_c, n_sys, X, shift, out);
  } else {
    if (ct || reg) apply_h_impl<double, 24>(L, ecut, N, vloc_c, n_sys, X, shift, out, reg);
    else apply_h_impl<double>(L, ecut, N, vloc_c, n_sys, X, shift, out);
  }
  return 0;
}

// Compile-time-N line transforms (N in {24, 32, 48, 64, 96}); dir as emu_fft_line.
int emu_fft_line_ct(int N, int dir, const double* in, double* out) {
  FftPlan pl;
  if (!make_plan(N, pl)) return 1;
  auto tw = twiddles<double>(N);
  std::vector<cplx<double>> b(N);
  for (int i = 0; i < N; ++i) b[i] = mk<double>(in[2 * i], in[2 * i + 1]);
#define EMU_CT(NN)                                                                             \
  case NN:                                                                                     \
    if (dir == 0) fft_dif_n<double, NN>(b.data(), pl, tw.data(), +1, 1, N, 1, -1, kOne);       \
    else fft_dit_n<double, NN>(b.data(), pl, tw.data(), -1, 1, N, 1, -1, kOne);                \
    break;
  switch (N) {
    EMU_CT(24) EMU_CT(32) EMU_CT(48) EMU_CT(64) EMU_CT(96)
    default: return 1;
  }
#undef EMU_CT
  for (int i = 0; i < N; ++i) { out[2 * i] = b[i].re; out[2 * i + 1] = b[i].im; }
  return 0;
}

// Right-hand sides [psi_a(r) f_b(r)] on the wavefunction sphere (real basis) for pairs (a_idx[s], b_idx[s]);
// psi_c: wfc-sphere complex (n_psi columns), f_c: rho-sphere complex (n_f columns).
int emu_products(double L, double ecut, int N, int n_psi, const double* psi_c, int n_f, const double* f_c,
                 int n_sys, const int* a_idx, const int* b_idx, double* out) {
  Sph w, r;
  build_sphere(L, ecut, N, w.h);
  build_sphere(L, 4 * ecut, N, r.h);
  FftPlan pl;
  make_plan(N, pl);
  auto tw = twiddles<double>(N);
  const long N3 = (long)N * N * N;
  const int nw = w.h.nrb(), nr = r.h.nrb();
  std::vector<double> prb((size_t)n_psi * nw), frb((size_t)n_f * nr), pr((size_t)n_psi * N3), fr((size_t)n_f * N3);
  sphere_to_rb_host<double>(w, n_psi, psi_c, 2L * w.h.n, nullptr, 0, prb.data(), nw);
  sphere_to_rb_host<double>(r, n_f, f_c, 2L * r.h.n, nullptr, 0, frb.data(), nr);
  to_real<double>(w, pl, tw, prb.data(), nw, n_psi, pr.data());
  to_real<double>(r, pl, tw, frb.data(), nr, n_f, fr.data());
  const int NP = 2 * w.h.m + 1, pairs = (n_sys + 1) / 2;
  std::vector<cplx<double>> Tb((size_t)pairs * NP * N * N), B((size_t)N * (N + 1)), Zp(w.h.npt_max + 1);
  XArgs<double> a{};
  a.mode = XM_FROM_REAL; a.A = pr.data(); a.lda = N3; a.a_index = a_idx; a.Bm = fr.data(); a.ldb = N3;
  a.b_index = b_idx; a.n_sys = n_sys;
  for (int q = 0; q < pairs; ++q) run_xline<double>(q, w.h.m, pl, tw, Tb.data(), a, B.data());
  Epi<double> e{};
  e.out = out; e.ldo = nw; e.vcoef = 1.0; e.n_sys = n_sys;
  for (int q = 0; q < pairs; ++q)
    for (int hp = 0; hp <= w.h.m; ++hp) run_r2g<double>(q, hp, w, pl, tw, Tb.data(), e, B.data(), Zp.data());
  return 0;
}

// drho of n_pert perturbations: coef * sum_v psi_v(r) x_{p n_v + v}(r) on the density sphere (real basis).
int emu_drho(double L, double ecut, int N, int n_v, const double* psi_c, int n_pert, const double* Xd,
             double coef, double* out) {
  Sph w, r;
  build_sphere(L, ecut, N, w.h);
  build_sphere(L, 4 * ecut, N, r.h);
  FftPlan pl;
  make_plan(N, pl);
  auto tw = twiddles<double>(N);
  const long N3 = (long)N * N * N;
  const int nw = w.h.nrb(), nr = r.h.nrb();
  const int n_sys = n_v * n_pert;
  std::vector<double> prb((size_t)n_v * nw), pr((size_t)n_v * N3), D((size_t)n_pert * N3);
  sphere_to_rb_host<double>(w, n_v, psi_c, 2L * w.h.n, nullptr, 0, prb.data(), nw);
  to_real<double>(w, pl, tw, prb.data(), nw, n_v, pr.data());
  const int NP = 2 * w.h.m + 1, pairs = (n_sys + 1) / 2;
  std::vector<cplx<double>> Tb((size_t)pairs * NP * N * N), B((size_t)N * (N + 1));
  std::vector<double> acc((size_t)N * N);
  for (int q = 0; q < pairs; ++q)
    for (int hi = 0; hi < NP; ++hi)
      run_g2r<double>(q, hi, w, pl, tw, Xd, nw, n_sys, Tb.data(), B.data());
  for (int p = 0; p < n_pert; ++p)
    for (int y = 0; y < N; ++y)
      drho_xline_body<double>(p, y, w.h.m, pl, tw.data(), Tb.data(), pr.data(), N3, n_v, n_sys, coef,
                              D.data(), N3, B.data(), acc.data(), kOne);
  const int NPr = 2 * r.h.m + 1, rpairs = (n_pert + 1) / 2;
  std::vector<cplx<double>> Tr((size_t)rpairs * NPr * N * N), Zp(r.h.npt_max + 1);
  XArgs<double> a{};
  a.mode = XM_FROM_REAL; a.A = D.data(); a.lda = N3; a.n_sys = n_pert;
  for (int q = 0; q < rpairs; ++q) run_xline<double>(q, r.h.m, pl, tw, Tr.data(), a, B.data());
  Epi<double> e{};
  e.out = out; e.ldo = nr; e.vcoef = 1.0; e.n_sys = n_pert;
  for (int q = 0; q < rpairs; ++q)
    for (int hp = 0; hp <= r.h.m; ++hp) run_r2g<double>(q, hp, r, pl, tw, Tr.data(), e, B.data(), Zp.data());
  return 0;
}

// Y <- Y - Psi Psi^T Y through the tiled projector body.
int emu_pc(int n, int nv, int n_sys, const double* Psi, double* Y) {
  std::vector<double> sm((size_t)nv * kPcTS + (size_t)kPcKC * nv + kPcKC * kPcTS);
  for (int t = 0; t * kPcTS < n_sys; ++t) pc_body<double>(t, Y, n, n_sys, Psi, n, n, nv, nullptr, sm.data(), kOne);
  return 0;
}

// Real basis <-> complex sphere round trip: out = rb_to_sphere(sphere_to_rb(c, part 0), sphere_to_rb(c, part 1)).
int emu_rb_roundtrip(double L, double ecut, int N, int n_sys, const double* c, double* rb, double* out) {
  Sph s;
  build_sphere(L, ecut, N, s.h);
  const int nb = s.h.nrb();
  std::vector<double> both((size_t)2 * n_sys * nb);
  for (int q = 0; q < n_sys; ++q)
    for (int i = 0; i < nb; ++i) {
      sphere_to_rb(q, c, 2L * s.h.n, nullptr, s.map(), 0, both.data(), nb, i);
      sphere_to_rb(q, c, 2L * s.h.n, nullptr, s.map(), 1, both.data() + (size_t)n_sys * nb, nb, i);
    }
  std::memcpy(rb, both.data(), sizeof(double) * n_sys * nb);
  std::vector<int> brow(n_sys);
  for (int q = 0; q < n_sys; ++q) brow[q] = n_sys + q;
  for (int q = 0; q < n_sys; ++q)
    for (int j = 0; j <= s.h.n_pairs; ++j) rb_to_sphere(q, both.data(), nb, brow.data(), nullptr, s.map(), out, 2L * s.h.n, j);
  return 0;
}

}  // extern "C"
