// Bodies of the linear-algebra kernels: the projector P_c, the batched masked
// preconditioned CG of Eq. sternheimer, and conversions between the complex
// full-sphere layout of the public interface and the real plane-wave basis.
#pragma once

#include "common.cuh"

namespace wgw {

// Sum of v over the block.  Fixed reduction tree for a fixed block size, so
// the result of a system does not depend on the other systems in the launch.
// red: at least 32 doubles of shared memory.
WGW_HD double block_sum(double v, double* red, Thr th) {
#if defined(__CUDA_ARCH__)
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = th.tid >> 5, l = th.tid & 31, nw = (th.nth + 31) >> 5;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double s = l < nw ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) red[32] = s;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
#else
  (void)red; (void)th;
  return v;
#endif
}

// FP32 partial sums: reduced within each warp in FP32, across warps in FP64 (a warp-level
// FP64 tree would run on GB300's FP64 pipe, 1/64 of the FP32 rate, for every thread).
WGW_HD double block_sum(float v, double* red, Thr th) {
#if defined(__CUDA_ARCH__)
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = th.tid >> 5, l = th.tid & 31, nw = (th.nth + 31) >> 5;
  if (l == 0) red[w] = double(v);
  __syncthreads();
  if (th.tid == 0) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += red[k];
    red[32] = s;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
#else
  (void)red; (void)th;
  return double(v);
#endif
}

// A block-uniform scalar computed by thread 0 (in FP64) and handed to every thread in T, so
// that the FP64 arithmetic runs once per block instead of once per thread (GB300's FP64 pipe
// runs at 1/64 of the FP32 rate).  red: the shared scratch of block_sum.
template <typename T, typename F>
WGW_HD T block_scalar(F f, double* red, Thr th) {
#if defined(__CUDA_ARCH__)
  T* slot = reinterpret_cast<T*>(red + 32);
  if (th.tid == 0) *slot = T(f());
  __syncthreads();
  const T v = *slot;
  __syncthreads();
  return v;
#else
  (void)red; (void)th;
  return T(f());
#endif
}

// Dot product of two length-n vectors: per-thread partial sums in T, then block_sum.
// Rows start 16-byte aligned (row lengths are multiples of 32), so FP32 rows are read as float4.
template <typename T>
WGW_HD double block_dot(const T* a, const T* b, int n, double* red, Thr th) {
  T part = T(0);
  int i0 = 0;
  if constexpr (sizeof(T) == sizeof(float)) {
    const int n4 = n / 4;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    for (int q = th.tid; q < n4; q += th.nth) {
      const float4 x = a4[q], y = b4[q];
      part += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
    }
    i0 = 4 * n4;
  }
  for (int i = i0 + th.tid; i < n; i += th.nth) part += a[i] * b[i];
  return block_sum(part, red, th);
}

// ---------------------------------------------------------------- P_c = 1 - P_v
// Y[:, s] <- Y[:, s] - Psi (Psi^T Y[:, s]) for the TS systems of one tile
// (Sec. 3: P_c = 1 - P_v, applied with two products against the occupied block).
// smem: C[nv * TS] + Ps[KC * nv] + Ys[KC * TS] elements of T.
constexpr int kPcTS = 8;
constexpr int kPcKC = 32;

template <typename T>
WGW_HD void pc_body(int tile, T* Y, long ldy, int n_sys, const T* Psi, long ldp, int n, int nv,
                    const int* active, T* sm, Thr th) {
  const int TS = kPcTS, KC = kPcKC;
  T* C = sm;
  T* Ps = C + nv * TS;
  T* Ys = Ps + KC * nv;
  const int s_base = tile * TS;
  for (int e = th.tid; e < nv * TS; e += th.nth) C[e] = T(0);
  for (int i0 = 0; i0 < n; i0 += KC) {
    WGW_SYNC();
    for (int e = th.tid; e < KC * nv; e += th.nth) {
      const int r = e % KC, v = e / KC;
      Ps[r * nv + v] = (i0 + r < n) ? Psi[(size_t)v * ldp + i0 + r] : T(0);
    }
    for (int e = th.tid; e < KC * TS; e += th.nth) {
      const int r = e % KC, t = e / KC, s = s_base + t;
      Ys[r * TS + t] = (i0 + r < n && s < n_sys) ? Y[(size_t)s * ldy + i0 + r] : T(0);
    }
    WGW_SYNC();
    for (int e = th.tid; e < nv * TS; e += th.nth) {
      const int v = e / TS, t = e % TS;
      T acc = C[e];
      for (int r = 0; r < KC; ++r) acc += Ps[r * nv + v] * Ys[r * TS + t];
      C[e] = acc;
    }
  }
  for (int i0 = 0; i0 < n; i0 += KC) {
    WGW_SYNC();
    for (int e = th.tid; e < KC * nv; e += th.nth) {
      const int r = e % KC, v = e / KC;
      Ps[r * nv + v] = (i0 + r < n) ? Psi[(size_t)v * ldp + i0 + r] : T(0);
    }
    WGW_SYNC();
    for (int e = th.tid; e < KC * TS; e += th.nth) {
      const int r = e % KC, t = e / KC, s = s_base + t, i = i0 + r;
      if (i >= n || s >= n_sys || !(active == nullptr || active[s])) continue;
      T acc = Y[(size_t)s * ldy + i];
      for (int v = 0; v < nv; ++v) acc -= Ps[r * nv + v] * C[v * TS + t];
      Y[(size_t)s * ldy + i] = acc;
    }
  }
}

// ---------------------------------------------------------------- batched CG
// Per-system state of the preconditioned CG on A = P_c (H - e_v) P_c.
struct CgState {
  double* rz;      // r . z
  double* bb;      // ||b||^2
  double* rr;      // ||r||^2 after the last update
  int* active;     // 1 while the system iterates
  int* iters;      // iterations done
  // Stagnation test (null = off): smallest ||r||^2 so far and the iteration it was reached.
  double* rr_best;
  int* it_best;
};

// A system whose residual norm has not halved within this many iterations has reached the
// attainable accuracy of its arithmetic (FP32 inner solves: the FP64 refinement takes over).
constexpr int kStagnationWindow = 30;

// Diagonal preconditioner 1 / max(0.5|G|^2 - e_v, 1 Ha) (a reading: the paper
// says only that the CG is preconditioned).
template <typename T>
WGW_HD T precond(const SphereTab& sp, int i, double e) {
  const double d = sp.g2[i] - e;
  return T(1.0 / (d > 1.0 ? d : 1.0));
}
// FP32 solves evaluate it in FP32 (FP64 arithmetic per element would run on GB300's FP64 pipe,
// 1/64 of the FP32 rate); any fixed positive diagonal is a valid preconditioner.
template <>
WGW_HD float precond<float>(const SphereTab& sp, int i, double e) {
  const float d = sp.g2f[i] - static_cast<float>(e);
  return 1.0f / (d > 1.0f ? d : 1.0f);
}

// x = 0, r = b, z = M^-1 r, bb = ||b||^2; a system with b = 0 is inactive from the start.
template <typename T>
WGW_HD void cg_init_a_body(int s, const SphereTab& sp, int n, const T* Bv, T* X, T* R, T* Z,
                           long ld, const double* eps, CgState st, double* red, Thr th) {
  const T* b = Bv + (size_t)s * ld;
  T* x = X + (size_t)s * ld;
  T* r = R + (size_t)s * ld;
  T* z = Z + (size_t)s * ld;
  const double e = eps[s];
  for (int i = th.tid; i < n; i += th.nth) {
    const T bi = b[i];
    x[i] = T(0);
    r[i] = bi;
    z[i] = precond<T>(sp, i, e) * bi;
  }
  const double bb = block_dot(b, b, n, red, th);
  if (th.tid == 0) {
    st.bb[s] = bb;
    st.rr[s] = bb;
    st.active[s] = bb > 0.0 ? 1 : 0;
    st.iters[s] = 0;
    if (st.rr_best) { st.rr_best[s] = bb; st.it_best[s] = 0; }
  }
}

// rz = r . z, p = z.
template <typename T>
WGW_HD void cg_init_b_body(int s, int n, const T* R, const T* Z, T* P, long ld, CgState st,
                           double* red, Thr th) {
  if (!st.active[s]) return;
  const T* r = R + (size_t)s * ld;
  const T* z = Z + (size_t)s * ld;
  T* p = P + (size_t)s * ld;
  for (int i = th.tid; i < n; i += th.nth) p[i] = z[i];
  const double rz = block_dot(r, z, n, red, th);
  if (th.tid == 0) st.rz[s] = rz;
}

// alpha = rz / (p . q), x += alpha p, r -= alpha q, convergence test, z = M^-1 r.
template <typename T>
WGW_HD void cg_step_a_body(int s, const SphereTab& sp, int n, T* X, T* R, T* Z, const T* P,
                           const T* Q, long ld, const double* eps, CgState st, double tol2,
                           int max_iter, double* red, Thr th) {
  if (!st.active[s]) return;
  T* x = X + (size_t)s * ld;
  T* r = R + (size_t)s * ld;
  T* z = Z + (size_t)s * ld;
  const T* p = P + (size_t)s * ld;
  const T* q = Q + (size_t)s * ld;
  const double pq = block_dot(p, q, n, red, th);
  const double rz0 = st.rz[s];
  const T a = block_scalar<T>([&] { return pq != 0.0 ? rz0 / pq : 0.0; }, red, th);
  const double e = eps[s];
  T part = T(0);
  int i0 = 0;
  if constexpr (sizeof(T) == sizeof(float)) {
    const int n4 = n / 4;
    const float ef = static_cast<float>(e);
    for (int qd = th.tid; qd < n4; qd += th.nth) {
      const float4 pv = reinterpret_cast<const float4*>(p)[qd], qv = reinterpret_cast<const float4*>(q)[qd];
      float4 xv = reinterpret_cast<float4*>(x)[qd], rv = reinterpret_cast<float4*>(r)[qd];
      const float4 gv = reinterpret_cast<const float4*>(sp.g2f)[qd];
      xv.x += a * pv.x; xv.y += a * pv.y; xv.z += a * pv.z; xv.w += a * pv.w;
      rv.x -= a * qv.x; rv.y -= a * qv.y; rv.z -= a * qv.z; rv.w -= a * qv.w;
      float4 zv;
      // z = M^-1 r with M^-1 evaluated exactly as precond<float>
      zv.x = (1.0f / fmaxf(gv.x - ef, 1.0f)) * rv.x; zv.y = (1.0f / fmaxf(gv.y - ef, 1.0f)) * rv.y;
      zv.z = (1.0f / fmaxf(gv.z - ef, 1.0f)) * rv.z; zv.w = (1.0f / fmaxf(gv.w - ef, 1.0f)) * rv.w;
      reinterpret_cast<float4*>(x)[qd] = xv;
      reinterpret_cast<float4*>(r)[qd] = rv;
      reinterpret_cast<float4*>(z)[qd] = zv;
      part += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
    }
    i0 = 4 * n4;
  }
  for (int i = i0 + th.tid; i < n; i += th.nth) {
    x[i] += a * p[i];
    const T ri = r[i] - a * q[i];
    r[i] = ri;
    z[i] = precond<T>(sp, i, e) * ri;
    part += ri * ri;
  }
  const double rr = block_sum(part, red, th);
  if (th.tid == 0) {
    st.rr[s] = rr;
    const int it = st.iters[s] + 1;
    st.iters[s] = it;
    bool stalled = false;
    if (st.rr_best) {
      if (rr < 0.25 * st.rr_best[s]) { st.rr_best[s] = rr; st.it_best[s] = it; }
      else stalled = it - st.it_best[s] >= kStagnationWindow;
    }
    if (rr <= tol2 * st.bb[s] || it >= max_iter || !(pq > 0.0) || stalled) st.active[s] = 0;
  }
}

// rz' = r . z, beta = rz'/rz, p = z + beta p.
template <typename T>
WGW_HD void cg_step_b_body(int s, int n, const T* R, const T* Z, T* P, long ld, CgState st,
                           double* red, Thr th) {
  if (!st.active[s]) return;
  const T* r = R + (size_t)s * ld;
  const T* z = Z + (size_t)s * ld;
  T* p = P + (size_t)s * ld;
  const double rz = block_dot(r, z, n, red, th);
  const double rz_old = st.rz[s];
  const T bt = block_scalar<T>([&] { return rz_old != 0.0 ? rz / rz_old : 0.0; }, red, th);
  int i0 = 0;
  if constexpr (sizeof(T) == sizeof(float)) {
    const int n4 = n / 4;
    for (int qd = th.tid; qd < n4; qd += th.nth) {
      const float4 zv = reinterpret_cast<const float4*>(z)[qd];
      float4 pv = reinterpret_cast<float4*>(p)[qd];
      pv.x = zv.x + bt * pv.x; pv.y = zv.y + bt * pv.y; pv.z = zv.z + bt * pv.z; pv.w = zv.w + bt * pv.w;
      reinterpret_cast<float4*>(p)[qd] = pv;
    }
    i0 = 4 * n4;
  }
  for (int i = i0 + th.tid; i < n; i += th.nth) p[i] = z[i] + bt * p[i];
  if (th.tid == 0) st.rz[s] = rz;
}

// ---------------------------------------------------------------- complex-shifted CG (COCG)
// (P_c (H - e_v) P_c + i w) x = b for a complex x = u + i v kept as two consecutive real
// rows (u at row 2s, v at row 2s + 1 of every vector buffer).  With A = P_c (H - e_v) P_c
// real symmetric, A + i w is complex symmetric, so conjugate gradients with the bilinear
// form x^T y = (u.u' - v.v') + i (u.v' + v.u') (COCG, a reading: the paper names only a
// preconditioned CG) applies; for w = 0 it reduces to the PCG above.
struct CocgState {
  double* rz_re; double* rz_im;   // rho = r^T z
  double* bb; double* rr;
  int* active;
  int* iters;
  const double* omega;            // per complex system
};

// x = 0, r = b, z = M^-1 r (both rows); ||b||^2 = |b_u|^2 + |b_v|^2.
template <typename T>
WGW_HD void cocg_init_a_body(int s, const SphereTab& sp, int n, const T* Bv, T* X, T* R, T* Z, long ld,
                             const double* eps, CocgState st, double* red, Thr th) {
  const double e = eps[s];
  T part = T(0);
  for (int row = 2 * s; row <= 2 * s + 1; ++row) {
    const T* b = Bv + (size_t)row * ld;
    T* x = X + (size_t)row * ld;
    T* r = R + (size_t)row * ld;
    T* z = Z + (size_t)row * ld;
    for (int i = th.tid; i < n; i += th.nth) {
      const T bi = b[i];
      x[i] = T(0);
      r[i] = bi;
      z[i] = precond<T>(sp, i, e) * bi;
      part += bi * bi;
    }
  }
  const double bb = block_sum(part, red, th);
  if (th.tid == 0) {
    st.bb[s] = bb;
    st.rr[s] = bb;
    st.active[s] = bb > 0.0 ? 1 : 0;
    st.iters[s] = 0;
  }
}

// rho = r^T z, p = z.
template <typename T>
WGW_HD void cocg_init_b_body(int s, int n, const T* R, const T* Z, T* P, long ld, CocgState st,
                             double* red, Thr th) {
  if (!st.active[s]) return;
  const T* ru = R + (size_t)(2 * s) * ld; const T* rv = ru + ld;
  const T* zu = Z + (size_t)(2 * s) * ld; const T* zv = zu + ld;
  T* pu = P + (size_t)(2 * s) * ld; T* pv = pu + ld;
  T a = T(0), b = T(0);
  for (int i = th.tid; i < n; i += th.nth) {
    pu[i] = zu[i];
    pv[i] = zv[i];
    a += ru[i] * zu[i] - rv[i] * zv[i];
    b += ru[i] * zv[i] + rv[i] * zu[i];
  }
  const double re = block_sum(a, red, th);
  const double im = block_sum(b, red, th);
  if (th.tid == 0) { st.rz_re[s] = re; st.rz_im[s] = im; }
}

// q <- A p + i w p (in place on Q), alpha = rho / p^T q, x += alpha p, r -= alpha q,
// convergence test on |r|^2, z = M^-1 r.
template <typename T>
WGW_HD void cocg_step_a_body(int s, const SphereTab& sp, int n, T* X, T* R, T* Z, const T* P, T* Q,
                             long ld, const double* eps, CocgState st, double tol2, int max_iter,
                             double* red, Thr th) {
  if (!st.active[s]) return;
  const T w = T(st.omega[s]);
  const T* pu = P + (size_t)(2 * s) * ld; const T* pv = pu + ld;
  T* qu = Q + (size_t)(2 * s) * ld; T* qv = qu + ld;
  T a = T(0), b = T(0);
  for (int i = th.tid; i < n; i += th.nth) {
    const T qa = qu[i] - w * pv[i], qb = qv[i] + w * pu[i];
    qu[i] = qa;
    qv[i] = qb;
    a += pu[i] * qa - pv[i] * qb;
    b += pu[i] * qb + pv[i] * qa;
  }
  const double sr = block_sum(a, red, th);
  const double si = block_sum(b, red, th);
  const double d2 = sr * sr + si * si;
  const double rr0 = st.rz_re[s], ri0 = st.rz_im[s];
  const double ar = d2 > 0 ? (rr0 * sr + ri0 * si) / d2 : 0.0;   // alpha = rho / sigma
  const double ai = d2 > 0 ? (ri0 * sr - rr0 * si) / d2 : 0.0;
  const T Ar = T(ar), Ai = T(ai);
  T* xu = X + (size_t)(2 * s) * ld; T* xv = xu + ld;
  T* ru = R + (size_t)(2 * s) * ld; T* rv = ru + ld;
  T* zu = Z + (size_t)(2 * s) * ld; T* zv = zu + ld;
  const double e = eps[s];
  T part = T(0);
  for (int i = th.tid; i < n; i += th.nth) {
    xu[i] += Ar * pu[i] - Ai * pv[i];
    xv[i] += Ar * pv[i] + Ai * pu[i];
    const T nu = ru[i] - (Ar * qu[i] - Ai * qv[i]);
    const T nv = rv[i] - (Ar * qv[i] + Ai * qu[i]);
    ru[i] = nu;
    rv[i] = nv;
    const T m = precond<T>(sp, i, e);
    zu[i] = m * nu;
    zv[i] = m * nv;
    part += nu * nu + nv * nv;
  }
  const double rr = block_sum(part, red, th);
  if (th.tid == 0) {
    st.rr[s] = rr;
    const int it = st.iters[s] + 1;
    st.iters[s] = it;
    if (rr <= tol2 * st.bb[s] || it >= max_iter || !(d2 > 0.0)) st.active[s] = 0;
  }
}

// rho' = r^T z, beta = rho'/rho, p = z + beta p.
template <typename T>
WGW_HD void cocg_step_b_body(int s, int n, const T* R, const T* Z, T* P, long ld, CocgState st,
                             double* red, Thr th) {
  if (!st.active[s]) return;
  const T* ru = R + (size_t)(2 * s) * ld; const T* rv = ru + ld;
  const T* zu = Z + (size_t)(2 * s) * ld; const T* zv = zu + ld;
  T* pu = P + (size_t)(2 * s) * ld; T* pv = pu + ld;
  T a = T(0), b = T(0);
  for (int i = th.tid; i < n; i += th.nth) {
    a += ru[i] * zu[i] - rv[i] * zv[i];
    b += ru[i] * zv[i] + rv[i] * zu[i];
  }
  const double nr = block_sum(a, red, th);
  const double ni = block_sum(b, red, th);
  const double orr = st.rz_re[s], ori = st.rz_im[s];
  const double d2 = orr * orr + ori * ori;
  const double br = d2 > 0 ? (nr * orr + ni * ori) / d2 : 0.0;
  const double bi = d2 > 0 ? (ni * orr - nr * ori) / d2 : 0.0;
  const T Br = T(br), Bi = T(bi);
  for (int i = th.tid; i < n; i += th.nth) {
    const T ou = pu[i], ov = pv[i];
    pu[i] = zu[i] + Br * ou - Bi * ov;
    pv[i] = zv[i] + Br * ov + Bi * ou;
  }
  if (th.tid == 0) { st.rz_re[s] = nr; st.rz_im[s] = ni; }
}

// r = b - (q + i w x) for complex system s (q = A x already in Q), FP64.
WGW_HD void shifted_residual(int s, int i, const double* B, const double* Q, const double* X, double w,
                             double* R, long ld) {
  const size_t u = (size_t)(2 * s) * ld + i, v = u + ld;
  R[u] = B[u] - (Q[u] - w * X[v]);
  R[v] = B[v] - (Q[v] + w * X[u]);
}

// ---------------------------------------------------------------- conversions
// Index map of a sphere in real-basis form: idx[0] = canonical index of G = 0,
// idx_pos[j], idx_neg[j] (j >= 1) = canonical indices of G_j and -G_j.
struct RbMap {
  int n_pairs;
  const int* i0;
  const int* pos;   // n_pairs + 1 entries, [0] unused
  const int* neg;
};

// Real-basis form of the real-in-r part (part = 0: (c(G) + c(-G)^*)/2) or of the
// other part (part = 1: (c(G) - c(-G)^*)/(2i)) of complex full-sphere coefficients c
// (interleaved re, im), each coefficient first multiplied by scale[canonical index] (null = 1).
WGW_HD void sphere_to_rb(int s, const double* c, long ldc, const double* scale, RbMap mp, int part,
                         double* out, long ldo, int i) {
  const double* cs = c + (size_t)s * ldc;
  double* o = out + (size_t)s * ldo;
  if (i == 0) {
    const int g = *mp.i0;
    const double f = scale ? scale[g] : 1.0;
    o[0] = f * (part == 0 ? cs[2 * g] : cs[2 * g + 1]);
    return;
  }
  const int j = (i + 1) / 2;
  const int gp = mp.pos[j], gn = mp.neg[j];
  const double f = scale ? scale[gp] : 1.0;
  const double pr = cs[2 * gp], pi = cs[2 * gp + 1], nr = cs[2 * gn], ni = cs[2 * gn + 1];
  double re, im;
  if (part == 0) { re = 0.5 * (pr + nr); im = 0.5 * (pi - ni); }
  else { re = 0.5 * (pi + ni); im = -0.5 * (pr - nr); }
  o[i] = f * kSqrt2 * ((i & 1) ? re : im);
}

// Complex full-sphere coefficients (interleaved) of a + i b from real-basis
// forms: a = in[s], b = in[b_row[s]] (b_row null or < 0: b = 0), each
// multiplied by scale[canonical index] (null = 1).  Thread j writes the
// canonical entries of real-basis pair j (j = 0: G = 0).
WGW_HD void rb_to_sphere(int s, const double* in, long ldi, const int* b_row, const double* scale,
                         RbMap mp, double* c, long ldc, int j) {
  const double* as = in + (size_t)s * ldi;
  const int br = b_row ? b_row[s] : -1;
  const double* bs = br >= 0 ? in + (size_t)br * ldi : nullptr;
  double* cs = c + (size_t)s * ldc;
  if (j == 0) {
    const int g = *mp.i0;
    const double f = scale ? scale[g] : 1.0;
    cs[2 * g] = f * as[0];
    cs[2 * g + 1] = bs ? f * bs[0] : 0.0;
    return;
  }
  const int gp = mp.pos[j], gn = mp.neg[j];
  const double f = (scale ? scale[gp] : 1.0) * kInvSqrt2;
  const double a1 = as[2 * j - 1], a2 = as[2 * j];
  const double b1 = bs ? bs[2 * j - 1] : 0.0, b2 = bs ? bs[2 * j] : 0.0;
  cs[2 * gp] = f * (a1 - b2);
  cs[2 * gp + 1] = f * (a2 + b1);
  cs[2 * gn] = f * (a1 + b2);
  cs[2 * gn + 1] = f * (b1 - a2);
}

// out[s] = alpha * x[s] + beta * y[s] for active systems (element i).
WGW_HD void axpby(int s, int i, double alpha, const double* x, double beta, const double* y,
                  double* out, long ld) {
  const size_t o = (size_t)s * ld + i;
  out[o] = alpha * x[o] + (beta != 0.0 ? beta * y[o] : 0.0);
}

}  // namespace wgw
