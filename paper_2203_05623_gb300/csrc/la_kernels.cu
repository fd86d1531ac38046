// __global__ wrappers of the linear-algebra kernels (bodies in la_bodies.cuh).
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "internal.h"

namespace wgw {

namespace {

constexpr int kCgThreads = 256;

__device__ __forceinline__ Thr thr() { Thr t; t.tid = threadIdx.x; t.nth = blockDim.x; return t; }

template <typename T>
__global__ void k_pc(T* Y, long ldy, int n_sys, const T* Psi, long ldp, int n, int nv,
                     const int* active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tile = blockIdx.x;
  if (active) {
    bool any = false;
    for (int t = 0; t < kPcTS; ++t) {
      const int s = tile * kPcTS + t;
      any |= (s < n_sys && active[s]);
    }
    if (!any) return;
  }
  pc_body<T>(tile, Y, ldy, n_sys, Psi, ldp, n, nv, active, reinterpret_cast<T*>(smem_raw), thr());
}

template <typename T>
__global__ void k_cg_init_a(SphereTab sp, int n, const T* Bv, T* X, T* R, T* Z, long ld,
                            const double* eps, CgState cs, const int* list) {
  __shared__ double red[33];
  const int s = list ? list[blockIdx.x] : blockIdx.x;
  if (s < 0) return;   // past the count of a device-compacted list
  cg_init_a_body<T>(s, sp, n, Bv, X, R, Z, ld, eps, cs, red, thr());
}

template <typename T>
__global__ void k_cg_init_b(int n, const T* R, const T* Z, T* P, long ld, CgState cs, const int* list) {
  __shared__ double red[33];
  const int s = list ? list[blockIdx.x] : blockIdx.x;
  if (s < 0) return;
  cg_init_b_body<T>(s, n, R, Z, P, ld, cs, red, thr());
}

// out[j] = in[rows[j]] for j < n_rows (rows of length n).
__global__ void k_gather_rows(int n_rows, int n, const int* __restrict__ rows, const double* __restrict__ in,
                              long ldi, double* __restrict__ out, long ldo) {
  for (int j = blockIdx.y; j < n_rows; j += gridDim.y) {
    const double* src = in + (size_t)rows[j] * ldi;
    double* dst = out + (size_t)j * ldo;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
  }
}

template <typename T>
__global__ void k_cg_step_a(SphereTab sp, int n, T* X, T* R, T* Z, const T* P, const T* Q, long ld,
                            const double* eps, CgState cs, double tol2, int max_iter, const int* list) {
  __shared__ double red[33];
  const int s = list ? list[blockIdx.x] : blockIdx.x;
  if (s < 0) return;
  cg_step_a_body<T>(s, sp, n, X, R, Z, P, Q, ld, eps, cs, tol2, max_iter, red, thr());
}

template <typename T>
__global__ void k_cg_step_b(int n, const T* R, const T* Z, T* P, long ld, CgState cs, const int* list) {
  __shared__ double red[33];
  const int s = list ? list[blockIdx.x] : blockIdx.x;
  if (s < 0) return;
  cg_step_b_body<T>(s, n, R, Z, P, ld, cs, red, thr());
}

__global__ void k_sphere_to_rb(int n_sys, int n_el, const double* c, long ldc, const double* scale,
                               RbMap mp, int part, double* out, long ldo) {
  for (int s = blockIdx.y; s < n_sys; s += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_el; i += gridDim.x * blockDim.x)
      sphere_to_rb(s, c, ldc, scale, mp, part, out, ldo, i);
}

__global__ void k_rb_to_sphere(int n_sys, int n_pairs, const double* in, long ldi, const int* b_row,
                               const double* scale, RbMap mp, double* c, long ldc) {
  for (int s = blockIdx.y; s < n_sys; s += gridDim.y)
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= n_pairs; j += gridDim.x * blockDim.x)
      rb_to_sphere(s, in, ldi, b_row, scale, mp, c, ldc, j);
}

__global__ void k_axpby(int n_sys, int n, double alpha, const double* x, double beta, const double* y,
                        double* out, long ld, const int* active) {
  for (int s = blockIdx.y; s < n_sys; s += gridDim.y) {
    if (active && !active[s]) continue;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      axpby(s, i, alpha, x, beta, y, out, ld);
  }
}

template <typename Ti, typename To>
__global__ void k_copy_cast(int n_sys, int n, const Ti* in, long ldi, To* out, long ldo,
                            const int* active) {
  for (int s = blockIdx.y; s < n_sys; s += gridDim.y) {
    if (active && !active[s]) continue;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      out[(size_t)s * ldo + i] = To(in[(size_t)s * ldi + i]);
  }
}

template <typename T>
__global__ void k_add_to(int n_sys, int n, const T* x, long ldx, double* y, long ldy,
                         const int* active) {
  for (int s = blockIdx.y; s < n_sys; s += gridDim.y) {
    if (active && !active[s]) continue;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      y[(size_t)s * ldy + i] += double(x[(size_t)s * ldx + i]);
  }
}

// y[s] += p[s] - t[s] (FP32 inputs, difference and sum in FP64), active systems only.
__global__ void k_add_diff(int n_sys, int n, const float* p, const float* t, long ldx, double* y, long ldy,
                           const int* active) {
  for (int s = blockIdx.y; s < n_sys; s += gridDim.y) {
    if (active && !active[s]) continue;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const size_t q = (size_t)s * ldx + i;
      y[(size_t)s * ldy + i] += double(p[q]) - double(t[q]);
    }
  }
}

template <typename T>
__global__ void k_norm2(int n, const T* x, long ld, double* out) {
  __shared__ double red[33];
  const double v = block_dot(x + (size_t)blockIdx.x * ld, x + (size_t)blockIdx.x * ld, n, red, thr());
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

__global__ void k_count(const int* flags, int n, int* out) {
  __shared__ double red[33];
  double c = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) c += flags[i] != 0;
  c = block_sum(c, red, thr());
  if (threadIdx.x == 0) *out = int(c + 0.5);
}


// ---------------------------------------------------------------- P_c as two tiled GEMMs
// Y <- Y - Psi (Psi^T Y) on the systems of a list (column j of the batch is system
// s = list[j], identity when list is null).  Psi: n x nv (column v at Psi + v*ldp),
// system s at Y + s*ldy.
// Phase 1: Cpart[kb][v][j] = sum_{k in K-block kb} Psi[k][v] Y[k][s_j]   (64 x 64 tiles, 4x4 per thread)
// Reduce:  C[v][j] = sum_kb Cpart[kb][v][j], in fixed order, into slice 0
// Phase 2: Y[i][s_j] -= sum_v Psi[i][v] C[v][j]
// No atomics: the result does not depend on the launch geometry of other systems' tiles.
constexpr int kGT = 64;    // tile edge
constexpr int kGK = 16;    // K chunk of phase 1

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

// Float-float compute type for FP64 storage (T itself otherwise).
template <typename T> struct FfIfDouble { using type = T; };
template <> struct FfIfDouble<double> { using type = ff; };
template <typename T> using ff_if_double = typename FfIfDouble<T>::type;

// RAW: base holds float-float pairs in its 8-byte slots (C = ff, T = double): no conversion.
template <typename T, typename C, bool RAW = false>
__device__ __forceinline__ void load_kchunk(C (*dst)[kGT + 4], const T* __restrict__ base, long ld,
                                            const int* __restrict__ cols, int col0, int n_cols, int k0,
                                            int k_hi) {
  // dst[kk][c] = base[col(c) * ld + k0 + kk] for kk < kGK, c < kGT (zero outside).
  constexpr int V = Vec16<T>::n;
  using VT = typename Vec16<T>::type;
  for (int e = threadIdx.x; e < kGK * kGT / V; e += blockDim.x) {
    const int c = e / (kGK / V), kq = (e % (kGK / V)) * V, k = k0 + kq;
    const int cc = col0 + c;
    T vals[V];
    const int col = cc < n_cols ? (cols ? cols[cc] : cc) : -1;
    if (col >= 0) {
      const T* src = base + (size_t)col * ld + k;
      if (k + V <= k_hi) {
        const VT w = *reinterpret_cast<const VT*>(src);
        const T* wp = reinterpret_cast<const T*>(&w);
#pragma unroll
        for (int j = 0; j < V; ++j) vals[j] = wp[j];
      } else {
#pragma unroll
        for (int j = 0; j < V; ++j) vals[j] = (k + j < k_hi) ? src[j] : T(0);
      }
    } else {
#pragma unroll
      for (int j = 0; j < V; ++j) vals[j] = T(0);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) {
      if constexpr (RAW) dst[kq + j][c] = *reinterpret_cast<const C*>(&vals[j]);
      else dst[kq + j][c] = C(vals[j]);
    }
  }
}

// C = compute type (T, or ff for T = double: operands converted once while staged in shared
// memory, products accumulated in float-float).
template <typename T, typename C = T, bool PsiRaw = false>
__global__ void __launch_bounds__(256) k_pc_gemm1(const T* __restrict__ Psi, long ldp,
                                                  const T* __restrict__ Y, long ldy, int n, int nv,
                                                  int n_list, const int* __restrict__ list, int kblk,
                                                  T* __restrict__ Cpart) {
  __shared__ __align__(16) C As[kGK][kGT + 4];
  __shared__ __align__(16) C Bs[kGK][kGT + 4];
  const int j0 = blockIdx.x * kGT, v0 = blockIdx.z * kGT, kb = blockIdx.y;
  const int k_lo = kb * kblk, k_hi = min(n, k_lo + kblk);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;   // tx: systems, ty: states
  // Float-float sums are flushed into FP64 every kFlushK terms: the rounding of the float-float
  // accumulator grows with the number of terms it has taken (about n 2^-48 of the largest
  // partial sum), so over the 30k-term rows of large spheres it would cap the FP64 residuals of
  // the refinement near 1e-10; blocks of 512 keep it near 1e-13.
  constexpr bool kFf = std::is_same<C, ff>::value;
  constexpr int kFlushK = 512;
  C acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = C(0); acc64[i][j] = 0.0; }
  int since = 0;
  for (int k0 = k_lo; k0 < k_hi; k0 += kGK) {
    load_kchunk<T, C, PsiRaw>(As, Psi, ldp, nullptr, v0, nv, k0, k_hi);
    load_kchunk<T, C>(Bs, Y, ldy, list, j0, n_list, k0, k_hi);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = As[kk][ty * 4 + i]; b[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
    if constexpr (kFf) {
      since += kGK;
      if (since >= kFlushK) {
        since = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) { acc64[i][j] += static_cast<double>(acc[i][j]); acc[i][j] = C(0); }
      }
    }
  }
  const int nvp = gridDim.z * kGT;
  T* out = Cpart + (size_t)kb * nvp * n_list;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int v = v0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int jx = j0 + tx * 4 + j;
      if (jx < n_list) {
        if constexpr (kFf) out[(size_t)v * n_list + jx] = T(acc64[i][j] + static_cast<double>(acc[i][j]));
        else out[(size_t)v * n_list + jx] = T(acc[i][j]);
      }
    }
  }
}

// ---------------------------------------------------------------- FP32 P_c, wide tiles
// The FP32 projector of the inner solves: tiles of 128 systems x 64 states with 4 x 8 values
// per thread (three float4 shared-memory reads per 32 FMAs), K chunks of 32 double-buffered
// through registers.  Same partial-sum layout as k_pc_gemm1 (Cpart[kb][v][j], v padded to 64).
constexpr int kFS = 128, kFV = 64, kFK = 32, kFLA = kFV + 4, kFLB = kFS + 4;
constexpr size_t kF1Smem = sizeof(float) * 2 * kFK * (kFLA + kFLB);

__device__ __forceinline__ float4 ldg4z(const float* row, int k, int k_hi) {
  if (k + 4 <= k_hi) return *reinterpret_cast<const float4*>(row + k);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (k < k_hi) v.x = row[k];
  if (k + 1 < k_hi) v.y = row[k + 1];
  if (k + 2 < k_hi) v.z = row[k + 2];
  if (k + 3 < k_hi) v.w = row[k + 3];
  return v;
}

__global__ void __launch_bounds__(256) k_pcf_gemm1(const float* __restrict__ Psi, long ldp,
                                                   const float* __restrict__ Y, long ldy, int n, int nv,
                                                   int n_list, const int* __restrict__ list, int kblk,
                                                   float* __restrict__ Cpart) {
  extern __shared__ __align__(16) float fsm[];
  float* As = fsm;                        // [2][kFK][kFLA]  (k, state)
  float* Bs = fsm + 2 * kFK * kFLA;       // [2][kFK][kFLB]  (k, system)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int j0 = blockIdx.x * kFS, kb = blockIdx.y, v0 = blockIdx.z * kFV;
  const int k_lo = kb * kblk, k_hi = min(n, k_lo + kblk);
  const int lr = tid >> 3, lq = tid & 7;   // loader: row (of 32) and 16-byte column
  const float* brow[4];
  const float* arow[2];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int j = j0 + lr + 32 * r;
    const int sj = j < n_list ? (list ? list[j] : j) : -1;
    brow[r] = sj >= 0 ? Y + (size_t)sj * ldy : nullptr;
  }
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int v = v0 + lr + 32 * r;
    arow[r] = v < nv ? Psi + (size_t)v * ldp : nullptr;
  }
  float4 pa[2], pb[4];
  auto fetch = [&](int k0) {
    const int k = k0 + lq * 4;
#pragma unroll
    for (int r = 0; r < 2; ++r) pa[r] = arow[r] ? ldg4z(arow[r], k, k_hi) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < 4; ++r) pb[r] = brow[r] ? ldg4z(brow[r], k, k_hi) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto stash = [&](int st) {
    float* A = As + st * kFK * kFLA;
    float* B = Bs + st * kFK * kFLB;
    const int kk = lq * 4;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int v = lr + 32 * r;
      A[(kk + 0) * kFLA + v] = pa[r].x; A[(kk + 1) * kFLA + v] = pa[r].y;
      A[(kk + 2) * kFLA + v] = pa[r].z; A[(kk + 3) * kFLA + v] = pa[r].w;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int j = lr + 32 * r;
      B[(kk + 0) * kFLB + j] = pb[r].x; B[(kk + 1) * kFLB + j] = pb[r].y;
      B[(kk + 2) * kFLB + j] = pb[r].z; B[(kk + 3) * kFLB + j] = pb[r].w;
    }
  };
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  int st = 0;
  if (k_lo < k_hi) {
    fetch(k_lo);
    stash(0);
    __syncthreads();
  }
  for (int k0 = k_lo; k0 < k_hi; k0 += kFK) {
    const bool more = k0 + kFK < k_hi;
    if (more) fetch(k0 + kFK);
    const float* A = As + st * kFK * kFLA;
    const float* B = Bs + st * kFK * kFLB;
#pragma unroll 8
    for (int kk = 0; kk < kFK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(A + kk * kFLA + ty * 4);
      const float4 b0 = *reinterpret_cast<const float4*>(B + kk * kFLB + tx * 8);
      const float4 b1 = *reinterpret_cast<const float4*>(B + kk * kFLB + tx * 8 + 4);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      stash(st ^ 1);
      __syncthreads();
      st ^= 1;
    }
  }
  const int nvp = gridDim.z * kFV;
  float* out = Cpart + (size_t)kb * nvp * n_list;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int v = v0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int jx = j0 + tx * 8 + j;
      if (jx < n_list) out[(size_t)v * n_list + jx] = acc[i][j];
    }
  }
}

// Y[:, s_j] = beta Y + alpha Psi C for 64 rows x 128 systems per block, 4 rows x 8 systems per thread.
constexpr int kF2R = 64, kF2LP = kF2R + 4;
constexpr size_t kF2Smem = sizeof(float) * kFV * (kF2LP + kFLB);

__global__ void __launch_bounds__(256) k_pcf_gemm2(const float* __restrict__ Psi, long ldp, float* __restrict__ Y,
                                                   long ldy, int n, int nv, int n_list,
                                                   const int* __restrict__ list, const float* __restrict__ C,
                                                   long ldc, float alpha, float beta,
                                                   const int* __restrict__ active) {
  extern __shared__ __align__(16) float fsm[];
  float* Ps = fsm;                    // [kFV][kF2LP]  (state, row)
  float* Cs = fsm + kFV * kF2LP;      // [kFV][kFLB]   (state, system)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * kF2R, j0 = blockIdx.y * kFS;
  if (active) {
    int any = 0;
    for (int t = tid; t < kFS && j0 + t < n_list; t += 256) {
      const int st = list ? list[j0 + t] : j0 + t;
      any |= st >= 0 && active[st];
    }
    if (!__syncthreads_or(any)) return;
  }
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  for (int vc = 0; vc < nv; vc += kFV) {
    for (int e = tid; e < kFV * (kF2R / 4); e += 256) {   // Psi rows as float4 along k
      const int vv = e / (kF2R / 4), q = e % (kF2R / 4), v = vc + vv, i = i0 + q * 4;
      const float4 x = v < nv ? ldg4z(Psi + (size_t)v * ldp, i, n) : make_float4(0.f, 0.f, 0.f, 0.f);
      *reinterpret_cast<float4*>(Ps + vv * kF2LP + q * 4) = x;
    }
    for (int e = tid; e < kFV * kFS; e += 256) {
      const int vv = e / kFS, c = e % kFS, v = vc + vv, jx = j0 + c;
      Cs[vv * kFLB + c] = (v < nv && jx < n_list) ? C[(size_t)v * ldc + jx] : 0.f;
    }
    __syncthreads();
    const int vmax = min(kFV, nv - vc);
    for (int vv = 0; vv < vmax; ++vv) {
      const float4 a = *reinterpret_cast<const float4*>(Ps + vv * kF2LP + tx * 4);
      const float4 b0 = *reinterpret_cast<const float4*>(Cs + vv * kFLB + ty * 8);
      const float4 b1 = *reinterpret_cast<const float4*>(Cs + vv * kFLB + ty * 8 + 4);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  const int r0 = i0 + tx * 4;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int jx = j0 + ty * 8 + j;
    if (jx >= n_list) continue;
    const int sx = list ? list[jx] : jx;
    if (sx < 0 || (active && !active[sx])) continue;
    float* y = Y + (size_t)sx * ldy + r0;
    if (r0 + 4 <= n) {
      float4 w = beta != 0.f ? *reinterpret_cast<float4*>(y) : make_float4(0.f, 0.f, 0.f, 0.f);
      w.x = beta * w.x + alpha * acc[0][j]; w.y = beta * w.y + alpha * acc[1][j];
      w.z = beta * w.z + alpha * acc[2][j]; w.w = beta * w.w + alpha * acc[3][j];
      *reinterpret_cast<float4*>(y) = w;
    } else {
      for (int i = 0; i < 4 && r0 + i < n; ++i) y[i] = (beta != 0.f ? beta * y[i] : 0.f) + alpha * acc[i][j];
    }
  }
}

// C[e] = sum_kb Cpart[kb * slice + e] (fixed order).
__global__ void k_sum_slices(const double* __restrict__ Cpart, size_t slice, int n_kb, double* __restrict__ C) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < slice; e += (size_t)gridDim.x * blockDim.x) {
    double sum = Cpart[e];
    for (int kb = 1; kb < n_kb; ++kb) sum += Cpart[(size_t)kb * slice + e];
    C[e] = sum;
  }
}

template <typename T>
__global__ void k_pc_reduce(T* __restrict__ Cpart, size_t slice, int n_kb) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < slice; e += (size_t)gridDim.x * blockDim.x) {
    // Four independent partial sums keep four loads in flight; combined in a fixed order.
    T s0 = Cpart[e], s1 = T(0), s2 = T(0), s3 = T(0);
    int kb = 1;
    for (; kb + 3 < n_kb; kb += 4) {
      s1 += Cpart[(size_t)kb * slice + e];
      s2 += Cpart[(size_t)(kb + 1) * slice + e];
      s3 += Cpart[(size_t)(kb + 2) * slice + e];
      s0 += Cpart[(size_t)(kb + 3) * slice + e];
    }
    for (; kb < n_kb; ++kb) s1 += Cpart[(size_t)kb * slice + e];
    Cpart[e] = (s0 + s1) + (s2 + s3);
  }
}

// Y[:, s_j] = beta Y[:, s_j] + alpha sum_v Psi[:, v] C[v][j]   (C row length ldc; beta = 0 never reads Y).
template <typename T, typename CT = T, bool PsiRaw = false>
__global__ void __launch_bounds__(256) k_pc_gemm2(const T* __restrict__ Psi, long ldp, T* __restrict__ Y,
                                                  long ldy, int n, int nv, int n_list,
                                                  const int* __restrict__ list, const T* __restrict__ C,
                                                  long ldc, T alpha, T beta,
                                                  const int* __restrict__ active) {
  __shared__ __align__(16) CT Cs[kGT][kGT + 4];     // C[v][j] of one 64-state chunk
  __shared__ __align__(16) CT Ps[kGT][kGT + 4];     // Psi[i][v] stored as Ps[v][i]
  const int i0 = blockIdx.x * kGT, j0 = blockIdx.y * kGT;
  // tx: 4 consecutive rows i (vector access along the system's column), ty: 4 systems.
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  if (active) {
    bool any = false;
    for (int t = 0; t < kGT && j0 + t < n_list; ++t) {
      const int st = list ? list[j0 + t] : j0 + t;
      any |= st >= 0 && active[st] != 0;
    }
    if (!any) return;
  }
  CT acc[4][4];   // [row][system]
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = CT(0);
  for (int vc = 0; vc < nv; vc += kGT) {
    for (int e = tid; e < kGT * kGT; e += 256) {
      const int c = e % kGT, vv = e / kGT, v = vc + vv, jx = j0 + c;
      Cs[vv][c] = (jx < n_list && v < nv) ? CT(C[(size_t)v * ldc + jx]) : CT(0);
      const int i = i0 + c;
      if constexpr (PsiRaw)
        Ps[vv][c] = (v < nv && i < n) ? reinterpret_cast<const CT*>(Psi)[(size_t)v * ldp + i] : CT(0);
      else
        Ps[vv][c] = (v < nv && i < n) ? CT(Psi[(size_t)v * ldp + i]) : CT(0);
    }
    __syncthreads();
    const int vmax = min(kGT, nv - vc);
    for (int vv = 0; vv < vmax; ++vv) {
      CT a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = Ps[vv][tx * 4 + i]; b[i] = Cs[vv][ty * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  constexpr int V = Vec16<T>::n;
  using VT = typename Vec16<T>::type;
  const int r0 = i0 + tx * 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int jx = j0 + ty * 4 + j;
    if (jx >= n_list) continue;
    const int sx = list ? list[jx] : jx;
    if (sx < 0 || (active && !active[sx])) continue;
    T* y = Y + (size_t)sx * ldy + r0;
    if (r0 + 4 <= n) {
#pragma unroll
      for (int q = 0; q < 4; q += V) {
        VT w;
        if (beta != T(0)) w = *reinterpret_cast<VT*>(y + q);
        T* wp = reinterpret_cast<T*>(&w);
#pragma unroll
        for (int u = 0; u < V; ++u) wp[u] = (beta != T(0) ? beta * wp[u] : T(0)) + alpha * T(acc[q + u][j]);
        *reinterpret_cast<VT*>(y + q) = w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r0 + i < n) y[i] = (beta != T(0) ? beta * y[i] : T(0)) + alpha * T(acc[i][j]);
    }
  }
}

// Ordered list of the active systems (single block; prefix sums over chunks of 1024 flags).
__global__ void __launch_bounds__(1024) k_build_list(const int* __restrict__ active, int n_sys,
                                                     int* __restrict__ list, int* __restrict__ count) {
  __shared__ int warp_sums[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c0 = 0; c0 < n_sys; c0 += blockDim.x) {
    const int s = c0 + threadIdx.x;
    const int f = (s < n_sys && active[s]) ? 1 : 0;
    const unsigned mask = __ballot_sync(0xffffffffu, f);
    const int before = __popc(mask & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[w] = __popc(mask);
    __syncthreads();
    if (w == 0) {
      int v = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      warp_sums[lane] = v;   // inclusive
    }
    __syncthreads();
    const int woff = w ? warp_sums[w - 1] : 0;
    if (f) list[base + woff + before] = s;
    __syncthreads();
    if (threadIdx.x == 0) base += warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

// The control step of a device-driven CG loop (one block of 1024 threads), run after every
// window of iterations inside a conditional WHILE graph node: compacts the n_cap entries of
// `list` in place to the systems still flagged (keeping their order; entries past the new count
// become -1, and with rows != null the row list 2s, 2s+1 of each complex system is rebuilt the
// same way), stores the count, and sets the node's condition to keep looping while more than
// min_keep systems remain and fewer than max_windows windows have run.
__global__ void __launch_bounds__(1024) k_loop_ctl(const int* __restrict__ flags, int* __restrict__ list, int n_cap,
                                                   int* __restrict__ rows, int* __restrict__ count,
                                                   int* __restrict__ windows, int max_windows, int min_keep,
                                                   cudaGraphConditionalHandle cond) {
  __shared__ int warp_sums[32];
  __shared__ int base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n_cap; c0 += blockDim.x) {
    const int j = c0 + threadIdx.x;
    const int s = j < n_cap ? list[j] : -1;
    const int f = (s >= 0 && flags[s]) ? 1 : 0;
    const unsigned mask = __ballot_sync(0xffffffffu, f);
    const int before = __popc(mask & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[w] = __popc(mask);
    __syncthreads();   // every entry of this chunk is read before any is overwritten
    if (w == 0) {
      int v = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      warp_sums[lane] = v;
    }
    __syncthreads();
    const int pos = base + (w ? warp_sums[w - 1] : 0) + before;   // pos <= j: writes stay behind the reads
    if (f) {
      list[pos] = s;
      if (rows) { rows[2 * pos] = 2 * s; rows[2 * pos + 1] = 2 * s + 1; }
    }
    __syncthreads();
    if (threadIdx.x == 0) base += warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  const int n_left = base;
  for (int j = n_left + threadIdx.x; j < n_cap; j += blockDim.x) {
    list[j] = -1;
    if (rows) { rows[2 * j] = -1; rows[2 * j + 1] = -1; }
  }
  if (threadIdx.x == 0) {
    *count = n_left;
    const int done = ++*windows;
    cudaGraphSetConditional(cond, (n_left > min_keep && done < max_windows) ? 1u : 0u);
  }
}

template <typename T>
__global__ void k_cocg_init_a(SphereTab sp, int n, const T* Bv, T* X, T* R, T* Z, long ld, const double* eps,
                              CocgState cs) {
  __shared__ double red[33];
  cocg_init_a_body<T>(blockIdx.x, sp, n, Bv, X, R, Z, ld, eps, cs, red, thr());
}

template <typename T>
__global__ void k_cocg_init_b(int n, const T* R, const T* Z, T* P, long ld, CocgState cs) {
  __shared__ double red[33];
  cocg_init_b_body<T>(blockIdx.x, n, R, Z, P, ld, cs, red, thr());
}

template <typename T>
__global__ void k_cocg_step_a(SphereTab sp, int n, T* X, T* R, T* Z, const T* P, T* Q, long ld,
                              const double* eps, CocgState cs, double tol2, int max_iter, const int* list) {
  __shared__ double red[33];
  const int s = list ? list[blockIdx.x] : blockIdx.x;
  if (s < 0) return;
  cocg_step_a_body<T>(s, sp, n, X, R, Z, P, Q, ld, eps, cs, tol2, max_iter, red, thr());
}

template <typename T>
__global__ void k_cocg_step_b(int n, const T* R, const T* Z, T* P, long ld, CocgState cs, const int* list) {
  __shared__ double red[33];
  const int s = list ? list[blockIdx.x] : blockIdx.x;
  if (s < 0) return;
  cocg_step_b_body<T>(s, n, R, Z, P, ld, cs, red, thr());
}

__global__ void k_expand_rows(const int* __restrict__ sys, int n, int* __restrict__ rows) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    rows[2 * j] = 2 * sys[j];
    rows[2 * j + 1] = 2 * sys[j] + 1;
  }
}

__global__ void k_shifted_residual(int n_cs, int n, const double* B, const double* Q, const double* X,
                                   const double* omega, double* R, long ld, const int* active) {
  for (int s = blockIdx.y; s < n_cs; s += gridDim.y) {
    if (active && !active[s]) continue;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      shifted_residual(s, i, B, Q, X, omega[s], R, ld);
  }
}

__global__ void k_pair_norm2(int n, const double* x, long ld, double* out) {
  __shared__ double red[33];
  const double* u = x + (size_t)(2 * blockIdx.x) * ld;
  double part = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) part += u[i] * u[i] + u[ld + i] * u[ld + i];
  const double v = block_sum(part, red, thr());
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

template <typename T>
__global__ void k_scale_c_rows(T* __restrict__ C, int rows, int ncols, const T* __restrict__ d) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)rows * ncols;
       e += (size_t)gridDim.x * blockDim.x)
    C[e] *= d[e / ncols];
}

inline dim3 grid_el(int n, int n_sys) {
  int bx = (n + 255) / 256;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  return dim3(bx, n_sys < 65535 ? n_sys : 65535);
}

}  // namespace

cudaError_t ensure_smem_limit(const void* kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set_to;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set_to[std::make_pair(kernel, dev)];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t launch_loop_ctl(const int* flags, int* list, int n_cap, int* rows, int* count, int* windows,
                            int max_windows, int min_keep, cudaGraphConditionalHandle cond, cudaStream_t st) {
  k_loop_ctl<<<1, 1024, 0, st>>>(flags, list, n_cap, rows, count, windows, max_windows, min_keep, cond);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pc(T* Y, long ldy, int n_sys, const int* list, const T* Psi, long ldp, int n, int nv,
                      const int* active, T* work, cudaStream_t st, bool ffc, const unsigned char* tc_tiles,
                      const T* psi_ff, int* tc_err, int tc_split) {
  if (n_sys == 0 || nv == 0) return cudaSuccess;
  if constexpr (sizeof(T) == sizeof(float)) {
    if (tc_tiles && tc_pc_supported(nv))
      return launch_pc_tc(reinterpret_cast<float*>(Y), ldy, n_sys, list, tc_tiles, n, nv, active,
                          reinterpret_cast<float*>(work), st, tc_err, tc_split);
  }
  const int n_kb = pc_kblocks(n, n_sys);
  const int kblk = ((n + n_kb - 1) / n_kb + kGK - 1) / kGK * kGK;
  const int nvp = (nv + kGT - 1) / kGT * kGT;
  dim3 g1((n_sys + kGT - 1) / kGT, n_kb, nvp / kGT);
  const bool use_ff = ffc && sizeof(T) == sizeof(double);
  if constexpr (sizeof(T) == sizeof(float)) {
    // FP32: the wide-tile kernels, split over K so that even a short list of systems fills the
    // GPU (kblk a multiple of the 32-element K chunk).
    const int nkb_f = pcf_kblocks(n, n_sys);
    const int kblk32 = ((n + nkb_f - 1) / nkb_f + kFK - 1) / kFK * kFK;
    cudaError_t e = ensure_smem_limit((const void*)k_pcf_gemm1, kF1Smem);
    if (e != cudaSuccess) return e;
    e = ensure_smem_limit((const void*)k_pcf_gemm2, kF2Smem);
    if (e != cudaSuccess) return e;
    dim3 gf1((n_sys + kFS - 1) / kFS, (n + kblk32 - 1) / kblk32, nvp / kGT);
    const int n_kb32 = (int)gf1.y;
    k_pcf_gemm1<<<gf1, 256, kF1Smem, st>>>(reinterpret_cast<const float*>(Psi), ldp, reinterpret_cast<const float*>(Y),
                                           ldy, n, nv, n_sys, list, kblk32, reinterpret_cast<float*>(work));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n_kb32 > 1) {
      const size_t slice = (size_t)nvp * n_sys;
      k_pc_reduce<T><<<(int)std::min<size_t>((slice + 255) / 256, 4096), 256, 0, st>>>(work, slice, n_kb32);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    dim3 gf2((n + kF2R - 1) / kF2R, (n_sys + kFS - 1) / kFS);
    k_pcf_gemm2<<<gf2, 256, kF2Smem, st>>>(reinterpret_cast<const float*>(Psi), ldp, reinterpret_cast<float*>(Y), ldy,
                                           n, nv, n_sys, list, reinterpret_cast<const float*>(work), (long)n_sys,
                                           -1.f, 1.f, active);
    return cudaGetLastError();
  }
  const bool raw = use_ff && psi_ff != nullptr;
  if (raw) k_pc_gemm1<T, ff_if_double<T>, true><<<g1, 256, 0, st>>>(psi_ff, ldp, Y, ldy, n, nv, n_sys, list, kblk, work);
  else if (use_ff) k_pc_gemm1<T, ff_if_double<T>><<<g1, 256, 0, st>>>(Psi, ldp, Y, ldy, n, nv, n_sys, list, kblk, work);
  else k_pc_gemm1<T><<<g1, 256, 0, st>>>(Psi, ldp, Y, ldy, n, nv, n_sys, list, kblk, work);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if (n_kb > 1) {
    const size_t slice = (size_t)nvp * n_sys;
    k_pc_reduce<T><<<(int)std::min<size_t>((slice + 255) / 256, 4096), 256, 0, st>>>(work, slice, n_kb);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  dim3 g2((n + kGT - 1) / kGT, (n_sys + kGT - 1) / kGT);
  if (raw)
    k_pc_gemm2<T, ff_if_double<T>, true><<<g2, 256, 0, st>>>(psi_ff, ldp, Y, ldy, n, nv, n_sys, list, work,
                                                              (long)n_sys, T(-1), T(1), active);
  else if (use_ff)
    k_pc_gemm2<T, ff_if_double<T>><<<g2, 256, 0, st>>>(Psi, ldp, Y, ldy, n, nv, n_sys, list, work, (long)n_sys,
                                                        T(-1), T(1), active);
  else
    k_pc_gemm2<T><<<g2, 256, 0, st>>>(Psi, ldp, Y, ldy, n, nv, n_sys, list, work, (long)n_sys, T(-1), T(1),
                                      active);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tn(const double* A, long lda, const double* B, long ldb, int K, int m, int n, double* C,
                           double* work, cudaStream_t st, const int* cols, bool ffc) {
  if (m == 0 || n == 0) return cudaSuccess;
  const int n_kb = pc_kblocks(K, n);
  const int kblk = ((K + n_kb - 1) / n_kb + kGK - 1) / kGK * kGK;
  const int mp = (m + kGT - 1) / kGT * kGT;
  dim3 g1((n + kGT - 1) / kGT, n_kb, mp / kGT);
  if (ffc) k_pc_gemm1<double, ff><<<g1, 256, 0, st>>>(A, lda, B, ldb, K, m, n, cols, kblk, work);
  else k_pc_gemm1<double><<<g1, 256, 0, st>>>(A, lda, B, ldb, K, m, n, cols, kblk, work);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const size_t slice = (size_t)mp * n;
  k_sum_slices<<<(int)std::min<size_t>((slice + 255) / 256, 4096), 256, 0, st>>>(work, slice, n_kb, C);
  return cudaGetLastError();
}

size_t gemm_tn_work_elems(int K, int m, int n) {
  const int mp = (m + kGT - 1) / kGT * kGT;
  return (size_t)pc_kblocks(K, n) * mp * n;
}

cudaError_t launch_gemm_nn(const double* A, long lda, int n, int k, const double* C, long ldc, int ncols,
                           double* Y, long ldy, double alpha, double beta, cudaStream_t st) {
  if (ncols == 0 || n == 0) return cudaSuccess;
  if (k == 0) {
    if (beta == 1.0) return cudaSuccess;
    return cudaErrorInvalidValue;
  }
  dim3 g2((n + kGT - 1) / kGT, (ncols + kGT - 1) / kGT);
  k_pc_gemm2<double><<<g2, 256, 0, st>>>(A, lda, Y, ldy, n, k, ncols, nullptr, C, ldc, alpha, beta, nullptr);
  return cudaGetLastError();
}

__global__ void k_to_ff(size_t n, const double* __restrict__ in, ff* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = ff(in[i]);
}

cudaError_t launch_to_ff(size_t n, const double* in, double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_to_ff<<<(int)std::min<size_t>((n + 255) / 256, 8192), 256, 0, st>>>(n, in, reinterpret_cast<ff*>(out));
  return cudaGetLastError();
}

cudaError_t launch_build_list(const int* active, int n_sys, int* list, int* count, cudaStream_t st) {
  k_build_list<<<1, 1024, 0, st>>>(active, n_sys, list, count);
  return cudaGetLastError();
}

// K blocks of the FP32 wide-tile P_c: about two CTAs per SM, each at least one 32-element chunk.
int pcf_kblocks(int n, int n_sys) {
  const int tiles = (n_sys + 127) / 128;
  const int nkc = std::max(1, (n + 31) / 32);
  return std::max(1, std::min(std::min(nkc, 32), (2 * 152 + tiles - 1) / tiles));
}

int pc_kblocks(int n, int n_sys) {
  // Enough K blocks that phase 1 has >= ~4 CTAs per SM, each block >= 256 rows.
  const int s_tiles = (n_sys + kGT - 1) / kGT;
  int kb = (4 * 152 + s_tiles - 1) / s_tiles;
  kb = std::max(1, std::min(kb, std::max(1, n / 256)));
  return kb;
}

size_t pc_work_elems(int n, int n_sys, int nv) {
  const int nvp = (nv + kGT - 1) / kGT * kGT;
  return (size_t)std::max(pc_kblocks(n, n_sys), pcf_kblocks(n, n_sys)) * nvp * n_sys;
}

template <typename T>
cudaError_t launch_cg_init_a(const SphereTab& sp, int n, int n_sys, const T* Bv, T* X, T* R, T* Z,
                             long ld, const double* eps, CgState cs, cudaStream_t st, const int* list) {
  if (n_sys == 0) return cudaSuccess;
  k_cg_init_a<T><<<n_sys, kCgThreads, 0, st>>>(sp, n, Bv, X, R, Z, ld, eps, cs, list);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_init_b(int n, int n_sys, const T* R, const T* Z, T* P, long ld, CgState cs,
                             cudaStream_t st, const int* list) {
  if (n_sys == 0) return cudaSuccess;
  k_cg_init_b<T><<<n_sys, kCgThreads, 0, st>>>(n, R, Z, P, ld, cs, list);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_step_a(const SphereTab& sp, int n, int n_sys, const int* list, T* X, T* R, T* Z,
                             const T* P, const T* Q, long ld, const double* eps, CgState cs, double tol2,
                             int max_iter, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_cg_step_a<T><<<n_sys, kCgThreads, 0, st>>>(sp, n, X, R, Z, P, Q, ld, eps, cs, tol2, max_iter, list);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_step_b(int n, int n_sys, const int* list, const T* R, const T* Z, T* P, long ld,
                             CgState cs, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_cg_step_b<T><<<n_sys, kCgThreads, 0, st>>>(n, R, Z, P, ld, cs, list);
  return cudaGetLastError();
}

cudaError_t launch_sphere_to_rb(int n_sys, const double* c, long ldc, const double* scale, RbMap mp,
                                int part, double* out, long ldo, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  const int n_el = 2 * mp.n_pairs + 1;
  k_sphere_to_rb<<<grid_el(n_el, n_sys), 256, 0, st>>>(n_sys, n_el, c, ldc, scale, mp, part, out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_rb_to_sphere(int n_sys, const double* in, long ldi, const int* b_row,
                                const double* scale, RbMap mp, double* c, long ldc, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_rb_to_sphere<<<grid_el(mp.n_pairs + 1, n_sys), 256, 0, st>>>(n_sys, mp.n_pairs, in, ldi, b_row, scale, mp, c, ldc);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(int n_rows, int n, const int* rows, const double* in, long ldi, double* out, long ldo,
                               cudaStream_t st) {
  if (n_rows == 0) return cudaSuccess;
  k_gather_rows<<<grid_el(n, n_rows), 256, 0, st>>>(n_rows, n, rows, in, ldi, out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_axpby(int n_sys, int n, double alpha, const double* x, double beta,
                         const double* y, double* out, long ld, const int* active, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_axpby<<<grid_el(n, n_sys), 256, 0, st>>>(n_sys, n, alpha, x, beta, y, out, ld, active);
  return cudaGetLastError();
}

template <typename Ti, typename To>
cudaError_t launch_copy_cast(int n_sys, int n, const Ti* in, long ldi, To* out, long ldo,
                             const int* active, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_copy_cast<Ti, To><<<grid_el(n, n_sys), 256, 0, st>>>(n_sys, n, in, ldi, out, ldo, active);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add_to(int n_sys, int n, const T* x, long ldx, double* y, long ldy,
                          const int* active, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_add_to<T><<<grid_el(n, n_sys), 256, 0, st>>>(n_sys, n, x, ldx, y, ldy, active);
  return cudaGetLastError();
}

cudaError_t launch_add_diff(int n_sys, int n, const float* p, const float* t, long ldx, double* y, long ldy,
                            const int* active, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_add_diff<<<grid_el(n, n_sys), 256, 0, st>>>(n_sys, n, p, t, ldx, y, ldy, active);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_norm2(int n_sys, int n, const T* x, long ld, double* out, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_norm2<T><<<n_sys, 256, 0, st>>>(n, x, ld, out);
  return cudaGetLastError();
}

cudaError_t launch_count(const int* flags, int n, int* out, cudaStream_t st) {
  k_count<<<1, 256, 0, st>>>(flags, n, out);
  return cudaGetLastError();
}


template <typename T>
cudaError_t launch_cocg_init_a(const SphereTab& sp, int n, int n_cs, const T* Bv, T* X, T* R, T* Z, long ld,
                               const double* eps, CocgState cs, cudaStream_t st) {
  if (n_cs == 0) return cudaSuccess;
  k_cocg_init_a<T><<<n_cs, kCgThreads, 0, st>>>(sp, n, Bv, X, R, Z, ld, eps, cs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cocg_init_b(int n, int n_cs, const T* R, const T* Z, T* P, long ld, CocgState cs,
                               cudaStream_t st) {
  if (n_cs == 0) return cudaSuccess;
  k_cocg_init_b<T><<<n_cs, kCgThreads, 0, st>>>(n, R, Z, P, ld, cs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cocg_step_a(const SphereTab& sp, int n, int n_list, const int* list, T* X, T* R, T* Z,
                               const T* P, T* Q, long ld, const double* eps, CocgState cs, double tol2,
                               int max_iter, cudaStream_t st) {
  if (n_list == 0) return cudaSuccess;
  k_cocg_step_a<T><<<n_list, kCgThreads, 0, st>>>(sp, n, X, R, Z, P, Q, ld, eps, cs, tol2, max_iter, list);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cocg_step_b(int n, int n_list, const int* list, const T* R, const T* Z, T* P, long ld,
                               CocgState cs, cudaStream_t st) {
  if (n_list == 0) return cudaSuccess;
  k_cocg_step_b<T><<<n_list, kCgThreads, 0, st>>>(n, R, Z, P, ld, cs, list);
  return cudaGetLastError();
}

cudaError_t launch_expand_rows(const int* sys, int n, int* rows, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_expand_rows<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(sys, n, rows);
  return cudaGetLastError();
}

cudaError_t launch_shifted_residual(int n_cs, int n, const double* B, const double* Q, const double* X,
                                    const double* omega, double* R, long ld, const int* active, cudaStream_t st) {
  if (n_cs == 0) return cudaSuccess;
  k_shifted_residual<<<grid_el(n, n_cs), 256, 0, st>>>(n_cs, n, B, Q, X, omega, R, ld, active);
  return cudaGetLastError();
}

cudaError_t launch_pair_norm2(int n_cs, int n, const double* x, long ld, double* out, cudaStream_t st) {
  if (n_cs == 0) return cudaSuccess;
  k_pair_norm2<<<n_cs, 256, 0, st>>>(n, x, ld, out);
  return cudaGetLastError();
}

#define WGW_INST_COCG(T)                                                                           \
  template cudaError_t launch_cocg_init_a<T>(const SphereTab&, int, int, const T*, T*, T*, T*, long, \
                                             const double*, CocgState, cudaStream_t);               \
  template cudaError_t launch_cocg_init_b<T>(int, int, const T*, const T*, T*, long, CocgState,     \
                                             cudaStream_t);                                         \
  template cudaError_t launch_cocg_step_a<T>(const SphereTab&, int, int, const int*, T*, T*, T*,    \
                                             const T*, T*, long, const double*, CocgState, double,  \
                                             int, cudaStream_t);                                    \
  template cudaError_t launch_cocg_step_b<T>(int, int, const int*, const T*, const T*, T*, long,    \
                                             CocgState, cudaStream_t);
WGW_INST_COCG(float)
WGW_INST_COCG(double)

// Q[:, s_j] += B diag(D) B^T P[:, s_j]  (Kleinman-Bylander term, Sec. 3: V_NL = sum_p |beta_p> D_p <beta_p|).
template <typename T>
cudaError_t launch_kb(T* Q, const T* P, long ld, int n_sys, const int* list, const T* B, long ldb, int n, int n_proj,
                      const T* D, T* work, cudaStream_t st, bool ffc) {
  const bool use_ff = ffc && sizeof(T) == sizeof(double);
  if (n_sys == 0 || n_proj == 0) return cudaSuccess;
  const int n_kb = pc_kblocks(n, n_sys);
  const int kblk = ((n + n_kb - 1) / n_kb + kGK - 1) / kGK * kGK;
  const int nvp = (n_proj + kGT - 1) / kGT * kGT;
  dim3 g1((n_sys + kGT - 1) / kGT, n_kb, nvp / kGT);
  if (use_ff) k_pc_gemm1<T, ff_if_double<T>><<<g1, 256, 0, st>>>(B, ldb, P, ld, n, n_proj, n_sys, list, kblk, work);
  else k_pc_gemm1<T><<<g1, 256, 0, st>>>(B, ldb, P, ld, n, n_proj, n_sys, list, kblk, work);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const size_t slice = (size_t)nvp * n_sys;
  if (n_kb > 1) {
    k_pc_reduce<T><<<(int)std::min<size_t>((slice + 255) / 256, 4096), 256, 0, st>>>(work, slice, n_kb);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  k_scale_c_rows<T><<<(int)std::min<size_t>(((size_t)n_proj * n_sys + 255) / 256, 4096), 256, 0, st>>>(
      work, n_proj, n_sys, D);
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  dim3 g2((n + kGT - 1) / kGT, (n_sys + kGT - 1) / kGT);
  if (use_ff)
    k_pc_gemm2<T, ff_if_double<T>><<<g2, 256, 0, st>>>(B, ldb, Q, ld, n, n_proj, n_sys, list, work, (long)n_sys,
                                                        T(1), T(1), nullptr);
  else
    k_pc_gemm2<T><<<g2, 256, 0, st>>>(B, ldb, Q, ld, n, n_proj, n_sys, list, work, (long)n_sys, T(1), T(1), nullptr);
  return cudaGetLastError();
}
template cudaError_t launch_kb<float>(float*, const float*, long, int, const int*, const float*, long, int, int,
                                      const float*, float*, cudaStream_t, bool);
template cudaError_t launch_kb<double>(double*, const double*, long, int, const int*, const double*, long, int, int,
                                       const double*, double*, cudaStream_t, bool);

#define WGW_INST_LA(T)                                                                             \
  template cudaError_t launch_pc<T>(T*, long, int, const int*, const T*, long, int, int,           \
                                    const int*, T*, cudaStream_t, bool, const unsigned char*,      \
                                    const T*, int*, int);                                          \
  template cudaError_t launch_cg_init_a<T>(const SphereTab&, int, int, const T*, T*, T*, T*, long, \
                                           const double*, CgState, cudaStream_t, const int*);     \
  template cudaError_t launch_cg_init_b<T>(int, int, const T*, const T*, T*, long, CgState,       \
                                           cudaStream_t, const int*);                             \
  template cudaError_t launch_cg_step_a<T>(const SphereTab&, int, int, const int*, T*, T*, T*,     \
                                           const T*, const T*, long, const double*, CgState,      \
                                           double, int, cudaStream_t);                            \
  template cudaError_t launch_cg_step_b<T>(int, int, const int*, const T*, const T*, T*, long,    \
                                           CgState, cudaStream_t);                                \
  template cudaError_t launch_add_to<T>(int, int, const T*, long, double*, long, const int*,      \
                                        cudaStream_t);                                            \
  template cudaError_t launch_norm2<T>(int, int, const T*, long, double*, cudaStream_t);
WGW_INST_LA(float)
WGW_INST_LA(double)
template cudaError_t launch_copy_cast<double, float>(int, int, const double*, long, float*, long,
                                                     const int*, cudaStream_t);
template cudaError_t launch_copy_cast<float, double>(int, int, const float*, long, double*, long,
                                                     const int*, cudaStream_t);
template cudaError_t launch_copy_cast<double, double>(int, int, const double*, long, double*, long,
                                                      const int*, cudaStream_t);

}  // namespace wgw
