// __global__ wrappers of the pruned 3D FFT pipeline (bodies in fft_bodies.cuh).
#include "internal.h"

namespace wgw {

int fft_threads(int n) { return n >= 40 ? 256 : 128; }

namespace {

__device__ __forceinline__ Thr thr() { Thr t; t.tid = threadIdx.x; t.nth = blockDim.x; return t; }

__device__ __forceinline__ bool pair_idle(const int* active, int pair, int n_sys) {
  if (active == nullptr) return false;
  const int s0 = 2 * pair, s1 = 2 * pair + 1;
  return !active[s0] && (s1 >= n_sys || !active[s1]);
}

template <typename T>
__global__ void k_plane_g2r(SphereTab sp, FftPlan pl, const cplx<T>* tw, const T* X, long ldx,
                            int n_sys, const int* active, cplx<T>* Tbuf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int pair = blockIdx.x, hi = blockIdx.y;
  if (pair_idle(active, pair, n_sys)) return;
  cplx<T>* tws = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* B = tws + pl.n;
  for (int i = threadIdx.x; i < pl.n; i += blockDim.x) tws[i] = tw[i];
  __syncthreads();
  plane_g2r_body<T>(pair, hi, sp, pl, tws, X, ldx, n_sys, active, Tbuf, B, thr());
}

template <typename T>
__global__ void k_xline(int m, FftPlan pl, const cplx<T>* tw, cplx<T>* Tbuf, XArgs<T> a,
                        const int* active) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int pair = blockIdx.x, y = blockIdx.y;
  if (pair_idle(active, pair, a.n_sys)) return;
  cplx<T>* tws = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* S = tws + pl.n;
  for (int i = threadIdx.x; i < pl.n; i += blockDim.x) tws[i] = tw[i];
  __syncthreads();
  xline_body<T>(pair, y, m, pl, tws, Tbuf, a, S, thr());
}

template <typename T>
__global__ void k_plane_r2g(SphereTab sp, FftPlan pl, const cplx<T>* tw, const cplx<T>* Tbuf,
                            Epi<T> e) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int pair = blockIdx.x, hp = blockIdx.y;
  if (pair_idle(e.active, pair, e.n_sys)) return;
  cplx<T>* tws = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* B = tws + pl.n;
  cplx<T>* Zp = B + pl.n * (pl.n + 1);
  for (int i = threadIdx.x; i < pl.n; i += blockDim.x) tws[i] = tw[i];
  __syncthreads();
  plane_r2g_body<T>(pair, hp, sp, pl, tws, Tbuf, e, B, Zp, thr());
}

template <typename T>
__global__ void k_drho_xline(int m, FftPlan pl, const cplx<T>* tw, const cplx<T>* Tbuf,
                             const T* psi_r, long ldpsi, int n_v, int n_sys, T coef, T* D, long ldd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x, y = blockIdx.y;
  cplx<T>* tws = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* S = tws + pl.n;
  T* acc = reinterpret_cast<T*>(S + pl.n * (pl.n + 1));
  for (int i = threadIdx.x; i < pl.n; i += blockDim.x) tws[i] = tw[i];
  __syncthreads();
  drho_xline_body<T>(p, y, m, pl, tws, Tbuf, psi_r, ldpsi, n_v, n_sys, coef, D, ldd, S, acc, thr());
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

template <typename T>
cudaError_t launch_plane_g2r(const SphereTab& sp, FftCtx<T> f, const T* X, long ldx, int n_sys,
                             const int* active, cplx<T>* Tbuf, cudaStream_t st) {
  const int N = f.plan.n, pairs = (n_sys + 1) / 2;
  if (pairs == 0) return cudaSuccess;
  const size_t smem = sizeof(cplx<T>) * (size_t)(N + N * (N + 1));
  cudaError_t err = set_smem(k_plane_g2r<T>, smem);
  if (err != cudaSuccess) return err;
  dim3 grid(pairs, 2 * sp.m + 1);
  k_plane_g2r<T><<<grid, fft_threads(N), smem, st>>>(sp, f.plan, f.tw, X, ldx, n_sys, active, Tbuf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_xline(int m, FftCtx<T> f, cplx<T>* Tbuf, const XArgs<T>& a, const int* active,
                         cudaStream_t st) {
  const int N = f.plan.n, pairs = (a.n_sys + 1) / 2;
  if (pairs == 0) return cudaSuccess;
  const size_t smem = sizeof(cplx<T>) * (size_t)(N + N * (N + 1));
  cudaError_t err = set_smem(k_xline<T>, smem);
  if (err != cudaSuccess) return err;
  dim3 grid(pairs, N);
  k_xline<T><<<grid, fft_threads(N), smem, st>>>(m, f.plan, f.tw, Tbuf, a, active);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_plane_r2g(const SphereTab& sp, int npt_max, FftCtx<T> f, const cplx<T>* Tbuf,
                             const Epi<T>& e, cudaStream_t st) {
  const int N = f.plan.n, pairs = (e.n_sys + 1) / 2;
  if (pairs == 0) return cudaSuccess;
  const size_t smem = sizeof(cplx<T>) * (size_t)(N + N * (N + 1) + npt_max);
  cudaError_t err = set_smem(k_plane_r2g<T>, smem);
  if (err != cudaSuccess) return err;
  dim3 grid(pairs, sp.m + 1);
  k_plane_r2g<T><<<grid, fft_threads(N), smem, st>>>(sp, f.plan, f.tw, Tbuf, e);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_drho_xline(int m, FftCtx<T> f, const cplx<T>* Tbuf, const T* psi_r, long ldpsi,
                              int n_v, int n_sys, int n_pert, T coef, T* D, long ldd,
                              cudaStream_t st) {
  const int N = f.plan.n;
  if (n_pert == 0) return cudaSuccess;
  const size_t smem = sizeof(cplx<T>) * (size_t)(N + N * (N + 1)) + sizeof(T) * (size_t)N * N;
  cudaError_t err = set_smem(k_drho_xline<T>, smem);
  if (err != cudaSuccess) return err;
  dim3 grid(n_pert, N);
  k_drho_xline<T><<<grid, fft_threads(N), smem, st>>>(m, f.plan, f.tw, Tbuf, psi_r, ldpsi, n_v,
                                                       n_sys, coef, D, ldd);
  return cudaGetLastError();
}

#define WGW_INST_FFT(T)                                                                            \
  template cudaError_t launch_plane_g2r<T>(const SphereTab&, FftCtx<T>, const T*, long, int,      \
                                           const int*, cplx<T>*, cudaStream_t);                   \
  template cudaError_t launch_xline<T>(int, FftCtx<T>, cplx<T>*, const XArgs<T>&, const int*,     \
                                       cudaStream_t);                                             \
  template cudaError_t launch_plane_r2g<T>(const SphereTab&, int, FftCtx<T>, const cplx<T>*,      \
                                           const Epi<T>&, cudaStream_t);                          \
  template cudaError_t launch_drho_xline<T>(int, FftCtx<T>, const cplx<T>*, const T*, long, int,  \
                                            int, int, T, T*, long, cudaStream_t);
WGW_INST_FFT(float)
WGW_INST_FFT(double)

}  // namespace wgw
