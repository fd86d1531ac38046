// __global__ wrappers of the linear-algebra kernels (bodies in la_bodies.cuh).
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
                            const double* eps, CgState cs) {
  __shared__ double red[33];
  cg_init_a_body<T>(blockIdx.x, sp, n, Bv, X, R, Z, ld, eps, cs, red, thr());
}

template <typename T>
__global__ void k_cg_init_b(int n, const T* R, const T* Z, T* P, long ld, CgState cs) {
  __shared__ double red[33];
  cg_init_b_body<T>(blockIdx.x, n, R, Z, P, ld, cs, red, thr());
}

template <typename T>
__global__ void k_cg_step_a(SphereTab sp, int n, T* X, T* R, T* Z, const T* P, const T* Q, long ld,
                            const double* eps, CgState cs, double tol2, int max_iter) {
  __shared__ double red[33];
  cg_step_a_body<T>(blockIdx.x, sp, n, X, R, Z, P, Q, ld, eps, cs, tol2, max_iter, red, thr());
}

template <typename T>
__global__ void k_cg_step_b(int n, const T* R, const T* Z, T* P, long ld, CgState cs) {
  __shared__ double red[33];
  cg_step_b_body<T>(blockIdx.x, n, R, Z, P, ld, cs, red, thr());
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

inline dim3 grid_el(int n, int n_sys) {
  int bx = (n + 255) / 256;
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  return dim3(bx, n_sys < 65535 ? n_sys : 65535);
}

}  // namespace

template <typename T>
cudaError_t launch_pc(T* Y, long ldy, int n_sys, const T* Psi, long ldp, int n, int nv,
                      const int* active, cudaStream_t st) {
  if (n_sys == 0 || nv == 0) return cudaSuccess;
  const size_t smem = sizeof(T) * (size_t)(nv * kPcTS + kPcKC * nv + kPcKC * kPcTS);
  if (smem > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(k_pc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  k_pc<T><<<(n_sys + kPcTS - 1) / kPcTS, 256, smem, st>>>(Y, ldy, n_sys, Psi, ldp, n, nv, active);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_init_a(const SphereTab& sp, int n, int n_sys, const T* Bv, T* X, T* R, T* Z,
                             long ld, const double* eps, CgState cs, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_cg_init_a<T><<<n_sys, kCgThreads, 0, st>>>(sp, n, Bv, X, R, Z, ld, eps, cs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_init_b(int n, int n_sys, const T* R, const T* Z, T* P, long ld, CgState cs,
                             cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_cg_init_b<T><<<n_sys, kCgThreads, 0, st>>>(n, R, Z, P, ld, cs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_step_a(const SphereTab& sp, int n, int n_sys, T* X, T* R, T* Z, const T* P,
                             const T* Q, long ld, const double* eps, CgState cs, double tol2,
                             int max_iter, cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_cg_step_a<T><<<n_sys, kCgThreads, 0, st>>>(sp, n, X, R, Z, P, Q, ld, eps, cs, tol2, max_iter);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_step_b(int n, int n_sys, const T* R, const T* Z, T* P, long ld, CgState cs,
                             cudaStream_t st) {
  if (n_sys == 0) return cudaSuccess;
  k_cg_step_b<T><<<n_sys, kCgThreads, 0, st>>>(n, R, Z, P, ld, cs);
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

#define WGW_INST_LA(T)                                                                             \
  template cudaError_t launch_pc<T>(T*, long, int, const T*, long, int, int, const int*,           \
                                    cudaStream_t);                                                 \
  template cudaError_t launch_cg_init_a<T>(const SphereTab&, int, int, const T*, T*, T*, T*, long, \
                                           const double*, CgState, cudaStream_t);                 \
  template cudaError_t launch_cg_init_b<T>(int, int, const T*, const T*, T*, long, CgState,       \
                                           cudaStream_t);                                         \
  template cudaError_t launch_cg_step_a<T>(const SphereTab&, int, int, T*, T*, T*, const T*,      \
                                           const T*, long, const double*, CgState, double, int,   \
                                           cudaStream_t);                                         \
  template cudaError_t launch_cg_step_b<T>(int, int, const T*, const T*, T*, long, CgState,       \
                                           cudaStream_t);                                         \
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
