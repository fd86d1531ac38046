// Small dense FP64 kernels of the PDEP Davidson (Sec. 3 and Sec. 4.2): the symmetric
// eigensolver of the Rayleigh-Ritz step and the elementwise helpers of the subspace
// updates.  The tall-skinny products use the tiled GEMMs of la_kernels.cu.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/wgw.h"
#include "internal.h"

namespace wgw {

namespace {

// Symmetric eigenproblem A = Z diag(w) Z^T for n <= kSyevMax, in one thread block.
//
// Householder tridiagonalisation: for k = 0 .. n-3 the reflector H = I - 2 v v^T
// (|v| = 1) maps column k below the diagonal onto a multiple of e_{k+1}; the
// trailing block becomes H A H = A - v w^T - w v^T with p = A v, w = 2p - 2(v.p)v,
// and Z <- Z H accumulates the transformations.  The tridiagonal matrix (d, e) is
// then diagonalised by the implicit-shift QL iteration (Wilkinson-type shift from
// the leading 2x2 block, chase of Givens rotations from the bottom of the
// unreduced block up to l); thread 0 computes each sweep's rotations and every
// thread applies them to its own rows of Z.  Eigenvalues are sorted ascending.
// A (column-major, lda) is overwritten.  work: n*n + 4n doubles.  info[0] = 0, or
// the index+1 of an eigenvalue that did not converge in 64 sweeps.
constexpr int kSyevMax = 2048;

__global__ void __launch_bounds__(1024) k_syev(int n, double* __restrict__ A, int lda, double* __restrict__ w,
                                               double* __restrict__ Z, int ldz, double* __restrict__ work,
                                               int* __restrict__ info) {
  __shared__ double red[33];
  __shared__ int sh_int[4];
  extern __shared__ double rot[];            // 2 * n: cosines and sines of one QL sweep
  const int tid = threadIdx.x, nth = blockDim.x;
  Thr th{tid, nth};
  double* v = work;                          // n
  double* p = work + n;                      // n
  double* d = work + 2 * n;                  // n
  double* e = work + 3 * n;                  // n
  double* Zs = work + 4 * n;                 // n * n
  for (int i = tid; i < n * n; i += nth) {
    const int r = i % n, c = i / n;
    Z[(size_t)c * ldz + r] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;   // length of the column below the diagonal
    double part = 0.0;
    for (int i = tid; i < m; i += nth) {
      const double x = A[(size_t)k * lda + k + 1 + i];
      part += x * x;
    }
    const double nx2 = block_sum(part, red, th);
    if (nx2 == 0.0) continue;
    const double x0 = A[(size_t)k * lda + k + 1];
    const double alpha = x0 > 0 ? -sqrt(nx2) : sqrt(nx2);
    const double vn = sqrt(nx2 - x0 * x0 + (x0 - alpha) * (x0 - alpha));
    for (int i = tid; i < m; i += nth) {
      const double x = A[(size_t)k * lda + k + 1 + i];
      v[i] = (i == 0 ? x - alpha : x) / vn;
    }
    __syncthreads();
    // p = A22 v (column j of A22 dotted with v: A22 is symmetric, columns are contiguous).
    const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
    for (int j = warp; j < m; j += nw) {
      const double* col = A + (size_t)(k + 1 + j) * lda + k + 1;
      double s = 0.0;
      for (int i = lane; i < m; i += 32) s += col[i] * v[i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) p[j] = s;
    }
    __syncthreads();
    double pc = 0.0;
    for (int i = tid; i < m; i += nth) pc += v[i] * p[i];
    const double c = block_sum(pc, red, th);
    for (int i = tid; i < m; i += nth) p[i] = 2.0 * p[i] - 2.0 * c * v[i];   // w
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += nth) {
      const int i = idx % m, j = idx / m;
      A[(size_t)(k + 1 + j) * lda + k + 1 + i] -= v[i] * p[j] + p[i] * v[j];
    }
    for (int i = tid; i < m; i += nth) {
      const double val = i == 0 ? alpha : 0.0;
      A[(size_t)k * lda + k + 1 + i] = val;
      A[(size_t)(k + 1 + i) * lda + k] = val;
    }
    __syncthreads();
    // Z <- Z H:  u = Z[:, k+1:] v,  Z[:, k+1:] -= 2 u v^T  (u stored in Zs[0..n)).
    for (int r = tid; r < n; r += nth) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += Z[(size_t)(k + 1 + j) * ldz + r] * v[j];
      Zs[r] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < n * m; idx += nth) {
      const int r = idx % n, j = idx / n;
      Z[(size_t)(k + 1 + j) * ldz + r] -= 2.0 * Zs[r] * v[j];
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nth) {
    d[i] = A[(size_t)i * lda + i];
    e[i] = i + 1 < n ? A[(size_t)i * lda + i + 1] : 0.0;
  }
  if (tid == 0) info[0] = 0;
  __syncthreads();
  // Implicit-shift QL on (d, e).
  double* cs = rot;
  double* sn = rot + n;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      if (tid == 0) {
        int m = l;
        for (; m < n - 1; ++m) {
          const double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= 2.220446049250313e-16 * dd) break;
        }
        int lo = m;   // rotations i = m-1 .. lo were recorded
        if (m != l && iter < 64) {
          double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
          double r = hypot(g, 1.0);
          g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
          double s = 1.0, c = 1.0, pp = 0.0;
          int i = m - 1;
          bool underflow = false;
          for (; i >= l; --i) {
            const double f = s * e[i], b = c * e[i];
            r = hypot(f, g);
            e[i + 1] = r;
            if (r == 0.0) {
              d[i + 1] -= pp;
              e[m] = 0.0;
              underflow = true;
              break;
            }
            s = f / r;
            c = g / r;
            g = d[i + 1] - pp;
            r = (d[i] - g) * s + 2.0 * c * b;
            pp = s * r;
            d[i + 1] = g + pp;
            g = c * r - b;
            cs[i] = c;
            sn[i] = s;
          }
          lo = underflow ? i + 1 : l;
          if (!underflow) {
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
          }
        }
        if (m != l && iter >= 64 && info[0] == 0) info[0] = l + 1;
        sh_int[0] = m;
        sh_int[1] = lo;
        sh_int[2] = (m == l || iter >= 64) ? 1 : 0;
      }
      __syncthreads();
      const int m = sh_int[0], lo = sh_int[1], done = sh_int[2];
      if (done) break;
      for (int r = tid; r < n; r += nth) {
        for (int i = m - 1; i >= lo; --i) {
          double* zi = Z + (size_t)i * ldz + r;
          double* zi1 = Z + (size_t)(i + 1) * ldz + r;
          const double f = *zi1;
          *zi1 = sn[i] * *zi + cs[i] * f;
          *zi = cs[i] * *zi - sn[i] * f;
        }
      }
      __syncthreads();
    }
  }
  // Sort ascending (selection order computed by thread 0, columns permuted through Zs).
  if (tid == 0) {
    for (int i = 0; i < n; ++i) p[i] = i;
    for (int i = 0; i < n; ++i) {
      int best = i;
      for (int j = i + 1; j < n; ++j)
        if (d[(int)p[j]] < d[(int)p[best]]) best = j;
      const double t = p[i]; p[i] = p[best]; p[best] = t;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nth) {
    const int r = idx % n, c = idx / n;
    Zs[idx] = Z[(size_t)((int)p[c]) * ldz + r];
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += nth) {
    const int r = idx % n, c = idx / n;
    Z[(size_t)c * ldz + r] = Zs[idx];
  }
  for (int i = tid; i < n; i += nth) w[i] = d[(int)p[i]];
}

// R[:, j] = AX[:, j] - theta[j] X[:, j]; rnorm[j] = ||R[:, j]||.
__global__ void k_ritz_residual(int n, int nb, const double* __restrict__ X, const double* __restrict__ AX,
                                long ld, const double* __restrict__ theta, double* __restrict__ R,
                                double* __restrict__ rnorm) {
  __shared__ double red[33];
  const int j = blockIdx.x;
  Thr th{(int)threadIdx.x, (int)blockDim.x};
  double part = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = AX[(size_t)j * ld + i] - theta[j] * X[(size_t)j * ld + i];
    R[(size_t)j * ld + i] = r;
    part += r * r;
  }
  const double s = block_sum(part, red, th);
  if (threadIdx.x == 0) rnorm[j] = sqrt(s);
}

// Symmetrise an m x m matrix stored row-major with row length ldt: T = (T + T^T)/2.
__global__ void k_symmetrise(int m, double* T, int ldt) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * m; idx += gridDim.x * blockDim.x) {
    const int i = idx / m, j = idx % m;
    if (j > i) {
      const double a = 0.5 * (T[(size_t)i * ldt + j] + T[(size_t)j * ldt + i]);
      T[(size_t)i * ldt + j] = a;
      T[(size_t)j * ldt + i] = a;
    }
  }
}

// C[j][c] = Y[j][idx[c]] * scale[c]: select and scale eigenvector columns (row-major k x kk input).
__global__ void k_select_scale(int k, const double* __restrict__ Zc, int ldz, const int* __restrict__ cols,
                               const double* __restrict__ scale, int nc, double* __restrict__ out, int ldo) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < k * nc; idx += gridDim.x * blockDim.x) {
    const int j = idx % k, c = idx / k;
    out[(size_t)j * ldo + c] = Zc[(size_t)cols[c] * ldz + j] * (scale ? scale[c] : 1.0);
  }
}

}  // namespace

cudaError_t launch_syev(int n, double* A, int lda, double* w, double* Z, int ldz, double* work, int* info,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kSyevMax) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * 2 * (size_t)n;
  if (smem > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(k_syev, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
  }
  k_syev<<<1, 1024, smem, st>>>(n, A, lda, w, Z, ldz, work, info);
  return cudaGetLastError();
}

size_t syev_work_elems(int n) { return (size_t)n * n + 4 * (size_t)n; }

cudaError_t launch_ritz_residual(int n, int nb, const double* X, const double* AX, long ld, const double* theta,
                                 double* R, double* rnorm, cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  k_ritz_residual<<<nb, 256, 0, st>>>(n, nb, X, AX, ld, theta, R, rnorm);
  return cudaGetLastError();
}

cudaError_t launch_symmetrise(int m, double* T, int ldt, cudaStream_t st) {
  k_symmetrise<<<std::max(1, std::min(1024, (m * m + 255) / 256)), 256, 0, st>>>(m, T, ldt);
  return cudaGetLastError();
}

cudaError_t launch_select_scale(int k, const double* Zc, int ldz, const int* cols, const double* scale, int nc,
                                double* out, int ldo, cudaStream_t st) {
  if (nc == 0 || k == 0) return cudaSuccess;
  k_select_scale<<<std::max(1, std::min(1024, (k * nc + 255) / 256)), 256, 0, st>>>(k, Zc, ldz, cols, scale, nc,
                                                                                     out, ldo);
  return cudaGetLastError();
}

}  // namespace wgw

// ---------------------------------------------------------------- scratch-free variant
// Work space of wgw_symm_eig_noalloc_dev: a file-scope device array sized for the largest
// accepted n.  Every GPU that loads the library holds it (about 2.1 MB) until the process
// exits, and every call shares it.
namespace {

constexpr int kNoAllocMaxN = 512;
constexpr size_t kNoAllocElems = (size_t)kNoAllocMaxN * kNoAllocMaxN + 4 * kNoAllocMaxN + 2;
static __device__ __align__(256) double g_syev_scratch[kNoAllocElems];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_syev_scratch on the current device.  The host-side symbol is only a
// stand-in and must never reach a kernel; the address is looked up once per device (with
// that device current) and cached.
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return wgw::report_error(WGW_ERR_CUDA, cudaGetErrorString(err));
  if (dev < 0 || dev >= kMaxDevices) return wgw::report_error(WGW_ERR_STATE, "device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_syev_scratch);
    if (err != cudaSuccess || !p)
      return wgw::report_error(WGW_ERR_CUDA, "cudaGetSymbolAddress of the eigensolver scratch failed");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return WGW_OK;
}

}  // namespace

extern "C" int wgw_symm_eig_noalloc_dev(int n, double* A_dev, double* w_dev, double* Z_dev, void* stream) {
  wgw::clear_error();
  if (n < 1 || n > kNoAllocMaxN)
    return wgw::report_error(WGW_ERR_ARG, "wgw_symm_eig_noalloc_dev accepts 1 <= n <= 512");
  if (!A_dev || !w_dev || !Z_dev) return wgw::report_error(WGW_ERR_ARG, "null device pointer");
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != WGW_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // The kernel writes every work entry before reading it and sets info itself, so the
  // previous call's contents need no clearing.
  int* info = reinterpret_cast<int*>(scratch + wgw::syev_work_elems(n));
  cudaError_t err = wgw::launch_syev(n, A_dev, n, w_dev, Z_dev, n, scratch, info, st);
  if (err != cudaSuccess) return wgw::report_error(WGW_ERR_CUDA, cudaGetErrorString(err));
  int h = 0;
  err = cudaMemcpyAsync(&h, info, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err != cudaSuccess) return wgw::report_error(WGW_ERR_CUDA, cudaGetErrorString(err));
  return h == 0 ? WGW_OK : wgw::report_error(WGW_ERR_NOCONV, "dense eigensolver did not converge");
}
