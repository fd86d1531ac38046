// Small dense FP64 kernels of the PDEP Davidson (Sec. 3 and Sec. 4.2): the symmetric
// eigensolver of the Rayleigh-Ritz step and the elementwise helpers of the subspace
// updates.  The tall-skinny products use the tiled GEMMs of la_kernels.cu.
#include <algorithm>
#include <cmath>
#include <mutex>

#include <cuda.h>   // CUcontext / CUresult types only

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
                                               int* __restrict__ info, int tridiagonal) {
  __shared__ double red[33];
  __shared__ int sh_int[4];
  extern __shared__ double rot[];            // 2 * n: cosines and sines of one QL sweep
  const int tid = threadIdx.x, nth = blockDim.x;
  Thr th{tid, nth};
  // Batched use: block b works on matrix b (consecutive n x n blocks of A, Z, work, w, info).
  A += (size_t)blockIdx.x * lda * n;
  Z += (size_t)blockIdx.x * ldz * n;
  w += (size_t)blockIdx.x * n;
  work += (size_t)blockIdx.x * ((size_t)n * n + 4 * (size_t)n);
  info += blockIdx.x;
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
  // A tridiagonal input is already in the form the Householder stage produces (Z = I).
  for (int k = 0; !tridiagonal && k + 2 < n; ++k) {
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

// ---------------------------------------------------------------- Lanczos chains (Sec. 3, Eq. lanczos)
// Chain s holds q^l at Q + (l * n_ch + s) * ld.

// Split Gram-Schmidt: chain s = blockIdx.x, chunk blockIdx.y of the n reals (gridDim.y chunks),
// so that a few hundred chains still fill the GPU.  Partial sums go to part[(s nb + b)(l+1) + j]
// and are summed in chunk order by the consumer (deterministic).  The arithmetic type C is
// double (native FP64) or ff (float-float on the FP32 units, for GPUs whose FP64 rate is a small
// fraction of FP32): with C = ff the previous Lanczos vectors are read from a float-float copy
// (8 bytes per real, like a double) and the vectors in and out stay double.
__device__ __forceinline__ void lz_chunk(int n, int& i0, int& i1) {
  const int per = (n + (int)gridDim.y - 1) / (int)gridDim.y;
  i0 = (int)blockIdx.y * per;
  i1 = min(n, i0 + per);
}

template <typename C> __device__ __forceinline__ C lz_c(double v);
template <> __device__ __forceinline__ double lz_c<double>(double v) { return v; }
template <> __device__ __forceinline__ ff lz_c<ff>(double v) { return ff(v); }
__device__ __forceinline__ double lz_d(double v) { return v; }
__device__ __forceinline__ double lz_d(ff v) { return double(v); }
__device__ __forceinline__ void lz_warp_sum(double& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
}
__device__ __forceinline__ void lz_warp_sum(ff& a) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    a = a + ff(__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off));
}

constexpr int kLzJ = 8;   // dot products accumulated per sweep over the chunk
constexpr int kLzE = 4;   // elements per thread per sweep (256-thread blocks)
constexpr int kLzChunkMax = 4096;   // reals per chunk (32 KB of shared memory in the dots kernel)

// part[(s nb + b)(l+1) + j] = sum over chunk b of q^j[i] x[i], j = 0..l.  256 threads; each thread
// holds kLzE elements of x so that kLzJ x kLzE independent loads are in flight per sweep.  The
// chunk of x is converted to C once into shared memory (dynamic, chunk x sizeof(C) bytes): a
// double -> float-float conversion runs on the FP64 unit.
template <typename C>
__global__ void __launch_bounds__(256) k_lz_gs_dots(int n, int l, int n_ch, const C* __restrict__ Qg, long ld,
                                                    const double* X, double* __restrict__ part) {
  __shared__ double red[8][kLzJ];
  extern __shared__ __align__(16) unsigned char lz_smem[];
  C* xs = reinterpret_cast<C*>(lz_smem);
  const int s = blockIdx.x, nb = gridDim.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int i0, i1;
  lz_chunk(n, i0, i1);
  const double* x = X + (size_t)s * ld;
  for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) xs[i - i0] = lz_c<C>(x[i]);
  __syncthreads();
  for (int j0 = 0; j0 <= l; j0 += kLzJ) {
    const int nj = min(kLzJ, l + 1 - j0);
    C acc[kLzJ];
#pragma unroll
    for (int jj = 0; jj < kLzJ; ++jj) acc[jj] = lz_c<C>(0.0);
    for (int base = i0 + (int)threadIdx.x; base < i1; base += kLzE * 256) {
      C xv[kLzE];
#pragma unroll
      for (int e = 0; e < kLzE; ++e) {
        const int i = base + e * 256;
        xv[e] = i < i1 ? xs[i - i0] : lz_c<C>(0.0);
      }
#pragma unroll
      for (int jj = 0; jj < kLzJ; ++jj) {
        if (jj < nj) {
          const C* q = Qg + ((size_t)(j0 + jj) * n_ch + s) * ld;
#pragma unroll
          for (int e = 0; e < kLzE; ++e) {
            const int i = base + e * 256;
            if (i < i1) mac(acc[jj], q[i], xv[e]);
          }
        }
      }
    }
#pragma unroll
    for (int jj = 0; jj < kLzJ; ++jj) lz_warp_sum(acc[jj]);
    if (lane == 0) {
#pragma unroll
      for (int jj = 0; jj < kLzJ; ++jj) red[warp][jj] = lz_d(acc[jj]);
    }
    __syncthreads();
    if ((int)threadIdx.x < nj) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
      part[((size_t)s * nb + blockIdx.y) * (l + 1) + j0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// r = x - sum_j c_j q^j on chunk b, c_j = sum over chunks of part (x may alias r).  With alpha,
// block (s, 0) stores alpha_l = c_l (the first pass, over x = H q^l, is the three-term step and
// the first Gram-Schmidt pass at once); alpha_only stops there.  With npart, the chunk's
// partial |r|^2 goes to npart[s nb + b].  256 threads.
template <typename C>
__global__ void __launch_bounds__(256) k_lz_gs_update(int n, int l, int n_ch, const C* __restrict__ Qg, long ld,
                                                      const double* X, double* R, const double* __restrict__ part,
                                                      double* __restrict__ alpha, int n_steps, int alpha_only,
                                                      double* __restrict__ npart) {
  __shared__ C ncoef[256];
  __shared__ double red[33];
  const int s = blockIdx.x, nb = gridDim.y;
  for (int j = threadIdx.x; j <= l; j += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[((size_t)s * nb + b) * (l + 1) + j];
    ncoef[j] = lz_c<C>(-t);
    if (j == l && alpha && blockIdx.y == 0) alpha[(size_t)s * n_steps + l] = t;
  }
  __syncthreads();
  if (alpha_only) return;
  int i0, i1;
  lz_chunk(n, i0, i1);
  const double* x = X + (size_t)s * ld;
  double* r = R + (size_t)s * ld;
  C nn = lz_c<C>(0.0);
  // kLzE elements per thread, j outermost: kLzE independent loads per j, four j unrolled.
  for (int base = i0 + (int)threadIdx.x; base < i1; base += kLzE * 256) {
    C acc[kLzE];
#pragma unroll
    for (int e = 0; e < kLzE; ++e) {
      const int i = base + e * 256;
      acc[e] = lz_c<C>(i < i1 ? x[i] : 0.0);
    }
#pragma unroll 4
    for (int j = 0; j <= l; ++j) {
      const C cj = ncoef[j];
      const C* q = Qg + ((size_t)j * n_ch + s) * ld;
#pragma unroll
      for (int e = 0; e < kLzE; ++e) {
        const int i = base + e * 256;
        if (i < i1) mac(acc[e], cj, q[i]);
      }
    }
#pragma unroll
    for (int e = 0; e < kLzE; ++e) {
      const int i = base + e * 256;
      if (i < i1) {
        r[i] = lz_d(acc[e]);
        mac(nn, acc[e], acc[e]);
      }
    }
  }
  if (npart) {
    Thr th{(int)threadIdx.x, (int)blockDim.x};
    const double t = block_sum(lz_d(nn), red, th);
    if (threadIdx.x == 0) npart[(size_t)s * nb + blockIdx.y] = t;
  }
}

// beta_{l+1} = |r|, q^{l+1} = r / beta_{l+1} on chunk b; a chain whose |r| fell to 1e-14 beta_0
// or below stops (q^{l+1} = 0, beta_{l+1} = 0).  |r|^2 comes from the partial norms npart, or,
// with npart null and a single chunk, from the block itself.  With C = ff the float-float copy
// Qf of q^{l+1} is written too.
template <typename C>
__global__ void __launch_bounds__(256) k_lz_normalise_split(int n, int l, int n_ch, const double* __restrict__ R,
                                                            double* __restrict__ Q, C* __restrict__ Qf, long ld,
                                                            double* __restrict__ beta, int n_steps,
                                                            const double* __restrict__ npart) {
  __shared__ double red[33];
  const int s = blockIdx.x, nb = gridDim.y;
  const double* r = R + (size_t)s * ld;
  int i0, i1;
  lz_chunk(n, i0, i1);
  double t = 0.0;
  if (npart) {
    for (int b = 0; b < nb; ++b) t += npart[(size_t)s * nb + b];
  } else {
    double part = 0.0;
    for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) part = fma(r[i], r[i], part);
    Thr th{(int)threadIdx.x, (int)blockDim.x};
    t = block_sum(part, red, th);
  }
  const double nrm = sqrt(t);
  const double b0 = beta[(size_t)s * n_steps];
  const bool stop = !(nrm > 1e-14 * b0);
  const double inv = stop ? 0.0 : 1.0 / nrm;
  const size_t off = ((size_t)(l + 1) * n_ch + s) * ld;
  for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) {
    const double qv = r[i] * inv;
    Q[off + i] = qv;
    if (Qf) Qf[off + i] = lz_c<C>(qv);
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) beta[(size_t)s * n_steps + l + 1] = stop ? 0.0 : nrm;
}

// beta_0 = |b|, q^0 = b / beta_0.
__global__ void k_lz_start(int n, const double* __restrict__ B, double* __restrict__ Q, long ld,
                           double* __restrict__ beta, int n_steps) {
  __shared__ double red[33];
  const int s = blockIdx.x;
  Thr th{(int)threadIdx.x, (int)blockDim.x};
  const double* b = B + (size_t)s * ld;
  double part = 0.0;
  for (int i = th.tid; i < n; i += th.nth) part += b[i] * b[i];
  const double nb = sqrt(block_sum(part, red, th));
  double* q = Q + (size_t)s * ld;
  for (int i = th.tid; i < n; i += th.nth) q[i] = nb > 0 ? b[i] / nb : 0.0;
  if (th.tid == 0) beta[(size_t)s * n_steps] = nb;
}

// Dense tridiagonal matrix of each chain: alpha on the diagonal, beta_1.. off it.
__global__ void k_lz_tridiag(int n_ch, int n_steps, const double* __restrict__ alpha, const double* __restrict__ beta,
                             double* __restrict__ T) {
  const size_t total = (size_t)n_ch * n_steps * n_steps;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ((size_t)n_steps * n_steps));
    const int rem = (int)(e % ((size_t)n_steps * n_steps));
    const int i = rem % n_steps, j = rem / n_steps;
    double v = 0.0;
    if (i == j) v = alpha[(size_t)s * n_steps + i];
    else if (j == i + 1) v = beta[(size_t)s * n_steps + j];
    else if (i == j + 1) v = beta[(size_t)s * n_steps + i];
    T[e] = v;
  }
}

// y[(k, s, l)] = beta_0 sum_l' U_{l l'} U_{0 l'} g_k(d_l'), g = 1/(e_v - d - i w) + 1/(e_v - d + i w)
// = 2 (e_v - d) / ((e_v - d)^2 + w^2), for chain s = m * n_v + v.
__global__ void k_lz_resolvent(int n_ch, int n_steps, int n_v, int n_om, const double* __restrict__ d,
                               const double* __restrict__ U, const double* __restrict__ beta,
                               const double* __restrict__ e_v, const double* __restrict__ omega,
                               double* __restrict__ y) {
  const size_t total = (size_t)n_om * n_ch * n_steps;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(e % n_steps);
    const int s = (int)((e / n_steps) % n_ch);
    const int k = (int)(e / ((size_t)n_steps * n_ch));
    const double ev = e_v[s % n_v], w = omega[k];
    const double* Us = U + (size_t)s * n_steps * n_steps;   // column-major: U(i, j) at j * n_steps + i
    const double* ds = d + (size_t)s * n_steps;
    double acc = 0.0;
    for (int lp = 0; lp < n_steps; ++lp) {
      const double x = ev - ds[lp];
      acc += Us[(size_t)lp * n_steps + l] * Us[(size_t)lp * n_steps] * (2.0 * x / (x * x + w * w));
    }
    y[e] = beta[(size_t)s * n_steps] * acc;
  }
}

// chi0[k][m][n] = coef sum_v sum_l ov_v[n][l * n_pdep + m] y[k][m n_v + v][l].
__global__ void k_lz_assemble(int n_pdep, int n_v, int n_steps, int n_om, const double* __restrict__ ov,
                              const double* __restrict__ y, double coef, double* __restrict__ chi) {
  const int n_ch = n_pdep * n_v;
  const size_t total = (size_t)n_om * n_pdep * n_pdep;
  const size_t ovs = (size_t)((n_pdep + 63) / 64 * 64) * n_steps * n_pdep;   // per-v block of gemm output
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(e % n_pdep);
    const int m = (int)((e / n_pdep) % n_pdep);
    const int k = (int)(e / ((size_t)n_pdep * n_pdep));
    double acc = 0.0;
    for (int v = 0; v < n_v; ++v) {
      const double* o = ov + (size_t)v * ovs + (size_t)n * n_steps * n_pdep;
      const double* yy = y + ((size_t)k * n_ch + (size_t)m * n_v + v) * n_steps;
      for (int l = 0; l < n_steps; ++l) acc += o[(size_t)l * n_pdep + m] * yy[l];
    }
    chi[e] = coef * acc;
  }
}
// G0 chains (Eq. ISR): residues C[v][n][l'][m] = beta_1 U_{0 l'} sum_l ov_v[n][l n_pdep + m] U_{l l'}
// for chain s = m n_v + v (v indexes the list of states).
__global__ void k_lz_residues(int n_pdep, int n_v, int n_steps, const double* __restrict__ ov,
                              const double* __restrict__ U, const double* __restrict__ beta, double* __restrict__ C) {
  const size_t total = (size_t)n_v * n_pdep * n_steps * n_pdep;
  const size_t ovs = (size_t)((n_pdep + 63) / 64 * 64) * n_steps * n_pdep;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % n_pdep);
    const int lp = (int)((e / n_pdep) % n_steps);
    const int nn = (int)((e / ((size_t)n_pdep * n_steps)) % n_pdep);
    const int v = (int)(e / ((size_t)n_pdep * n_steps * n_pdep));
    const int s = m * n_v + v;
    const double* Us = U + (size_t)s * n_steps * n_steps + (size_t)lp * n_steps;   // column l'
    const double* o = ov + (size_t)v * ovs + (size_t)nn * n_steps * n_pdep + m;
    double acc = 0.0;
    for (int l = 0; l < n_steps; ++l) acc += o[(size_t)l * n_pdep] * Us[l];
    C[e] = beta[(size_t)s * n_steps] * Us[0] * acc;
  }
}

// g0[v][k][n][m] = sum_l' C[v][n][l'][m] / (d_s[l'] - z_k), complex (interleaved), s = m n_v + v.
__global__ void k_lz_g0_eval(int n_pdep, int n_v, int n_steps, int n_z, const double* __restrict__ C,
                             const double* __restrict__ d, const double* __restrict__ z, double* __restrict__ g) {
  const size_t total = (size_t)n_v * n_z * n_pdep * n_pdep;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(e % n_pdep);
    const int nn = (int)((e / n_pdep) % n_pdep);
    const int k = (int)((e / ((size_t)n_pdep * n_pdep)) % n_z);
    const int v = (int)(e / ((size_t)n_pdep * n_pdep * n_z));
    const double zr = z[2 * k], zi = z[2 * k + 1];
    const double* ds = d + (size_t)(m * n_v + v) * n_steps;
    const double* c = C + ((size_t)v * n_pdep + nn) * n_steps * n_pdep + m;
    double re = 0.0, im = 0.0;
    for (int lp = 0; lp < n_steps; ++lp) {
      // 1 / (x - i zi) = (x + i zi) / (x^2 + zi^2), x = d - zr
      const double x = ds[lp] - zr, den = x * x + zi * zi, cv = c[(size_t)lp * n_pdep];
      re += cv * x / den;
      im += cv * zi / den;
    }
    g[2 * e] = re;
    g[2 * e + 1] = im;
  }
}
// Eq. ISR by quadrature: out[i][j] = coef sum_k (w_k / 2 pi) sum_nm lam[k][n][m]
// (g[i][(j nk + k) 2][n][m] + g[i][(j nk + k) 2 + 1][n][m]), complex.  One block per (i, j).
__global__ void __launch_bounds__(256) k_lz_isr(int n_pdep, int n_states, int n_omega, int n_nodes,
                                                const double* __restrict__ g, const double* __restrict__ lam,
                                                const double* __restrict__ w, double coef, double* __restrict__ out) {
  __shared__ double red[33];
  const int i = blockIdx.x / n_omega, j = blockIdx.x % n_omega;
  const int nz = 2 * n_omega * n_nodes;
  const size_t mm = (size_t)n_pdep * n_pdep;
  Thr th{(int)threadIdx.x, (int)blockDim.x};
  double re = 0.0, im = 0.0;
  for (size_t e = threadIdx.x; e < (size_t)n_nodes * mm; e += blockDim.x) {
    const int k = (int)(e / mm);
    const size_t nm = e % mm;
    const double f = lam[e] * w[k] * (0.5 / 3.14159265358979323846);
    const size_t zp = (size_t)(j * n_nodes + k) * 2;
    const double* gp = g + 2 * (((size_t)i * nz + zp) * mm + nm);
    const double* gm = g + 2 * (((size_t)i * nz + zp + 1) * mm + nm);
    re += f * (gp[0] + gm[0]);
    im += f * (gp[1] + gm[1]);
  }
  re = block_sum(re, red, th);
  im = block_sum(im, red, th);
  if (threadIdx.x == 0) {
    out[2 * ((size_t)i * n_omega + j)] = coef * re;
    out[2 * ((size_t)i * n_omega + j) + 1] = coef * im;
  }
}
}  // namespace

cudaError_t launch_syev(int n, double* A, int lda, double* w, double* Z, int ldz, double* work, int* info,
                        cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kSyevMax) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * 2 * (size_t)n;
  {
    cudaError_t err = ensure_smem_limit((const void*)k_syev, smem);
    if (err != cudaSuccess) return err;
  }
  k_syev<<<1, 1024, smem, st>>>(n, A, lda, w, Z, ldz, work, info, 0);
  return cudaGetLastError();
}

cudaError_t launch_syev_batched(int n, int batch, double* A, double* w, double* Z, double* work, int* info,
                                cudaStream_t st, bool tridiagonal) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  if (n > kSyevMax) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * 2 * (size_t)n;
  {
    cudaError_t err = ensure_smem_limit((const void*)k_syev, smem);
    if (err != cudaSuccess) return err;
  }
  k_syev<<<batch, n <= 128 ? 128 : 1024, smem, st>>>(n, A, n, w, Z, n, work, info, tridiagonal ? 1 : 0);
  return cudaGetLastError();
}

#define WGW_G1D(total) std::max<size_t>(1, std::min<size_t>(4096, ((size_t)(total) + 255) / 256))

cudaError_t launch_lz_start(int n, int n_ch, const double* B, double* Q, long ld, double* beta, int n_steps,
                            cudaStream_t st) {
  k_lz_start<<<n_ch, 256, 0, st>>>(n, B, Q, ld, beta, n_steps);
  return cudaGetLastError();
}

cudaError_t launch_lz_tridiag(int n_ch, int n_steps, const double* alpha, const double* beta, double* T,
                              cudaStream_t st) {
  k_lz_tridiag<<<WGW_G1D((size_t)n_ch * n_steps * n_steps), 256, 0, st>>>(n_ch, n_steps, alpha, beta, T);
  return cudaGetLastError();
}
cudaError_t launch_lz_resolvent(int n_ch, int n_steps, int n_v, int n_om, const double* d, const double* U,
                                const double* beta, const double* e_v, const double* omega, double* y,
                                cudaStream_t st) {
  k_lz_resolvent<<<WGW_G1D((size_t)n_om * n_ch * n_steps), 256, 0, st>>>(n_ch, n_steps, n_v, n_om, d, U, beta,
                                                                          e_v, omega, y);
  return cudaGetLastError();
}
cudaError_t launch_lz_assemble(int n_pdep, int n_v, int n_steps, int n_om, const double* ov, const double* y,
                               double coef, double* chi, cudaStream_t st) {
  k_lz_assemble<<<WGW_G1D((size_t)n_om * n_pdep * n_pdep), 256, 0, st>>>(n_pdep, n_v, n_steps, n_om, ov, y,
                                                                          coef, chi);
  return cudaGetLastError();
}

int lz_split(int n, int n_ch) {
  const int want = (4 * 304 + n_ch - 1) / n_ch;      // about eight 256-thread blocks per SM
  // Chunks of 512 .. 4096 reals (the dots kernel stages a chunk in 32 KB of shared memory).
  return std::max((n + kLzChunkMax - 1) / kLzChunkMax, std::max(1, std::min(want, (n + 511) / 512)));
}

cudaError_t launch_lz_gs_dots(int n, int l, int n_ch, const double* Q, const double* Qf, long ld, const double* X,
                              double* part, int nb, cudaStream_t st) {
  if (l > 255) return cudaErrorInvalidValue;
  const int per = (n + nb - 1) / nb;
  if (per > kLzChunkMax) return cudaErrorInvalidValue;
  const size_t smem = sizeof(double) * (size_t)per;   // sizeof(ff) == sizeof(double)
  if (Qf)
    k_lz_gs_dots<ff><<<dim3(n_ch, nb), 256, smem, st>>>(n, l, n_ch, reinterpret_cast<const ff*>(Qf), ld, X, part);
  else
    k_lz_gs_dots<double><<<dim3(n_ch, nb), 256, smem, st>>>(n, l, n_ch, Q, ld, X, part);
  return cudaGetLastError();
}

cudaError_t launch_lz_gs_update(int n, int l, int n_ch, const double* Q, const double* Qf, long ld, const double* X,
                                double* R, const double* part, double* alpha, int n_steps, bool alpha_only,
                                double* npart, int nb, cudaStream_t st) {
  if (l > 255) return cudaErrorInvalidValue;
  if (Qf)
    k_lz_gs_update<ff><<<dim3(n_ch, nb), 256, 0, st>>>(n, l, n_ch, reinterpret_cast<const ff*>(Qf), ld, X, R, part,
                                                       alpha, n_steps, alpha_only ? 1 : 0, npart);
  else
    k_lz_gs_update<double><<<dim3(n_ch, nb), 256, 0, st>>>(n, l, n_ch, Q, ld, X, R, part, alpha, n_steps,
                                                           alpha_only ? 1 : 0, npart);
  return cudaGetLastError();
}

cudaError_t launch_lz_normalise(int n, int l, int n_ch, const double* R, double* Q, double* Qf, long ld,
                                double* beta, int n_steps, const double* npart, int nb, cudaStream_t st) {
  if (!npart) nb = 1;   // the norm is then reduced inside the one block of each chain
  if (Qf)
    k_lz_normalise_split<ff><<<dim3(n_ch, nb), 256, 0, st>>>(n, l, n_ch, R, Q, reinterpret_cast<ff*>(Qf), ld, beta,
                                                             n_steps, npart);
  else
    k_lz_normalise_split<double><<<dim3(n_ch, nb), 256, 0, st>>>(n, l, n_ch, R, Q, nullptr, ld, beta, n_steps,
                                                                 npart);
  return cudaGetLastError();
}

cudaError_t launch_lz_residues(int n_pdep, int n_v, int n_steps, const double* ov, const double* U, const double* beta,
                               double* C, cudaStream_t st) {
  k_lz_residues<<<WGW_G1D((size_t)n_v * n_pdep * n_steps * n_pdep), 256, 0, st>>>(n_pdep, n_v, n_steps, ov, U, beta,
                                                                                   C);
  return cudaGetLastError();
}

cudaError_t launch_lz_isr(int n_pdep, int n_states, int n_omega, int n_nodes, const double* g, const double* lam,
                          const double* w, double coef, double* out, cudaStream_t st) {
  k_lz_isr<<<n_states * n_omega, 256, 0, st>>>(n_pdep, n_states, n_omega, n_nodes, g, lam, w, coef, out);
  return cudaGetLastError();
}

cudaError_t launch_lz_g0_eval(int n_pdep, int n_v, int n_steps, int n_z, const double* C, const double* d,
                              const double* z, double* g, cudaStream_t st) {
  k_lz_g0_eval<<<WGW_G1D((size_t)n_v * n_z * n_pdep * n_pdep), 256, 0, st>>>(n_pdep, n_v, n_steps, n_z, C, d, z, g);
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

// ---------------------------------------------------------------- Dyson equation
// X = (1 - A)^-1 A for one n x n matrix per block (row-major, batch over imaginary
// frequencies): Gaussian elimination of M = 1 - A with partial pivoting (ties to the lower
// row), applied to the right-hand side X = A, then back substitution.  M is work space.
// info[k] = 1 if frequency k met a zero pivot.
__global__ void __launch_bounds__(256) k_dyson(int n, const double* __restrict__ A, double* __restrict__ X,
                                               double* __restrict__ M, int* __restrict__ info) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int piv;
  const size_t off = (size_t)blockIdx.x * n * n;
  const double* a = A + off;
  double* x = X + off;
  double* m = M + off;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, w = tid >> 5, nw = (nth + 31) >> 5;
  for (int e = tid; e < n * n; e += nth) {
    m[e] = (e / n == e % n ? 1.0 : 0.0) - a[e];
    x[e] = a[e];
  }
  if (tid == 0) info[blockIdx.x] = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += nth) {
      const double v = fabs(m[(size_t)i * n + k]);
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { rv[w] = best; ri[w] = bi; }
    __syncthreads();
    if (tid == 0) {
      double b = -1.0;
      int p = n;
      for (int q = 0; q < nw; ++q)
        if (rv[q] > b || (rv[q] == b && ri[q] < p)) { b = rv[q]; p = ri[q]; }
      piv = p;
      if (!(b > 0.0)) info[blockIdx.x] = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != k && p < n) {
      for (int j = tid; j < n; j += nth) {
        const double t = m[(size_t)k * n + j]; m[(size_t)k * n + j] = m[(size_t)p * n + j]; m[(size_t)p * n + j] = t;
        const double u = x[(size_t)k * n + j]; x[(size_t)k * n + j] = x[(size_t)p * n + j]; x[(size_t)p * n + j] = u;
      }
    }
    __syncthreads();
    const double d = m[(size_t)k * n + k];
    if (d != 0.0) {
      const int rows = n - k - 1, cols = (n - k - 1) + n;   // M columns k+1.. then all X columns
      for (int e = tid; e < rows * cols; e += nth) {
        const int i = k + 1 + e / cols, c = e % cols;
        const double f = m[(size_t)i * n + k] / d;
        if (c < n - k - 1) m[(size_t)i * n + k + 1 + c] -= f * m[(size_t)k * n + k + 1 + c];
        else x[(size_t)i * n + (c - (n - k - 1))] -= f * x[(size_t)k * n + (c - (n - k - 1))];
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const double d = m[(size_t)k * n + k];
    for (int j = tid; j < n; j += nth) x[(size_t)k * n + j] = d != 0.0 ? x[(size_t)k * n + j] / d : 0.0;
    __syncthreads();
    for (int e = tid; e < k * n; e += nth) {
      const int i = e / n, j = e % n;
      x[(size_t)i * n + j] -= m[(size_t)i * n + k] * x[(size_t)k * n + j];
    }
    __syncthreads();
  }
}

cudaError_t launch_dyson(int n, int n_omega, const double* A, double* X, double* M, int* info, cudaStream_t st) {
  if (n <= 0 || n_omega <= 0) return cudaSuccess;
  k_dyson<<<n_omega, 256, 0, st>>>(n, A, X, M, info);
  return cudaGetLastError();
}

}  // namespace wgw

// ---------------------------------------------------------------- scratch-free variant
// Work space of wgw_symm_eig_noalloc_dev: a file-scope device array sized for the largest
// accepted n (about 2.1 MB).  It exists on a GPU once this file's device code is loaded there
// (wgw_setup on that device loads it, and so does the first call of the entry point), stays
// until the process exits, and is shared by every call.
namespace {

constexpr int kNoAllocMaxN = 512;
constexpr size_t kNoAllocElems = (size_t)kNoAllocMaxN * kNoAllocMaxN + 4 * kNoAllocMaxN + 2;
static __device__ __align__(256) double g_syev_scratch[kNoAllocElems];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
// Per device: the array's device address and the CUDA context it was looked up in.  A context
// created after a cudaDeviceReset (or another context made current through the driver API)
// holds its own copy of the array, so a different current context means a fresh lookup.
struct ScratchSlot {
  CUcontext ctx = nullptr;
  double* ptr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// The context current on the calling thread (null if none), through the driver entry point the
// runtime hands out, so the library needs no link against the driver library.
CUcontext current_context() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of g_syev_scratch on the current device.  The host-side symbol is only a
// stand-in and must never reach a kernel; the address is looked up with the device current
// (which also loads this file's device code there if nothing has yet) and cached per device
// and context.
int scratch_address(double** out) {
  int dev = -1;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return wgw::report_error(WGW_ERR_CUDA, cudaGetErrorString(err));
  if (dev < 0 || dev >= kMaxDevices) return wgw::report_error(WGW_ERR_STATE, "device index out of range");
  const CUcontext cur = current_context();
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchSlot& slot = g_scratch[dev];
  if (!slot.ptr || !cur || cur != slot.ctx) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_syev_scratch);
    if (err != cudaSuccess || !p)
      return wgw::report_error(WGW_ERR_CUDA, "cudaGetSymbolAddress of the eigensolver scratch failed");
    slot.ptr = static_cast<double*>(p);
    slot.ctx = current_context();
  }
  *out = slot.ptr;
  return WGW_OK;
}

}  // namespace

namespace wgw {
// Loads the scratch-free eigensolver's work array on the current device and caches its address
// (called by wgw_setup, so that a context's device is prepared before its memory fills up).
int noalloc_prepare() {
  double* p = nullptr;
  return scratch_address(&p);
}
}  // namespace wgw

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
