// Kernels of the correlation self-energy at real frequencies (Sec. 2, Eq. sigmacIR with its
// parts Eq. ISR and Eq. Rfac; Sec. 3, Eq. lanczos for the frequency dependence): the response in
// the basis at complex frequencies from the residues of the chi0 Lanczos chains, the Dyson step
// at complex frequencies, I^SR at one real frequency per evaluation point, and the residue term's
// contraction.  All FP64; these are small dense problems next to the chains that feed them.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace wgw {

namespace {

constexpr double kPi = 3.14159265358979323846;

// chi[e][m][n] = coef sum_v sum_l' W[v][n][l'][m] g(e_v - d_(m n_v + v)[l'], z_e),
// g(a, z) = 1/(a - z) + 1/(a + z): the i w of Eq. lanczos replaced by the complex z_e.
// W: residues of the chains of P_c H P_c (the G0 residue layout with v over every occupied
// state).  One thread per (e, m, n); complex values interleaved.
__global__ void k_chi_z(int n_pdep, int n_v, int n_steps, int n_e, const double* __restrict__ W,
                        const double* __restrict__ d, const double* __restrict__ e_v, const double* __restrict__ z,
                        double coef, double* __restrict__ chi) {
  const size_t total = (size_t)n_e * n_pdep * n_pdep;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(t % n_pdep);
    const int m = (int)((t / n_pdep) % n_pdep);
    const int e = (int)(t / ((size_t)n_pdep * n_pdep));
    const double zr = z[2 * e], zi = z[2 * e + 1];
    double re = 0.0, im = 0.0;
    for (int v = 0; v < n_v; ++v) {
      const double* ds = d + (size_t)(m * n_v + v) * n_steps;
      const double* w = W + ((size_t)v * n_pdep + n) * n_steps * n_pdep + m;
      const double ev = e_v[v];
      for (int lp = 0; lp < n_steps; ++lp) {
        const double a = ev - ds[lp], c = w[(size_t)lp * n_pdep];
        // 1/((a - zr) - i zi) + 1/((a + zr) + i zi)
        const double x1 = a - zr, x2 = a + zr;
        const double q1 = 1.0 / (x1 * x1 + zi * zi), q2 = 1.0 / (x2 * x2 + zi * zi);
        re += c * (x1 * q1 + x2 * q2);
        im += c * (zi * q1 - zi * q2);
      }
    }
    chi[2 * t] = coef * re;
    chi[2 * t + 1] = coef * im;
  }
}

// X = (1 - A)^-1 A for one complex n x n row-major matrix per block (interleaved): Gaussian
// elimination of M = 1 - A with partial pivoting on |M_ik|^2 (ties to the lower row), applied to
// the right-hand side X = A, then back substitution.  info[b] = 1 on a zero pivot.
__global__ void __launch_bounds__(256) k_dyson_z(int n, const double* __restrict__ A, double* __restrict__ X,
                                                 double* __restrict__ M, int* __restrict__ info) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int piv;
  const size_t off = 2 * (size_t)blockIdx.x * n * n;
  const double* a = A + off;
  double* x = X + off;
  double* mm = M + off;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, w = tid >> 5, nw = (nth + 31) >> 5;
  for (int e = tid; e < n * n; e += nth) {
    mm[2 * e] = (e / n == e % n ? 1.0 : 0.0) - a[2 * e];
    mm[2 * e + 1] = -a[2 * e + 1];
    x[2 * e] = a[2 * e];
    x[2 * e + 1] = a[2 * e + 1];
  }
  if (tid == 0) info[blockIdx.x] = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += nth) {
      const size_t q = 2 * ((size_t)i * n + k);
      const double v = mm[q] * mm[q] + mm[q + 1] * mm[q + 1];
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
      for (int j = tid; j < 2 * n; j += nth) {
        const size_t rk = 2 * (size_t)k * n + j, rp = 2 * (size_t)p * n + j;
        const double t = mm[rk]; mm[rk] = mm[rp]; mm[rp] = t;
        const double u = x[rk]; x[rk] = x[rp]; x[rp] = u;
      }
    }
    __syncthreads();
    const size_t kk = 2 * ((size_t)k * n + k);
    const double dr = mm[kk], di = mm[kk + 1], dn = dr * dr + di * di;
    if (dn > 0.0) {
      const double ir = dr / dn, ii = -di / dn;   // 1 / d
      const int rows = n - k - 1, cols = (n - k - 1) + n;   // M columns k+1.. then all X columns
      for (int e = tid; e < rows * cols; e += nth) {
        const int i = k + 1 + e / cols, c = e % cols;
        const size_t ik = 2 * ((size_t)i * n + k);
        const double fr = mm[ik] * ir - mm[ik + 1] * ii, fi = mm[ik] * ii + mm[ik + 1] * ir;   // f = M_ik / d
        double* dst;
        const double* src;
        if (c < n - k - 1) {
          dst = mm + 2 * ((size_t)i * n + k + 1 + c);
          src = mm + 2 * ((size_t)k * n + k + 1 + c);
        } else {
          dst = x + 2 * ((size_t)i * n + (c - (n - k - 1)));
          src = x + 2 * ((size_t)k * n + (c - (n - k - 1)));
        }
        dst[0] -= fr * src[0] - fi * src[1];
        dst[1] -= fr * src[1] + fi * src[0];
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const size_t kk = 2 * ((size_t)k * n + k);
    const double dr = mm[kk], di = mm[kk + 1], dn = dr * dr + di * di;
    const double ir = dn > 0.0 ? dr / dn : 0.0, ii = dn > 0.0 ? -di / dn : 0.0;
    for (int j = tid; j < n; j += nth) {
      double* xv = x + 2 * ((size_t)k * n + j);
      const double r = xv[0] * ir - xv[1] * ii, im = xv[0] * ii + xv[1] * ir;
      xv[0] = r;
      xv[1] = im;
    }
    __syncthreads();
    for (int e = tid; e < k * n; e += nth) {
      const int i = e / n, j = e % n;
      const double* mv = mm + 2 * ((size_t)i * n + k);
      const double* xk = x + 2 * ((size_t)k * n + j);
      double* xi = x + 2 * ((size_t)i * n + j);
      xi[0] -= mv[0] * xk[0] - mv[1] * xk[1];
      xi[1] -= mv[0] * xk[1] + mv[1] * xk[0];
    }
    __syncthreads();
  }
}

// I^SR of Eq. ISR at one real frequency per point p (state list index i_p, frequency w_p):
//   out[p] = coef sum_k (wt_k / 2 pi) sum_nm Lambda_k[m][n] [g0_nm(w_p + i w'_k) + g0_nm(w_p - i w'_k)],
//   g0_nm(z) = sum_l' C[i][n][l'][m] / (d_(m n_s + i)[l'] - z),
// where the two terms add to 2 (d - w) / ((d - w)^2 + w'^2) (real).  Lambda_k: the complex Dyson
// output at z = i w'_k (row = chain vector m, column = bra n; its real part is used).  One block
// per point.
__global__ void __launch_bounds__(256) k_isr_points(int n_pdep, int n_states, int n_steps, int n_nodes, int n_pts,
                                                    const double* __restrict__ C, const double* __restrict__ d,
                                                    const int* __restrict__ pt_state, const double* __restrict__ pt_w,
                                                    const double* __restrict__ lam, const double* __restrict__ nodes,
                                                    const double* __restrict__ wts, double coef,
                                                    double* __restrict__ out) {
  __shared__ double red[33];
  const int p = blockIdx.x;
  const int i = pt_state[p];
  const double w = pt_w[p];
  const size_t mm = (size_t)n_pdep * n_pdep;
  Thr th{(int)threadIdx.x, (int)blockDim.x};
  double acc = 0.0;
  for (size_t e = threadIdx.x; e < (size_t)n_nodes * mm; e += blockDim.x) {
    const int k = (int)(e / mm);
    const int m = (int)((e % mm) / n_pdep), n = (int)(e % n_pdep);
    const double wp = nodes[k];
    const double* ds = d + (size_t)(m * n_states + i) * n_steps;
    const double* c = C + ((size_t)i * n_pdep + n) * n_steps * n_pdep + m;
    double g = 0.0;
    for (int lp = 0; lp < n_steps; ++lp) {
      const double x = ds[lp] - w;
      g += c[(size_t)lp * n_pdep] * (2.0 * x / (x * x + wp * wp));
    }
    acc += lam[2 * ((size_t)k * mm + (size_t)m * n_pdep + n)] * wts[k] * (0.5 / kPi) * g;
  }
  acc = block_sum(acc, red, th);
  if (threadIdx.x == 0) out[p] = coef * acc;
}

// Residue-term contraction (Eq. Rfac), one block per entry e = (state list index i_e, occupied
// state j_e, occupation factor f_e, Lambda_e at e_j - w + i eta):
//   out[e] = f_e sum_nm Lambda_e[m][n] Y[i_e][j_e][n] Y[i_e][j_e][m]   (complex),
// Y[i][j][m] = <psi_j | psi_(states i) phi~_m> (rows of length n_pdep, ys per state).
__global__ void __launch_bounds__(256) k_residue_entries(int n_pdep, int n_e, const double* __restrict__ lam,
                                                         const double* __restrict__ Y, long ys,
                                                         const int* __restrict__ e_state, const int* __restrict__ e_j,
                                                         const double* __restrict__ e_f, double* __restrict__ out) {
  __shared__ double red[33];
  const int e = blockIdx.x;
  const double* y = Y + (size_t)e_state[e] * ys + (size_t)e_j[e] * n_pdep;
  const double* L = lam + 2 * (size_t)e * n_pdep * n_pdep;
  Thr th{(int)threadIdx.x, (int)blockDim.x};
  double re = 0.0, im = 0.0;
  for (int t = threadIdx.x; t < n_pdep * n_pdep; t += blockDim.x) {
    const int m = t / n_pdep, n = t % n_pdep;
    const double yy = y[n] * y[m];
    re += L[2 * t] * yy;
    im += L[2 * t + 1] * yy;
  }
  re = block_sum(re, red, th);
  im = block_sum(im, red, th);
  if (threadIdx.x == 0) {
    out[2 * e] = e_f[e] * re;
    out[2 * e + 1] = e_f[e] * im;
  }
}

size_t grid1d(size_t total) { return std::max<size_t>(1, std::min<size_t>(8192, (total + 255) / 256)); }

}  // namespace

cudaError_t launch_chi_z(int n_pdep, int n_v, int n_steps, int n_e, const double* W, const double* d,
                         const double* e_v, const double* z, double coef, double* chi, cudaStream_t st) {
  if (n_e <= 0) return cudaSuccess;
  k_chi_z<<<grid1d((size_t)n_e * n_pdep * n_pdep), 256, 0, st>>>(n_pdep, n_v, n_steps, n_e, W, d, e_v, z, coef, chi);
  return cudaGetLastError();
}

cudaError_t launch_dyson_z(int n, int batch, const double* A, double* X, double* M, int* info, cudaStream_t st) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  k_dyson_z<<<batch, 256, 0, st>>>(n, A, X, M, info);
  return cudaGetLastError();
}

cudaError_t launch_isr_points(int n_pdep, int n_states, int n_steps, int n_nodes, int n_pts, const double* C,
                              const double* d, const int* pt_state, const double* pt_w, const double* lam,
                              const double* nodes, const double* wts, double coef, double* out, cudaStream_t st) {
  if (n_pts <= 0) return cudaSuccess;
  k_isr_points<<<n_pts, 256, 0, st>>>(n_pdep, n_states, n_steps, n_nodes, n_pts, C, d, pt_state, pt_w, lam, nodes,
                                      wts, coef, out);
  return cudaGetLastError();
}

cudaError_t launch_residue_entries(int n_pdep, int n_e, const double* lam, const double* Y, long ys,
                                   const int* e_state, const int* e_j, const double* e_f, double* out,
                                   cudaStream_t st) {
  if (n_e <= 0) return cudaSuccess;
  k_residue_entries<<<n_e, 256, 0, st>>>(n_pdep, n_e, lam, Y, ys, e_state, e_j, e_f, out);
  return cudaGetLastError();
}

}  // namespace wgw
