// Launchers shared between the translation units of the wgw library.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "fft_bodies.cuh"
#include "la_bodies.cuh"

namespace wgw {

// Kernel choice per stage of the FFT pipeline (G -> r planes, x-lines, r -> G planes) on the
// lengths with register-resident kernels (24, 32, 48, 64, and 96 in FP32): kFftRegScalar,
// kFftRegPacked (packed FP32 butterflies; FP32 compute only) or kFftShared (the shared-memory
// kernel); -1 = the built-in default kFftDefault (kFftDefault96 at 96).  Other lengths always run
// the shared-memory kernels.
constexpr int kFftRegScalar = 0, kFftRegPacked = 1, kFftShared = 2, kFftChoices = 3;
struct FftKern {
  int g2r = -1, xline = -1, r2g = -1;
};
// Built-in choice until tuned, from GB300 measurements on the 48^3 block (register-resident kernels,
// median of three): G -> r 0.199 ms packed against 0.248 scalar, x-line 0.362 against 0.418,
// r -> G 0.252 against 0.264; the shared-memory kernels 2-4x slower.
constexpr FftKern kFftDefault{kFftRegPacked, kFftRegPacked, kFftRegPacked};
// N = 96 (FP32; 65536 systems of the 96^3 model): G -> r 30.4 ms packed, 36.2 scalar, 31.0 shared;
// x-line 39.0 scalar, 40.2 packed, 106.5 shared; r -> G 23.1 packed, 24.2 scalar, 40.6 shared.
constexpr FftKern kFftDefault96{kFftRegPacked, kFftRegScalar, kFftRegPacked};

template <typename T>
struct FftCtx {
  FftPlan plan;
  const cplx<T>* tw;              // exp(+2 pi i k / N), k < N
  const cplx<ff>* twe = nullptr;  // the same in float-float; non-null selects float-float
                                  // compute for T = double (pair buffers then hold cplx<ff>)
  FftKern kern{};                 // kernel choice per stage
};

int fft_threads(int n);

// Record a failure for wgw_last_error() and return `status` (wgw_api.cu).
int report_error(int status, const char* msg);
void clear_error();

// Pruned 3D FFT pipeline (fft_kernels_*.cu), storage type T and compute type C.
template <typename T, typename C>
cudaError_t launch_plane_g2r_c(const SphereTab& sp, const FftPlan& plan, const cplx<C>* tw, const T* X, long ldx,
                               int n_sys, const int* list, const int* active, cplx<C>* Tbuf, cudaStream_t st,
                               int kern);
template <typename T, typename C>
cudaError_t launch_xline_c(int m, const FftPlan& plan, const cplx<C>* tw, cplx<C>* Tbuf, const XArgs<T>& a,
                           const int* active, cudaStream_t st, int kern);
template <typename T, typename C>
cudaError_t launch_plane_r2g_c(const SphereTab& sp, int npt_max, const FftPlan& plan, const cplx<C>* tw,
                               const cplx<C>* Tbuf, const Epi<T>& e, cudaStream_t st, int kern);
template <typename T, typename C>
cudaError_t launch_drho_xline_c(int m, const FftPlan& plan, const cplx<C>* tw, const cplx<C>* Tbuf,
                                const T* psi_r, long ldpsi, int n_v, int n_sys, int n_pert, T coef, T* D,
                                long ldd, cudaStream_t st);

// Dispatch on the context's compute type: T = float and T = double compute in T, or, when
// f.twe is set (T = double only), in float-float with the pair buffer Tbuf holding cplx<ff>
// (the same size as cplx<double>).
inline bool ff_grid_supported(int n) { return n == 24 || n == 32 || n == 48 || n == 64 || n == 96; }
template <typename T>
inline bool use_ff(const FftCtx<T>& f) {
  return sizeof(T) == sizeof(double) && f.twe != nullptr && ff_grid_supported(f.plan.n);
}

template <typename T>
cudaError_t launch_plane_g2r(const SphereTab& sp, FftCtx<T> f, const T* X, long ldx, int n_sys,
                             const int* list, const int* active, cplx<T>* Tbuf, cudaStream_t st) {
  if (use_ff(f))
    return launch_plane_g2r_c<T, ff>(sp, f.plan, f.twe, X, ldx, n_sys, list, active,
                                     reinterpret_cast<cplx<ff>*>(Tbuf), st, f.kern.g2r);
  return launch_plane_g2r_c<T, T>(sp, f.plan, f.tw, X, ldx, n_sys, list, active, Tbuf, st, f.kern.g2r);
}
template <typename T>
cudaError_t launch_xline(int m, FftCtx<T> f, cplx<T>* Tbuf, const XArgs<T>& a, const int* active,
                         cudaStream_t st) {
  if (use_ff(f))
    return launch_xline_c<T, ff>(m, f.plan, f.twe, reinterpret_cast<cplx<ff>*>(Tbuf), a, active, st, f.kern.xline);
  return launch_xline_c<T, T>(m, f.plan, f.tw, Tbuf, a, active, st, f.kern.xline);
}
template <typename T>
cudaError_t launch_plane_r2g(const SphereTab& sp, int npt_max, FftCtx<T> f, const cplx<T>* Tbuf,
                             const Epi<T>& e, cudaStream_t st) {
  if (use_ff(f))
    return launch_plane_r2g_c<T, ff>(sp, npt_max, f.plan, f.twe, reinterpret_cast<const cplx<ff>*>(Tbuf), e, st,
                                     f.kern.r2g);
  return launch_plane_r2g_c<T, T>(sp, npt_max, f.plan, f.tw, Tbuf, e, st, f.kern.r2g);
}
template <typename T>
cudaError_t launch_drho_xline(int m, FftCtx<T> f, const cplx<T>* Tbuf, const T* psi_r, long ldpsi,
                              int n_v, int n_sys, int n_pert, T coef, T* D, long ldd, cudaStream_t st) {
  if (use_ff(f))
    return launch_drho_xline_c<T, ff>(m, f.plan, f.twe, reinterpret_cast<const cplx<ff>*>(Tbuf), psi_r, ldpsi,
                                      n_v, n_sys, n_pert, coef, D, ldd, st);
  return launch_drho_xline_c<T, T>(m, f.plan, f.tw, Tbuf, psi_r, ldpsi, n_v, n_sys, n_pert, coef, D, ldd, st);
}

// Fused FP32 H application (hpsi_fused.cu): plane g2r, x-line with V(r) and plane r2g of the
// systems of a list in one kernel, the pair intermediate in (distributed) shared memory.  Same
// arguments and results as the three separate launches with XM_APPLY_V; supported for the grid
// sizes and sphere radii hpsi_fused_supported accepts.
bool hpsi_fused_supported(int N, int m);
cudaError_t launch_hpsi_fused(const SphereTab& sp, int N, const float* P, long ldp, int n_list, const int* list,
                              const int* active, const float* V, const Epi<float>& e, cudaStream_t st);

// Linear algebra (la_kernels.cu).
// Y <- Y - Psi Psi^T Y for the active systems of a list (null = systems 0..n_sys-1);
// work holds pc_work_elems(n, n_sys, nv) elements of T.
// ffc: for T = double, compute in float-float (operands rounded to float-float pairs).
// tc_tiles: for T = float, the tensor-core kernels (tc_kernels.cu) with Psi pre-split into these
// tiles (launch_tc_tile_psi); null selects the CUDA-core GEMMs.
// psi_ff: with ffc, Psi as float-float pairs in 8-byte slots (no per-load conversion), or null.
// tc_err: device int the tensor-core kernels set when a wait times out (required with tc_tiles).
template <typename T>
cudaError_t launch_pc(T* Y, long ldy, int n_sys, const int* list, const T* Psi, long ldp, int n, int nv,
                      const int* active, T* work, cudaStream_t st, bool ffc = false,
                      const unsigned char* tc_tiles = nullptr, const T* psi_ff = nullptr, int* tc_err = nullptr,
                      int tc_split = 8);
// P_c on the tensor cores (3xTF32 products, FP32 accumulation in tensor memory); work holds
// tc_pc_work_elems(n, n_sys, nv) floats; tiles from launch_tc_tile_psi; *err (device) is set to 1
// when a wait on an MMA or copy barrier times out.
// split: phase-1 CTAs per SM the K dimension is cut for (1..kTcSplitMax; picked by the autotuner).
constexpr int kTcSplitDefault = 8, kTcSplitMax = 16;
cudaError_t launch_pc_tc(float* Y, long ldy, int n_sys, const int* list, const unsigned char* tiles, int n, int nv,
                         const int* active, float* work, cudaStream_t st, int* err, int split = kTcSplitDefault);
size_t tc_pc_work_elems(int n, int n_sys, int nv);
// Kleinman-Bylander term on the tensor cores: Q[s] += B diag(D) B^T P[s] for the systems of a list
// (active only), B (n x n_proj, n_proj <= 256) as operand tiles from launch_tc_tile_psi, D on the
// device; 3xTF32 products with FP32 accumulation, work and err as for launch_pc_tc.
cudaError_t launch_kb_tc(float* Q, const float* P, long ld, int n_sys, const int* list, const unsigned char* tiles,
                         int n, int n_proj, const float* D, const int* active, float* work, cudaStream_t st, int* err,
                         int split = kTcSplitDefault);
bool tc_pc_supported(int nv);
// Psi (n x nv, column v at Psi + v ldp) split into TF32 hi/lo parts and laid out as the operand
// tiles of both phases; tc_psi_tile_bytes(n, nv) bytes.
size_t tc_psi_tile_bytes(int n, int nv);
cudaError_t launch_tc_tile_psi(const float* Psi, long ldp, int n, int nv, unsigned char* tiles, cudaStream_t st);
// One bounded mbarrier wait that nothing completes: sets *dev_flag after about one second.
cudaError_t tc_wait_selftest(int* dev_flag, cudaStream_t st);
// Reads (and clears) a tensor-core wait-timeout flag (device int dev_flag); synchronises st.
cudaError_t tc_error_read_and_clear(int* flag, int* dev_flag, cudaStream_t st);
// C = A^T B: A is K x m (column j at A + j*lda), B is K x n (column j at B + c_j * ldb with
// c_j = cols[j], or j when cols is null); C is written row-major with rows of length n, padded
// to a multiple of 64 rows.  work: gemm_tn_work_elems(K, m, n) doubles.  ffc: float-float
// products and sums (operands converted once into shared memory) instead of native FP64.
cudaError_t launch_gemm_tn(const double* A, long lda, const double* B, long ldb, int K, int m, int n, double* C,
                           double* work, cudaStream_t st, const int* cols = nullptr, bool ffc = false);
size_t gemm_tn_work_elems(int K, int m, int n);
// Y[:, j] = beta Y[:, j] + alpha sum_v A[:, v] C[v][j]: A is n x k, C row-major k x ncols (row length ldc).
cudaError_t launch_gemm_nn(const double* A, long lda, int n, int k, const double* C, long ldc, int ncols,
                           double* Y, long ldy, double alpha, double beta, cudaStream_t st);
// Dense symmetric eigensolver (dense_kernels.cu): A = Z diag(w) Z^T, w ascending, n <= 2048.
cudaError_t launch_syev(int n, double* A, int lda, double* w, double* Z, int ldz, double* work, int* info,
                        cudaStream_t st);
size_t syev_work_elems(int n);
cudaError_t launch_ritz_residual(int n, int nb, const double* X, const double* AX, long ld, const double* theta,
                                 double* R, double* rnorm, cudaStream_t st);
cudaError_t launch_symmetrise(int m, double* T, int ldt, cudaStream_t st);
cudaError_t launch_select_scale(int k, const double* Zc, int ldz, const int* cols, const double* scale, int nc,
                                double* out, int ldo, cudaStream_t st);
// Complex-shifted CG (la_bodies.cuh): complex system s occupies rows 2s (real) and 2s+1 (imaginary).
template <typename T>
cudaError_t launch_cocg_init_a(const SphereTab& sp, int n, int n_cs, const T* Bv, T* X, T* R, T* Z, long ld,
                               const double* eps, CocgState cs, cudaStream_t st);
template <typename T>
cudaError_t launch_cocg_init_b(int n, int n_cs, const T* R, const T* Z, T* P, long ld, CocgState cs,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_cocg_step_a(const SphereTab& sp, int n, int n_list, const int* list, T* X, T* R, T* Z,
                               const T* P, T* Q, long ld, const double* eps, CocgState cs, double tol2,
                               int max_iter, cudaStream_t st);
template <typename T>
cudaError_t launch_cocg_step_b(int n, int n_list, const int* list, const T* R, const T* Z, T* P, long ld,
                               CocgState cs, cudaStream_t st);
// rows[2j] = 2 sys[j], rows[2j+1] = 2 sys[j] + 1.
cudaError_t launch_expand_rows(const int* sys, int n, int* rows, cudaStream_t st);
// R = B - (Q + i w X) per complex system (active only).
cudaError_t launch_shifted_residual(int n_cs, int n, const double* B, const double* Q, const double* X,
                                    const double* omega, double* R, long ld, const int* active, cudaStream_t st);
// out[s] = |x_{2s}|^2 + |x_{2s+1}|^2.
cudaError_t launch_pair_norm2(int n_cs, int n, const double* x, long ld, double* out, cudaStream_t st);
// Lanczos chains (dense_kernels.cu); chain s keeps q^l at Q + (l * n_ch + s) * ld.
// tridiagonal: the input matrices are tridiagonal (the Householder stage is skipped).
cudaError_t launch_syev_batched(int n, int batch, double* A, double* w, double* Z, double* work, int* info,
                                cudaStream_t st, bool tridiagonal = false);
cudaError_t launch_lz_start(int n, int n_ch, const double* B, double* Q, long ld, double* beta, int n_steps,
                            cudaStream_t st);
cudaError_t launch_lz_tridiag(int n_ch, int n_steps, const double* alpha, const double* beta, double* T,
                              cudaStream_t st);
cudaError_t launch_lz_resolvent(int n_ch, int n_steps, int n_v, int n_om, const double* d, const double* U,
                                const double* beta, const double* e_v, const double* omega, double* y,
                                cudaStream_t st);
cudaError_t launch_lz_assemble(int n_pdep, int n_v, int n_steps, int n_om, const double* ov, const double* y,
                               double coef, double* chi, cudaStream_t st);
// Split Gram-Schmidt of the Lanczos chains: gridDim.y = nb chunks of the n reals per chain.
// Qf: float-float copy of the chain vectors (ff pairs in double-sized slots), or null for
// native FP64 arithmetic.
int lz_split(int n, int n_ch);
cudaError_t launch_lz_gs_dots(int n, int l, int n_ch, const double* Q, const double* Qf, long ld, const double* X,
                              double* part, int nb, cudaStream_t st);
cudaError_t launch_lz_gs_update(int n, int l, int n_ch, const double* Q, const double* Qf, long ld, const double* X,
                                double* R, const double* part, double* alpha, int n_steps, bool alpha_only,
                                double* npart, int nb, cudaStream_t st);
// q^{l+1} = r / |r| (and its float-float copy); npart null: one block per chain reduces |r|.
cudaError_t launch_lz_normalise(int n, int l, int n_ch, const double* R, double* Q, double* Qf, long ld,
                                double* beta, int n_steps, const double* npart, int nb, cudaStream_t st);
cudaError_t launch_lz_residues(int n_pdep, int n_v, int n_steps, const double* ov, const double* U, const double* beta,
                               double* C, cudaStream_t st);
cudaError_t launch_lz_isr(int n_pdep, int n_states, int n_omega, int n_nodes, const double* g, const double* lam,
                          const double* w, double coef, double* out, cudaStream_t st);
cudaError_t launch_lz_g0_eval(int n_pdep, int n_v, int n_steps, int n_z, const double* C, const double* d,
                              const double* z, double* g, cudaStream_t st);
// Q[:, s] += B diag(D) B^T P[:, s] for the systems of a list (Kleinman-Bylander term); B is n x n_proj.
// work: pc_work_elems(n, n_sys, n_proj) elements of T.
template <typename T>
cudaError_t launch_kb(T* Q, const T* P, long ld, int n_sys, const int* list, const T* B, long ldb, int n, int n_proj,
                      const T* D, T* work, cudaStream_t st, bool ffc = false);
// Ordered list of the systems s < n_sys with active[s] != 0, and their count.
cudaError_t launch_build_list(const int* active, int n_sys, int* list, int* count, cudaStream_t st);
int pc_kblocks(int n, int n_sys);
int pcf_kblocks(int n, int n_sys);
size_t pc_work_elems(int n, int n_sys, int nv);
// Systems 0..n_sys-1, or list[0..n_sys) when a list is given.
template <typename T>
cudaError_t launch_cg_init_a(const SphereTab& sp, int n, int n_sys, const T* Bv, T* X, T* R, T* Z,
                             long ld, const double* eps, CgState cs, cudaStream_t st, const int* list = nullptr);
template <typename T>
cudaError_t launch_cg_init_b(int n, int n_sys, const T* R, const T* Z, T* P, long ld, CgState cs,
                             cudaStream_t st, const int* list = nullptr);
// out[j] = in[rows[j]] for j < n_rows, rows of n doubles.
// Raises the dynamic shared-memory limit of a kernel on the current device to at least `bytes`
// and never lowers it: contexts of different sizes launch the same kernels from several host
// threads, and a lower setting made by one between another's setting and its launch would make
// that launch fail.
cudaError_t ensure_smem_limit(const void* kernel, size_t bytes);
// Control step of the device-driven CG loop (see k_loop_ctl in la_kernels.cu).
cudaError_t launch_loop_ctl(const int* flags, int* list, int n_cap, int* rows, int* count, int* windows,
                            int max_windows, int min_keep, cudaGraphConditionalHandle cond, cudaStream_t st);
cudaError_t launch_gather_rows(int n_rows, int n, const int* rows, const double* in, long ldi, double* out, long ldo,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_cg_step_a(const SphereTab& sp, int n, int n_sys, const int* list, T* X, T* R, T* Z,
                             const T* P, const T* Q, long ld, const double* eps, CgState cs, double tol2,
                             int max_iter, cudaStream_t st);
template <typename T>
cudaError_t launch_cg_step_b(int n, int n_sys, const int* list, const T* R, const T* Z, T* P, long ld,
                             CgState cs, cudaStream_t st);
cudaError_t launch_sphere_to_rb(int n_sys, const double* c, long ldc, const double* scale, RbMap mp,
                                int part, double* out, long ldo, cudaStream_t st);
cudaError_t launch_rb_to_sphere(int n_sys, const double* in, long ldi, const int* b_row,
                                const double* scale, RbMap mp, double* c, long ldc, cudaStream_t st);
cudaError_t launch_axpby(int n_sys, int n, double alpha, const double* x, double beta,
                         const double* y, double* out, long ld, const int* active, cudaStream_t st);
template <typename Ti, typename To>
cudaError_t launch_copy_cast(int n_sys, int n, const Ti* in, long ldi, To* out, long ldo,
                             const int* active, cudaStream_t st);
// y[s] += x[s] (x cast to double), for active systems (null = all).
template <typename T>
cudaError_t launch_add_to(int n_sys, int n, const T* x, long ldx, double* y, long ldy,
                          const int* active, cudaStream_t st);
// y[s] += p[s] - t[s] for active systems (FP32 inputs, FP64 difference and sum).
cudaError_t launch_add_diff(int n_sys, int n, const float* p, const float* t, long ldx, double* y, long ldy,
                            const int* active, cudaStream_t st);
// Per-system norms ||x_s||^2 into out[s].
template <typename T>
cudaError_t launch_norm2(int n_sys, int n, const T* x, long ld, double* out, cudaStream_t st);
// out[i] = in[i] as a float-float pair stored in the 8-byte slot i of out.
cudaError_t launch_to_ff(size_t n, const double* in, double* out, cudaStream_t st);
// X = (1 - A)^-1 A per n x n row-major matrix of a batch (dense_kernels.cu); M: work of the same size.
cudaError_t launch_dyson(int n, int n_omega, const double* A, double* X, double* M, int* info, cudaStream_t st);
// Self-energy at real frequencies (sigma_kernels.cu).
// chi[e][m][n] = coef sum_v sum_l' W[v][n][l'][m] [1/(e_v - d - z_e) + 1/(e_v - d + z_e)], complex.
cudaError_t launch_chi_z(int n_pdep, int n_v, int n_steps, int n_e, const double* W, const double* d,
                         const double* e_v, const double* z, double coef, double* chi, cudaStream_t st);
// X = (1 - A)^-1 A per complex n x n row-major matrix of a batch; M: work of the same size.
cudaError_t launch_dyson_z(int n, int batch, const double* A, double* X, double* M, int* info, cudaStream_t st);
// I^SR at one real frequency per point from the G0 residues C, Ritz values d and Lambda at the nodes.
cudaError_t launch_isr_points(int n_pdep, int n_states, int n_steps, int n_nodes, int n_pts, const double* C,
                              const double* d, const int* pt_state, const double* pt_w, const double* lam,
                              const double* nodes, const double* wts, double coef, double* out, cudaStream_t st);
// Residue-term contraction per entry: f_e sum_nm Lambda_e[m][n] Y_n Y_m (complex).
cudaError_t launch_residue_entries(int n_pdep, int n_e, const double* lam, const double* Y, long ys,
                                   const int* e_state, const int* e_j, const double* e_f, double* out,
                                   cudaStream_t st);
// Loads the work array of wgw_symm_eig_noalloc_dev on the current device and caches its device
// address (dense_kernels.cu); returns a WGW status.
int noalloc_prepare();
// Count of nonzero entries of flags[0..n) into *out (one block).
cudaError_t launch_count(const int* flags, int n, int* out, cudaStream_t st);

}  // namespace wgw
