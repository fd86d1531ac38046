/*
 * wgw -- batched DFPT response chi0 for plane-wave full-frequency GW on one GPU.
 *
 * C interface of libwgw.so.  The library applies the independent-particle
 * density response chi0 of a Gamma-point, spin-unpolarised Kohn-Sham system to
 * a batch of perturbations without empty states (Sec. 3 of Yu & Govoni,
 * "GPU Acceleration of Large-Scale Full-Frequency GW Calculations",
 * arXiv:2203.05623):
 *   for every occupied state v and perturbation dV_p, solve the Sternheimer
 *   equation  P_c (H - e_v) P_c dpsi_vp = -P_c dV_p psi_v   (Eq. sternheimer,
 *   P_c = 1 - P_v) by batched preconditioned CG, with H = T + V_loc applied in
 *   dual space through FFTs (Sec. 4.1), then accumulate
 *   drho_p = sum_sigma sum_v [psi_v^* dpsi_vp + c.c.]                (Eq. dfpt).
 *
 * Units are Hartree atomic units.  The cell is cubic with side L (bohr),
 * volume Omega = L^3.  Plane waves G = (2 pi / L)(h, k, l).  The wavefunction
 * sphere is 0.5|G|^2 <= ecut, the density sphere 0.5|G|^2 <= 4 ecut.  Both are
 * in CANONICAL ORDER: ascending h^2+k^2+l^2, ties broken by (h, k, l) compared
 * lexicographically as signed integers; wgw_get_gvectors returns the order.
 *
 * Complex arrays are interleaved (re, im) doubles.  Coefficient conventions:
 * potentials and densities f(r) = sum_G f(G) e^{iG.r}; orbitals
 * psi(r) = Omega^{-1/2} sum_G psi(G) e^{iG.r} with sum_G |psi(G)|^2 = 1.
 * With these, drho(G) = sum_G' chi0_GG' dV(G'), chi0_GG' = (1/Omega) FT FT chi0(r, r').
 *
 * Ownership: every pointer argument is owned by the caller and only read (or
 * written, for outputs) during the call.  The context owns all device memory
 * it allocates (occupied states, potential, work space) until wgw_destroy.
 * Host-pointer entry points copy inputs in and results out within the call.
 * *_dev entry points take device pointers and a CUDA stream (cudaStream_t
 * passed as void*), enqueue their work on that stream and return after it
 * completes.
 *
 * Errors: every function returns a status code and never aborts or exits.
 * wgw_last_error() describes the last failure of the calling thread.
 * A context that returned WGW_ERR_CUDA should be destroyed.
 */
#ifndef WGW_H
#define WGW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WGW_OK 0
#define WGW_ERR_ARG 1      /* invalid argument (sizes, layout, symmetry) */
#define WGW_ERR_NOMEM 2    /* device allocation failed */
#define WGW_ERR_NOCONV 3   /* some Sternheimer system missed cg_tol; outputs are still written */
#define WGW_ERR_CUDA 4     /* a CUDA call failed */
#define WGW_ERR_TIMEOUT 5  /* a bounded device wait gave up */
#define WGW_ERR_STATE 6    /* call not valid in the context's state */
#define WGW_ERR_CANCELLED 7  /* the request was cancelled (wgw_cancel) */

#define WGW_FP64 0   /* every step in FP64 */
#define WGW_MIXED 1  /* FP32 inner CG + FP64 residual refinement (Sec. 5.1, mixed precision) */

#define WGW_SPHERE_WFC 0
#define WGW_SPHERE_RHO 1

typedef struct wgw_ctx wgw_ctx;

typedef struct wgw_options {
  int precision;       /* WGW_FP64 or WGW_MIXED */
  double cg_tol;       /* per system: ||b - A x||_2 <= cg_tol ||b||_2, residual in FP64 */
  int max_cg_iter;     /* CG iterations per solve (FP64) or per inner solve (MIXED) */
  int max_refine;      /* MIXED: FP64 refinement steps */
  double inner_tol;    /* MIXED: relative residual reduction of each inner FP32 solve */
  double f_s;          /* occupation of each state (2 = spin-unpolarised, the sum over sigma of Eq. dfpt) */
  int check_every;     /* CG iterations between two compactions of the list of iterating systems */
  double dav_tol;      /* Davidson: max |lambda_i(k) - lambda_i(k-1)| <= dav_tol and every Ritz residual
                          norm <= sqrt(dav_tol) */
  int dav_max_iter;    /* Davidson iterations */
  int dav_factor;      /* Davidson subspace limit = dav_factor * n_pdep (Sec. 4.2: 4) */
  int seed;            /* start block seed when none is given */
  int fp64_emulation;  /* MIXED: 1 = the FP64-accuracy FFT passes (right-hand sides, refinement
                          residuals, drho) compute in float-float (two FP32 values per number, about
                          48 significant bits) because GB300's FP64 rate is 1/64 of its FP32 rate;
                          0 = native FP64.  Storage stays FP64 either way. */
  int tensor_cores;    /* MIXED: 1 = the projector P_c of the FP32 inner solves runs on the tcgen05
                          tensor cores (TF32 products split three ways, hi*hi + hi*lo + lo*hi, FP32
                          accumulation: FP32 accuracy); 0 = FP32 CUDA-core GEMMs. */
  int cuda_graphs;     /* 2 = device-driven loop: after the first window of check_every iterations (run
                          directly), each graph launch holds a conditional WHILE node that repeats a
                          window and a device-side compaction of the list of systems still iterating
                          (finished systems drop out of the launches without a host poll); the host
                          waits only when half of the list has finished, to launch smaller grids.
                          The same kernels as 1, with FP32 K splits sized for the captured list, so
                          results agree with 1 to rounding.  1 = each window between two host polls
                          is captured as one CUDA graph and replayed (bit-identical to 0); 0 = direct
                          launches.  Graphs are not used while profiling is on. */
  int max_batch_systems;  /* most Sternheimer systems (complex-shifted: twice their count) solved as one
                             batch; larger applies run in chunks of whole perturbations.  0 = as many as
                             fit 85 % of the free device memory (the default). */
  int fused_h;            /* MIXED: the FP32 H application.  1 = one kernel per pair with the FFT
                             intermediate in (distributed) shared memory, on the grids it supports (24, 32,
                             48); 0 = three kernels with the intermediate in device memory; 2 = the faster of
                             the two on the context's first list of >= 256 systems (autotuned, the default;
                             wgw_autotune_info reports the choice).  The same operations: results agree to
                             FP32 rounding. */
  int tc_split;           /* MIXED, tensor_cores: phase-1 CTAs per SM the K dimension of the tensor-core
                             projector and KB products is cut for, 1..16; 0 = picked by the autotuner on
                             the context's first large projection (the default).  A fixed split gives
                             bit-identical results from run to run. */
  int fft_kernels[3];     /* MIXED: the kernel of each FP32 FFT stage of the H application (G -> r planes,
                             x-lines with V(r), r -> G planes) on the grids with register-resident kernels
                             (24, 32, 48, 64, 96): WGW_FFT_REG (one line per thread in registers), WGW_FFT_REG_PACKED
                             (the same with packed FP32 butterflies), WGW_FFT_SHARED (lines in shared
                             memory), or WGW_FFT_AUTO (the default: every candidate of the stage is timed on
                             the context's first application to >= 256 systems and the fastest kept;
                             wgw_autotune_fft reports the choice).  The same transforms: results agree to
                             FP32 rounding, and a fixed choice is bit-identical from run to run. */
  int h_chunk_pairs;      /* MIXED: the FP32 three-kernel H application runs its pairs in groups of this
                             many through a pair intermediate of that size, so that what one kernel
                             writes is still in L2 when the next reads it; 0 = all pairs at once; -1 =
                             autotuned (the default: no chunking and chunks of 32 MB and 64 MB of
                             intermediate are timed on the context's first application to >= 256 systems;
                             wgw_autotune_chunk reports the choice).  Results are bit-identical for any
                             value. */
} wgw_options;

#define WGW_FFT_AUTO (-1)
#define WGW_FFT_REG 0
#define WGW_FFT_REG_PACKED 1
#define WGW_FFT_SHARED 2

typedef struct wgw_stats {
  int n_systems;            /* real Sternheimer systems solved (states x real perturbation parts) */
  int n_converged;          /* systems that met cg_tol */
  int max_iters;            /* most CG iterations of one system (sum over refinement steps) */
  int refinements;          /* MIXED: FP64 refinement steps taken */
  double max_rel_residual;  /* max over systems of ||b - A x|| / ||b|| (FP64) */
} wgw_stats;

/* Fills *opt with defaults: WGW_FP64, cg_tol 1e-12, max_cg_iter 2000, max_refine 8,
 * inner_tol 5e-6, f_s 2, check_every 8, dav_tol 1e-8, dav_max_iter 100, dav_factor 4, seed 12345,
 * fp64_emulation 1, tensor_cores 1, cuda_graphs 2, max_batch_systems 0, fused_h 2, tc_split 0,
 * fft_kernels WGW_FFT_AUTO x 3, h_chunk_pairs -1. */
int wgw_default_options(wgw_options* opt);

/*
 * Creates a context for one ground state (the output of the DFT run that
 * precedes the response calculation, Sec. 3).
 *   L        cubic cell side [bohr], > 0.
 *   ecut     wavefunction cutoff [Ha], > 0.
 *   grid     FFT points per axis; a product of 2, 3, 5; must exceed 2 m_rho where m_rho is the
 *            largest |Miller index| of the density sphere (then H psi by FFTs is alias-free).
 *   vloc_G   V_loc(G) on the density sphere, N_rho complex; must be real in r (V(-G) = V(G)^*).
 *   n_proj   number of Kleinman-Bylander projectors (>= 0); H gains sum_p |beta_p> D_p <beta_p| (Sec. 3).
 *   beta_G   N_pw x n_proj complex projectors on the wavefunction sphere (column-major), each real
 *            in r; may be NULL when n_proj = 0.
 *   d_proj   n_proj couplings D_p [Ha]; may be NULL when n_proj = 0.
 *   psi_v    occupied states, N_pw x n_v complex, column-major (state v at psi_v + 2 N_pw v);
 *            each must be real in r (psi(-G) = psi(G)^*) and the set orthonormal.
 *   e_v      their eigenvalues [Ha], n_v entries.
 *   opt      options (NULL = defaults); copied.
 * On success *out holds the new context.
 */
int wgw_setup(wgw_ctx** out, double L, double ecut, int grid, const double* vloc_G, int n_proj,
              const double* beta_G, const double* d_proj, const double* psi_v, const double* e_v,
              int n_v, const wgw_options* opt);

/* Number of plane waves of a sphere (which = WGW_SPHERE_WFC or WGW_SPHERE_RHO). */
int wgw_sphere_size(const wgw_ctx* ctx, int which, int* n);

/* Miller indices (3 int32 per G, canonical order) of a sphere; miller has room for 3 * size. */
int wgw_get_gvectors(const wgw_ctx* ctx, int which, int32_t* miller);

/* Replaces the options of a context (precision, tolerances, f_s, ...). */
int wgw_set_options(wgw_ctx* ctx, const wgw_options* opt);

/*
 * drho = chi0(i omega) dV for a batch of perturbations (Eq. sternheimer + Eq. dfpt).
 *   dV      N_rho x n_pert complex (perturbation p at dV + 2 N_rho p), density-sphere order.
 *           A perturbation need not be real in r: it is applied by linearity as
 *           dV = A + i B with A, B real in r (B is skipped when it is zero).
 *   omega   n_omega imaginary frequencies omega >= 0 [Ha] (host array).  omega = 0 solves the
 *           static Eq. sternheimer by PCG; every omega > 0 is solved, batched over frequencies,
 *           as P_c (H - e_v + i omega) P_c x = -P_c dV psi_v by complex-symmetric CG (COCG), and
 *           drho = f_s sum_v 2 Re(psi_v^* x) (the -i omega partner is the complex conjugate).
 *   drho    N_rho x n_pert x n_omega complex output (p fastest after G).
 *   st      optional statistics (may be NULL).
 * Returns WGW_ERR_NOCONV (with drho written) when a system missed cg_tol.
 */
int wgw_apply_chi0(wgw_ctx* ctx, const double* dV, int n_pert, const double* omega, int n_omega,
                   double* drho, wgw_stats* st);

/* As wgw_apply_chi0 with dV and drho in device memory; work is enqueued on `stream`. */
int wgw_apply_chi0_dev(wgw_ctx* ctx, const double* dV_dev, int n_pert, const double* omega,
                       int n_omega, double* drho_dev, void* stream, wgw_stats* st);

/* As wgw_apply_chibar0_dev (below) with host arrays, copied in and out within the call. */
int wgw_apply_chibar0(wgw_ctx* ctx, const double* phi, int n_pert, const double* omega, int n_omega,
                      double* out, wgw_stats* st);

/*
 * Spin-polarised response: the sum over spin channels sigma of Eq. dfpt (Sec. 3; the
 * Sternheimer systems of every channel and state are independent).  Each context is one channel
 * of the same system: the same cell, cutoff and grid, its own V_sigma, psi_sigma, e_sigma and
 * options, normally f_s = 1 (wgw_options.f_s).  Then
 *   out = sum_sigma chi0_sigma(i omega) dV       (symmetrized = 0, arguments as wgw_apply_chi0)
 *   out = sum_sigma chi0bar_sigma(i omega) phi   (symmetrized = 1, as wgw_apply_chibar0),
 * host arrays, summed in the order of ctxs.  The channels run concurrently, each on its own
 * context's stream from its own host thread.  st: n_systems and n_converged summed, the other
 * fields the maximum over channels.
 * Returns WGW_ERR_ARG for n_ctx outside 1..8, a context listed twice, or contexts that differ in
 * cell, cutoff or grid; WGW_ERR_NOCONV (out written) when a channel missed cg_tol.
 */
int wgw_apply_channels(wgw_ctx* const* ctxs, int n_ctx, int symmetrized, const double* dV, int n_pert,
                       const double* omega, int n_omega, double* out, wgw_stats* st);

/*
 * Symmetrised response chi0bar phi = v^1/2 chi0 v^1/2 phi (Sec. 2.1), v^1/2(G) = sqrt(4 pi)/|G|,
 * zero at G = 0.  phi and out are dimensionless density-sphere coefficients; layout as for
 * wgw_apply_chi0_dev (device pointers, work on `stream`).
 */
int wgw_apply_chibar0_dev(wgw_ctx* ctx, const double* phi_dev, int n_pert, const double* omega,
                          int n_omega, double* out_dev, void* stream, wgw_stats* st);

/*
 * Kernel timing (no counterpart in the paper; used to report roofline fractions).
 * When enabled, every kernel launch of the context is bracketed by CUDA events on
 * its stream and accumulated per kernel class; enabling resets the counters.
 * Classes 0..8: plane_g2r, xline, plane_r2g, drho_xline, pc_project, cg_update, convert,
 * other, hpsi_fused, for the kernels on FP32 arrays; classes 9..17: the same names with "_f64",
 * for the kernels on FP64 arrays (native FP64 or float-float compute).  wgw_profile_read returns, for one class, the summed
 * device milliseconds, the launch count and the summed algorithmic bytes and flops
 * (each launch's own compulsory inputs and outputs); any output pointer may be NULL.
 */
#define WGW_PROF_KINDS 18
int wgw_profile_enable(wgw_ctx* ctx, int on);
/* Restricts recording to the classes whose bit is set in mask (bit k = class k; default all),
 * so that a timed run can bracket only the launches of one class. */
int wgw_profile_classes(wgw_ctx* ctx, unsigned mask);
int wgw_profile_read(wgw_ctx* ctx, int kind, double* ms, long* launches, double* bytes, double* flops);
const char* wgw_profile_kind_name(int kind);

/*
 * Per-system diagnostics of the last batched solve of this context (the last apply call, or
 * the last block application of a Davidson run).  Static systems (omega = 0) are ordered
 * s = r * n_v + v, where r runs over the real-in-r parts of the batch (the perturbations' real
 * parts, then their non-zero imaginary parts); when the call had frequencies omega > 0 the
 * records are those of its complex-shifted systems, q = (k * n_real + r) * n_v + v over those
 * frequencies k.  Writes min(n, n_systems) entries: CG iterations summed over refinement
 * steps, the final FP64 relative residual, and converged[s] = 1 if the system met cg_tol, else
 * 0 (the systems behind a WGW_ERR_NOCONV); any output pointer may be NULL.  Returns the number
 * of entries written, or WGW_ERR_ARG (with nothing written) on a NULL context or negative n.
 */
int wgw_system_info(const wgw_ctx* ctx, int n, int* iters, double* rel_residual, int* converged);

/*
 * Sampled solutions (no counterpart in the paper; they let a caller check single Sternheimer
 * systems of a large batch, Eq. sternheimer, one by one).  wgw_sample_solutions selects static
 * systems, numbered as in wgw_system_info (s = r * n_v + v), whose solutions dpsi_s the following
 * static applies (omega = 0) of the context keep; n = 0 clears the selection.  Indices beyond a
 * batch's systems are ignored for that batch.  wgw_read_samples copies the kept solutions of the
 * last static apply, in the selection's order, to dpsi: N_pw x n complex, wavefunction-sphere
 * canonical order (the psi_v layout of wgw_setup), each in range(P_c); a system not in the last
 * batch reads as zeros.  Returns WGW_ERR_ARG for n above the selection.
 */
int wgw_sample_solutions(wgw_ctx* ctx, int n, const int* systems);
int wgw_read_samples(wgw_ctx* ctx, int n, double* dpsi);

/*
 * PDEP basis (Sec. 3): the n_pdep leading (most negative) eigenpairs of chi0bar(omega = 0) by a
 * block Davidson iteration.  Start from an orthonormalised block, apply chi0bar (batched
 * Sternheimer solves in the context's precision), Rayleigh-Ritz in FP64 on the GPU, expand with
 * the residuals of unconverged pairs orthogonalised in FP64, restart from the Ritz vectors
 * when the subspace would exceed dav_factor * n_pdep (Sec. 4.2).  Converged when the eigenvalues
 * moved by at most dav_tol and every Ritz residual norm is at most sqrt(dav_tol).
 *   x0     host, N_rho x n_pdep complex start block (its real-in-r part is used), or NULL for
 *          a seeded block of uniform numbers weighted by v^1/2 (opt.seed).
 *   eig    host, n_pdep eigenvalues, ascending (most negative first).
 *   basis  host, N_rho x n_pdep complex eigenvectors (orthonormal in sum_G conj(a) b), or NULL.
 *   st     n_systems = Sternheimer systems solved, n_converged = converged pairs,
 *          max_iters = Davidson iterations, refinements = chi0bar block applications,
 *          max_rel_residual = largest Ritz residual norm.
 * Returns WGW_ERR_NOCONV (outputs written) if not converged in dav_max_iter iterations.
 */
int wgw_pdep_davidson(wgw_ctx* ctx, int n_pdep, const double* x0, double* eig, double* basis,
                      wgw_stats* st);

/*
 * PDEP basis of a spin-polarised system: as wgw_pdep_davidson, for the spin-summed response
 * chi0bar = sum_sigma chi0bar_sigma, with one context per spin channel (as for
 * wgw_apply_channels).  Every block application runs the channels concurrently (the first on
 * ctxs[0]'s stream, the others on their own) and sums them; the Davidson options (dav_tol,
 * dav_max_iter, dav_factor, seed) and the Rayleigh-Ritz work are those of ctxs[0].
 * Returns WGW_ERR_ARG as wgw_apply_channels does, otherwise as wgw_pdep_davidson.
 */
int wgw_pdep_davidson_channels(wgw_ctx* const* ctxs, int n_ctx, int n_pdep, const double* x0, double* eig,
                               double* basis, wgw_stats* st);

/*
 * Frequency dependence of chi0 in a basis by Lanczos chains (Sec. 3, the recurrence above
 * Eq. lanczos, and Eq. lanczos).  For every occupied state v and basis vector m, a chain on
 * P_c H P_c starts from b = P_c [phi~_m psi_v] (phi~ = v^1/2 phi), q^1 = b/|b|, beta_1 = |b|,
 * q^{l+1} = [(H - alpha_l) q^l - beta_l q^{l-1}] / beta_{l+1} with full reorthogonalisation
 * (two classical Gram-Schmidt passes, each followed by P_c), all in FP64 on the GPU.  With d, U
 * the eigenpairs of each chain's tridiagonal matrix,
 *   chi0_nm(i w) = (f_s/Omega) sum_v beta_1 sum_{l,l'} <P_c phi~_n psi_v|q^l> U_{l l'} U_{1 l'}
 *                  [1/(e_v - d_l' - i w) + 1/(e_v - d_l' + i w)]   (real).
 *   phi        host, N_rho x n_pdep complex basis (its real-in-r part is used), e.g. the PDEP basis.
 *   n_steps    chain length, 1..255.
 *   omega      host, n_omega >= 0 imaginary frequencies (may be NULL when n_omega = 0).
 *   alpha, beta  host outputs (or NULL), n_v x n_pdep x n_steps, l fastest; beta[..][0] = |b|.
 *   chi0_pdep  host output (or NULL), n_omega x n_pdep x n_pdep: chi0_nm(i w_k) at
 *              chi0_pdep[(k * n_pdep + m) * n_pdep + n].
 * A chain whose residual vanishes (Krylov space exhausted) continues with zero vectors.
 */
int wgw_lanczos(wgw_ctx* ctx, const double* phi, int n_pdep, int n_steps, const double* omega, int n_omega,
                double* alpha, double* beta, double* chi0_pdep, wgw_stats* st);

/*
 * Dense symmetric eigensolver of the Rayleigh-Ritz step (Sec. 4.2): A = Z diag(w) Z^T in FP64
 * on the GPU, one thread block (Householder tridiagonalisation, implicit-shift QL).  Device
 * pointers: A n x n column-major (overwritten), w n (ascending), Z n x n column-major.
 * 1 <= n <= 2048.  Work is enqueued on `stream` and the call returns when it completes.
 */
int wgw_symm_eig_dev(int n, double* A_dev, double* w_dev, double* Z_dev, void* stream);

/*
 * wgw_symm_eig_dev without any allocation (the paper has no counterpart; this serves callers
 * that cannot allocate device memory at the point of the call: a host process whose device
 * memory is all reserved up front by another allocator, or code that must not pay for the
 * device-wide synchronisation a cudaMalloc/cudaFree implies).  Same arguments, result and
 * error codes as wgw_symm_eig_dev, for 1 <= n <= 512; larger n returns WGW_ERR_ARG.
 * Its work space is one fixed array in device memory (about 2.1 MB), part of the library's
 * device code: it comes into existence on a GPU when that code is loaded there, which wgw_setup
 * does for the device it runs on and the first call of this function does otherwise, and it
 * stays until the process exits.  Loading takes device memory, so a caller that reserves all
 * device memory up front should create a context with wgw_setup, or make one call (n = 1 will
 * do), on that device first.  The first call on a device (in a CUDA context) also looks up the
 * array's device address with the device current, so make that first call before any stream
 * capture.  The call returns once its stream has finished the work (it reads the solver's
 * status back).  All calls share the array: calls whose work overlaps on a GPU (different
 * streams or host threads at the same time) race and must be serialised by the caller.
 */
int wgw_symm_eig_noalloc_dev(int n, double* A_dev, double* w_dev, double* Z_dev, void* stream);

/*
 * G0 Lanczos chains for the short-range correlation integral (Sec. 3, Eq. ISR, the Lanczos
 * recurrence under it and Eq. lanczos).  For every listed occupied state i and basis vector m a
 * chain of H itself (NOT projected) starts from b = [psi_i phi~_m] (phi~ = v^1/2 phi, the product
 * taken on the wavefunction sphere), q^1 = b/|b|, beta_1 = |b|, with full reorthogonalisation
 * (two classical Gram-Schmidt passes), in FP64 on the GPU.  With d, U the eigenpairs of each
 * chain's tridiagonal matrix, the frequency-independent residues
 *   C[i][n][l'][m] = beta_1 U_{1 l'} sum_l <psi_i phi~_n | q^l_m> U_{l l'}
 * give the resolvent matrices at any complex frequency z = w + i w' analytically:
 *   g0[i][k][n][m] = <psi_i phi~_n | (H - z_k)^-1 | psi_i phi~_m> = sum_l' C[i][n][l'][m] / (d_l' - z_k).
 *   phi        host, N_rho x n_pdep complex basis (its real-in-r part is used), e.g. the PDEP basis.
 *   states     host, n_states indices of occupied states (0..n_v-1, as given to wgw_setup).
 *   n_steps    chain length, 1..255.
 *   z          host, n_z complex frequencies, interleaved (re, im); may be NULL when n_z = 0.
 *   alpha, beta, d  host outputs (or NULL), n_states x n_pdep x n_steps, l fastest; beta[..][0] = |b|;
 *              d ascending per chain.
 *   residues   host output (or NULL), n_states x n_pdep x n_steps x n_pdep reals, C[i][n][l'][m].
 *   g0         host output (or NULL), n_states x n_z x n_pdep x n_pdep complex, interleaved.
 *   st         n_systems = chains, max_iters = n_steps.
 * A chain whose residual vanishes (Krylov space exhausted) continues with zero vectors.
 * Returns WGW_ERR_ARG for a state index outside 0..n_v-1 or n_steps outside 1..255.
 */
int wgw_g0_lanczos(wgw_ctx* ctx, const double* phi, int n_pdep, const int* states, int n_states, int n_steps,
                   const double* z, int n_z, double* alpha, double* beta, double* d, double* residues,
                   double* g0, wgw_stats* st);

/*
 * Kohn-Sham Hamiltonian on wavefunctions (Sec. 4.1: kinetic term on the sphere, V_loc by FFT to
 * the real-space grid and back, KB projectors): out = H psi for n_psi wavefunctions that are
 * real in r, on device memory, work enqueued on `stream` (as for wgw_apply_chi0_dev).
 *   psi_dev, out_dev  N_pw x n_psi complex, wavefunction-sphere canonical order (psi_v layout of
 *                     wgw_setup); only the real-in-r part of psi is used.
 *   fp32     1: the FP32 kernels of the inner CG (mixed-precision context only); 0: FP64
 *            accuracy (float-float on a mixed context with fp64_emulation, else native FP64).
 */
int wgw_apply_h_dev(wgw_ctx* ctx, const double* psi_dev, int n_psi, double* out_dev, int fp32, void* stream);

/*
 * Exchange self-energy of occupied states (Sec. 2, Eq. sigmacIR: Sigma_X is Eq. self_energy_gw
 * with the bare Coulomb potential v in place of W_0):
 *   sigma_x[k] = <psi_i|Sigma_X|psi_i> = -(1/Omega) sum_{j occ} sum_{G != 0} (4 pi/|G|^2) |FT[psi_i psi_j](G)|^2
 * for i = states[k], psi(r) = sum_G c(G) e^{iG.r} as given to wgw_setup (Omega^{-1/2} normalisation),
 * FT the density-sphere coefficients (1/N_grid) sum_r; one spin channel (no factor 2); the
 * G = 0 head is left out (it belongs to the long-range part).  Pair densities are formed in real
 * space and transformed with the library's FFT kernels at FP64 accuracy (float-float on a
 * mixed context with fp64_emulation).  Result in Ha.
 * Returns WGW_ERR_ARG for a state index outside 0..n_v-1.
 */
int wgw_sigma_x(wgw_ctx* ctx, const int* states, int n_states, double* sigma_x);

/*
 * Autotuner record of a context.  Two choices are made on the context's own shapes.  The K
 * split of the tensor-core projector (how many phase-1 CTAs per SM the contraction over plane
 * waves is cut into): at the first projection of at least 256 systems every candidate runs on a
 * scratch copy of the vectors and the fastest median time wins; *tc_split = the choice (0: not
 * tuned yet); splits[k], ms[k] = each candidate and its median time for up to n_max candidates.
 * The FP32 H kernel (options.fused_h = 2): at the first application to at least 256 systems the
 * three-kernel pipeline and the fused kernel both run on scratch output; *fused_h = the choice
 * (-1: not tuned, 0: three kernels, 1: fused), h_ms[0], h_ms[1] = their median times [ms].  Any
 * output may be NULL.  Returns the number of split candidates written, or -WGW_ERR_ARG for a
 * null context or negative n_max.
 */
int wgw_autotune_info(const wgw_ctx* ctx, int* tc_split, int* splits, double* ms, int n_max, int* fused_h,
                      double* h_ms);

/*
 * FFT autotuner record of a context (the choice of fft_kernels, Sec. 4.1's FFTs): choice[s] = the
 * kernel of stage s (0: G -> r planes, 1: x-lines, 2: r -> G planes) in effect for the FP32 H
 * application, WGW_FFT_REG / WGW_FFT_REG_PACKED / WGW_FFT_SHARED, or WGW_FFT_AUTO while it has not
 * been tuned yet; ms[3 s + k] = the median time [ms] of candidate k of stage s on the context's first
 * large list (0 when not timed: a fixed option, a grid without register-resident kernels, or not
 * tuned yet).  Either output may be NULL.  Returns WGW_ERR_ARG for a null context.
 */
int wgw_autotune_fft(const wgw_ctx* ctx, int* choice, double* ms);

/*
 * Chunk autotuner record of a context (h_chunk_pairs): *chunk_pairs = the chunk in effect (0: no
 * chunking; -1: not tuned yet); candidates[k], ms[k] = each timed chunk size and the median time
 * [ms] of the FP32 three-kernel H application on the context's first large list, for up to n_max
 * candidates.  Any output may be NULL.  Returns the number of candidates written, or -WGW_ERR_ARG
 * for a null context or negative n_max.
 */
int wgw_autotune_chunk(const wgw_ctx* ctx, int* chunk_pairs, int* candidates, double* ms, int n_max);

/*
 * Failure-detection self-test (no counterpart in the paper).  Every wait of the library's
 * kernels on a device barrier is bounded to about one second of wall time, after which the
 * kernel sets an error flag, releases what it holds and returns; the host turns the flag into
 * WGW_ERR_TIMEOUT.  This call runs one such wait on a barrier that nothing completes, on the
 * current device, and stores the flag the kernel left (1: the wait gave up as designed) in
 * *timed_out.  Takes about one second; the device stays usable.
 */
int wgw_selftest_wait_timeout(int* timed_out);

/*
 * Short-range correlation integral of Eq. ISR on the imaginary axis, for listed occupied states
 * i and real frequencies w:
 *   isr[i][j] = (1/Omega) int_0^inf dw'/(2 pi) sum_nm Lambda_nm(i w') [g0_nm(w_j + i w') + g0_nm(w_j - i w')]
 * (the integral over the whole axis folded with Lambda even in w'), taken by the caller's
 * quadrature (nodes w'_k >= 0, weights), with g0 the G0 Lanczos resolvent of wgw_g0_lanczos
 * (same phi, states and n_steps) and Lambda_nm(i w'_k) given at the nodes (e.g. wgw_dyson of the
 * PDEP-basis chibar0 from wgw_lanczos).  The contraction runs on the GPU.
 *   lam      host, n_nodes x n_pdep x n_pdep (row-major per node).
 *   isr      host output, n_states x n_omega complex, interleaved.
 * Returns WGW_ERR_ARG for a state outside 0..n_v-1, a negative node or missing arrays.
 */
int wgw_isr(wgw_ctx* ctx, const double* phi, int n_pdep, const int* states, int n_states, int n_steps,
            const double* omega, int n_omega, const double* lam, const double* nodes, const double* weights,
            int n_nodes, double* isr, wgw_stats* st);

/*
 * Dyson equation in a basis (Sec. 2: the screened response from the independent-particle one,
 * epsilon^-1 - 1 = (1 - chibar0)^-1 chibar0 for the symmetrised responses), for every frequency
 * of a batch, in FP64 on the GPU (Gaussian elimination with partial pivoting, one CTA per
 * frequency).  No context is needed.
 *   chi0bar  host, n_omega matrices n x n, row-major, frequency-major (the layout of
 *            wgw_lanczos's chi0_pdep; a transposed layout gives the transposed result, since
 *            the two factors commute).
 *   chibar   host output, same layout: (1 - chi0bar)^-1 chi0bar.
 * Returns WGW_ERR_ARG for n outside 1..4096 or when 1 - chi0bar is singular.
 */
int wgw_dyson(int n, int n_omega, const double* chi0bar, double* chibar);

/*
 * Response and screened response in a basis at complex frequencies (Sec. 2, the Dyson step;
 * Sec. 3, Eq. lanczos with the i w of the resolvent replaced by a complex z): from the chains of
 * wgw_lanczos (same phi and n_steps, run inside this call),
 *   chi0_z[k][m][n] = (f_s/Omega) sum_v sum_l' W[v][n][l'][m] [1/(e_v - d_l' - z_k) + 1/(e_v - d_l' + z_k)],
 *   W[v][n][l'][m] = beta_1 U_{1 l'} sum_l <P_c phi~_n psi_v|q^l> U_{l l'}   (chain of (v, m)),
 * and lam_z[k] = (1 - chi0_z[k])^-1 chi0_z[k] (complex Gaussian elimination with partial
 * pivoting, one CTA per frequency), all in FP64 on the GPU.  z = w + i eta is a real frequency
 * w with a broadening eta (the frequencies the residue term of Eq. Rfac needs); z = i w gives
 * wgw_lanczos's chi0_pdep.
 *   z          host, n_z complex frequencies, interleaved (re, im).
 *   chi0_z, lam_z  host outputs (either may be NULL), n_z x n_pdep x n_pdep complex, interleaved,
 *              element (m, n) of frequency k at 2 ((k n_pdep + m) n_pdep + n).
 * Returns WGW_ERR_ARG for bad sizes or when 1 - chi0_z is singular at one of the frequencies.
 */
int wgw_lanczos_z(wgw_ctx* ctx, const double* phi, int n_pdep, int n_steps, const double* z, int n_z,
                  double* chi0_z, double* lam_z, wgw_stats* st);

/*
 * Parameters of the correlation self-energy (wgw_sigma, wgw_qp).
 *   n_steps_chi  length of the chi0 Lanczos chains in the basis (Eq. lanczos), 1..255.
 *   n_steps_g0   length of the G0 chains (Eq. ISR), 1..255.
 *   nodes, weights, n_nodes  quadrature of the imaginary-axis integral over [0, inf) (host).
 *   e_fermi      Fermi energy [Ha]: at least the highest occupied e_v.
 *   eta          broadening of Lambda at the real frequencies of the residue term [Ha], >= 0.
 */
typedef struct wgw_sigma_params {
  int n_steps_chi;
  int n_steps_g0;
  const double* nodes;
  const double* weights;
  int n_nodes;
  double e_fermi;
  double eta;
} wgw_sigma_params;

/*
 * Diagonal self-energy of occupied states at real frequencies by contour deformation (Sec. 2,
 * Eq. sigmacIR: Sigma(w) = Sigma_X + I(w) + R(w)), every part on the GPU from chains run once
 * inside the call:
 *   sigma_x[i]   as wgw_sigma_x.
 *   isr[i][j]    I^SR_i(w_j) of Eq. ISR as wgw_isr (real), with Lambda(i w'_k) at the quadrature
 *                nodes from the chi0 chains of the basis (wgw_lanczos_z at z = i w'_k).
 *   res[i][j]    R_i(w_j) of Eq. Rfac in the basis (complex, interleaved):
 *                  (1/Omega) sum_j' f_ij'(w) sum_nm Lambda_nm(e_j' - w + i eta) <b_n|j'><j'|b_m>,
 *                  f_ij'(w) = theta(e_j' - e_F) theta(w - e_j') - theta(e_F - e_j') theta(e_j' - w),
 *                b_n = psi_i phi~_n, Lambda from the chi0 chains (wgw_lanczos_z at e_j' - w + i eta).
 * The context holds the occupied states only, so every w_j must be <= e_fermi: there f vanishes
 * for every empty state and the sum runs over the occupied j' with e_j' > w (the Kohn-Sham
 * energies stand in for the quasiparticle energies in f).
 *   states     host, n_states indices of occupied states.
 *   omega      host, n_omega real frequencies [Ha], each <= e_fermi.
 *   sigma_x    host output (or NULL), n_states.
 *   isr        host output (or NULL), n_states x n_omega.
 *   res        host output (or NULL), n_states x n_omega complex, interleaved.
 * Returns WGW_ERR_ARG for bad sizes, a state outside 0..n_v-1, e_fermi below an occupied energy,
 * a frequency above e_fermi, or when 1 - chi0 is singular at a frequency it needs.
 */
int wgw_sigma(wgw_ctx* ctx, const double* phi, int n_pdep, const int* states, int n_states,
              const wgw_sigma_params* prm, const double* omega, int n_omega, double* sigma_x, double* isr,
              double* res, wgw_stats* st);

/*
 * Quasiparticle energies of occupied states (Sec. 2, Eq. e_qp):
 *   e_qp = e_i + Re <psi_i|Sigma(e_qp)|psi_i> - <psi_i|v_xc|psi_i>,
 * solved by the secant method from e_i and e_i + 0.01 Ha (Sec. 3: a root-finding algorithm such
 * as the secant method), stopping when two iterates differ by at most tol * max(1, |e|); Sigma as
 * wgw_sigma, its chains run once for all iterations and the states of a call iterate together.
 *   v_xc       host, n_states expectation values of the exchange-correlation potential (NULL = 0).
 *   e_qp       host output, n_states.
 *   sigma_qp   host output (or NULL), n_states complex (interleaved): Sigma_i(e_qp).
 *   iters      host output (or NULL), n_states: secant steps taken.
 * Returns WGW_ERR_NOCONV when a state has not converged in max_iter steps (or its secant
 * stalls), WGW_ERR_ARG as wgw_sigma, also when an iterate rises above e_fermi.
 */
int wgw_qp(wgw_ctx* ctx, const double* phi, int n_pdep, const int* states, int n_states,
           const wgw_sigma_params* prm, const double* v_xc, double tol, int max_iter, double* e_qp,
           double* sigma_qp, int* iters, wgw_stats* st);

/*
 * Serving (no counterpart in the paper, which runs one calculation per job): non-blocking
 * requests on a context.  wgw_submit copies the request's inputs and returns a ticket at once;
 * one worker thread per context runs queued requests on the context's stream.
 *   - On a mixed-precision context, static requests (one frequency, omega = 0) are batched
 *     continuously: every Sternheimer system of an admitted request takes a slot of a device
 *     pool (up to 16384 slots, 60 % of the free memory), the FP32 inner CG of all slots runs in
 *     windows of check_every iterations, and between two windows finished systems are retired
 *     (FP64-accurate residual, next refinement or done), finished requests return their results,
 *     and queued requests are admitted into the free slots.  A request that arrives while others
 *     are on the GPU joins at the next window and its systems iterate in the same launches.
 *   - Other requests (frequencies other than the single 0, or an FP64 context) run as batched
 *     applies: queued requests with the same kind and frequency set are merged (as many as 80 %
 *     of the free device memory admits); such a request waits until the continuous engine is idle.
 * Requests on different contexts (different systems or grids) run on different streams and
 * overlap on the GPU.  The result of a request equals its result alone up to the rounding of the
 * batched reductions (tests bound it by the path's tolerance).  While a context has requests in
 * flight, its other entry points wait until they are done.
 */
#define WGW_REQ_CHI0 0     /* out = chi0(i omega) dV, as wgw_apply_chi0 */
#define WGW_REQ_CHIBAR0 1  /* out = chi0bar(i omega) phi, as wgw_apply_chibar0 */
#define WGW_REQ_PDEP 2     /* PDEP basis, as wgw_pdep_davidson: n_pert = n_pdep eigenpairs, dV = start block
                              (N_rho x n_pdep complex) or NULL, no frequencies (omega may be NULL,
                              n_omega 0); out = n_pdep eigenvalues followed by the basis (N_rho x n_pdep
                              complex).  The Davidson runs on its own host thread and stream, and each of
                              its chi0bar block applications is served like a WGW_REQ_CHIBAR0 request of
                              the queue (batched with the other requests); result.batch_requests = block
                              applications, result.batch_systems = Sternheimer systems solved. */

typedef struct wgw_request {
  int kind;               /* WGW_REQ_CHI0, WGW_REQ_CHIBAR0 or WGW_REQ_PDEP */
  const double* dV;       /* host, N_rho x n_pert complex; copied during wgw_submit */
  int n_pert;
  const double* omega;    /* host, n_omega >= 1 frequencies >= 0; copied */
  int n_omega;
  double* out;            /* host, N_rho x n_pert x n_omega complex; written by the library before the
                             request is reported done; must stay valid until then */
} wgw_request;

typedef struct wgw_result {
  int status;             /* status of the batched apply that served the request */
  double latency_s;       /* submission -> results written */
  double queue_s;         /* submission -> start of its batch */
  int batch_requests;     /* requests merged into that batch; continuous batching: most requests it
                             shared the slot pool with */
  int batch_systems;      /* Sternheimer systems of that batch (continuous batching: its own) */
} wgw_result;

/* Checks and copies the request, queues it and returns its ticket at once.  Returns WGW_ERR_ARG
 * (nothing queued) for an unknown kind, n_pert < 1, n_omega outside 1..4096, a frequency that is
 * negative or not finite, a null buffer, or perturbation coefficients that are not finite.  A
 * request whose least memory need (one perturbation at a time, plus its inputs and outputs)
 * exceeds 80 % of the free device memory waits; on an idle context it completes with
 * WGW_ERR_NOMEM. */
int wgw_submit(wgw_ctx* ctx, const wgw_request* req, uint64_t* ticket);
/* Cancels a request: a queued one completes at once, a running one when its batch ends, with
 * status WGW_ERR_CANCELLED and its output left unwritten.  WGW_ERR_ARG for an unknown or
 * already finished ticket.  The ticket is still released by wgw_poll / wgw_wait. */
int wgw_cancel(wgw_ctx* ctx, uint64_t ticket);
/* *done = 1 (and *res filled, ticket released) when the request has finished, else 0.  For a
 * request that finished with res->status != WGW_OK, wgw_last_error on the calling thread then
 * says what failed (as wgw_wait). */
int wgw_poll(wgw_ctx* ctx, uint64_t ticket, int* done, wgw_result* res);
/* Blocks until the request has finished; fills *res (may be NULL) and releases the ticket. */
int wgw_wait(wgw_ctx* ctx, uint64_t ticket, wgw_result* res);

/* Releases the context and all device memory it owns (after finishing queued requests).
 * NULL is allowed. */
void wgw_destroy(wgw_ctx* ctx);

/* Static description of a status code. */
const char* wgw_status_string(int status);

/* Description of the last failure of the calling thread ("" if none). */
const char* wgw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* WGW_H */
