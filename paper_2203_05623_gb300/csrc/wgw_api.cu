// Host side of libwgw: plane-wave spheres, context set-up, and the chi0 apply
// driver (Eq. sternheimer solved by batched CG, then Eq. dfpt).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/wgw.h"
#include "internal.h"
#include "serve_sched.h"
#include "tables.h"

using namespace wgw;

namespace {

thread_local std::string g_last_error;

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

#define WGW_CK(expr)                                                                         \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(WGW_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));         \
  } while (0)

#define WGW_TRY(expr)                 \
  do {                                \
    int s_ = (expr);                  \
    if (s_ != WGW_OK) return s_;      \
  } while (0)

// Device buffer that only grows; freed when it goes out of scope (move-only).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  int ensure(size_t need) {
    if (need <= bytes) return WGW_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(WGW_ERR_NOMEM, "cudaMalloc of " + std::to_string(need) + " bytes failed");
    }
    bytes = need;
    return WGW_OK;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
  void release() { if (p) cudaFree(p); p = nullptr; bytes = 0; }
};

long pad32(long n) { return (n + 31) / 32 * 32; }

// A plane-wave sphere (host tables from tables.h) with device copies.
struct HostSphere : SphereHostTables {
  DevBuf d_off, d_ent, d_g2, d_g2f, d_i0, d_pos, d_neg, d_vsqrt;
  SphereTab tab() const {
    SphereTab t;
    t.m = m; t.n_pairs = n_pairs;
    t.plane_off = d_off.as<int>(); t.ent = d_ent.as<int2>(); t.g2 = d_g2.as<double>();
    t.g2f = d_g2f.as<float>();
    return t;
  }
  RbMap map() const {
    RbMap r; r.n_pairs = n_pairs; r.i0 = d_i0.as<int>(); r.pos = d_pos.as<int>(); r.neg = d_neg.as<int>();
    return r;
  }
  void release() { d_off.release(); d_ent.release(); d_g2.release(); d_g2f.release(); d_i0.release(); d_pos.release(); d_neg.release(); d_vsqrt.release(); }
};

template <typename T>
int upload(DevBuf& d, const std::vector<T>& h) {
  WGW_TRY(d.ensure(sizeof(T) * std::max<size_t>(h.size(), 1)));
  if (!h.empty()) WGW_CK(cudaMemcpy(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
  return WGW_OK;
}

int upload_sphere(HostSphere& s) {
  WGW_TRY(upload(s.d_off, s.plane_off));
  WGW_TRY(upload(s.d_ent, s.ent));
  WGW_TRY(upload(s.d_g2, s.g2));
  WGW_TRY(upload(s.d_g2f, s.g2f));
  WGW_TRY(upload(s.d_i0, std::vector<int>{s.i0}));
  WGW_TRY(upload(s.d_pos, s.pos));
  WGW_TRY(upload(s.d_neg, s.neg));
  WGW_TRY(upload(s.d_vsqrt, s.vsqrt));
  return WGW_OK;
}

// Per-precision device state of a context.
template <typename T>
struct Prec {
  DevBuf tw;        // N twiddles
  DevBuf twe;       // the same in float-float (T = double)
  bool use_ff = false;   // FFT passes compute in float-float (T = double)
  DevBuf psi;       // occupied states, real basis, n_v x ld_w
  DevBuf psi_r;     // occupied states in real space, n_v x N^3
  DevBuf v_r;       // V_loc in real space
  DevBuf psi_r_ff, v_r_ff, psi_ff;   // T = double: float-float copies for the float-float passes
  // work
  DevBuf X, R, Z, P, Q, Bv, Tw, shift;
  DevBuf kbB, kbD;  // KB projectors in the real basis (n_proj x ld_w) and couplings
  // Real-space inputs of the FFT passes in the storage their compute type reads.
  const T* psi_r_fft() const { return use_ff ? psi_r_ff.as<T>() : psi_r.as<T>(); }
  const T* v_r_fft() const { return use_ff ? v_r_ff.as<T>() : v_r.as<T>(); }
  FftCtx<T> fft(const FftPlan& pl) const {
    FftCtx<T> f;
    f.plan = pl;
    f.tw = tw.as<cplx<T>>();
    f.twe = use_ff ? twe.as<cplx<ff>>() : nullptr;
    return f;
  }
  void release() {
    DevBuf* all[] = {&tw, &twe, &psi, &psi_r, &v_r, &psi_r_ff, &v_r_ff, &psi_ff, &X, &R, &Z, &P, &Q, &Bv, &Tw, &shift, &kbB, &kbD};
    for (DevBuf* b : all) b->release();
  }
};

// Per-kernel-class timing with CUDA events recorded on the launching stream
// (enabled by wgw_profile_enable).  Each record brackets one launch.
// Classes 0..7 time the FP32 kernels, 8..15 the same kernels on FP64 arrays (native FP64 or
// float-float compute).
constexpr int kProfHalf = 9, kProfKinds = 2 * kProfHalf;
const char* const kProfNames[kProfKinds] = {"plane_g2r", "xline", "plane_r2g", "drho_xline",
                                            "pc_project", "cg_update", "convert", "other", "hpsi_fused",
                                            "plane_g2r_f64", "xline_f64", "plane_r2g_f64", "drho_xline_f64",
                                            "pc_project_f64", "cg_update_f64", "convert_f64", "other_f64",
                                            "hpsi_fused_f64"};
enum ProfKind { PK_G2R = 0, PK_XLINE, PK_R2G, PK_DRHO, PK_PC, PK_CG, PK_CONV, PK_OTHER, PK_HPSI };

struct Prof {
  bool on = false;
  unsigned mask = (1u << kProfKinds) - 1;   // classes recorded while on
  bool f64 = true;    // storage precision of the launches being recorded
  struct Rec { int kind; cudaEvent_t a, b; double bytes, flops; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  double ms[kProfKinds] = {}, bytes[kProfKinds] = {}, flops[kProfKinds] = {};
  long n[kProfKinds] = {};
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  template <typename F>
  cudaError_t run(int kind, double by, double fl, cudaStream_t st, F&& f) {
    const int k = kind + (f64 ? kProfHalf : 0);
    if (!on || !((mask >> k) & 1u)) return f();
    Rec r{k, get(), get(), by, fl};
    cudaEventRecord(r.a, st);
    cudaError_t err = f();
    cudaEventRecord(r.b, st);
    recs.push_back(r);
    return err;
  }
  void flush() {
    for (Rec& r : recs) {
      float t = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
        ms[r.kind] += t; n[r.kind] += 1; bytes[r.kind] += r.bytes; flops[r.kind] += r.flops;
      }
      pool.push_back(r.a); pool.push_back(r.b);
    }
    recs.clear();
  }
  void reset() {
    flush();
    for (int k = 0; k < kProfKinds; ++k) { ms[k] = bytes[k] = flops[k] = 0; n[k] = 0; }
  }
  void release() {
    flush();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// Sets the precision recorded by a Prof for the lifetime of the guard.
struct ProfPrec {
  Prof& p;
  bool old;
  ProfPrec(Prof& prof, bool f64) : p(prof), old(prof.f64) { p.f64 = f64; }
  ~ProfPrec() { p.f64 = old; }
};

}  // namespace

struct wgw_ctx {
  double L = 0, ecut = 0, omega_cell = 0;
  int N = 0, n_v = 0, n_proj = 0;
  long ld_w = 0, ld_r = 0, grid3 = 0;
  wgw_options opt{};
  FftPlan plan{};
  HostSphere wfc, rho;
  std::vector<double> e_v;
  Prec<double> d;
  Prec<float> f;
  DevBuf e_v_d;
  // apply work space (double unless noted)
  DevBuf dvin, dv_rb, dv_r, Trho, Dr, drho_rb, eps, a_idx, b_idx, brow, cg_rz, cg_bb, cg_rr,
      cg_act, cg_it, cnt, rr64, act64, norms, pc_work, sys_list, list64, cg_rzi, omg, row_list, rowact,
      drho_all, psi_tc, kb_tc, cg_best, cg_itbest, lz_q, lz_qf, tc_err, loop_ctr;
  cudaStream_t stream = nullptr;
  Prof prof;
  // Autotuner results: the K split of the tensor-core P_c (phase-1 CTAs per SM; 0 = not tuned
  // yet) and the median time of each candidate on this context's shapes.
  int tc_split = 0;
  std::vector<std::pair<int, double>> tc_tune;
  // The FP32 H kernel choice (-1: not tuned yet; 0: three kernels; 1: fused) and the median time
  // of each variant on this context's first large list.
  int h_choice = -1;
  double h_ms[2] = {0.0, 0.0};
  // The FFT stage kernels of the FP32 H application (G -> r, x-line, r -> G; -1 entries: the
  // built-in default until tuned) and each candidate's median time (0: not timed).
  FftKern fft_kern{};
  bool fft_tuned = false;
  // Pairs per L2-resident chunk of the FP32 three-kernel H pipeline (0: all pairs at once) and the
  // tuned candidates' median times.
  int h_chunk = 0;
  bool chunk_tuned = false;
  std::vector<std::pair<int, double>> chunk_ms;
  double fft_ms[3][kFftChoices] = {};
  std::vector<int> last_iters;      // per system of the last apply: CG iterations (all refinements)
  std::vector<double> last_relres;  // per system of the last apply: final FP64 ||b - A x|| / ||b||
  std::vector<int> last_conv;       // per system of the last apply: 1 if it met cg_tol
  // Sampled solutions (wgw_sample_solutions): static systems whose dpsi the applies keep, and
  // their values from the last static apply (N_pw complex each, canonical order).
  std::vector<int> sample_sys;
  std::vector<double> sample_out;
  DevBuf sample_buf;
  std::vector<int> blk_iters;       // the same for the batched solve that just ran (one chunk)
  std::vector<double> blk_relres;
  std::vector<int> blk_conv;
  // Serialises every entry point that uses the context's device state (callers and the
  // request worker).
  std::recursive_mutex mu;
  // Request queue of wgw_submit (see the serving section below), guarded by qmu.
  std::mutex qmu;
  std::condition_variable qcv;
  serve::Queue sq;
  bool stop = false;
  // Served Davidson requests: one host thread each while it runs (its block applications are
  // requests of the queue); the worker stays up while any is running.
  int pdep_active = 0;
  std::vector<std::thread> pdep_threads;
  // Continuous-batching engine of the served static requests (worker thread only).
  DevBuf eng_in, eng_out, eng_xc, eng_list, eng_mask, eng_pool;
  long eng_requests = 0, eng_windows = 0;
  std::thread worker;
  int device = 0;
  ~wgw_ctx() {
    {
      std::lock_guard<std::mutex> lk(qmu);
      stop = true;
    }
    qcv.notify_all();
    if (worker.joinable()) worker.join();
    for (std::thread& t : pdep_threads)
      if (t.joinable()) t.join();
    prof.release();
    d.release(); f.release(); wfc.release(); rho.release();
    DevBuf* eng[] = {&eng_in, &eng_out, &eng_xc, &eng_list, &eng_mask, &eng_pool};
    for (DevBuf* b : eng) b->release();
    DevBuf* all[] = {&e_v_d, &dvin, &dv_rb, &dv_r, &Trho, &Dr, &drho_rb, &eps, &a_idx, &b_idx, &brow,
                     &cg_rz, &cg_bb, &cg_rr, &cg_act, &cg_it, &cnt, &rr64, &act64, &norms, &pc_work, &sys_list, &list64, &cg_rzi, &omg,
                     &row_list, &rowact, &drho_all, &psi_tc, &kb_tc, &cg_best, &cg_itbest, &lz_q, &lz_qf, &tc_err};
    for (DevBuf* b : all) b->release();
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

// Algorithmic bytes of the FFT-pipeline kernels (their own inputs and outputs).
template <typename T>
double t_bytes(const wgw_ctx* c, int m, int pairs) {
  return (double)pairs * (2 * m + 1) * c->N * c->N * sizeof(cplx<T>);
}

// Real-space function(s) of a batch of real-basis vectors of one sphere:
// out[s] (N^3 reals, digit-reversed positions) for s < n_sys.
template <typename T>
int to_real(wgw_ctx* c, Prec<T>& pr, const HostSphere& sp, const T* X, long ldx, int n_sys, T* out,
            DevBuf& tbuf, cudaStream_t st) {
  ProfPrec pp(c->prof, sizeof(T) == 8);
  const int N = c->N, NP = 2 * sp.m + 1, pairs = (n_sys + 1) / 2;
  WGW_TRY(tbuf.ensure(sizeof(cplx<T>) * (size_t)pairs * NP * N * N));
  FftCtx<T> f = pr.fft(c->plan);
  const double tb = t_bytes<T>(c, sp.m, pairs);
  WGW_CK(c->prof.run(PK_G2R, tb + (double)n_sys * sp.nrb() * sizeof(T), 0, st, [&] {
    return launch_plane_g2r<T>(sp.tab(), f, X, ldx, n_sys, nullptr, nullptr, tbuf.as<cplx<T>>(), st); }));
  XArgs<T> a{};
  a.mode = XM_TO_REAL; a.R0 = out; a.R1 = out; a.ldr = c->grid3; a.n_sys = n_sys;
  WGW_CK(c->prof.run(PK_XLINE, tb + (double)n_sys * c->grid3 * sizeof(T), 0, st, [&] {
    return launch_xline<T>(sp.m, f, tbuf.as<cplx<T>>(), a, nullptr, st); }));
  return WGW_OK;
}

// FFT stage kernels of the FP32 H application: the option where fixed, else the autotuner's
// choice (the built-in default until it has run).
FftKern fft_choice(const wgw_ctx* c) {
  FftKern k = c->fft_kern;
  if (c->opt.fft_kernels[0] != WGW_FFT_AUTO) k.g2r = c->opt.fft_kernels[0];
  if (c->opt.fft_kernels[1] != WGW_FFT_AUTO) k.xline = c->opt.fft_kernels[1];
  if (c->opt.fft_kernels[2] != WGW_FFT_AUTO) k.r2g = c->opt.fft_kernels[2];
  return k;
}

// Autotuner of the tensor-core P_c: at the first projection of at least 256 systems (never
// inside a graph capture) every candidate K split runs three times on a scratch copy of the
// vectors and the fastest median wins for the life of the context.
constexpr int kTcSplitCandidates[] = {2, 4, 8, 16};

int tune_tc_split(wgw_ctx* c, const float* Y, int n_list, float* work, cudaStream_t st) {
  const int n = c->wfc.nrb();
  DevBuf scratch;
  WGW_TRY(scratch.ensure(sizeof(float) * (size_t)n_list * c->ld_w));
  WGW_CK(cudaMemcpyAsync(scratch.p, Y, sizeof(float) * (size_t)n_list * c->ld_w, cudaMemcpyDeviceToDevice, st));
  cudaEvent_t a = nullptr, b = nullptr;
  WGW_CK(cudaEventCreate(&a));
  WGW_CK(cudaEventCreate(&b));
  int best = kTcSplitDefault;
  double best_ms = 1e300;
  c->tc_tune.clear();
  for (int split : kTcSplitCandidates) {
    std::vector<float> ts;
    for (int r = 0; r < 4; ++r) {
      WGW_CK(cudaEventRecord(a, st));
      WGW_CK(launch_pc_tc(scratch.as<float>(), c->ld_w, n_list, nullptr, c->psi_tc.as<unsigned char>(), n, c->n_v,
                          nullptr, work, st, c->tc_err.as<int>(), split));
      WGW_CK(cudaEventRecord(b, st));
      WGW_CK(cudaEventSynchronize(b));
      float ms = 0.f;
      WGW_CK(cudaEventElapsedTime(&ms, a, b));
      if (r > 0) ts.push_back(ms);   // the first run warms up
    }
    std::sort(ts.begin(), ts.end());
    const double med = ts[ts.size() / 2];
    c->tc_tune.emplace_back(split, med);
    if (med < best_ms) { best_ms = med; best = split; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->tc_split = best;
  return WGW_OK;
}

// Autotuner of the FFT stage kernels of the FP32 H application (grids with register-resident
// kernels; stages the options leave to it), at the context's first application to at least 256
// systems: each candidate of a stage is timed (median of three after a warm-up) on the first
// n_list rows of P, with the other stages at their current choice; the G -> r (and x-line) stages
// run untimed before each x-line (r -> G) timing, so every timed launch sees a freshly written
// intermediate.  Output goes to scratch.
int tune_fft(wgw_ctx* c, Prec<float>& pr, const float* P, int n_list, cudaStream_t st) {
  c->fft_tuned = true;
  const int N = c->N, NP = 2 * c->wfc.m + 1, pairs = (n_list + 1) / 2;
  if (!(N == 24 || N == 32 || N == 48 || N == 64 || N == 96)) return WGW_OK;
  DevBuf out;
  WGW_TRY(out.ensure(sizeof(float) * (size_t)n_list * c->ld_w));
  WGW_TRY(pr.Tw.ensure(sizeof(cplx<float>) * (size_t)pairs * NP * N * N));
  Epi<float> e{};
  e.out = out.as<float>(); e.ldo = c->ld_w; e.pin = P; e.ldp = c->ld_w; e.vcoef = 1.f; e.kin = 1.f;
  e.shift = pr.shift.as<float>(); e.n_sys = n_list; e.active = nullptr; e.list = nullptr;
  const int* list = nullptr;
  const int* active = nullptr;
  FftCtx<float> f = pr.fft(c->plan);
  cplx<float>* Tb = pr.Tw.as<cplx<float>>();
  XArgs<float> xa{};
  xa.mode = XM_APPLY_V; xa.V = pr.v_r_fft(); xa.n_sys = n_list; xa.list = list;
  cudaEvent_t a = nullptr, b = nullptr;
  WGW_CK(cudaEventCreate(&a));
  WGW_CK(cudaEventCreate(&b));
  FftKern k = fft_choice(c);
  int* sel[3] = {&k.g2r, &k.xline, &k.r2g};
  int rc = WGW_OK;
  for (int stage = 0; stage < 3 && rc == WGW_OK; ++stage) {
    if (c->opt.fft_kernels[stage] != WGW_FFT_AUTO) continue;
    double best = 1e300;
    int pick = *sel[stage];
    for (int cand = 0; cand < kFftChoices && rc == WGW_OK; ++cand) {
      *sel[stage] = cand;
      f.kern = k;
      std::vector<float> ts;
      for (int r = 0; r < 4; ++r) {
        cudaError_t err = cudaSuccess;
        if (stage >= 1) err = launch_plane_g2r<float>(c->wfc.tab(), f, P, c->ld_w, n_list, list, active, Tb, st);
        if (err == cudaSuccess && stage == 2) err = launch_xline<float>(c->wfc.m, f, Tb, xa, active, st);
        if (err == cudaSuccess) err = cudaEventRecord(a, st);
        if (err == cudaSuccess && stage == 0)
          err = launch_plane_g2r<float>(c->wfc.tab(), f, P, c->ld_w, n_list, list, active, Tb, st);
        if (err == cudaSuccess && stage == 1) err = launch_xline<float>(c->wfc.m, f, Tb, xa, active, st);
        if (err == cudaSuccess && stage == 2)
          err = launch_plane_r2g<float>(c->wfc.tab(), c->wfc.npt_max, f, Tb, e, st);
        if (err == cudaSuccess) err = cudaEventRecord(b, st);
        if (err == cudaSuccess) err = cudaEventSynchronize(b);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
        if (err != cudaSuccess) {
          rc = fail(WGW_ERR_CUDA, std::string("FFT autotuner: ") + cudaGetErrorString(err));
          break;
        }
        if (r > 0) ts.push_back(ms);
      }
      if (rc != WGW_OK) break;
      std::sort(ts.begin(), ts.end());
      c->fft_ms[stage][cand] = ts[ts.size() / 2];
      if (c->fft_ms[stage][cand] < best) { best = c->fft_ms[stage][cand]; pick = cand; }
    }
    *sel[stage] = pick;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc == WGW_OK) c->fft_kern = k;
  return rc;
}

// Autotuner of the FP32 H application: the three-kernel pipeline and the fused kernel each run
// four times (the first warms up) on the context's first list of at least 256 systems, writing a
// scratch output, and the faster median wins for the life of the context (wgw_autotune_info).
int tune_h(wgw_ctx* c, Prec<float>& pr, const float* P, int n_list, const int* list, const int* active,
           cudaStream_t st) {
  const int N = c->N, NP = 2 * c->wfc.m + 1, pairs = (n_list + 1) / 2;
  DevBuf out;
  WGW_TRY(out.ensure(sizeof(float) * (size_t)n_list * c->ld_w));
  WGW_TRY(pr.Tw.ensure(sizeof(cplx<float>) * (size_t)pairs * NP * N * N));
  Epi<float> e{};
  e.out = out.as<float>(); e.ldo = c->ld_w; e.pin = P; e.ldp = c->ld_w; e.vcoef = 1.f; e.kin = 1.f;
  e.shift = pr.shift.as<float>(); e.n_sys = n_list; e.active = nullptr; e.list = nullptr;
  // The same amount of work on the first n_list rows of P (valid rows of the batch), every
  // system active, so that the scratch output needs n_list rows whatever the list holds.
  (void)list;
  (void)active;
  list = nullptr;
  active = nullptr;
  FftCtx<float> f = pr.fft(c->plan);
  cplx<float>* Tb = pr.Tw.as<cplx<float>>();
  cudaEvent_t a = nullptr, b = nullptr;
  WGW_CK(cudaEventCreate(&a));
  WGW_CK(cudaEventCreate(&b));
  XArgs<float> xa{};
  xa.mode = XM_APPLY_V; xa.V = pr.v_r_fft(); xa.n_sys = n_list; xa.list = list;
  f.kern = fft_choice(c);
  double med[2] = {0, 0};
  for (int variant = 0; variant < 2; ++variant) {
    std::vector<float> ts;
    for (int r = 0; r < 4; ++r) {
      WGW_CK(cudaEventRecord(a, st));
      if (variant == 1) {
        WGW_CK(launch_hpsi_fused(c->wfc.tab(), N, P, c->ld_w, n_list, list, active, pr.v_r_fft(), e, st));
      } else {
        WGW_CK(launch_plane_g2r<float>(c->wfc.tab(), f, P, c->ld_w, n_list, list, active, Tb, st));
        WGW_CK(launch_xline<float>(c->wfc.m, f, Tb, xa, active, st));
        WGW_CK(launch_plane_r2g<float>(c->wfc.tab(), c->wfc.npt_max, f, Tb, e, st));
      }
      WGW_CK(cudaEventRecord(b, st));
      WGW_CK(cudaEventSynchronize(b));
      float ms = 0.f;
      WGW_CK(cudaEventElapsedTime(&ms, a, b));
      if (r > 0) ts.push_back(ms);
    }
    std::sort(ts.begin(), ts.end());
    med[variant] = ts[ts.size() / 2];
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->h_ms[0] = med[0];
  c->h_ms[1] = med[1];
  c->h_choice = med[1] < med[0] ? 1 : 0;
  return WGW_OK;
}

// P_c applied to the systems of a list (null = 0..n_list-1), timed as pc_project.
template <typename T>
int run_pc(wgw_ctx* c, T* Y, int n_list, const int* list, const T* Psi, const int* active, cudaStream_t st) {
  ProfPrec pp(c->prof, sizeof(T) == 8);
  const double n = c->wfc.nrb(), nv = c->n_v;
  const bool tcores = sizeof(T) == sizeof(float) && c->opt.tensor_cores != 0 && tc_pc_supported(c->n_v) &&
                      Psi == reinterpret_cast<const T*>(c->f.psi.p);
  WGW_TRY(c->pc_work.ensure(sizeof(T) * std::max(pc_work_elems((int)n, n_list, std::max(c->n_v, c->n_proj)),
                                                 tc_pc_work_elems((int)n, n_list, c->n_v))));
  T* work = c->pc_work.as<T>();
  if (tcores && !c->psi_tc.p) {   // operand tiles of the occupied block and the wait flag, once per context
    WGW_TRY(c->psi_tc.ensure(tc_psi_tile_bytes((int)n, c->n_v)));
    WGW_CK(launch_tc_tile_psi(c->f.psi.as<float>(), c->ld_w, (int)n, c->n_v, c->psi_tc.as<unsigned char>(), st));
    if (!c->tc_err.p) {
      WGW_TRY(c->tc_err.ensure(sizeof(int)));
      WGW_CK(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), st));
    }
  }
  const unsigned char* tiles = tcores ? c->psi_tc.as<unsigned char>() : nullptr;
  if (tcores && c->opt.tc_split > 0) c->tc_split = c->opt.tc_split;
  if (tcores && c->tc_split == 0 && n_list >= 256) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    WGW_CK(cudaStreamIsCapturing(st, &cap));
    if (cap == cudaStreamCaptureStatusNone)
      WGW_TRY(tune_tc_split(c, reinterpret_cast<const float*>(Y), n_list, reinterpret_cast<float*>(work), st));
  }
  const int split = c->tc_split > 0 ? c->tc_split : kTcSplitDefault;
  WGW_CK(c->prof.run(PK_PC, 2.0 * n_list * n * sizeof(T) + n * nv * sizeof(T), 4.0 * n * nv * n_list, st, [&] {
    const bool ffc = sizeof(T) == 8 && c->d.use_ff;
    const T* psi_ff = (ffc && Psi == reinterpret_cast<const T*>(c->d.psi.p)) ? reinterpret_cast<const T*>(c->d.psi_ff.p)
                                                                             : nullptr;
    return launch_pc<T>(Y, c->ld_w, n_list, list, Psi, c->ld_w, (int)n, c->n_v, active, work, st, ffc, tiles,
                        psi_ff, tcores ? c->tc_err.as<int>() : nullptr, split); }));
  return WGW_OK;
}

// The three FFT kernels of the local part of H on a list (g2r, x-line with V(r), r2g with the
// kinetic and shift epilogue), Q = (T + V - e_v) P.  chunk > 0: the pairs run in consecutive groups
// of `chunk` pairs through a pair intermediate of that size, so that an intermediate written by
// g2r is still in L2 when the x-line and r2g kernels read it (a 48^3 pair holds 387 KB; 128 pairs
// hold 50 MB of the 129 MB L2).  The same kernels on the same pairs: results are bit-identical to
// chunk = 0.
template <typename T>
int h_pipeline(wgw_ctx* c, Prec<T>& pr, const FftCtx<T>& f, const T* P, T* Q, int n_list, const int* list,
               const int* active, cplx<T>* Tb, int chunk, cudaStream_t st) {
  const int pairs = (n_list + 1) / 2, nrb = c->wfc.nrb();
  if (chunk <= 0 || chunk >= pairs) chunk = pairs;
  for (int p0 = 0; p0 < pairs; p0 += chunk) {
    const int nc = std::min(n_list - 2 * p0, 2 * chunk), pc = (nc + 1) / 2;
    // A chunk of an explicit list is a sub-list; without a list its systems are 2 p0.. of the
    // batch, so the per-system arrays move with it.
    const long so = list ? 0 : 2L * p0;
    const int* lc = list ? list + 2 * p0 : nullptr;
    const int* ac = (active && !list) ? active + so : active;
    const T* Pc = P + so * c->ld_w;
    const double tb = t_bytes<T>(c, c->wfc.m, pc);
    Epi<T> e{};
    e.out = Q + so * c->ld_w; e.ldo = c->ld_w; e.pin = Pc; e.ldp = c->ld_w; e.vcoef = T(1); e.kin = T(1);
    e.shift = pr.shift.template as<T>() + so; e.n_sys = nc; e.active = ac; e.list = lc;
    WGW_CK(c->prof.run(PK_G2R, tb + (double)nc * nrb * sizeof(T), 0, st, [&] {
      return launch_plane_g2r<T>(c->wfc.tab(), f, Pc, c->ld_w, nc, lc, ac, Tb, st); }));
    XArgs<T> a{};
    a.mode = XM_APPLY_V; a.V = pr.v_r_fft(); a.n_sys = nc; a.list = lc;
    WGW_CK(c->prof.run(PK_XLINE, 2 * tb + (double)c->grid3 * sizeof(T), 0, st, [&] {
      return launch_xline<T>(c->wfc.m, f, Tb, a, ac, st); }));
    WGW_CK(c->prof.run(PK_R2G, tb + 2.0 * nc * nrb * sizeof(T), 0, st, [&] {
      return launch_plane_r2g<T>(c->wfc.tab(), c->wfc.npt_max, f, Tb, e, st); }));
  }
  return WGW_OK;
}

// Autotuner of the chunk size of the FP32 H pipeline (options.h_chunk_pairs = -1), at the context's
// first application to >= 256 systems, after the FFT stage kernels: no chunking and chunks whose
// pair intermediate holds 32 MB and 64 MB each run the pipeline four times on the first n_list
// rows of P (scratch output, the first run a warm-up), and the fastest median wins.
int tune_chunk(wgw_ctx* c, Prec<float>& pr, const float* P, int n_list, cudaStream_t st) {
  c->chunk_tuned = true;
  const int pairs = (n_list + 1) / 2;
  const double per_pair = t_bytes<float>(c, c->wfc.m, 1);   // one pair's intermediate
  std::vector<int> cands = {0};
  for (double mb : {32.0, 64.0}) {
    const int k = std::max(1, (int)(mb * 1048576.0 / per_pair));
    if (k < pairs && (cands.size() == 1 || k != cands.back())) cands.push_back(k);
  }
  if (cands.size() == 1) return WGW_OK;
  DevBuf out;
  WGW_TRY(out.ensure(sizeof(float) * (size_t)n_list * c->ld_w));
  const int NP = 2 * c->wfc.m + 1, N = c->N;
  WGW_TRY(pr.Tw.ensure(sizeof(cplx<float>) * (size_t)pairs * NP * N * N));
  FftCtx<float> f = pr.fft(c->plan);
  f.kern = fft_choice(c);
  cudaEvent_t a = nullptr, b = nullptr;
  WGW_CK(cudaEventCreate(&a));
  WGW_CK(cudaEventCreate(&b));
  int rc = WGW_OK, best = 0;
  double best_ms = 1e300;
  c->chunk_ms.clear();
  for (int k : cands) {
    std::vector<float> ts;
    for (int r = 0; r < 4 && rc == WGW_OK; ++r) {
      cudaError_t err = cudaEventRecord(a, st);
      if (err == cudaSuccess) {
        rc = h_pipeline<float>(c, pr, f, P, out.as<float>(), n_list, nullptr, nullptr, pr.Tw.as<cplx<float>>(), k, st);
        if (rc != WGW_OK) break;
        err = cudaEventRecord(b, st);
      }
      if (err == cudaSuccess) err = cudaEventSynchronize(b);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, a, b);
      if (err != cudaSuccess) rc = fail(WGW_ERR_CUDA, std::string("chunk autotuner: ") + cudaGetErrorString(err));
      if (r > 0) ts.push_back(ms);
    }
    if (rc != WGW_OK) break;
    std::sort(ts.begin(), ts.end());
    const double med = ts[ts.size() / 2];
    c->chunk_ms.push_back({k, med});
    if (med < best_ms) { best_ms = med; best = k; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc == WGW_OK) c->h_chunk = best;
  return rc;
}

// Q = P_c (H - e_v) P for the active systems of a list (P already in range(P_c)).
template <typename T>
int apply_A(wgw_ctx* c, Prec<T>& pr, const T* P, T* Q, int n_list, const int* list, const int* active,
            cudaStream_t st, bool project_out = true) {
  ProfPrec pp(c->prof, sizeof(T) == 8);
  const int N = c->N, NP = 2 * c->wfc.m + 1, pairs = (n_list + 1) / 2;
  if (pairs == 0) return WGW_OK;
  bool fused = false;
  if constexpr (std::is_same<T, float>::value) {
    if (!c->fft_tuned && n_list >= 256) {   // FFT stage kernels, once per context on its first large list
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      WGW_CK(cudaStreamIsCapturing(st, &cap));
      if (cap == cudaStreamCaptureStatusNone) WGW_TRY(tune_fft(c, pr, P, n_list, st));
    }
    if (c->opt.fused_h != 0 && hpsi_fused_supported(N, c->wfc.m)) {
      if (c->opt.fused_h == 1) {
        fused = true;
      } else {   // 2: the autotuner's choice, made once per context on its first large list
        if (c->h_choice < 0 && n_list >= 256) {
          cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
          WGW_CK(cudaStreamIsCapturing(st, &cap));
          if (cap == cudaStreamCaptureStatusNone) WGW_TRY(tune_h(c, pr, P, n_list, list, active, st));
        }
        fused = c->h_choice == 1;
      }
    }
  }
  if (!fused) WGW_TRY(pr.Tw.ensure(sizeof(cplx<T>) * (size_t)pairs * NP * N * N));
  FftCtx<T> f = pr.fft(c->plan);
  if constexpr (std::is_same<T, float>::value) f.kern = fft_choice(c);
  cplx<T>* Tb = pr.Tw.template as<cplx<T>>();
  const int nrb = c->wfc.nrb();
  const double tb = t_bytes<T>(c, c->wfc.m, pairs);
  Epi<T> e{};
  e.out = Q; e.ldo = c->ld_w; e.pin = P; e.ldp = c->ld_w; e.vcoef = T(1); e.kin = T(1);
  e.shift = pr.shift.template as<T>(); e.n_sys = n_list; e.active = active; e.list = list;
  if constexpr (std::is_same<T, float>::value) {
    if (fused) {
      // Algorithmic work: p in, q out and V(r); flops 5 n log2 n per line transform (rows and
      // columns of the 2m+1 planes both ways, N^2 x-lines both ways) and the V(r) product.
      const double nl = 5.0 * N * std::log2((double)N);
      const double fl = (double)pairs * (2.0 * NP * NP * nl + 2.0 * NP * N * nl + 2.0 * N * N * nl + 2.0 * c->grid3);
      WGW_CK(c->prof.run(PK_HPSI, 2.0 * n_list * nrb * sizeof(T) + (double)c->grid3 * sizeof(T), fl, st, [&] {
        return launch_hpsi_fused(c->wfc.tab(), N, P, c->ld_w, n_list, list, active, pr.v_r_fft(), e, st); }));
    }
  }
  if (!fused) {
    (void)tb;
    int chunk = 0;
    if constexpr (std::is_same<T, float>::value) {
      if (c->opt.h_chunk_pairs >= 0) {
        chunk = c->opt.h_chunk_pairs;
      } else {
        if (!c->chunk_tuned && n_list >= 256) {
          cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
          WGW_CK(cudaStreamIsCapturing(st, &cap));
          if (cap == cudaStreamCaptureStatusNone) WGW_TRY(tune_chunk(c, pr, P, n_list, st));
        }
        chunk = c->h_chunk;
      }
    }
    WGW_TRY(h_pipeline<T>(c, pr, f, P, Q, n_list, list, active, Tb, chunk, st));
  }
  if (c->n_proj > 0) {
    WGW_TRY(c->pc_work.ensure(sizeof(T) * std::max(pc_work_elems(nrb, n_list, std::max(c->n_v, c->n_proj)),
                                                   tc_pc_work_elems(nrb, n_list, std::max(c->n_v, c->n_proj)))));
    const bool kb_tc = sizeof(T) == sizeof(float) && c->opt.tensor_cores != 0 && tc_pc_supported(c->n_proj);
    if (kb_tc && !c->kb_tc.p) {   // operand tiles of the projectors, once per context
      WGW_TRY(c->kb_tc.ensure(tc_psi_tile_bytes(nrb, c->n_proj)));
      WGW_CK(launch_tc_tile_psi(c->f.kbB.as<float>(), c->ld_w, nrb, c->n_proj, c->kb_tc.as<unsigned char>(), st));
      if (!c->tc_err.p) {
        WGW_TRY(c->tc_err.ensure(sizeof(int)));
        WGW_CK(cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), st));
      }
    }
    WGW_CK(c->prof.run(PK_PC, 3.0 * n_list * nrb * sizeof(T), 4.0 * nrb * c->n_proj * n_list, st, [&] {
      if constexpr (std::is_same<T, float>::value) {
        if (kb_tc)
          return launch_kb_tc(Q, P, c->ld_w, n_list, list, c->kb_tc.as<unsigned char>(), nrb, c->n_proj,
                              c->f.kbD.as<float>(), active, c->pc_work.as<float>(), st, c->tc_err.as<int>(),
                              c->opt.tc_split > 0 ? c->opt.tc_split
                                                  : (c->tc_split > 0 ? c->tc_split : kTcSplitDefault));
      }
      return launch_kb<T>(Q, P, c->ld_w, n_list, list, pr.kbB.template as<T>(), c->ld_w, nrb, c->n_proj,
                          pr.kbD.template as<T>(), c->pc_work.template as<T>(), st,
                          sizeof(T) == 8 && c->d.use_ff); }));
  }
  if (project_out) WGW_TRY(run_pc<T>(c, Q, n_list, list, pr.psi.template as<T>(), active, st));
  return WGW_OK;
}

// The FP32 inner solves skip the projection of (H - e_v) p: the occupied states are eigenvectors
// of H, so H maps range(P_c) into itself and, for p in range(P_c), P_c (H - e_v) p = (H - e_v) p
// up to the FP32 rounding of H p (~1e-7 relative).  The search directions stay in range(P_c)
// because z = P_c M^-1 r is projected; what leaks into r is rounding noise far below the inner
// tolerance, and the FP64 residual of the refinement uses the full projections.
constexpr bool kProjectInnerOutput = false;

// stagnation: stop a system whose residual has stopped decreasing (FP32 inner solves only).
CgState cg_state(wgw_ctx* c, bool stagnation = false) {
  CgState s;
  s.rz = c->cg_rz.as<double>(); s.bb = c->cg_bb.as<double>(); s.rr = c->cg_rr.as<double>();
  s.active = c->cg_act.as<int>(); s.iters = c->cg_it.as<int>();
  s.rr_best = stagnation ? c->cg_best.as<double>() : nullptr;
  s.it_best = stagnation ? c->cg_itbest.as<int>() : nullptr;
  return s;
}

// Ordered list of the systems with flags[s] != 0 into `list`; returns the count on the host.
int build_list(wgw_ctx* c, const int* flags, int n, int* list, cudaStream_t st, int* out) {
  WGW_CK(c->prof.run(PK_OTHER, 8.0 * n, 0, st, [&] { return launch_build_list(flags, n, list, c->cnt.as<int>(), st); }));
  WGW_CK(cudaMemcpyAsync(out, c->cnt.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  return WGW_OK;
}

// The device-driven CG loop (cuda_graphs = 2): one graph launch whose conditional WHILE node runs
// `window` (check_every iterations over the list of n_cap entries it was captured with) and then
// the control step k_loop_ctl, which compacts the list on the device (entries past the count
// become -1, which every list kernel skips) and repeats the body while more than min_keep systems
// are still iterating and fewer than max_windows windows have run.  The host waits once at the
// end, for the count and the windows run, and captures the next launch with the shorter list:
// no host poll between windows.  rows: the row list of the complex-shifted solve (null for CG).
int device_loop(wgw_ctx* c, cudaStream_t st, const int* flags, int* list, int* rows, int n_cap, int max_windows,
                int min_keep, const std::function<int(cudaStream_t)>& window, int* n_left, int* n_windows) {
  WGW_TRY(c->loop_ctr.ensure(2 * sizeof(int)));
  int* ctr = c->loop_ctr.as<int>();
  // A default stream cannot be captured: the loop then runs on the context's stream, ordered
  // after and before the caller's stream by events.
  const bool side = st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
  const cudaStream_t gst = side ? c->stream : st;
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t x) { if (e == cudaSuccess) e = x; return e == cudaSuccess; };
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  if (side) {
    ck(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
    ck(cudaEventRecord(ev_in, st));
    ck(cudaStreamWaitEvent(gst, ev_in, 0));
  }
  ck(cudaMemsetAsync(ctr, 0, 2 * sizeof(int), gst));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  int status = WGW_OK;
  ck(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h{};
  ck(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) ck(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  if (e == cudaSuccess && ck(cudaStreamBeginCaptureToGraph(gst, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeRelaxed))) {
    status = window(gst);
    const cudaError_t le = status == WGW_OK
        ? launch_loop_ctl(flags, list, n_cap, rows, ctr, ctr + 1, max_windows, min_keep, h, gst) : cudaSuccess;
    cudaGraph_t body = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(gst, &body);
    ck(le);
    ck(ce);
  }
  int hc[2] = {0, 0};
  if (status == WGW_OK && e == cudaSuccess) {
    ck(cudaGraphInstantiate(&exec, g, 0));
    ck(cudaGraphLaunch(exec, gst));
    ck(cudaMemcpyAsync(hc, ctr, sizeof hc, cudaMemcpyDeviceToHost, gst));
    ck(cudaStreamSynchronize(gst));
    if (side) {
      ck(cudaEventRecord(ev_out, gst));
      ck(cudaStreamWaitEvent(st, ev_out, 0));
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (g) cudaGraphDestroy(g);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (status != WGW_OK) return status;
  if (e != cudaSuccess) return fail(WGW_ERR_CUDA, cudaGetErrorString(e));
  *n_left = hc[0];
  *n_windows = hc[1];
  return WGW_OK;
}

// Preconditioned CG on A x = b for all systems (b in pr.Bv, x into pr.X), to relative residual tol.
// Every check_every iterations the host rebuilds the list of systems still iterating, and the
// following iterations launch over that list only.
template <typename T>
int cg_solve(wgw_ctx* c, Prec<T>& pr, int n_sys, double tol, int max_iter, cudaStream_t st) {
  ProfPrec pp(c->prof, sizeof(T) == 8);
  const int n = c->wfc.nrb();
  const long ld = c->ld_w;
  T* X = pr.X.template as<T>();
  T* R = pr.R.template as<T>();
  T* Z = pr.Z.template as<T>();
  T* P = pr.P.template as<T>();
  T* Q = pr.Q.template as<T>();
  const T* Bv = pr.Bv.template as<T>();
  const T* Psi = pr.psi.template as<T>();
  const double* eps = c->eps.as<double>();
  CgState cs = cg_state(c, sizeof(T) == sizeof(float));
  const int* act = cs.active;
  const double vb = (double)n_sys * n * sizeof(T);
  WGW_CK(c->prof.run(PK_CG, 4 * vb, 0, st, [&] {
    return launch_cg_init_a<T>(c->wfc.tab(), n, n_sys, Bv, X, R, Z, ld, eps, cs, st); }));
  WGW_TRY(run_pc<T>(c, Z, n_sys, nullptr, Psi, act, st));
  WGW_CK(c->prof.run(PK_CG, 3 * vb, 0, st, [&] { return launch_cg_init_b<T>(n, n_sys, R, Z, P, ld, cs, st); }));
  int* lbuf = c->sys_list.as<int>();
  int n_list = 0;
  WGW_TRY(build_list(c, act, n_sys, lbuf, st, &n_list));
  const int every = std::max(1, c->opt.check_every);
  const bool proj_q = sizeof(T) == sizeof(double) || kProjectInnerOutput;
  // The iterations between two list rebuilds (a window): the launches depend on the window only
  // through n_list, so every window but the first (which also sizes the work buffers) is
  // captured as a CUDA graph and replayed, updating the previous executable graph in place.
  auto window = [&](int it0, int w, cudaStream_t st) -> int {
    const double lb = (double)n_list * n * sizeof(T);
    for (int k = 0; k < w; ++k) {
      WGW_TRY(apply_A<T>(c, pr, P, Q, n_list, lbuf, act, st, proj_q));
      WGW_CK(c->prof.run(PK_CG, 7 * lb, 0, st, [&] {
        return launch_cg_step_a<T>(c->wfc.tab(), n, n_list, lbuf, X, R, Z, P, Q, ld, eps, cs, tol * tol,
                                   max_iter, st); }));
      WGW_TRY(run_pc<T>(c, Z, n_list, lbuf, Psi, act, st));
      WGW_CK(c->prof.run(PK_CG, 4 * lb, 0, st, [&] {
        return launch_cg_step_b<T>(n, n_list, lbuf, R, Z, P, ld, cs, st); }));
    }
    // Without the projection of q, rounding noise collects in the occupied part of r, where the
    // iteration cannot remove it; clear it before the convergence test settles on it.
    if (!proj_q && (it0 + w) % every == 0) WGW_TRY(run_pc<T>(c, R, n_list, lbuf, Psi, act, st));
    return WGW_OK;
  };
  const bool graphs = c->opt.cuda_graphs != 0 && !c->prof.on;
  // A default stream cannot be captured: the graph then runs on the context's stream, ordered
  // after and before the caller's stream by events.
  const bool side = st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
  const cudaStream_t gst = side ? c->stream : st;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  if (graphs && side) {
    cudaError_t ee = cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming);
    if (ee == cudaSuccess) ee = cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming);
    if (ee != cudaSuccess) {
      if (ev_in) cudaEventDestroy(ev_in);
      return fail(WGW_ERR_CUDA, cudaGetErrorString(ee));
    }
  }
  cudaGraphExec_t exec = nullptr;
  int status = WGW_OK;
  const bool dev_loop = graphs && c->opt.cuda_graphs == 2;
  for (int it = 0; it < max_iter && n_list > 0;) {
    const int w = std::min(every - it % every, max_iter - it);
    if (dev_loop && it > 0 && it % every == 0) {
      // Halve the grids: return to the host when half of the captured list has finished.
      int left = 0, ran = 0;
      status = device_loop(c, st, act, lbuf, nullptr, n_list, (max_iter - it + every - 1) / every,
                           n_list > 64 ? n_list / 2 : 0, [&](cudaStream_t s) { return window(it, every, s); },
                           &left, &ran);
      if (status != WGW_OK) break;
      it += ran * every;
      n_list = left;
      continue;
    }
    if (graphs && it > 0) {
      // Failures set status and leave the loop, so that the executable graph and the events
      // are destroyed below on every path.
      cudaError_t pe = cudaSuccess;
      if (side) {
        pe = cudaEventRecord(ev_in, st);
        if (pe == cudaSuccess) pe = cudaStreamWaitEvent(gst, ev_in, 0);
      }
      if (pe == cudaSuccess) pe = cudaStreamBeginCapture(gst, cudaStreamCaptureModeRelaxed);
      if (pe != cudaSuccess) { status = fail(WGW_ERR_CUDA, cudaGetErrorString(pe)); break; }
      const int rc = window(it, w, gst);
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(gst, &g);
      if (rc != WGW_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        status = rc != WGW_OK ? rc : fail(WGW_ERR_CUDA, cudaGetErrorString(ce));
        break;
      }
      cudaGraphExecUpdateResultInfo info;
      if (!exec || cudaGraphExecUpdate(exec, g, &info) != cudaSuccess) {
        (void)cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
        if (ie != cudaSuccess) {
          cudaGraphDestroy(g);
          status = fail(WGW_ERR_CUDA, cudaGetErrorString(ie));
          break;
        }
      }
      cudaGraphDestroy(g);
      cudaError_t le = cudaGraphLaunch(exec, gst);
      if (le == cudaSuccess && side) {
        le = cudaEventRecord(ev_out, gst);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(st, ev_out, 0);
      }
      if (le != cudaSuccess) { status = fail(WGW_ERR_CUDA, cudaGetErrorString(le)); break; }
    } else {
      status = window(it, w, st);
      if (status != WGW_OK) break;
    }
    it += w;
    if (it % every == 0) {
      status = build_list(c, act, n_sys, lbuf, st, &n_list);
      if (status != WGW_OK) break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (status != WGW_OK) return status;
  if (sizeof(T) == sizeof(float) && c->tc_err.p) {
    int flag = 0;
    WGW_CK(tc_error_read_and_clear(&flag, c->tc_err.as<int>(), st));
    if (flag) return fail(WGW_ERR_TIMEOUT, "tensor-core P_c: a wait on the MMA completion barrier timed out");
  }
  return WGW_OK;
}

int ensure_work(wgw_ctx* c, int n_sys, int n_real) {
  const size_t vb = (size_t)n_sys * c->ld_w;
  DevBuf* dv[] = {&c->d.X, &c->d.R, &c->d.Z, &c->d.P, &c->d.Q, &c->d.Bv};
  for (DevBuf* b : dv) WGW_TRY(b->ensure(sizeof(double) * vb));
  WGW_TRY(c->d.shift.ensure(sizeof(double) * n_sys));
  if (c->opt.precision == WGW_MIXED) {
    DevBuf* fv[] = {&c->f.X, &c->f.R, &c->f.Z, &c->f.P, &c->f.Q, &c->f.Bv};
    for (DevBuf* b : fv) WGW_TRY(b->ensure(sizeof(float) * vb));
    WGW_TRY(c->f.shift.ensure(sizeof(float) * n_sys));
  }
  WGW_TRY(c->eps.ensure(sizeof(double) * n_sys));
  WGW_TRY(c->a_idx.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->b_idx.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->cg_rz.ensure(sizeof(double) * n_sys));
  WGW_TRY(c->cg_bb.ensure(sizeof(double) * n_sys));
  WGW_TRY(c->cg_rr.ensure(sizeof(double) * n_sys));
  WGW_TRY(c->cg_act.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->cg_it.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->cg_best.ensure(sizeof(double) * n_sys));
  WGW_TRY(c->cg_itbest.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->rr64.ensure(sizeof(double) * n_sys));
  WGW_TRY(c->act64.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->sys_list.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->cg_rzi.ensure(sizeof(double) * n_sys));
  WGW_TRY(c->omg.ensure(sizeof(double) * n_sys));
  WGW_TRY(c->row_list.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->list64.ensure(sizeof(int) * n_sys));
  WGW_TRY(c->cnt.ensure(sizeof(int) * 4));
  WGW_TRY(c->dv_r.ensure(sizeof(double) * (size_t)n_real * c->grid3));
  WGW_TRY(c->Dr.ensure(sizeof(double) * (size_t)n_real * c->grid3));
  return WGW_OK;
}

__global__ void k_residual_flags(int n_sys, const double* rr, const double* bb, double tol2, int* act) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n_sys) act[s] = (bb[s] > 0.0 && rr[s] > tol2 * bb[s]) ? 1 : 0;
}

// The residual of each refinement is projected with the FP32 tensor-core P_c (see solve_all).
constexpr bool kRefineResidualFp32Pc = true;

// Solve all systems to cg_tol.  Right-hand sides in d.Bv; solutions into d.X.
int solve_all(wgw_ctx* c, int n_sys, cudaStream_t st, wgw_stats* stats) {
  const int n = c->wfc.nrb();
  const long ld = c->ld_w;
  const double tol = c->opt.cg_tol;
  std::vector<int> iters_total(n_sys, 0);
  int refinements = 0;
  if (c->opt.precision == WGW_FP64) {
    WGW_TRY(cg_solve<double>(c, c->d, n_sys, tol, c->opt.max_cg_iter, st));
    WGW_CK(cudaMemcpyAsync(iters_total.data(), c->cg_it.p, sizeof(int) * n_sys, cudaMemcpyDeviceToHost, st));
  } else {
    // Iterative refinement: x = 0, r = b; repeat { inner FP32 CG on A e = r; x += e; r = b - A x (FP64) }.
    double* X = c->d.X.as<double>();
    double* R = c->d.R.as<double>();
    double* Q = c->d.Q.as<double>();
    const double* Bv = c->d.Bv.as<double>();
    WGW_CK(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)n_sys * ld, st));
    WGW_CK(cudaMemcpyAsync(R, Bv, sizeof(double) * (size_t)n_sys * ld, cudaMemcpyDeviceToDevice, st));
    WGW_CK(c->prof.run(PK_OTHER, 8.0 * n_sys * n, 0, st, [&] { return launch_norm2<double>(n_sys, n, Bv, ld, c->cg_bb.as<double>(), st); }));
    std::vector<int> it_host(n_sys);
    // Keep the FP64 |b|^2 aside: the inner solves overwrite cg_bb.
    WGW_TRY(c->norms.ensure(sizeof(double) * n_sys));
    double* bb64 = c->norms.as<double>();
    WGW_CK(cudaMemcpyAsync(bb64, c->cg_bb.p, sizeof(double) * n_sys, cudaMemcpyDeviceToDevice, st));
    int* act64 = c->act64.as<int>();
    for (int k = 0; k < c->opt.max_refine; ++k) {
      WGW_CK(c->prof.run(PK_OTHER, 8.0 * n_sys * n, 0, st, [&] { return launch_norm2<double>(n_sys, n, R, ld, c->rr64.as<double>(), st); }));
      WGW_CK(c->prof.run(PK_OTHER, 20.0 * n_sys, 0, st, [&] {
        k_residual_flags<<<(n_sys + 255) / 256, 256, 0, st>>>(n_sys, c->rr64.as<double>(), bb64, tol * tol, act64);
        return cudaGetLastError(); }));
      int na = 0;
      int* l64 = c->list64.as<int>();
      WGW_TRY(build_list(c, act64, n_sys, l64, st, &na));
      if (na == 0) break;
      ++refinements;
      // Inner right-hand side: the FP32 image of r (only active systems; others get b = 0).
      WGW_CK(cudaMemsetAsync(c->f.Bv.p, 0, sizeof(float) * (size_t)n_sys * ld, st));
      WGW_CK(c->prof.run(PK_CONV, 12.0 * n_sys * n, 0, st, [&] { return launch_copy_cast<double, float>(n_sys, n, R, ld, c->f.Bv.as<float>(), ld, act64, st); }));
      WGW_TRY(cg_solve<float>(c, c->f, n_sys, c->opt.inner_tol, c->opt.max_cg_iter, st));
      WGW_CK(cudaMemcpyAsync(it_host.data(), c->cg_it.p, sizeof(int) * n_sys, cudaMemcpyDeviceToHost, st));
      WGW_CK(cudaStreamSynchronize(st));
      for (int s = 0; s < n_sys; ++s) iters_total[s] += it_host[s];
      WGW_CK(c->prof.run(PK_CONV, 20.0 * n_sys * n, 0, st, [&] { return launch_add_to<float>(n_sys, n, c->f.X.as<float>(), ld, X, ld, act64, st); }));
      // r = b - A x in FP64 for the systems that moved.  The FP32 corrections carry an
      // O(eps_32) component along the occupied states; P_c (H - e_v) maps it to zero (the
      // occupied states are eigenvectors of H), so the residual does not see it and it is
      // projected out once, after the last refinement.
      //
      // P_c of the residual: (H - e_v) x is formed at FP64 accuracy and left unprojected;
      // r = b - (H - e_v) x then differs from P_c r only by o = P_v (H - e_v) x, small with
      // the occupied component of x (FP32 rounding of the corrections).  That component is
      // removed with the FP32 tensor-core projector applied twice to the FP32 image t of r:
      //   r += P_c(P_c(t)) - t.
      // One FP32 pass leaves an occupied error of about eps |t| ~ eps |o| (the overlaps are
      // formed from all of t), which the inner solves cannot reduce and which stalled the
      // refinement above cg_tol = 1e-11 with 256 occupied states; the second pass takes it to
      // eps^2 |o|.  What remains is the FP32 rounding of the subtraction, eps_32 |o|, far below
      // cg_tol |b|.  The FP64-accuracy projector stays on the right-hand sides and the final x.
      WGW_TRY(apply_A<double>(c, c->d, X, Q, na, l64, act64, st, !kRefineResidualFp32Pc));
      WGW_CK(c->prof.run(PK_CONV, 24.0 * n_sys * n, 0, st, [&] { return launch_axpby(n_sys, n, 1.0, Bv, -1.0, Q, R, ld, act64, st); }));
      if (kRefineResidualFp32Pc) {
        float* t32 = c->f.Bv.as<float>();
        float* p32 = c->f.X.as<float>();
        WGW_CK(c->prof.run(PK_CONV, 24.0 * na * n, 0, st, [&] {
          cudaError_t e = launch_copy_cast<double, float>(n_sys, n, R, ld, t32, ld, act64, st);
          if (e == cudaSuccess) e = launch_copy_cast<double, float>(n_sys, n, R, ld, p32, ld, act64, st);
          return e; }));
        for (int pass = 0; pass < 2; ++pass) WGW_TRY(run_pc<float>(c, p32, na, l64, c->f.psi.as<float>(), act64, st));
        WGW_CK(c->prof.run(PK_CONV, 24.0 * na * n, 0, st, [&] {
          return launch_add_diff(n_sys, n, p32, t32, ld, R, ld, act64, st); }));
      }
    }
    // The solution lies in range(P_c): remove the occupied component in FP64.
    WGW_TRY(run_pc<double>(c, X, n_sys, nullptr, c->d.psi.as<double>(), nullptr, st));
  }
  if (c->opt.precision == WGW_FP64) {
    // Final FP64 residual of every system (independent check of the CG's recursive residual).
    double* X = c->d.X.as<double>();
    double* Q = c->d.Q.as<double>();
    double* R = c->d.R.as<double>();
    WGW_TRY(apply_A<double>(c, c->d, X, Q, n_sys, nullptr, nullptr, st));
    WGW_CK(c->prof.run(PK_CONV, 24.0 * n_sys * n, 0, st, [&] { return launch_axpby(n_sys, n, 1.0, c->d.Bv.as<double>(), -1.0, Q, R, ld, nullptr, st); }));
    WGW_CK(c->prof.run(PK_OTHER, 8.0 * n_sys * n, 0, st, [&] { return launch_norm2<double>(n_sys, n, R, ld, c->rr64.as<double>(), st); }));
    WGW_CK(c->prof.run(PK_OTHER, 8.0 * n_sys * n, 0, st, [&] { return launch_norm2<double>(n_sys, n, c->d.Bv.as<double>(), ld, c->cg_bb.as<double>(), st); }));
  } else {
    // R holds b - A x in FP64 for every system's final x (recomputed after its last
    // update); ||b||^2 was kept in norms.
    WGW_CK(c->prof.run(PK_OTHER, 8.0 * n_sys * n, 0, st, [&] {
      return launch_norm2<double>(n_sys, n, c->d.R.as<double>(), ld, c->rr64.as<double>(), st); }));
    WGW_CK(cudaMemcpyAsync(c->cg_bb.p, c->norms.p, sizeof(double) * n_sys, cudaMemcpyDeviceToDevice, st));
  }
  std::vector<double> rr(n_sys), bb(n_sys);
  WGW_CK(cudaMemcpyAsync(rr.data(), c->rr64.p, sizeof(double) * n_sys, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaMemcpyAsync(bb.data(), c->cg_bb.p, sizeof(double) * n_sys, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  int conv = 0, maxit = 0;
  double maxrel = 0.0;
  c->blk_iters = iters_total;
  c->blk_relres.assign(n_sys, 0.0);
  c->blk_conv.assign(n_sys, 0);
  for (int s = 0; s < n_sys; ++s) {
    const double rel = bb[s] > 0 ? std::sqrt(rr[s] / bb[s]) : 0.0;
    c->blk_relres[s] = rel;
    maxrel = std::max(maxrel, rel);
    if (rel <= tol * (1.0 + 1e-6) || bb[s] == 0.0) { ++conv; c->blk_conv[s] = 1; }
    maxit = std::max(maxit, iters_total[s]);
  }
  if (stats) {
    stats->n_systems += n_sys;
    stats->n_converged += conv;
    stats->max_iters = std::max(stats->max_iters, maxit);
    stats->refinements = std::max(stats->refinements, refinements);
    stats->max_rel_residual = std::max(stats->max_rel_residual, maxrel);
  }
  return conv == n_sys ? WGW_OK : fail(WGW_ERR_NOCONV, "some Sternheimer systems missed cg_tol");
}

__global__ void k_rows_from_systems(int n_cs, const int* __restrict__ act, int* __restrict__ rows) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_cs; s += gridDim.x * blockDim.x)
    rows[2 * s] = rows[2 * s + 1] = act[s];
}

CocgState cocg_state(wgw_ctx* c) {
  CocgState s;
  s.rz_re = c->cg_rz.as<double>(); s.rz_im = c->cg_rzi.as<double>(); s.bb = c->cg_bb.as<double>();
  s.rr = c->cg_rr.as<double>(); s.active = c->cg_act.as<int>(); s.iters = c->cg_it.as<int>();
  s.omega = c->omg.as<double>();
  return s;
}

// List of active complex systems into c->sys_list and the matching row list into c->row_list.
int build_cs_lists(wgw_ctx* c, const int* flags, int n_cs, cudaStream_t st, int* n_out) {
  WGW_TRY(build_list(c, flags, n_cs, c->sys_list.as<int>(), st, n_out));
  WGW_CK(launch_expand_rows(c->sys_list.as<int>(), *n_out, c->row_list.as<int>(), st));
  return WGW_OK;
}

// COCG on (A + i w_s) x = b for n_cs complex systems (rows 2s, 2s+1 of pr.Bv / pr.X).
template <typename T>
int cocg_solve(wgw_ctx* c, Prec<T>& pr, int n_cs, double tol, int max_iter, cudaStream_t st) {
  ProfPrec pp(c->prof, sizeof(T) == 8);
  const int n = c->wfc.nrb();
  const long ld = c->ld_w;
  T* X = pr.X.template as<T>();
  T* R = pr.R.template as<T>();
  T* Z = pr.Z.template as<T>();
  T* P = pr.P.template as<T>();
  T* Q = pr.Q.template as<T>();
  const T* Bv = pr.Bv.template as<T>();
  const T* Psi = pr.psi.template as<T>();
  const double* eps = c->eps.as<double>();
  CocgState cs = cocg_state(c);
  const double vb = 2.0 * n_cs * n * sizeof(T);
  WGW_CK(c->prof.run(PK_CG, 4 * vb, 0, st, [&] {
    return launch_cocg_init_a<T>(c->wfc.tab(), n, n_cs, Bv, X, R, Z, ld, eps, cs, st); }));
  WGW_TRY(run_pc<T>(c, Z, 2 * n_cs, nullptr, Psi, nullptr, st));
  WGW_CK(c->prof.run(PK_CG, 3 * vb, 0, st, [&] { return launch_cocg_init_b<T>(n, n_cs, R, Z, P, ld, cs, st); }));
  int n_list = 0;
  WGW_TRY(build_cs_lists(c, cs.active, n_cs, st, &n_list));
  const int* lbuf = c->sys_list.as<int>();
  const int* rbuf = c->row_list.as<int>();
  const int every = std::max(1, c->opt.check_every);
  const bool proj_q = sizeof(T) == sizeof(double) || kProjectInnerOutput;
  auto iteration = [&](cudaStream_t s) -> int {
    const double lb = 2.0 * n_list * n * sizeof(T);
    WGW_TRY(apply_A<T>(c, pr, P, Q, 2 * n_list, rbuf, nullptr, s, proj_q));
    WGW_CK(c->prof.run(PK_CG, 9 * lb, 0, s, [&] {
      return launch_cocg_step_a<T>(c->wfc.tab(), n, n_list, lbuf, X, R, Z, P, Q, ld, eps, cs, tol * tol,
                                   max_iter, s); }));
    WGW_TRY(run_pc<T>(c, Z, 2 * n_list, rbuf, Psi, nullptr, s));
    WGW_CK(c->prof.run(PK_CG, 4 * lb, 0, s, [&] {
      return launch_cocg_step_b<T>(n, n_list, lbuf, R, Z, P, ld, cs, s); }));
    return WGW_OK;
  };
  const bool dev_loop = c->opt.cuda_graphs == 2 && !c->prof.on;
  for (int it = 0; it < max_iter && n_list > 0;) {
    if (dev_loop && it > 0 && it % every == 0) {   // as in cg_solve, after a first direct window
      int left = 0, ran = 0;
      WGW_TRY(device_loop(c, st, cs.active, c->sys_list.as<int>(), c->row_list.as<int>(), n_list,
                          (max_iter - it + every - 1) / every, n_list > 64 ? n_list / 2 : 0,
                          [&](cudaStream_t s) -> int {
                            for (int k = 0; k < every; ++k) WGW_TRY(iteration(s));
                            if (!proj_q) WGW_TRY(run_pc<T>(c, R, 2 * n_list, rbuf, Psi, nullptr, s));
                            return WGW_OK;
                          },
                          &left, &ran));
      it += ran * every;
      n_list = left;
      continue;
    }
    WGW_TRY(iteration(st));
    ++it;
    if (it % every == 0) {
      if (!proj_q) WGW_TRY(run_pc<T>(c, R, 2 * n_list, rbuf, Psi, nullptr, st));   // as in cg_solve
      WGW_TRY(build_cs_lists(c, cs.active, n_cs, st, &n_list));
    }
  }
  return WGW_OK;
}

// Solve all complex-shifted systems to cg_tol (right-hand sides in d.Bv rows, solutions into d.X).
int solve_shifted(wgw_ctx* c, int n_cs, cudaStream_t st, wgw_stats* stats) {
  const int n = c->wfc.nrb();
  const long ld = c->ld_w;
  const double tol = c->opt.cg_tol;
  std::vector<int> iters_total(n_cs, 0), it_host(n_cs);
  int refinements = 0;
  double* X = c->d.X.as<double>();
  double* R = c->d.R.as<double>();
  double* Q = c->d.Q.as<double>();
  const double* Bv = c->d.Bv.as<double>();
  const double* omega = c->omg.as<double>();
  WGW_TRY(c->norms.ensure(sizeof(double) * n_cs));
  double* bb64 = c->norms.as<double>();
  WGW_CK(launch_pair_norm2(n_cs, n, Bv, ld, bb64, st));
  if (c->opt.precision == WGW_FP64) {
    WGW_TRY(cocg_solve<double>(c, c->d, n_cs, tol, c->opt.max_cg_iter, st));
    WGW_CK(cudaMemcpyAsync(iters_total.data(), c->cg_it.p, sizeof(int) * n_cs, cudaMemcpyDeviceToHost, st));
    WGW_TRY(run_pc<double>(c, X, 2 * n_cs, nullptr, c->d.psi.as<double>(), nullptr, st));
    WGW_TRY(apply_A<double>(c, c->d, X, Q, 2 * n_cs, nullptr, nullptr, st));
    WGW_CK(launch_shifted_residual(n_cs, n, Bv, Q, X, omega, R, ld, nullptr, st));
  } else {
    WGW_CK(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)2 * n_cs * ld, st));
    WGW_CK(cudaMemcpyAsync(R, Bv, sizeof(double) * (size_t)2 * n_cs * ld, cudaMemcpyDeviceToDevice, st));
    int* act64 = c->act64.as<int>();
    WGW_TRY(c->rowact.ensure(sizeof(int) * 2 * n_cs));
    int* rowact = c->rowact.as<int>();
    for (int k = 0; k < c->opt.max_refine; ++k) {
      WGW_CK(launch_pair_norm2(n_cs, n, R, ld, c->rr64.as<double>(), st));
      k_residual_flags<<<(n_cs + 255) / 256, 256, 0, st>>>(n_cs, c->rr64.as<double>(), bb64, tol * tol, act64);
      WGW_CK(cudaGetLastError());
      int na = 0;
      WGW_TRY(build_cs_lists(c, act64, n_cs, st, &na));
      if (na == 0) break;
      ++refinements;
      // Keep the list of this refinement step: cocg_solve rebuilds sys_list / row_list.
      WGW_TRY(c->list64.ensure(sizeof(int) * 2 * n_cs));
      WGW_CK(cudaMemcpyAsync(c->list64.p, c->row_list.p, sizeof(int) * 2 * na, cudaMemcpyDeviceToDevice, st));
      k_rows_from_systems<<<(n_cs + 255) / 256, 256, 0, st>>>(n_cs, act64, rowact);
      WGW_CK(cudaGetLastError());
      WGW_CK(cudaMemsetAsync(c->f.Bv.p, 0, sizeof(float) * (size_t)2 * n_cs * ld, st));
      WGW_CK((launch_copy_cast<double, float>(2 * n_cs, n, R, ld, c->f.Bv.as<float>(), ld, rowact, st)));
      WGW_TRY(cocg_solve<float>(c, c->f, n_cs, c->opt.inner_tol, c->opt.max_cg_iter, st));
      WGW_CK(cudaMemcpyAsync(it_host.data(), c->cg_it.p, sizeof(int) * n_cs, cudaMemcpyDeviceToHost, st));
      WGW_CK(cudaStreamSynchronize(st));
      for (int q = 0; q < n_cs; ++q) iters_total[q] += it_host[q];
      WGW_CK(launch_add_to<float>(2 * n_cs, n, c->f.X.as<float>(), ld, X, ld, rowact, st));
      const int* l64 = c->list64.as<int>();
      WGW_TRY(run_pc<double>(c, X, 2 * na, l64, c->d.psi.as<double>(), nullptr, st));
      WGW_TRY(apply_A<double>(c, c->d, X, Q, 2 * na, l64, nullptr, st));
      WGW_CK(launch_shifted_residual(n_cs, n, Bv, Q, X, omega, R, ld, act64, st));
    }
  }
  WGW_CK(launch_pair_norm2(n_cs, n, R, ld, c->rr64.as<double>(), st));
  std::vector<double> rr(n_cs), bb(n_cs);
  WGW_CK(cudaMemcpyAsync(rr.data(), c->rr64.p, sizeof(double) * n_cs, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaMemcpyAsync(bb.data(), bb64, sizeof(double) * n_cs, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  int conv = 0, maxit = 0;
  double maxrel = 0.0;
  c->blk_iters = iters_total;
  c->blk_relres.assign(n_cs, 0.0);
  c->blk_conv.assign(n_cs, 0);
  for (int q = 0; q < n_cs; ++q) {
    const double rel = bb[q] > 0 ? std::sqrt(rr[q] / bb[q]) : 0.0;
    c->blk_relres[q] = rel;
    maxrel = std::max(maxrel, rel);
    if (rel <= tol * (1.0 + 1e-6) || bb[q] == 0.0) { ++conv; c->blk_conv[q] = 1; }
    maxit = std::max(maxit, iters_total[q]);
  }
  if (stats) {
    stats->n_systems += n_cs;
    stats->n_converged += conv;
    stats->max_iters = std::max(stats->max_iters, maxit);
    stats->refinements = std::max(stats->refinements, refinements);
    stats->max_rel_residual = std::max(stats->max_rel_residual, maxrel);
  }
  return conv == n_cs ? WGW_OK : fail(WGW_ERR_NOCONV, "some complex-shifted Sternheimer systems missed cg_tol");
}

// Device bytes one batched solve needs per system and per perturbation (vectors, the FFT pair
// intermediates of both precisions, projector work, real-space perturbation and drho).
void solve_bytes(const wgw_ctx* c, double* per_sys, double* per_pert) {
  const double N2 = (double)c->N * c->N;
  const bool mixed = c->opt.precision == WGW_MIXED;
  const int nv = std::max(c->n_v, c->n_proj), nvp = (nv + 63) / 64 * 64;
  *per_sys = (6.0 * 8 + (mixed ? 6.0 * 4 : 0.0)) * c->ld_w + 0.5 * (2 * c->wfc.m + 1) * N2 * (16.0 + (mixed ? 8.0 : 0.0)) +
             8.0 * nvp * 2 + 128.0;
  *per_pert = 2.0 * 8.0 * c->grid3 + 8.0 * c->ld_r + 0.5 * (2 * c->rho.m + 1) * N2 * 16.0;
}

// Bytes held by the grow-only work buffers of the batched solves (reused or regrown by the next one).
double held_work_bytes(const wgw_ctx* c) {
  const DevBuf* bufs[] = {&c->d.X, &c->d.R, &c->d.Z, &c->d.P, &c->d.Q, &c->d.Bv, &c->d.Tw,
                          &c->f.X, &c->f.R, &c->f.Z, &c->f.P, &c->f.Q, &c->f.Bv, &c->f.Tw,
                          &c->pc_work, &c->dv_r, &c->Dr, &c->Trho};
  double b = 0.0;
  for (const DevBuf* d : bufs) b += (double)d->bytes;
  return b;
}

// Perturbations per batched solve: all of them when they fit, else as many as fit 85 % of the
// free device memory (plus the work buffers the context already holds), or the option's cap.
int chunk_perts(wgw_ctx* c, int n_real, int sys_per_pert) {
  double per_sys = 0, per_pert = 0;
  solve_bytes(c, &per_sys, &per_pert);
  const double per = per_sys * sys_per_pert + per_pert;
  int by_mem = n_real;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
    const double budget = 0.85 * ((double)free_b + held_work_bytes(c));
    by_mem = (int)std::max(1.0, std::floor(budget / per));
  } else {
    cudaGetLastError();
  }
  int cap = n_real;
  if (c->opt.max_batch_systems > 0) cap = std::max(1, c->opt.max_batch_systems / std::max(1, sys_per_pert));
  return std::max(1, std::min(n_real, std::min(by_mem, cap)));
}

// drho_r(r) = (2 f_s / Omega) sum_v psi_v(r) x_{r v}(r) for the solutions X (systems s = r n_v + v,
// rows of length ldx), then to the density sphere: real-basis rows of drho_out (length ld_r).
int drho_pass(wgw_ctx* c, const double* X, long ldx, int n_real, double* drho_out, cudaStream_t st) {
  ProfPrec pp(c->prof, true);
  const int N = c->N, n_v = c->n_v, n_sys = n_real * n_v;
  const HostSphere& rs = c->rho;
  const int NP = 2 * c->wfc.m + 1, pairs = (n_sys + 1) / 2;
  WGW_TRY(c->d.Tw.ensure(sizeof(cplx<double>) * (size_t)pairs * NP * N * N));
  WGW_TRY(c->Dr.ensure(sizeof(double) * (size_t)n_real * c->grid3));
  FftCtx<double> f = c->d.fft(c->plan);
  const double tb = t_bytes<double>(c, c->wfc.m, pairs);
  WGW_CK(c->prof.run(PK_G2R, tb + (double)n_sys * c->wfc.nrb() * sizeof(double), 0, st, [&] {
    return launch_plane_g2r<double>(c->wfc.tab(), f, X, ldx, n_sys, nullptr, nullptr, c->d.Tw.as<cplx<double>>(),
                                    st); }));
  const double coef = 2.0 * c->opt.f_s / c->omega_cell;
  WGW_CK(c->prof.run(PK_DRHO, tb + (double)(n_v + n_real) * c->grid3 * sizeof(double), 0, st, [&] {
    return launch_drho_xline<double>(c->wfc.m, f, c->d.Tw.as<cplx<double>>(), c->d.psi_r_fft(), c->grid3, n_v,
                                     n_sys, n_real, coef, c->Dr.as<double>(), c->grid3, st); }));
  const int NPr = 2 * rs.m + 1, rpairs = (n_real + 1) / 2;
  WGW_TRY(c->Trho.ensure(sizeof(cplx<double>) * (size_t)rpairs * NPr * N * N));
  XArgs<double> a{};
  a.mode = XM_FROM_REAL; a.A = c->Dr.as<double>(); a.lda = c->grid3; a.n_sys = n_real;
  const double tr = t_bytes<double>(c, rs.m, rpairs);
  WGW_CK(c->prof.run(PK_XLINE, tr + (double)n_real * c->grid3 * sizeof(double), 0, st, [&] {
    return launch_xline<double>(rs.m, f, c->Trho.as<cplx<double>>(), a, nullptr, st); }));
  Epi<double> e{};
  e.out = drho_out; e.ldo = c->ld_r; e.vcoef = 1.0; e.n_sys = n_real;
  WGW_CK(c->prof.run(PK_R2G, tr + (double)n_real * rs.nrb() * sizeof(double), 0, st, [&] {
    return launch_plane_r2g<double>(rs.tab(), rs.npt_max, f, c->Trho.as<cplx<double>>(), e, st); }));
  return WGW_OK;
}

// drho = chi0 dV for n_real perturbations that are real in r, given and returned in
// real-basis form (rows of length ld_r): dV in dvrb, drho into drho_out.  Steps 2-6
// of the apply for one batched solve: system tables, dV(r), right-hand sides, Sternheimer
// solves, drho.
int chi0_rb_block(wgw_ctx* c, const double* dvrb, int n_real, double* drho_out, cudaStream_t st,
                  wgw_stats* stats) {
  const int N = c->N, n_v = c->n_v;
  const long ldr = c->ld_r, ldw = c->ld_w;
  const HostSphere& rs = c->rho;
  const int n_sys = n_real * n_v;
  WGW_TRY(ensure_work(c, n_sys, n_real));
  // 2. System tables: s = r * n_v + v.
  std::vector<double> eps(n_sys), shift(n_sys);
  std::vector<float> shiftf(n_sys);
  std::vector<int> ai(n_sys), bi(n_sys);
  for (int r = 0; r < n_real; ++r)
    for (int v = 0; v < n_v; ++v) {
      const int s = r * n_v + v;
      eps[s] = c->e_v[v];
      shift[s] = -c->e_v[v];
      shiftf[s] = (float)shift[s];
      ai[s] = v;
      bi[s] = r;
    }
  WGW_CK(cudaMemcpyAsync(c->eps.p, eps.data(), sizeof(double) * n_sys, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemcpyAsync(c->d.shift.p, shift.data(), sizeof(double) * n_sys, cudaMemcpyHostToDevice, st));
  if (c->opt.precision == WGW_MIXED)
    WGW_CK(cudaMemcpyAsync(c->f.shift.p, shiftf.data(), sizeof(float) * n_sys, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemcpyAsync(c->a_idx.p, ai.data(), sizeof(int) * n_sys, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemcpyAsync(c->b_idx.p, bi.data(), sizeof(int) * n_sys, cudaMemcpyHostToDevice, st));
  // 3. dV_r(r) for every real perturbation.
  double* dvr = c->dv_r.as<double>();
  WGW_TRY(to_real<double>(c, c->d, rs, dvrb, ldr, n_real, dvr, c->Trho, st));
  // 4. Right-hand sides b_s = -P_c [psi_v(r) dV_r(r)] on the wavefunction sphere.
  {
    const int NP = 2 * c->wfc.m + 1, pairs = (n_sys + 1) / 2;
    WGW_TRY(c->d.Tw.ensure(sizeof(cplx<double>) * (size_t)pairs * NP * N * N));
    FftCtx<double> f = c->d.fft(c->plan);
    XArgs<double> a{};
    a.mode = XM_FROM_REAL; a.A = c->d.psi_r_fft(); a.lda = c->grid3; a.a_index = c->a_idx.as<int>();
    a.Bm = dvr; a.ldb = c->grid3; a.b_index = c->b_idx.as<int>(); a.n_sys = n_sys;
    const double tb = t_bytes<double>(c, c->wfc.m, pairs);
    WGW_CK(c->prof.run(PK_XLINE, tb + 2.0 * n_sys * c->grid3 * sizeof(double), 0, st, [&] {
      return launch_xline<double>(c->wfc.m, f, c->d.Tw.as<cplx<double>>(), a, nullptr, st); }));
    Epi<double> e{};
    e.out = c->d.Bv.as<double>(); e.ldo = ldw; e.vcoef = -1.0; e.n_sys = n_sys;
    WGW_CK(c->prof.run(PK_R2G, tb + (double)n_sys * c->wfc.nrb() * sizeof(double), 0, st, [&] {
      return launch_plane_r2g<double>(c->wfc.tab(), c->wfc.npt_max, f, c->d.Tw.as<cplx<double>>(), e, st); }));
    WGW_TRY(run_pc<double>(c, c->d.Bv.as<double>(), n_sys, nullptr, c->d.psi.as<double>(), nullptr, st));
  }
  // 5. Sternheimer solves.
  const int solve_status = solve_all(c, n_sys, st, stats);
  if (solve_status != WGW_OK && solve_status != WGW_ERR_NOCONV) return solve_status;
  // 6. drho_r(r) = (2 f_s / Omega) sum_v psi_v(r) x_{v r}(r), then to the density sphere.
  WGW_TRY(drho_pass(c, c->d.X.as<double>(), ldw, n_real, drho_out, st));
  return solve_status;
}

// Copies the solutions of the sampled systems among [s0, s0 + n) (rows s - s0 of d.X, real basis)
// to the host as wavefunction-sphere coefficients.
int keep_samples(wgw_ctx* c, int s0, int n, cudaStream_t st) {
  const int n_pw = c->wfc.n;
  if (c->sample_out.size() != c->sample_sys.size() * 2 * (size_t)n_pw)
    c->sample_out.assign(c->sample_sys.size() * 2 * (size_t)n_pw, 0.0);
  for (size_t k = 0; k < c->sample_sys.size(); ++k) {
    const int sys = c->sample_sys[k];
    if (sys < s0 || sys >= s0 + n) continue;
    WGW_TRY(c->sample_buf.ensure(sizeof(double) * 2 * (size_t)n_pw));
    WGW_CK(launch_rb_to_sphere(1, c->d.X.as<double>() + (size_t)(sys - s0) * c->ld_w, c->ld_w, nullptr, nullptr,
                               c->wfc.map(), c->sample_buf.as<double>(), 2L * n_pw, st));
    WGW_CK(cudaMemcpyAsync(c->sample_out.data() + k * 2 * (size_t)n_pw, c->sample_buf.p,
                           sizeof(double) * 2 * (size_t)n_pw, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
  }
  return WGW_OK;
}

// chi0_rb_block over chunks of perturbations that fit the device (drho into c->drho_rb); the
// per-system records of wgw_system_info follow the batch order s = r n_v + v.
int chi0_rb(wgw_ctx* c, const double* dvrb, int n_real, cudaStream_t st, wgw_stats* stats) {
  WGW_TRY(c->drho_rb.ensure(sizeof(double) * (size_t)std::max(n_real, 1) * c->ld_r));
  const int per = chunk_perts(c, n_real, c->n_v);
  c->last_iters.assign((size_t)n_real * c->n_v, 0);
  c->last_relres.assign((size_t)n_real * c->n_v, 0.0);
  c->last_conv.assign((size_t)n_real * c->n_v, 0);
  int status = WGW_OK;
  for (int r0 = 0; r0 < n_real; r0 += per) {
    const int nr = std::min(per, n_real - r0);
    const int s1 = chi0_rb_block(c, dvrb + (size_t)r0 * c->ld_r, nr, c->drho_rb.as<double>() + (size_t)r0 * c->ld_r,
                                 st, stats);
    if (s1 != WGW_OK && s1 != WGW_ERR_NOCONV) return s1;
    if (s1 == WGW_ERR_NOCONV) status = s1;
    std::copy(c->blk_iters.begin(), c->blk_iters.end(), c->last_iters.begin() + (size_t)r0 * c->n_v);
    std::copy(c->blk_relres.begin(), c->blk_relres.end(), c->last_relres.begin() + (size_t)r0 * c->n_v);
    std::copy(c->blk_conv.begin(), c->blk_conv.end(), c->last_conv.begin() + (size_t)r0 * c->n_v);
    WGW_TRY(keep_samples(c, r0 * c->n_v, nr * c->n_v, st));
  }
  return status == WGW_OK ? WGW_OK : fail(status, "some Sternheimer systems missed cg_tol");
}

// drho(i w_k) = chi0(i w_k) dV for n_real real-in-r perturbations (real-basis rows of dvrb) and
// every w_k > 0, batched over frequencies: complex system (k, r, v) -> rows 2s, 2s+1 with
// s = (k n_real + r) n_v + v.  Results for frequency k at out + k * kstride (rows r, length ld_r).
int chi0_rb_shifted_block(wgw_ctx* c, const double* dvrb, int n_real, const std::vector<double>& oms,
                          double* out, size_t kstride, cudaStream_t st, wgw_stats* stats) {
  const int N = c->N, n_v = c->n_v, n_om = (int)oms.size();
  const long ldr = c->ld_r, ldw = c->ld_w;
  const HostSphere& rs = c->rho;
  const int n_rs = n_real * n_v, n_cs = n_om * n_rs, rows = 2 * n_cs;
  WGW_TRY(ensure_work(c, std::max(rows, n_rs), n_real));
  std::vector<int> ai(n_rs), bi(n_rs);
  for (int r = 0; r < n_real; ++r)
    for (int v = 0; v < n_v; ++v) { ai[r * n_v + v] = v; bi[r * n_v + v] = r; }
  std::vector<double> eps(n_cs), om(n_cs), shift(rows);
  std::vector<float> shiftf(rows);
  for (int k = 0; k < n_om; ++k)
    for (int q = 0; q < n_rs; ++q) {
      const int s = k * n_rs + q, v = q % n_v;
      eps[s] = c->e_v[v];
      om[s] = oms[k];
      shift[2 * s] = shift[2 * s + 1] = -c->e_v[v];
      shiftf[2 * s] = shiftf[2 * s + 1] = (float)-c->e_v[v];
    }
  WGW_CK(cudaMemcpyAsync(c->a_idx.p, ai.data(), sizeof(int) * n_rs, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemcpyAsync(c->b_idx.p, bi.data(), sizeof(int) * n_rs, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemcpyAsync(c->eps.p, eps.data(), sizeof(double) * n_cs, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemcpyAsync(c->omg.p, om.data(), sizeof(double) * n_cs, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemcpyAsync(c->d.shift.p, shift.data(), sizeof(double) * rows, cudaMemcpyHostToDevice, st));
  if (c->opt.precision == WGW_MIXED)
    WGW_CK(cudaMemcpyAsync(c->f.shift.p, shiftf.data(), sizeof(float) * rows, cudaMemcpyHostToDevice, st));
  double* dvr = c->dv_r.as<double>();
  WGW_TRY(to_real<double>(c, c->d, rs, dvrb, ldr, n_real, dvr, c->Trho, st));
  FftCtx<double> f = c->d.fft(c->plan);
  {
    // Real right-hand sides -P_c [psi_v dV_r] of the n_rs (r, v) pairs into d.Q, then copied to
    // the real row of every frequency's complex system (imaginary rows are zero).
    const int NP = 2 * c->wfc.m + 1, pairs = (n_rs + 1) / 2;
    WGW_TRY(c->d.Tw.ensure(sizeof(cplx<double>) * (size_t)pairs * NP * N * N));
    XArgs<double> a{};
    a.mode = XM_FROM_REAL; a.A = c->d.psi_r_fft(); a.lda = c->grid3; a.a_index = c->a_idx.as<int>();
    a.Bm = dvr; a.ldb = c->grid3; a.b_index = c->b_idx.as<int>(); a.n_sys = n_rs;
    const double tb = t_bytes<double>(c, c->wfc.m, pairs);
    WGW_CK(c->prof.run(PK_XLINE, tb + 2.0 * n_rs * c->grid3 * sizeof(double), 0, st, [&] {
      return launch_xline<double>(c->wfc.m, f, c->d.Tw.as<cplx<double>>(), a, nullptr, st); }));
    Epi<double> e{};
    e.out = c->d.Q.as<double>(); e.ldo = ldw; e.vcoef = -1.0; e.n_sys = n_rs;
    WGW_CK(c->prof.run(PK_R2G, tb + (double)n_rs * c->wfc.nrb() * sizeof(double), 0, st, [&] {
      return launch_plane_r2g<double>(c->wfc.tab(), c->wfc.npt_max, f, c->d.Tw.as<cplx<double>>(), e, st); }));
    WGW_TRY(run_pc<double>(c, c->d.Q.as<double>(), n_rs, nullptr, c->d.psi.as<double>(), nullptr, st));
    WGW_CK(cudaMemsetAsync(c->d.Bv.p, 0, sizeof(double) * (size_t)rows * ldw, st));
    for (int k = 0; k < n_om; ++k)
      WGW_CK(cudaMemcpy2DAsync(c->d.Bv.as<double>() + (size_t)2 * k * n_rs * ldw, 2 * ldw * sizeof(double),
                               c->d.Q.p, ldw * sizeof(double), ldw * sizeof(double), n_rs,
                               cudaMemcpyDeviceToDevice, st));
  }
  const int solve_status = solve_shifted(c, n_cs, st, stats);
  if (solve_status != WGW_OK && solve_status != WGW_ERR_NOCONV) return solve_status;
  const int pairs = (n_rs + 1) / 2;
  const int NPr = 2 * rs.m + 1, rpairs = (n_real + 1) / 2;
  WGW_TRY(c->Trho.ensure(sizeof(cplx<double>) * (size_t)rpairs * NPr * N * N));
  const double coef = 2.0 * c->opt.f_s / c->omega_cell;
  for (int k = 0; k < n_om; ++k) {
    // drho = (f_s/Omega) sum_v 2 Re(psi_v x_v) uses the real rows of frequency k (stride 2 ld).
    const double* Xk = c->d.X.as<double>() + (size_t)2 * k * n_rs * ldw;
    const double tb = t_bytes<double>(c, c->wfc.m, pairs);
    WGW_CK(c->prof.run(PK_G2R, tb + (double)n_rs * c->wfc.nrb() * sizeof(double), 0, st, [&] {
      return launch_plane_g2r<double>(c->wfc.tab(), f, Xk, 2 * ldw, n_rs, nullptr, nullptr,
                                      c->d.Tw.as<cplx<double>>(), st); }));
    WGW_CK(c->prof.run(PK_DRHO, tb + (double)(n_v + n_real) * c->grid3 * sizeof(double), 0, st, [&] {
      return launch_drho_xline<double>(c->wfc.m, f, c->d.Tw.as<cplx<double>>(), c->d.psi_r_fft(),
                                       c->grid3, n_v, n_rs, n_real, coef, c->Dr.as<double>(), c->grid3, st); }));
    XArgs<double> a{};
    a.mode = XM_FROM_REAL; a.A = c->Dr.as<double>(); a.lda = c->grid3; a.n_sys = n_real;
    const double tr = t_bytes<double>(c, rs.m, rpairs);
    WGW_CK(c->prof.run(PK_XLINE, tr + (double)n_real * c->grid3 * sizeof(double), 0, st, [&] {
      return launch_xline<double>(rs.m, f, c->Trho.as<cplx<double>>(), a, nullptr, st); }));
    Epi<double> e{};
    e.out = out + (size_t)k * kstride; e.ldo = ldr; e.vcoef = 1.0; e.n_sys = n_real;
    WGW_CK(c->prof.run(PK_R2G, tr + (double)n_real * rs.nrb() * sizeof(double), 0, st, [&] {
      return launch_plane_r2g<double>(rs.tab(), rs.npt_max, f, c->Trho.as<cplx<double>>(), e, st); }));
  }
  return solve_status;
}

// chi0_rb_shifted_block over chunks of perturbations that fit the device; results into
// c->drho_all (row k n_real + r), per-system records in the order q = (k n_real + r) n_v + v.
int chi0_rb_shifted(wgw_ctx* c, const double* dvrb, int n_real, const std::vector<double>& oms, cudaStream_t st,
                    wgw_stats* stats) {
  const int n_om = (int)oms.size(), n_v = c->n_v;
  const long ldr = c->ld_r;
  WGW_TRY(c->drho_all.ensure(sizeof(double) * (size_t)std::max(1, n_om * n_real) * ldr));
  const int per = chunk_perts(c, n_real, 2 * n_v * n_om);
  const size_t n_cs = (size_t)n_om * n_real * n_v;
  c->last_iters.assign(n_cs, 0);
  c->last_relres.assign(n_cs, 0.0);
  c->last_conv.assign(n_cs, 0);
  int status = WGW_OK;
  for (int r0 = 0; r0 < n_real; r0 += per) {
    const int nr = std::min(per, n_real - r0);
    const int s1 = chi0_rb_shifted_block(c, dvrb + (size_t)r0 * ldr, nr, oms, c->drho_all.as<double>() + (size_t)r0 * ldr,
                                         (size_t)n_real * ldr, st, stats);
    if (s1 != WGW_OK && s1 != WGW_ERR_NOCONV) return s1;
    if (s1 == WGW_ERR_NOCONV) status = s1;
    for (int k = 0; k < n_om; ++k)
      for (int r = 0; r < nr; ++r)
        for (int v = 0; v < n_v; ++v) {
          const size_t q = ((size_t)k * nr + r) * n_v + v, g = ((size_t)k * n_real + r0 + r) * n_v + v;
          c->last_iters[g] = c->blk_iters[q];
          c->last_relres[g] = c->blk_relres[q];
          c->last_conv[g] = c->blk_conv[q];
        }
  }
  return status == WGW_OK ? WGW_OK : fail(status, "some complex-shifted Sternheimer systems missed cg_tol");
}

// Float-float FP64-accuracy passes: the mixed path on the compiled grids.
void set_ff(wgw_ctx* c) {
  c->d.use_ff = c->opt.precision == WGW_MIXED && c->opt.fp64_emulation != 0 && ff_grid_supported(c->N);
}

// Core of chi0 / chibar0 application; dV and drho in device memory.
int apply_core(wgw_ctx* c, const double* dV, int n_pert, const double* omega, int n_omega,
               double* drho, bool symmetrized, cudaStream_t st, wgw_stats* stats) {
  if (!c) return fail(WGW_ERR_ARG, "null context");
  // Float-float kernels exist for the compiled grid sizes only; other grids run native FP64.
  set_ff(c);
  if (n_pert < 0 || n_omega < 1 || !omega) return fail(WGW_ERR_ARG, "need n_pert >= 0 and n_omega >= 1");
  std::vector<int> k_zero, k_pos;
  std::vector<double> w_pos;
  for (int k = 0; k < n_omega; ++k) {
    if (!(omega[k] >= 0.0)) return fail(WGW_ERR_ARG, "imaginary frequencies must be >= 0");
    if (omega[k] == 0.0) k_zero.push_back(k);
    else { k_pos.push_back(k); w_pos.push_back(omega[k]); }
  }
  if (n_pert == 0) return WGW_OK;
  if (!dV || !drho) return fail(WGW_ERR_ARG, "null dV or drho");
  const long ldr = c->ld_r;
  const HostSphere& rs = c->rho;
  const double* scale = symmetrized ? rs.d_vsqrt.as<double>() : nullptr;
  // 1. Real-in-r parts of each perturbation: rows [0, n_pert) = Hermitian parts,
  //    rows n_pert + k = the non-zero anti-Hermitian parts.
  WGW_TRY(c->dv_rb.ensure(sizeof(double) * (size_t)2 * n_pert * ldr));
  double* dvrb = c->dv_rb.as<double>();
  WGW_CK(cudaMemsetAsync(dvrb, 0, sizeof(double) * (size_t)2 * n_pert * ldr, st));
  const double cb = 16.0 * n_pert * rs.n + 8.0 * n_pert * rs.nrb();
  WGW_CK(c->prof.run(PK_CONV, cb, 0, st, [&] { return launch_sphere_to_rb(n_pert, dV, 2L * rs.n, scale, rs.map(), 0, dvrb, ldr, st); }));
  WGW_CK(c->prof.run(PK_CONV, cb, 0, st, [&] { return launch_sphere_to_rb(n_pert, dV, 2L * rs.n, scale, rs.map(), 1, dvrb + (size_t)n_pert * ldr, ldr, st); }));
  WGW_TRY(c->norms.ensure(sizeof(double) * 2 * n_pert));
  WGW_CK(c->prof.run(PK_OTHER, 16.0 * n_pert * rs.nrb(), 0, st, [&] { return launch_norm2<double>(2 * n_pert, rs.nrb(), dvrb, ldr, c->norms.as<double>(), st); }));
  std::vector<double> nrm(2 * n_pert);
  WGW_CK(cudaMemcpyAsync(nrm.data(), c->norms.p, sizeof(double) * 2 * n_pert, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  std::vector<int> brow(n_pert, -1);
  int n_real = n_pert;
  for (int p = 0; p < n_pert; ++p) {
    if (nrm[n_pert + p] > 0.0) {
      if (n_real != n_pert + p)
        WGW_CK(cudaMemcpyAsync(dvrb + (size_t)n_real * ldr, dvrb + (size_t)(n_pert + p) * ldr,
                               sizeof(double) * ldr, cudaMemcpyDeviceToDevice, st));
      brow[p] = n_real++;
    }
  }
  WGW_TRY(c->brow.ensure(sizeof(int) * n_pert));
  WGW_CK(cudaMemcpyAsync(c->brow.p, brow.data(), sizeof(int) * n_pert, cudaMemcpyHostToDevice, st));
  if (stats) *stats = wgw_stats{};
  int solve_status = WGW_OK;
  if (!k_zero.empty()) {
    solve_status = chi0_rb(c, dvrb, n_real, st, stats);
    if (solve_status != WGW_OK && solve_status != WGW_ERR_NOCONV) return solve_status;
  }
  // 7. Complex output drho_p = chi0 A_p + i chi0 B_p for every frequency.
  for (int k : k_zero)
    WGW_CK(c->prof.run(PK_CONV, 16.0 * n_pert * rs.n + 8.0 * n_pert * rs.nrb(), 0, st, [&] {
      return launch_rb_to_sphere(n_pert, c->drho_rb.as<double>(), ldr, c->brow.as<int>(), scale, rs.map(),
                                 drho + (size_t)k * n_pert * 2 * rs.n, 2L * rs.n, st); }));
  if (!k_pos.empty()) {
    const int s2 = chi0_rb_shifted(c, dvrb, n_real, w_pos, st, stats);
    if (s2 != WGW_OK && s2 != WGW_ERR_NOCONV) return s2;
    if (s2 == WGW_ERR_NOCONV) solve_status = s2;
    for (size_t j = 0; j < k_pos.size(); ++j)
      WGW_CK(c->prof.run(PK_CONV, 16.0 * n_pert * rs.n + 8.0 * n_pert * rs.nrb(), 0, st, [&] {
        return launch_rb_to_sphere(n_pert, c->drho_all.as<double>() + j * n_real * ldr, ldr, c->brow.as<int>(),
                                   scale, rs.map(), drho + (size_t)k_pos[j] * n_pert * 2 * rs.n, 2L * rs.n, st); }));
  }
  WGW_CK(cudaStreamSynchronize(st));
  c->prof.flush();
  return solve_status;
}


// ---------------------------------------------------------------- PDEP Davidson (Sec. 3, Sec. 4.2)
__global__ void k_scale_rows(int n, int nb, const double* __restrict__ in, long ldi, const double* __restrict__ sc,
                             double* __restrict__ out, long ldo) {
  for (int j = blockIdx.y; j < nb; j += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      out[(size_t)j * ldo + i] = (sc ? sc[i] : 1.0) * in[(size_t)j * ldi + i];
}

// Start vectors when none are given: uniform numbers in (-1, 1) from a counter-based
// hash (splitmix64 of seed and element index), weighted by v^1/2 so that the block
// leans towards long wavelengths.
__global__ void k_start_block(int n, int nb, unsigned long long seed, const double* __restrict__ vs,
                              double* __restrict__ out, long ld) {
  for (int j = blockIdx.y; j < nb; j += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      unsigned long long z = seed + 0x9E3779B97F4A7C15ull * ((unsigned long long)j * n + i + 1);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
      out[(size_t)j * ld + i] = (2.0 * u - 1.0) * vs[i];
    }
}

struct Davidson {
  wgw_ctx* c;
  std::vector<wgw_ctx*> chans;   // further spin channels (chibar0 is the sum over c and these)
  cudaStream_t st;
  int nr;           // real-basis length of the density sphere
  long ld;
  DevBuf vs_rb, gwork, Cbuf, Gbuf, Ubuf, sbuf, syw, info, cols, scl, Ysel;
  Prof* pf = nullptr;   // the context's profiler, or an idle one off the context's thread

  int gemm_tn(const double* A, int m, const double* B, int n, double* C) {
    WGW_TRY(gwork.ensure(sizeof(double) * gemm_tn_work_elems(nr, m, n)));
    WGW_CK(pf->run(PK_OTHER, 8.0 * (double)nr * (m + n), 2.0 * nr * m * n, st, [&] {
      return launch_gemm_tn(A, ld, B, ld, nr, m, n, C, gwork.as<double>(), st); }));
    return WGW_OK;
  }
  int gemm_nn(const double* A, int k, const double* C, int ldc, int ncols, double* Y, double alpha, double beta) {
    WGW_CK(pf->run(PK_OTHER, 8.0 * (double)nr * (k + 2 * ncols), 2.0 * nr * k * ncols, st, [&] {
      return launch_gemm_nn(A, ld, nr, k, C, ldc, ncols, Y, ld, alpha, beta, st); }));
    return WGW_OK;
  }
  int syev(int n, double* A, double* w, double* Z) {
    WGW_TRY(syw.ensure(sizeof(double) * syev_work_elems(n)));
    WGW_TRY(info.ensure(sizeof(int)));
    WGW_CK(pf->run(PK_OTHER, 16.0 * n * n, 3.0 * n * n * n, st, [&] {
      return launch_syev(n, A, n, w, Z, n, syw.as<double>(), info.as<int>(), st); }));
    int h = 0;
    WGW_CK(cudaMemcpyAsync(&h, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    if (h != 0) return fail(WGW_ERR_NOCONV, "dense eigensolver did not converge");
    return WGW_OK;
  }
  // B <- B - V (V^T B), twice.
  int orth_against(double* B, int nb, const double* V, int size) {
    if (size == 0 || nb == 0) return WGW_OK;
    const int mp = (size + 63) / 64 * 64;
    WGW_TRY(Cbuf.ensure(sizeof(double) * (size_t)mp * nb));
    for (int pass = 0; pass < 2; ++pass) {
      WGW_TRY(gemm_tn(V, size, B, nb, Cbuf.as<double>()));
      WGW_TRY(gemm_nn(V, size, Cbuf.as<double>(), nb, nb, B, -1.0, 1.0));
    }
    return WGW_OK;
  }
  // dest <- B U_keep diag(s_keep^-1/2) from the Gram matrix B^T B = U diag(s) U^T, dropping
  // directions with s below 1e-12 s_max.  dest must not alias B.  Returns the kept count.
  int orthonormalize(const double* B, int nb, double* dest, int* kept) {
    *kept = 0;
    if (nb == 0) return WGW_OK;
    const int mp = (nb + 63) / 64 * 64;
    WGW_TRY(Gbuf.ensure(sizeof(double) * (size_t)mp * nb));
    WGW_TRY(Ubuf.ensure(sizeof(double) * (size_t)nb * nb));
    WGW_TRY(sbuf.ensure(sizeof(double) * nb));
    WGW_TRY(gemm_tn(B, nb, B, nb, Gbuf.as<double>()));
    WGW_CK(launch_symmetrise(nb, Gbuf.as<double>(), nb, st));
    WGW_TRY(syev(nb, Gbuf.as<double>(), sbuf.as<double>(), Ubuf.as<double>()));
    std::vector<double> sv(nb);
    WGW_CK(cudaMemcpyAsync(sv.data(), sbuf.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    const double smax = sv[nb - 1];
    std::vector<int> keep;
    std::vector<double> sc;
    for (int i = nb - 1; i >= 0; --i)
      if (smax > 0 && sv[i] > 1e-12 * smax) { keep.push_back(i); sc.push_back(1.0 / std::sqrt(sv[i])); }
    const int nk = (int)keep.size();
    if (nk == 0) return WGW_OK;
    WGW_TRY(cols.ensure(sizeof(int) * nk));
    WGW_TRY(scl.ensure(sizeof(double) * nk));
    WGW_TRY(Ysel.ensure(sizeof(double) * (size_t)nb * nk));
    WGW_CK(cudaMemcpyAsync(cols.p, keep.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(scl.p, sc.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, st));
    WGW_CK(launch_select_scale(nb, Ubuf.as<double>(), nb, cols.as<int>(), scl.as<double>(), nk, Ysel.as<double>(), nk, st));
    WGW_TRY(gemm_nn(B, nb, Ysel.as<double>(), nk, nk, dest, 1.0, 0.0));
    *kept = nk;
    return WGW_OK;
  }
  // out = chibar0 in for nb vectors (real basis): v^1/2 chi0 v^1/2.
  // Block application supplied from outside (the served Davidson routes it through the request
  // queue); null = the context's own batched solve below.
  std::function<int(const double* in, int nb, double* out, wgw_stats* acc)> ext;

  int chibar0(const double* in, int nb, double* out, wgw_stats* acc) {
    if (ext) return ext(in, nb, out, acc);
    WGW_TRY(c->dv_rb.ensure(sizeof(double) * (size_t)nb * ld));
    double* dv = c->dv_rb.as<double>();
    dim3 g(std::max(1, std::min(64, (nr + 255) / 256)), std::min(nb, 65535));
    k_scale_rows<<<g, 256, 0, st>>>(nr, nb, in, ld, vs_rb.as<double>(), dv, ld);
    WGW_CK(cudaGetLastError());
    wgw_stats s1{};
    if (!chans.empty()) WGW_CK(cudaStreamSynchronize(st));   // dv is read on the channels' streams
    // The further channels run on their own contexts and streams from their own host threads,
    // concurrently with the first.
    const size_t nch = chans.size();
    std::vector<int> rcs(nch, WGW_OK);
    std::vector<wgw_stats> ss(nch);
    std::vector<std::string> errs(nch);
    std::vector<std::thread> th;
    for (size_t k = 0; k < nch; ++k)
      th.emplace_back([&, k] {
        wgw_ctx* ck = chans[k];
        if (cudaSetDevice(ck->device) != cudaSuccess) { rcs[k] = WGW_ERR_CUDA; errs[k] = "cudaSetDevice"; return; }
        std::lock_guard<std::recursive_mutex> lk(ck->mu);
        set_ff(ck);
        rcs[k] = chi0_rb(ck, dv, nb, ck->stream, &ss[k]);
        if ((rcs[k] == WGW_OK || rcs[k] == WGW_ERR_NOCONV) && cudaStreamSynchronize(ck->stream) != cudaSuccess)
          rcs[k] = WGW_ERR_CUDA;
        errs[k] = g_last_error;
      });
    const int rc = chi0_rb(c, dv, nb, st, &s1);
    for (std::thread& t : th) t.join();
    if (rc != WGW_OK && rc != WGW_ERR_NOCONV) return rc;
    for (size_t k = 0; k < nch; ++k) {
      if (rcs[k] != WGW_OK && rcs[k] != WGW_ERR_NOCONV) return fail(rcs[k], errs[k].c_str());
      WGW_CK(launch_axpby(nb, nr, 1.0, c->drho_rb.as<double>(), 1.0, chans[k]->drho_rb.as<double>(),
                          c->drho_rb.as<double>(), ld, nullptr, st));
      s1.n_systems += ss[k].n_systems;
      s1.max_rel_residual = std::max(s1.max_rel_residual, ss[k].max_rel_residual);
    }
    k_scale_rows<<<g, 256, 0, st>>>(nr, nb, c->drho_rb.as<double>(), ld, vs_rb.as<double>(), out, ld);
    WGW_CK(cudaGetLastError());
    acc->n_systems += s1.n_systems;
    acc->max_rel_residual = std::max(acc->max_rel_residual, s1.max_rel_residual);
    return WGW_OK;
  }
};

int davidson_impl(wgw_ctx* c, int npd, const double* x0, double* eig, double* basis, wgw_stats* out_st,
                  const std::vector<wgw_ctx*>& chans = {},
                  std::function<int(const double*, int, double*, wgw_stats*)> ext = nullptr,
                  cudaStream_t own_stream = nullptr) {
  Davidson D;
  D.c = c;
  D.chans = chans;
  D.ext = ext;
  Prof idle;
  D.pf = ext ? &idle : &c->prof;
  if (!ext) set_ff(c);
  D.st = own_stream ? own_stream : c->stream;
  D.nr = c->rho.nrb();
  D.ld = c->ld_r;
  cudaStream_t st = D.st;
  const long ld = D.ld;
  const int nr = D.nr;
  const int kmax = c->opt.dav_factor * npd;
  if (kmax > 2048) return fail(WGW_ERR_ARG, "Davidson subspace above 2048 vectors");
  // v^1/2 per real-basis element of the density sphere (0 at G = 0).
  {
    std::vector<double> vs(nr, 0.0);
    for (int j = 1; j <= c->rho.n_pairs; ++j) vs[2 * j - 1] = vs[2 * j] = c->rho.vsqrt[c->rho.pos[j]];
    WGW_TRY(D.vs_rb.ensure(sizeof(double) * nr));
    WGW_CK(cudaMemcpy(D.vs_rb.p, vs.data(), sizeof(double) * nr, cudaMemcpyHostToDevice));
  }
  DevBuf V, Wb, X, AX, R, Tmp, T, Z, theta, rn;
  WGW_TRY(V.ensure(sizeof(double) * (size_t)kmax * ld));
  WGW_TRY(Wb.ensure(sizeof(double) * (size_t)kmax * ld));
  DevBuf* nbufs[] = {&X, &AX, &R, &Tmp};
  for (DevBuf* b : nbufs) WGW_TRY(b->ensure(sizeof(double) * (size_t)npd * ld));
  const int kpad = (kmax + 63) / 64 * 64;
  WGW_TRY(T.ensure(sizeof(double) * (size_t)kpad * kmax));
  WGW_TRY(Z.ensure(sizeof(double) * (size_t)kmax * kmax));
  WGW_TRY(theta.ensure(sizeof(double) * kmax));
  WGW_TRY(rn.ensure(sizeof(double) * npd));
  WGW_CK(cudaMemsetAsync(V.p, 0, V.bytes, st));
  WGW_CK(cudaMemsetAsync(R.p, 0, R.bytes, st));
  // Start block.
  if (x0) {
    DevBuf xin;
    WGW_TRY(xin.ensure(sizeof(double) * 2 * (size_t)c->rho.n * npd));
    WGW_CK(cudaMemcpy(xin.p, x0, sizeof(double) * 2 * (size_t)c->rho.n * npd, cudaMemcpyHostToDevice));
    WGW_CK(launch_sphere_to_rb(npd, xin.as<double>(), 2L * c->rho.n, nullptr, c->rho.map(), 0, R.as<double>(), ld, st));
    WGW_CK(cudaStreamSynchronize(st));
  } else {
    dim3 g(std::max(1, std::min(64, (nr + 255) / 256)), std::min(npd, 65535));
    k_start_block<<<g, 256, 0, st>>>(nr, npd, (unsigned long long)c->opt.seed, D.vs_rb.as<double>(), R.as<double>(), ld);
    WGW_CK(cudaGetLastError());
  }
  wgw_stats acc{};
  int size = 0, nb = 0, kept = 0;
  WGW_TRY(D.orthonormalize(R.as<double>(), npd, Tmp.as<double>(), &kept));
  WGW_TRY(D.orthonormalize(Tmp.as<double>(), kept, V.as<double>(), &nb));
  if (nb < npd) return fail(WGW_ERR_ARG, "start block has rank below n_pdep");
  std::vector<double> th_prev, th(kmax), rnh(npd);
  int it = 0, converged = 0;
  double max_res = 0.0;
  for (it = 1; it <= c->opt.dav_max_iter && nb > 0; ++it) {
    WGW_TRY(D.chibar0(V.as<double>() + (size_t)size * ld, nb, Wb.as<double>() + (size_t)size * ld, &acc));
    acc.refinements += 1;
    size += nb;
    // Rayleigh-Ritz: T = V^T W, T = Z diag(theta) Z^T.
    WGW_TRY(D.gemm_tn(V.as<double>(), size, Wb.as<double>(), size, T.as<double>()));
    WGW_CK(launch_symmetrise(size, T.as<double>(), size, st));
    WGW_TRY(D.syev(size, T.as<double>(), theta.as<double>(), Z.as<double>()));
    // Ritz vectors and residuals of the npd lowest.
    std::vector<int> first(npd);
    for (int j = 0; j < npd; ++j) first[j] = j;
    WGW_TRY(D.cols.ensure(sizeof(int) * npd));
    WGW_TRY(D.Ysel.ensure(sizeof(double) * (size_t)size * npd));
    WGW_CK(cudaMemcpyAsync(D.cols.p, first.data(), sizeof(int) * npd, cudaMemcpyHostToDevice, st));
    WGW_CK(launch_select_scale(size, Z.as<double>(), size, D.cols.as<int>(), nullptr, npd, D.Ysel.as<double>(), npd, st));
    WGW_TRY(D.gemm_nn(V.as<double>(), size, D.Ysel.as<double>(), npd, npd, X.as<double>(), 1.0, 0.0));
    WGW_TRY(D.gemm_nn(Wb.as<double>(), size, D.Ysel.as<double>(), npd, npd, AX.as<double>(), 1.0, 0.0));
    WGW_CK(launch_ritz_residual(nr, npd, X.as<double>(), AX.as<double>(), ld, theta.as<double>(), R.as<double>(),
                                rn.as<double>(), st));
    WGW_CK(cudaMemcpyAsync(th.data(), theta.p, sizeof(double) * npd, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaMemcpyAsync(rnh.data(), rn.p, sizeof(double) * npd, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    const double tol = c->opt.dav_tol, rtol = std::sqrt(tol);
    double dth = 1e300;
    if (!th_prev.empty()) {
      dth = 0.0;
      for (int j = 0; j < npd; ++j) dth = std::max(dth, std::fabs(th[j] - th_prev[j]));
    }
    th_prev.assign(th.begin(), th.begin() + npd);
    max_res = 0.0;
    converged = 0;
    std::vector<int> sel;
    for (int j = 0; j < npd; ++j) {
      max_res = std::max(max_res, rnh[j]);
      if (rnh[j] <= rtol) ++converged;
      else sel.push_back(j);
    }
    if (dth <= tol && converged == npd) break;
    if (sel.empty()) { sel.resize(npd); for (int j = 0; j < npd; ++j) sel[j] = j; }
    // Gather the residuals to expand with into Tmp.
    for (size_t q = 0; q < sel.size(); ++q)
      WGW_CK(cudaMemcpyAsync(Tmp.as<double>() + q * ld, R.as<double>() + (size_t)sel[q] * ld, sizeof(double) * ld,
                             cudaMemcpyDeviceToDevice, st));
    const int nsel = (int)sel.size();
    if (size + nsel > kmax) {
      // Restart from the Ritz vectors and their images.
      WGW_CK(cudaMemcpyAsync(V.p, X.p, sizeof(double) * (size_t)npd * ld, cudaMemcpyDeviceToDevice, st));
      WGW_CK(cudaMemcpyAsync(Wb.p, AX.p, sizeof(double) * (size_t)npd * ld, cudaMemcpyDeviceToDevice, st));
      size = npd;
    }
    WGW_TRY(D.orth_against(Tmp.as<double>(), nsel, V.as<double>(), size));
    WGW_TRY(D.orthonormalize(Tmp.as<double>(), nsel, R.as<double>(), &kept));
    WGW_TRY(D.orth_against(R.as<double>(), kept, V.as<double>(), size));
    WGW_TRY(D.orthonormalize(R.as<double>(), kept, V.as<double>() + (size_t)size * ld, &nb));
  }
  if (eig) std::copy(th.begin(), th.begin() + npd, eig);
  if (basis) {
    DevBuf bout;
    WGW_TRY(bout.ensure(sizeof(double) * 2 * (size_t)c->rho.n * npd));
    WGW_CK(launch_rb_to_sphere(npd, X.as<double>(), ld, nullptr, nullptr, c->rho.map(), bout.as<double>(),
                               2L * c->rho.n, st));
    WGW_CK(cudaMemcpyAsync(basis, bout.p, sizeof(double) * 2 * (size_t)c->rho.n * npd, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
  }
  if (!ext) c->prof.flush();
  if (out_st) {
    out_st->n_systems = acc.n_systems;
    out_st->n_converged = converged;
    out_st->max_iters = std::min(it, c->opt.dav_max_iter);
    out_st->refinements = acc.refinements;
    out_st->max_rel_residual = max_res;
  }
  return converged == npd ? WGW_OK : fail(WGW_ERR_NOCONV, "Davidson did not converge");
}

// ---------------------------------------------------------------- Lanczos chains (Sec. 3)
// Chains on P_c H P_c for every (state v, basis vector m), started from P_c [phi~_m psi_v]
// (phi~ = v^1/2 phi), FP64 throughout; chi0_nm(i w) from the chains' tridiagonal spectra.
// G0 mode of the Lanczos chains (Eq. ISR): chains of h itself from [phi~_m psi_i], i over a list
// of occupied states, with the frequency-independent residues and the resolvent matrices at
// complex frequencies as outputs.
struct LzG0 {
  const int* states;
  int n_states;
  const double* z;   // n_z complex, interleaved
  int n_z;
  double* d;         // host outputs, or null
  double* C;
  double* g0;
  // Eq. ISR by quadrature (optional): z holds w_j +- i w'_k in the order (j, k, +/-).
  const double* lam = nullptr;      // host, n_nodes x n_pdep x n_pdep
  const double* weights = nullptr;  // host, n_nodes
  int n_omega = 0, n_nodes = 0;
  double* isr = nullptr;            // host output, n_states x n_omega complex
};

// Spectral data of a set of chains kept on the device for later evaluation at any frequency:
// the residues W[v][n][l'][m] = beta_1 U_{1 l'} sum_l <b_(n,v)|q^l_(m,v)> U_{l l'} and the Ritz
// values d of chain s = m n_v + v (v over the occupied states for the chi0 chains, over the
// listed states for the G0 chains); for the G0 chains also the overlaps
// Y[i][j][m] = <psi_j | psi_(states i) phi~_m> with every occupied j (rows of length n_pdep,
// ys doubles per listed state).
struct LzKeep {
  DevBuf W, d, Y;
  long ys = 0;
};

// Lanczos chains of every (state, basis vector) pair.  Without g0: chains of P_c H P_c from
// P_c [phi~_m psi_v], every occupied v, and chi0 in the basis.  With g0: chains of H.
int lanczos_impl(wgw_ctx* c, const double* phi, int npd, int n_steps, const double* omega, int n_om,
                 double* alpha_out, double* beta_out, double* chi_out, wgw_stats* st_out,
                 const LzG0* g0 = nullptr, LzKeep* keep = nullptr) {
  cudaStream_t st = c->stream;
  // FP64-accurate chains: float-float FFT passes on the mixed path (compiled grids), native FP64
  // otherwise.
  set_ff(c);
  const bool proj = g0 == nullptr;
  const int N = c->N, n_v = proj ? c->n_v : g0->n_states, n = c->wfc.nrb(), nr = c->rho.nrb();
  const long ldw = c->ld_w, ldr = c->ld_r;
  const int n_ch = npd * n_v;
  // Perturbations phi~_m = v^1/2 phi_m (real-in-r part), to real space.
  WGW_TRY(c->dv_rb.ensure(sizeof(double) * (size_t)npd * ldr));
  {
    DevBuf xin;
    WGW_TRY(xin.ensure(sizeof(double) * 2 * (size_t)c->rho.n * npd));
    WGW_CK(cudaMemcpy(xin.p, phi, sizeof(double) * 2 * (size_t)c->rho.n * npd, cudaMemcpyHostToDevice));
    WGW_CK(cudaMemsetAsync(c->dv_rb.p, 0, sizeof(double) * (size_t)npd * ldr, st));
    WGW_CK(launch_sphere_to_rb(npd, xin.as<double>(), 2L * c->rho.n, c->rho.d_vsqrt.as<double>(), c->rho.map(), 0,
                               c->dv_rb.as<double>(), ldr, st));
    WGW_CK(cudaStreamSynchronize(st));
  }
  WGW_TRY(ensure_work(c, n_ch, npd));
  std::vector<int> ai(n_ch), bi(n_ch);
  for (int m = 0; m < npd; ++m)
    for (int v = 0; v < n_v; ++v) { ai[m * n_v + v] = proj ? v : g0->states[v]; bi[m * n_v + v] = m; }
  WGW_CK(cudaMemcpyAsync(c->a_idx.p, ai.data(), sizeof(int) * n_ch, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemcpyAsync(c->b_idx.p, bi.data(), sizeof(int) * n_ch, cudaMemcpyHostToDevice, st));
  WGW_CK(cudaMemsetAsync(c->d.shift.p, 0, sizeof(double) * n_ch, st));   // A = (P_c) H (P_c)
  double* dvr = c->dv_r.as<double>();
  WGW_TRY(to_real<double>(c, c->d, c->rho, c->dv_rb.as<double>(), ldr, npd, dvr, c->Trho, st));
  FftCtx<double> f = c->d.fft(c->plan);
  double* S = c->d.Bv.as<double>();
  {
    const int NP = 2 * c->wfc.m + 1, pairs = (n_ch + 1) / 2;
    WGW_TRY(c->d.Tw.ensure(sizeof(cplx<double>) * (size_t)pairs * NP * N * N));
    XArgs<double> a{};
    a.mode = XM_FROM_REAL; a.A = c->d.psi_r_fft(); a.lda = c->grid3; a.a_index = c->a_idx.as<int>();
    a.Bm = dvr; a.ldb = c->grid3; a.b_index = c->b_idx.as<int>(); a.n_sys = n_ch;
    WGW_CK(launch_xline<double>(c->wfc.m, f, c->d.Tw.as<cplx<double>>(), a, nullptr, st));
    Epi<double> e{};
    e.out = S; e.ldo = ldw; e.vcoef = 1.0; e.n_sys = n_ch;
    WGW_CK(launch_plane_r2g<double>(c->wfc.tab(), c->wfc.npt_max, f, c->d.Tw.as<cplx<double>>(), e, st));
    if (proj) WGW_TRY(run_pc<double>(c, S, n_ch, nullptr, c->d.psi.as<double>(), nullptr, st));
  }
  // The chain vectors (and their float-float copy) stay with the context between calls.
  DevBuf& Qb = c->lz_q;
  DevBuf al, be, T, dd, U, wk, inf, ov, y, om, lists;
  WGW_TRY(Qb.ensure(sizeof(double) * (size_t)(n_steps + 1) * n_ch * ldw));
  WGW_TRY(al.ensure(sizeof(double) * (size_t)n_ch * n_steps));
  WGW_TRY(be.ensure(sizeof(double) * (size_t)n_ch * n_steps));
  WGW_CK(cudaMemsetAsync(al.p, 0, al.bytes, st));
  WGW_CK(cudaMemsetAsync(be.p, 0, be.bytes, st));
  double* Q = Qb.as<double>();
  double* HQ = c->d.Q.as<double>();
  double* R = c->d.R.as<double>();
  // Each step: r = Hq^l - sum_j c_j q^j with c_j = q^j . Hq^l over all previous vectors (the
  // three-term step, alpha_l = c_l, and the first Gram-Schmidt pass at once: with orthonormal q
  // the coefficients of q^l and q^(l-1) are alpha_l and beta_l), then a second classical
  // Gram-Schmidt pass (each pass followed by P_c on the projected chains), then beta_(l+1) = |r|.
  // Every pass is split over chunks of the n reals so that a few hundred chains fill the GPU; on
  // the float-float path the passes read a float-float copy of the chain vectors and compute on
  // the FP32 units.  The recurrence kernels are timed as other_f64; algorithmic bytes are the
  // vectors each reads and writes once.
  ProfPrec pp(c->prof, true);
  const double vb = (double)n_ch * n * sizeof(double);
  const int nb = lz_split(n, n_ch);
  DevBuf part, npart;
  DevBuf& Qfb = c->lz_qf;
  WGW_TRY(part.ensure(sizeof(double) * (size_t)n_ch * nb * n_steps));
  WGW_TRY(npart.ensure(sizeof(double) * (size_t)n_ch * nb));
  double* Qf = nullptr;
  if (c->d.use_ff) {
    WGW_TRY(Qfb.ensure(sizeof(double) * (size_t)(n_steps + 1) * n_ch * ldw));
    Qf = Qfb.as<double>();
  }
  double* pt = part.as<double>();
  WGW_CK(launch_lz_start(n, n_ch, S, Q, ldw, be.as<double>(), n_steps, st));
  if (Qf) WGW_CK(launch_to_ff((size_t)n_ch * ldw, Q, Qf, st));
  for (int l = 0; l < n_steps; ++l) {
    double* ql = Q + (size_t)l * n_ch * ldw;
    WGW_TRY(apply_A<double>(c, c->d, ql, HQ, n_ch, nullptr, nullptr, st, proj));
    const bool last = l + 1 == n_steps;
    for (int pass = 0; pass < 2; ++pass) {
      const double* X = pass == 0 ? HQ : R;
      WGW_CK(c->prof.run(PK_OTHER, (l + 2) * vb, 2.0 * (l + 1) * n * n_ch, st, [&] {
        return launch_lz_gs_dots(n, l, n_ch, Q, Qf, ldw, X, pt, nb, st); }));
      WGW_CK(c->prof.run(PK_OTHER, last ? 0.0 : (l + 3) * vb, last ? 0.0 : 2.0 * (l + 1) * n * n_ch, st, [&] {
        return launch_lz_gs_update(n, l, n_ch, Q, Qf, ldw, X, R, pt, pass == 0 ? al.as<double>() : nullptr,
                                   n_steps, last, (!proj && pass == 1) ? npart.as<double>() : nullptr, nb, st); }));
      if (last) break;
      if (proj) WGW_TRY(run_pc<double>(c, R, n_ch, nullptr, c->d.psi.as<double>(), nullptr, st));
    }
    if (last) break;
    // After P_c the partial norms of the update are stale: the projected chains reduce |r|
    // inside one block per chain.
    WGW_CK(c->prof.run(PK_OTHER, (Qf ? 3 : 2) * vb, 0, st, [&] {
      return launch_lz_normalise(n, l, n_ch, R, Q, Qf, ldw, be.as<double>(), n_steps,
                                 proj ? nullptr : npart.as<double>(), nb, st); }));
  }
  // Overlaps <(P_c) phi~_n psi_v | q^l_(m,v)>, one product per state v.
  const int mp = (npd + 63) / 64 * 64;
  const size_t ovs = (size_t)mp * n_steps * npd;
  WGW_TRY(ov.ensure(sizeof(double) * ovs * n_v));
  WGW_TRY(lists.ensure(sizeof(int) * (size_t)n_steps * npd));
  DevBuf gw;
  WGW_TRY(gw.ensure(sizeof(double) * gemm_tn_work_elems(n, npd, n_steps * npd)));
  std::vector<int> cols((size_t)n_steps * npd);
  for (int v = 0; v < n_v; ++v) {
    for (int l = 0; l < n_steps; ++l)
      for (int m = 0; m < npd; ++m) cols[(size_t)l * npd + m] = l * n_ch + m * n_v + v;
    WGW_CK(cudaMemcpyAsync(lists.p, cols.data(), sizeof(int) * cols.size(), cudaMemcpyHostToDevice, st));
    WGW_CK(launch_gemm_tn(S + (size_t)v * ldw, (long)n_v * ldw, Q, ldw, n, npd, n_steps * npd,
                          ov.as<double>() + (size_t)v * ovs, gw.as<double>(), st, lists.as<int>(), Qf != nullptr));
    WGW_CK(cudaStreamSynchronize(st));   // cols is reused for the next state
  }
  if (keep && !proj) {
    // Overlaps of every occupied state with the chain starts b_(m,i) = psi_i phi~_m (unnormalised).
    const int nv_all = c->n_v;
    keep->ys = (long)((nv_all + 63) / 64 * 64) * npd;
    WGW_TRY(keep->Y.ensure(sizeof(double) * (size_t)keep->ys * n_v));
    WGW_TRY(gw.ensure(sizeof(double) * gemm_tn_work_elems(n, nv_all, npd)));
    for (int v = 0; v < n_v; ++v) {
      for (int m = 0; m < npd; ++m) cols[m] = m * n_v + v;
      WGW_CK(cudaMemcpyAsync(lists.p, cols.data(), sizeof(int) * npd, cudaMemcpyHostToDevice, st));
      WGW_CK(launch_gemm_tn(c->d.psi.as<double>(), ldw, S, ldw, n, nv_all, npd,
                            keep->Y.as<double>() + (size_t)v * keep->ys, gw.as<double>(), st, lists.as<int>(),
                            c->d.use_ff));
      WGW_CK(cudaStreamSynchronize(st));
    }
  }
  // Tridiagonal spectra d, U of every chain.
  WGW_TRY(T.ensure(sizeof(double) * (size_t)n_ch * n_steps * n_steps));
  WGW_TRY(U.ensure(sizeof(double) * (size_t)n_ch * n_steps * n_steps));
  WGW_TRY(dd.ensure(sizeof(double) * (size_t)n_ch * n_steps));
  WGW_TRY(wk.ensure(sizeof(double) * (size_t)n_ch * syev_work_elems(n_steps)));
  WGW_TRY(inf.ensure(sizeof(int) * n_ch));
  WGW_CK(launch_lz_tridiag(n_ch, n_steps, al.as<double>(), be.as<double>(), T.as<double>(), st));
  WGW_CK(launch_syev_batched(n_steps, n_ch, T.as<double>(), dd.as<double>(), U.as<double>(), wk.as<double>(),
                             inf.as<int>(), st, true));
  std::vector<int> infh(n_ch);
  WGW_CK(cudaMemcpyAsync(infh.data(), inf.p, sizeof(int) * n_ch, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  for (int q = 0; q < n_ch; ++q)
    if (infh[q] != 0) return fail(WGW_ERR_NOCONV, "tridiagonal eigensolver did not converge");
  if (keep) {
    const size_t nW = (size_t)n_v * npd * n_steps * npd;
    WGW_TRY(keep->W.ensure(sizeof(double) * nW));
    WGW_TRY(keep->d.ensure(sizeof(double) * (size_t)n_ch * n_steps));
    WGW_CK(launch_lz_residues(npd, n_v, n_steps, ov.as<double>(), U.as<double>(), be.as<double>(),
                              keep->W.as<double>(), st));
    WGW_CK(cudaMemcpyAsync(keep->d.p, dd.p, sizeof(double) * (size_t)n_ch * n_steps, cudaMemcpyDeviceToDevice, st));
    WGW_CK(cudaStreamSynchronize(st));
  }
  if (!proj) {
    // Residues C[i][n][l'][m] = beta_1 U_{1 l'} sum_l <b_n|q^l_m> U_{l l'}, then the resolvent
    // matrices g0[i][k][n][m] = sum_l' C[i][n][l'][m] / (d_l' - z_k).
    DevBuf Cd, zd, gd;
    const size_t nC = (size_t)n_v * npd * n_steps * npd;
    WGW_TRY(Cd.ensure(sizeof(double) * nC));
    WGW_CK(launch_lz_residues(npd, n_v, n_steps, ov.as<double>(), U.as<double>(), be.as<double>(), Cd.as<double>(),
                              st));
    if (g0->C) WGW_CK(cudaMemcpyAsync(g0->C, Cd.p, sizeof(double) * nC, cudaMemcpyDeviceToHost, st));
    if ((g0->g0 || g0->isr) && g0->n_z > 0) {
      const size_t ng = (size_t)n_v * g0->n_z * npd * npd;
      WGW_TRY(zd.ensure(sizeof(double) * 2 * g0->n_z));
      WGW_TRY(gd.ensure(sizeof(double) * 2 * ng));
      WGW_CK(cudaMemcpyAsync(zd.p, g0->z, sizeof(double) * 2 * g0->n_z, cudaMemcpyHostToDevice, st));
      WGW_CK(launch_lz_g0_eval(npd, n_v, n_steps, g0->n_z, Cd.as<double>(), dd.as<double>(), zd.as<double>(),
                               gd.as<double>(), st));
      if (g0->g0) WGW_CK(cudaMemcpyAsync(g0->g0, gd.p, sizeof(double) * 2 * ng, cudaMemcpyDeviceToHost, st));
      if (g0->isr) {
        DevBuf lamd, wd, od;
        const size_t nl = (size_t)g0->n_nodes * npd * npd;
        WGW_TRY(lamd.ensure(sizeof(double) * nl));
        WGW_TRY(wd.ensure(sizeof(double) * g0->n_nodes));
        WGW_TRY(od.ensure(sizeof(double) * 2 * (size_t)n_v * g0->n_omega));
        WGW_CK(cudaMemcpyAsync(lamd.p, g0->lam, sizeof(double) * nl, cudaMemcpyHostToDevice, st));
        WGW_CK(cudaMemcpyAsync(wd.p, g0->weights, sizeof(double) * g0->n_nodes, cudaMemcpyHostToDevice, st));
        WGW_CK(launch_lz_isr(npd, n_v, g0->n_omega, g0->n_nodes, gd.as<double>(), lamd.as<double>(),
                             wd.as<double>(), 1.0 / c->omega_cell, od.as<double>(), st));
        WGW_CK(cudaMemcpyAsync(g0->isr, od.p, sizeof(double) * 2 * (size_t)n_v * g0->n_omega,
                               cudaMemcpyDeviceToHost, st));
        WGW_CK(cudaStreamSynchronize(st));   // lamd, wd, od leave scope
      }
    }
    if (g0->d) {
      std::vector<double> dh((size_t)n_ch * n_steps);
      WGW_CK(cudaMemcpyAsync(dh.data(), dd.p, sizeof(double) * dh.size(), cudaMemcpyDeviceToHost, st));
      WGW_CK(cudaStreamSynchronize(st));
      for (int v = 0; v < n_v; ++v)
        for (int m = 0; m < npd; ++m)
          for (int l = 0; l < n_steps; ++l)
            g0->d[((size_t)v * npd + m) * n_steps + l] = dh[((size_t)m * n_v + v) * n_steps + l];
    }
    WGW_CK(cudaStreamSynchronize(st));
  }
  if (proj && chi_out && n_om > 0) {
    WGW_TRY(om.ensure(sizeof(double) * n_om));
    WGW_CK(cudaMemcpyAsync(om.p, omega, sizeof(double) * n_om, cudaMemcpyHostToDevice, st));
    WGW_TRY(y.ensure(sizeof(double) * (size_t)n_om * n_ch * n_steps));
    WGW_CK(launch_lz_resolvent(n_ch, n_steps, n_v, n_om, dd.as<double>(), U.as<double>(), be.as<double>(),
                               c->e_v_d.as<double>(), om.as<double>(), y.as<double>(), st));
    DevBuf chi;
    WGW_TRY(chi.ensure(sizeof(double) * (size_t)n_om * npd * npd));
    WGW_CK(launch_lz_assemble(npd, n_v, n_steps, n_om, ov.as<double>(), y.as<double>(), c->opt.f_s / c->omega_cell,
                              chi.as<double>(), st));
    WGW_CK(cudaMemcpyAsync(chi_out, chi.p, sizeof(double) * (size_t)n_om * npd * npd, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
  }
  std::vector<double> ah((size_t)n_ch * n_steps), bh((size_t)n_ch * n_steps);
  WGW_CK(cudaMemcpyAsync(ah.data(), al.p, sizeof(double) * ah.size(), cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaMemcpyAsync(bh.data(), be.p, sizeof(double) * bh.size(), cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  for (int v = 0; v < n_v; ++v)
    for (int m = 0; m < npd; ++m)
      for (int l = 0; l < n_steps; ++l) {
        const size_t dst = ((size_t)v * npd + m) * n_steps + l, src = ((size_t)m * n_v + v) * n_steps + l;
        if (alpha_out) alpha_out[dst] = ah[src];
        if (beta_out) beta_out[dst] = bh[src];
      }
  c->prof.flush();
  if (st_out) {
    *st_out = wgw_stats{};
    st_out->n_systems = n_ch;
    st_out->n_converged = n_ch;
    st_out->max_iters = n_steps;
  }
  (void)nr;
  return WGW_OK;
}

// ---------------------------------------------------------------- continuous batching
// Served requests whose frequencies are all zero run through a slot engine.  Every Sternheimer
// system of an admitted request takes a slot (a row of the context's CG work arrays); the worker
// runs the FP32 inner CG of all slots together in windows of check_every iterations, and between
// two windows it (1) retires the systems whose inner solve ended: the FP32 correction is added,
// the FP64-accurate residual computed, and the system is done or starts its next refinement;
// (2) finishes the requests whose systems are all done (final P_c, drho, results to the host);
// (3) admits queued requests into the free slots (perturbations to real space, right-hand sides,
// inner CG set-up).  A request that arrives while others are on the GPU therefore joins at the
// next window, and its systems iterate in the same launches as theirs.  The arithmetic of a
// system is that of the batched solve (same kernels, refinement and stopping rule), so a request's
// result equals its result alone up to the rounding of the batched reductions.
struct EngReq {
  serve::Request rq;
  int n_real = 0;
  std::vector<int> brow;      // per perturbation: part row of its imaginary part, -1 if none
  int pbase = -1;             // first perturbation-pool row of its parts
  std::vector<int> slots;     // slot of system (r, v) at r n_v + v
  int n_done = 0, n_conv = 0, max_iters = 0, refinements = 0, peers = 1;
  double max_rel = 0.0;
  std::chrono::steady_clock::time_point t_admit;
};

struct Engine {
  enum { kFree = 0, kStart = 1, kInner = 2, kDone = 3 };
  wgw_ctx* c = nullptr;
  cudaStream_t st = nullptr;
  int cap = 0, pcap = 0;
  std::vector<int> phase, refine, iters, sys_r, sys_v;
  std::vector<uint64_t> owner;
  std::vector<int> free_slots;
  std::vector<char> pool_used;
  std::vector<int> a_idx, b_idx;
  std::vector<double> eps, shift;
  std::vector<float> shiftf;
  std::map<uint64_t, EngReq> live;

  int init(int n_cap, int n_pcap) {
    cap = n_cap;
    pcap = n_pcap;
    WGW_TRY(ensure_work(c, cap, 1));
    WGW_TRY(c->norms.ensure(sizeof(double) * cap));
    WGW_TRY(c->eng_mask.ensure(sizeof(int) * cap));
    WGW_TRY(c->eng_list.ensure(sizeof(int) * cap));
    WGW_TRY(c->eng_pool.ensure(sizeof(double) * (size_t)pcap * c->grid3));
    phase.assign(cap, kFree); refine.assign(cap, 0); iters.assign(cap, 0); sys_r.assign(cap, 0);
    sys_v.assign(cap, 0); owner.assign(cap, 0); a_idx.assign(cap, 0); b_idx.assign(cap, 0);
    eps.assign(cap, 0.0); shift.assign(cap, 0.0); shiftf.assign(cap, 0.f);
    free_slots.clear();
    for (int s = cap - 1; s >= 0; --s) free_slots.push_back(s);
    pool_used.assign(pcap, 0);
    WGW_CK(cudaMemsetAsync(c->d.X.p, 0, sizeof(double) * (size_t)cap * c->ld_w, st));
    WGW_CK(cudaMemsetAsync(c->cg_act.p, 0, sizeof(int) * cap, st));
    return WGW_OK;
  }
  int pool_alloc(int n) {
    for (int b = 0; b + n <= pcap; ++b) {
      bool ok = true;
      for (int k = 0; k < n && ok; ++k) ok = !pool_used[b + k];
      if (ok) {
        for (int k = 0; k < n; ++k) pool_used[b + k] = 1;
        return b;
      }
    }
    return -1;
  }
  // Uploads a host list and a matching mask over all slots; returns the device list.
  int upload_list(const std::vector<int>& l, int** dev_list, const int** dev_mask) {
    std::vector<int> mask(cap, 0);
    for (int s : l) mask[s] = 1;
    WGW_CK(cudaMemcpyAsync(c->eng_list.p, l.data(), sizeof(int) * l.size(), cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(c->eng_mask.p, mask.data(), sizeof(int) * cap, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaStreamSynchronize(st));   // the host vectors leave scope
    *dev_list = c->eng_list.as<int>();
    if (dev_mask) *dev_mask = c->eng_mask.as<int>();
    return WGW_OK;
  }
  int upload_tables() {
    WGW_CK(cudaMemcpyAsync(c->a_idx.p, a_idx.data(), sizeof(int) * cap, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(c->b_idx.p, b_idx.data(), sizeof(int) * cap, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(c->eps.p, eps.data(), sizeof(double) * cap, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(c->d.shift.p, shift.data(), sizeof(double) * cap, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(c->f.shift.p, shiftf.data(), sizeof(float) * cap, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaStreamSynchronize(st));
    return WGW_OK;
  }

  // Admits one request (slots and pool rows are available): perturbation parts, dV(r), the
  // right-hand sides of its systems, x = 0, r = b, |b|^2.
  int admit(serve::Request&& rq) {
    const int n_pert = rq.n_pert, n_v = c->n_v;
    const long ldr = c->ld_r;
    const HostSphere& rs = c->rho;
    const bool sym = rq.kind == WGW_REQ_CHIBAR0;
    const double* scale = sym ? rs.d_vsqrt.as<double>() : nullptr;
    WGW_TRY(c->eng_in.ensure(sizeof(double) * 2 * (size_t)rs.n * n_pert));
    WGW_CK(cudaMemcpyAsync(c->eng_in.p, rq.dV.data(), sizeof(double) * rq.dV.size(), cudaMemcpyHostToDevice, st));
    WGW_TRY(c->dv_rb.ensure(sizeof(double) * (size_t)2 * n_pert * ldr));
    double* dvrb = c->dv_rb.as<double>();
    WGW_CK(cudaMemsetAsync(dvrb, 0, sizeof(double) * (size_t)2 * n_pert * ldr, st));
    WGW_CK(launch_sphere_to_rb(n_pert, c->eng_in.as<double>(), 2L * rs.n, scale, rs.map(), 0, dvrb, ldr, st));
    WGW_CK(launch_sphere_to_rb(n_pert, c->eng_in.as<double>(), 2L * rs.n, scale, rs.map(), 1,
                               dvrb + (size_t)n_pert * ldr, ldr, st));
    WGW_TRY(c->rr64.ensure(sizeof(double) * std::max(cap, 2 * n_pert)));
    WGW_CK(launch_norm2<double>(2 * n_pert, rs.nrb(), dvrb, ldr, c->rr64.as<double>(), st));
    std::vector<double> nrm(2 * n_pert);
    WGW_CK(cudaMemcpyAsync(nrm.data(), c->rr64.p, sizeof(double) * 2 * n_pert, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    EngReq er;
    er.brow.assign(n_pert, -1);
    int n_real = n_pert;
    for (int p = 0; p < n_pert; ++p)
      if (nrm[n_pert + p] > 0.0) {
        if (n_real != n_pert + p)
          WGW_CK(cudaMemcpyAsync(dvrb + (size_t)n_real * ldr, dvrb + (size_t)(n_pert + p) * ldr, sizeof(double) * ldr,
                                 cudaMemcpyDeviceToDevice, st));
        er.brow[p] = n_real++;
      }
    er.n_real = n_real;
    er.pbase = pool_alloc(n_real);
    if (er.pbase < 0 || (int)free_slots.size() < n_real * n_v) return fail(WGW_ERR_STATE, "engine admission without room");
    double* pool = c->eng_pool.as<double>() + (size_t)er.pbase * c->grid3;
    WGW_TRY(to_real<double>(c, c->d, rs, dvrb, ldr, n_real, pool, c->Trho, st));
    std::vector<int> slots;
    for (int r = 0; r < n_real; ++r)
      for (int v = 0; v < n_v; ++v) {
        const int sl = free_slots.back();
        free_slots.pop_back();
        slots.push_back(sl);
        owner[sl] = rq.ticket; sys_r[sl] = r; sys_v[sl] = v; phase[sl] = kStart; refine[sl] = 0; iters[sl] = 0;
        a_idx[sl] = v; b_idx[sl] = er.pbase + r;
        eps[sl] = c->e_v[v]; shift[sl] = -c->e_v[v]; shiftf[sl] = (float)-c->e_v[v];
      }
    er.slots = slots;
    WGW_TRY(upload_tables());
    int* dl = nullptr;
    const int* dm = nullptr;
    WGW_TRY(upload_list(slots, &dl, &dm));
    // Right-hand sides b_s = -P_c [psi_v(r) dV_r(r)] of the new slots.
    const int n_new = (int)slots.size(), NP = 2 * c->wfc.m + 1, N = c->N, pairs = (n_new + 1) / 2;
    WGW_TRY(c->d.Tw.ensure(sizeof(cplx<double>) * (size_t)pairs * NP * N * N));
    FftCtx<double> f = c->d.fft(c->plan);
    XArgs<double> a{};
    a.mode = XM_FROM_REAL; a.A = c->d.psi_r_fft(); a.lda = c->grid3; a.a_index = c->a_idx.as<int>();
    a.Bm = c->eng_pool.as<double>(); a.ldb = c->grid3; a.b_index = c->b_idx.as<int>(); a.n_sys = n_new; a.list = dl;
    WGW_CK(launch_xline<double>(c->wfc.m, f, c->d.Tw.as<cplx<double>>(), a, nullptr, st));
    Epi<double> e{};
    e.out = c->d.Bv.as<double>(); e.ldo = c->ld_w; e.vcoef = -1.0; e.n_sys = n_new; e.list = dl;
    WGW_CK(launch_plane_r2g<double>(c->wfc.tab(), c->wfc.npt_max, f, c->d.Tw.as<cplx<double>>(), e, st));
    WGW_TRY(run_pc<double>(c, c->d.Bv.as<double>(), n_new, dl, c->d.psi.as<double>(), nullptr, st));
    const int n = c->wfc.nrb();
    const long ld = c->ld_w;
    WGW_CK(launch_axpby(cap, n, 0.0, c->d.Bv.as<double>(), 0.0, c->d.Bv.as<double>(), c->d.X.as<double>(), ld, dm, st));
    WGW_CK((launch_copy_cast<double, double>(cap, n, c->d.Bv.as<double>(), ld, c->d.R.as<double>(), ld, dm, st)));
    WGW_CK(launch_norm2<double>(cap, n, c->d.Bv.as<double>(), ld, c->norms.as<double>(), st));
    er.t_admit = std::chrono::steady_clock::now();
    er.rq = std::move(rq);
    er.peers = (int)live.size() + 1;
    for (auto& kv : live) kv.second.peers = std::max(kv.second.peers, (int)live.size() + 1);
    live.emplace(er.rq.ticket, std::move(er));
    c->eng_requests++;
    return WGW_OK;
  }

  // Starts the inner FP32 solves of the slots in phase kStart (right-hand side = FP64 residual).
  int start_inner() {
    std::vector<int> l;
    for (int s = 0; s < cap; ++s)
      if (phase[s] == kStart) l.push_back(s);
    if (l.empty()) return WGW_OK;
    int* dl = nullptr;
    const int* dm = nullptr;
    WGW_TRY(upload_list(l, &dl, &dm));
    const int n = c->wfc.nrb();
    const long ld = c->ld_w;
    CgState cs = cg_state(c, true);
    WGW_CK((launch_copy_cast<double, float>(cap, n, c->d.R.as<double>(), ld, c->f.Bv.as<float>(), ld, dm, st)));
    WGW_CK(launch_cg_init_a<float>(c->wfc.tab(), n, (int)l.size(), c->f.Bv.as<float>(), c->f.X.as<float>(),
                                   c->f.R.as<float>(), c->f.Z.as<float>(), ld, c->eps.as<double>(), cs, st, dl));
    WGW_TRY(run_pc<float>(c, c->f.Z.as<float>(), (int)l.size(), dl, c->f.psi.as<float>(), cs.active, st));
    WGW_CK(launch_cg_init_b<float>(n, (int)l.size(), c->f.R.as<float>(), c->f.Z.as<float>(), c->f.P.as<float>(), ld,
                                   cs, st, dl));
    for (int s : l) phase[s] = kInner;
    return WGW_OK;
  }

  // One window of check_every FP32 CG iterations over every slot in its inner solve; then the
  // systems whose inner solve ended are retired.
  int window() {
    std::vector<int> l;
    for (int s = 0; s < cap; ++s)
      if (phase[s] == kInner) l.push_back(s);
    if (l.empty()) return WGW_OK;
    int* dl = nullptr;
    WGW_TRY(upload_list(l, &dl, nullptr));
    const int n = c->wfc.nrb(), nl = (int)l.size();
    const long ld = c->ld_w;
    CgState cs = cg_state(c, true);
    const int* act = cs.active;
    float* P = c->f.P.as<float>();
    float* Q = c->f.Q.as<float>();
    for (int k = 0; k < std::max(1, c->opt.check_every); ++k) {
      WGW_TRY(apply_A<float>(c, c->f, P, Q, nl, dl, act, st, false));
      WGW_CK(launch_cg_step_a<float>(c->wfc.tab(), n, nl, dl, c->f.X.as<float>(), c->f.R.as<float>(),
                                     c->f.Z.as<float>(), P, Q, ld, c->eps.as<double>(), cs,
                                     c->opt.inner_tol * c->opt.inner_tol, c->opt.max_cg_iter, st));
      WGW_TRY(run_pc<float>(c, c->f.Z.as<float>(), nl, dl, c->f.psi.as<float>(), act, st));
      WGW_CK(launch_cg_step_b<float>(n, nl, dl, c->f.R.as<float>(), c->f.Z.as<float>(), P, ld, cs, st));
    }
    WGW_TRY(run_pc<float>(c, c->f.R.as<float>(), nl, dl, c->f.psi.as<float>(), act, st));
    c->eng_windows++;
    std::vector<int> ah(cap), ih(cap);
    WGW_CK(cudaMemcpyAsync(ah.data(), cs.active, sizeof(int) * cap, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaMemcpyAsync(ih.data(), cs.iters, sizeof(int) * cap, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    std::vector<int> ret;
    for (int s : l)
      if (!ah[s]) ret.push_back(s);
    if (ret.empty()) return WGW_OK;
    // Retire: x += e, r = b - A x at FP64 accuracy, then done or the next refinement.
    const int* dm = nullptr;
    WGW_TRY(upload_list(ret, &dl, &dm));
    double* X = c->d.X.as<double>();
    WGW_CK(launch_add_to<float>(cap, n, c->f.X.as<float>(), ld, X, ld, dm, st));
    WGW_TRY(apply_A<double>(c, c->d, X, c->d.Q.as<double>(), (int)ret.size(), dl, nullptr, st));
    WGW_CK(launch_axpby(cap, n, 1.0, c->d.Bv.as<double>(), -1.0, c->d.Q.as<double>(), c->d.R.as<double>(), ld, dm, st));
    WGW_CK(launch_norm2<double>(cap, n, c->d.R.as<double>(), ld, c->rr64.as<double>(), st));
    std::vector<double> rr(cap), bb(cap);
    WGW_CK(cudaMemcpyAsync(rr.data(), c->rr64.p, sizeof(double) * cap, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaMemcpyAsync(bb.data(), c->norms.p, sizeof(double) * cap, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    const double tol = c->opt.cg_tol;
    for (int s : ret) {
      iters[s] += ih[s];
      const double rel = bb[s] > 0 ? std::sqrt(rr[s] / bb[s]) : 0.0;
      const bool conv = rel <= tol * (1.0 + 1e-6) || bb[s] == 0.0;
      EngReq& er = live.at(owner[s]);
      if (conv || refine[s] + 1 >= c->opt.max_refine) {
        phase[s] = kDone;
        er.n_done++;
        if (conv) er.n_conv++;
        er.max_rel = std::max(er.max_rel, rel);
        er.max_iters = std::max(er.max_iters, iters[s]);
        er.refinements = std::max(er.refinements, refine[s] + 1);
      } else {
        refine[s]++;
        phase[s] = kStart;
      }
    }
    return WGW_OK;
  }

  // Releases a request's slots and pool rows.
  void release(EngReq& er) {
    for (int sl : er.slots) {
      phase[sl] = kFree;
      free_slots.push_back(sl);
    }
    for (int k = 0; k < er.n_real; ++k) pool_used[er.pbase + k] = 0;
  }

  // Final projection, drho and the results of a request whose systems are all done.
  int finish(EngReq& er) {
    const int n_pert = er.rq.n_pert, n_real = er.n_real, n_v = c->n_v;
    const HostSphere& rs = c->rho;
    int* dl = nullptr;
    WGW_TRY(upload_list(er.slots, &dl, nullptr));
    const int ns = (int)er.slots.size();
    WGW_TRY(run_pc<double>(c, c->d.X.as<double>(), ns, dl, c->d.psi.as<double>(), nullptr, st));
    WGW_TRY(c->eng_xc.ensure(sizeof(double) * (size_t)ns * c->ld_w));
    WGW_CK(launch_gather_rows(ns, (int)c->ld_w, dl, c->d.X.as<double>(), c->ld_w, c->eng_xc.as<double>(), c->ld_w, st));
    WGW_TRY(c->drho_rb.ensure(sizeof(double) * (size_t)n_real * c->ld_r));
    WGW_TRY(drho_pass(c, c->eng_xc.as<double>(), c->ld_w, n_real, c->drho_rb.as<double>(), st));
    const bool sym = er.rq.kind == WGW_REQ_CHIBAR0;
    WGW_TRY(c->brow.ensure(sizeof(int) * n_pert));
    WGW_CK(cudaMemcpyAsync(c->brow.p, er.brow.data(), sizeof(int) * n_pert, cudaMemcpyHostToDevice, st));
    WGW_TRY(c->eng_out.ensure(sizeof(double) * 2 * (size_t)rs.n * n_pert));
    WGW_CK(launch_rb_to_sphere(n_pert, c->drho_rb.as<double>(), c->ld_r, c->brow.as<int>(),
                               sym ? rs.d_vsqrt.as<double>() : nullptr, rs.map(), c->eng_out.as<double>(), 2L * rs.n, st));
    WGW_CK(cudaMemcpyAsync(er.rq.out, c->eng_out.p, sizeof(double) * 2 * (size_t)rs.n * n_pert,
                           cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    (void)n_v;
    return WGW_OK;
  }
};

// A request the engine takes: chi0 or chibar0 at the single frequency 0.
bool engine_eligible(const serve::Request& r) {
  return (r.kind == WGW_REQ_CHI0 || r.kind == WGW_REQ_CHIBAR0) && r.omega.size() == 1 && r.omega[0] == 0.0;
}

}  // namespace

namespace wgw {
int report_error(int status, const char* msg) { return fail(status, msg); }
void clear_error() { g_last_error.clear(); }
}  // namespace wgw

extern "C" {

int wgw_default_options(wgw_options* opt) {
  if (!opt) return fail(WGW_ERR_ARG, "null options");
  opt->precision = WGW_FP64;
  opt->fp64_emulation = 1;
  opt->tensor_cores = 1;
  opt->cuda_graphs = 2;
  opt->cg_tol = 1e-12;
  opt->max_cg_iter = 2000;
  opt->max_refine = 8;
  opt->inner_tol = 5e-6;
  opt->f_s = 2.0;
  opt->check_every = 8;
  opt->dav_tol = 1e-8;
  opt->dav_max_iter = 100;
  opt->dav_factor = 4;
  opt->seed = 12345;
  opt->max_batch_systems = 0;
  opt->fused_h = 2;
  opt->tc_split = 0;
  for (int k = 0; k < 3; ++k) opt->fft_kernels[k] = WGW_FFT_AUTO;
  opt->h_chunk_pairs = -1;
  return WGW_OK;
}

static int check_options(const wgw_options& o) {
  if (o.precision != WGW_FP64 && o.precision != WGW_MIXED) return fail(WGW_ERR_ARG, "bad precision");
  if (!(o.cg_tol > 0) || !(o.inner_tol > 0) || o.max_cg_iter < 1 || o.max_refine < 1 || !(o.f_s > 0))
    return fail(WGW_ERR_ARG, "bad tolerances or iteration limits");
  if (!(o.dav_tol > 0) || o.dav_max_iter < 1 || o.dav_factor < 2)
    return fail(WGW_ERR_ARG, "bad Davidson options");
  if (o.max_batch_systems < 0) return fail(WGW_ERR_ARG, "max_batch_systems < 0");
  if (o.tc_split < 0 || o.tc_split > kTcSplitMax) return fail(WGW_ERR_ARG, "tc_split outside 0..16");
  for (int k = 0; k < 3; ++k)
    if (o.fft_kernels[k] < WGW_FFT_AUTO || o.fft_kernels[k] > WGW_FFT_SHARED)
      return fail(WGW_ERR_ARG, "fft_kernels entries must be WGW_FFT_AUTO, _REG, _REG_PACKED or _SHARED");
  if (o.h_chunk_pairs < -1) return fail(WGW_ERR_ARG, "h_chunk_pairs must be -1 (autotuned), 0 or a pair count");
  return WGW_OK;
}

int wgw_set_options(wgw_ctx* c, const wgw_options* opt) {
  if (!c || !opt) return fail(WGW_ERR_ARG, "null argument");
  WGW_TRY(check_options(*opt));
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->opt = *opt;
  return WGW_OK;
}

static int setup_impl(wgw_ctx* c, const double* vloc_G, const double* psi_v, const double* e_v) {
  const int N = c->N;
  if (!make_plan(N, c->plan)) return fail(WGW_ERR_ARG, "grid must be a product of 2, 3 and 5");
  build_sphere(c->L, c->ecut, N, c->wfc);
  build_sphere(c->L, 4.0 * c->ecut, N, c->rho);
  if (N <= 2 * c->rho.m) return fail(WGW_ERR_ARG, "grid too small: need grid > 2 * max |Miller| of the density sphere");
  if (N > 255) return fail(WGW_ERR_ARG, "grid above 255 points per axis");
  if (c->n_v > c->wfc.n) return fail(WGW_ERR_ARG, "more occupied states than plane waves");
  c->ld_w = pad32(c->wfc.nrb());
  c->ld_r = pad32(c->rho.nrb());
  c->grid3 = (long)N * N * N;
  WGW_TRY(upload_sphere(c->wfc));
  WGW_TRY(upload_sphere(c->rho));
  WGW_CK(cudaGetDevice(&c->device));
  WGW_CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  WGW_TRY(noalloc_prepare());
  cudaStream_t st = c->stream;
  // Twiddles exp(+2 pi i k / N).
  std::vector<cplx<double>> twd(N);
  std::vector<cplx<float>> twf(N);
  std::vector<cplx<ff>> twff(N);
  for (int k = 0; k < N; ++k) {
    const double a = 2.0 * M_PI * k / N;
    twd[k] = mk<double>(std::cos(a), std::sin(a));
    twf[k] = mk<float>((float)twd[k].re, (float)twd[k].im);
    twff[k] = mk<ff>(ff(twd[k].re), ff(twd[k].im));
  }
  WGW_TRY(upload(c->d.tw, twd));
  WGW_TRY(upload(c->f.tw, twf));
  WGW_TRY(upload(c->d.twe, twff));
  c->e_v.assign(e_v, e_v + c->n_v);
  WGW_TRY(upload(c->e_v_d, c->e_v));
  // Occupied states: complex sphere -> real basis (checking they are real in r).
  const int n_v = c->n_v;
  DevBuf tmp;
  WGW_TRY(tmp.ensure(sizeof(double) * (size_t)2 * std::max(c->wfc.n * n_v, c->rho.n)));
  WGW_CK(cudaMemcpy(tmp.p, psi_v, sizeof(double) * 2 * (size_t)c->wfc.n * n_v, cudaMemcpyHostToDevice));
  WGW_TRY(c->d.psi.ensure(sizeof(double) * (size_t)n_v * c->ld_w));
  WGW_CK(cudaMemsetAsync(c->d.psi.p, 0, sizeof(double) * (size_t)n_v * c->ld_w, st));
  WGW_CK(launch_sphere_to_rb(n_v, tmp.as<double>(), 2L * c->wfc.n, nullptr, c->wfc.map(), 0, c->d.psi.as<double>(), c->ld_w, st));
  DevBuf anti;
  WGW_TRY(anti.ensure(sizeof(double) * (size_t)std::max(n_v, 1) * std::max(c->ld_w, c->ld_r)));
  WGW_CK(cudaMemsetAsync(anti.p, 0, anti.bytes, st));
  WGW_CK(launch_sphere_to_rb(n_v, tmp.as<double>(), 2L * c->wfc.n, nullptr, c->wfc.map(), 1, anti.as<double>(), c->ld_w, st));
  DevBuf nrm;
  WGW_TRY(nrm.ensure(sizeof(double) * 2 * (n_v + 1)));
  WGW_CK(launch_norm2<double>(n_v, c->wfc.nrb(), c->d.psi.as<double>(), c->ld_w, nrm.as<double>(), st));
  WGW_CK(launch_norm2<double>(n_v, c->wfc.nrb(), anti.as<double>(), c->ld_w, nrm.as<double>() + n_v, st));
  std::vector<double> h(2 * n_v);
  WGW_CK(cudaMemcpyAsync(h.data(), nrm.p, sizeof(double) * 2 * n_v, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  for (int v = 0; v < n_v; ++v) {
    if (std::fabs(h[v] - 1.0) > 1e-8) { tmp.release(); anti.release(); nrm.release(); return fail(WGW_ERR_ARG, "psi_v not normalised"); }
    if (h[n_v + v] > 1e-20) { tmp.release(); anti.release(); nrm.release(); return fail(WGW_ERR_ARG, "psi_v not real in r (psi(-G) != psi(G)^*)"); }
  }
  WGW_TRY(c->f.psi.ensure(sizeof(float) * (size_t)n_v * c->ld_w));
  WGW_CK((launch_copy_cast<double, float>(n_v, (int)c->ld_w, c->d.psi.as<double>(), c->ld_w, c->f.psi.as<float>(), c->ld_w, nullptr, st)));
  // psi_v(r).
  WGW_TRY(c->d.psi_r.ensure(sizeof(double) * (size_t)n_v * c->grid3));
  WGW_TRY(to_real<double>(c, c->d, c->wfc, c->d.psi.as<double>(), c->ld_w, n_v, c->d.psi_r.as<double>(), c->d.Tw, st));
  WGW_TRY(c->f.psi_r.ensure(sizeof(float) * (size_t)n_v * c->grid3));
  WGW_CK((launch_copy_cast<double, float>(n_v, (int)c->grid3, c->d.psi_r.as<double>(), c->grid3, c->f.psi_r.as<float>(), c->grid3, nullptr, st)));
  // V_loc(r).
  WGW_CK(cudaMemcpy(tmp.p, vloc_G, sizeof(double) * 2 * (size_t)c->rho.n, cudaMemcpyHostToDevice));
  DevBuf vrb;
  WGW_TRY(vrb.ensure(sizeof(double) * c->ld_r));
  WGW_CK(cudaMemsetAsync(vrb.p, 0, sizeof(double) * c->ld_r, st));
  WGW_CK(launch_sphere_to_rb(1, tmp.as<double>(), 2L * c->rho.n, nullptr, c->rho.map(), 0, vrb.as<double>(), c->ld_r, st));
  WGW_CK(cudaMemsetAsync(anti.p, 0, anti.bytes, st));
  WGW_CK(launch_sphere_to_rb(1, tmp.as<double>(), 2L * c->rho.n, nullptr, c->rho.map(), 1, anti.as<double>(), c->ld_r, st));
  WGW_CK(launch_norm2<double>(1, c->rho.nrb(), vrb.as<double>(), c->ld_r, nrm.as<double>(), st));
  WGW_CK(launch_norm2<double>(1, c->rho.nrb(), anti.as<double>(), c->ld_r, nrm.as<double>() + 1, st));
  WGW_CK(cudaMemcpyAsync(h.data(), nrm.p, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  if (h[1] > 1e-24 * std::max(1.0, h[0])) { tmp.release(); anti.release(); nrm.release(); vrb.release(); return fail(WGW_ERR_ARG, "vloc_G not real in r"); }
  WGW_TRY(c->d.v_r.ensure(sizeof(double) * c->grid3));
  DevBuf tr;
  WGW_TRY(to_real<double>(c, c->d, c->rho, vrb.as<double>(), c->ld_r, 1, c->d.v_r.as<double>(), tr, st));
  WGW_TRY(c->f.v_r.ensure(sizeof(float) * c->grid3));
  WGW_CK((launch_copy_cast<double, float>(1, (int)c->grid3, c->d.v_r.as<double>(), c->grid3, c->f.v_r.as<float>(), c->grid3, nullptr, st)));
  WGW_TRY(c->d.psi_r_ff.ensure(sizeof(double) * (size_t)n_v * c->grid3));
  WGW_CK(launch_to_ff((size_t)n_v * c->grid3, c->d.psi_r.as<double>(), c->d.psi_r_ff.as<double>(), st));
  WGW_TRY(c->d.v_r_ff.ensure(sizeof(double) * c->grid3));
  WGW_CK(launch_to_ff((size_t)c->grid3, c->d.v_r.as<double>(), c->d.v_r_ff.as<double>(), st));
  WGW_TRY(c->d.psi_ff.ensure(sizeof(double) * (size_t)n_v * c->ld_w));
  WGW_CK(launch_to_ff((size_t)n_v * c->ld_w, c->d.psi.as<double>(), c->d.psi_ff.as<double>(), st));
  WGW_CK(cudaStreamSynchronize(st));
  tmp.release(); anti.release(); nrm.release(); vrb.release(); tr.release();
  return WGW_OK;
}

static int setup_kb(wgw_ctx* c, const double* beta_G, const double* d_proj) {
  // Projectors beta_p(G) (wavefunction sphere, real in r) -> real basis, in FP64 and FP32.
  const int np = c->n_proj;
  cudaStream_t st = c->stream;
  DevBuf tmp, anti, nrm;
  WGW_TRY(tmp.ensure(sizeof(double) * 2 * (size_t)c->wfc.n * np));
  WGW_CK(cudaMemcpy(tmp.p, beta_G, sizeof(double) * 2 * (size_t)c->wfc.n * np, cudaMemcpyHostToDevice));
  WGW_TRY(c->d.kbB.ensure(sizeof(double) * (size_t)np * c->ld_w));
  WGW_TRY(anti.ensure(sizeof(double) * (size_t)np * c->ld_w));
  WGW_CK(cudaMemsetAsync(c->d.kbB.p, 0, c->d.kbB.bytes, st));
  WGW_CK(cudaMemsetAsync(anti.p, 0, anti.bytes, st));
  WGW_CK(launch_sphere_to_rb(np, tmp.as<double>(), 2L * c->wfc.n, nullptr, c->wfc.map(), 0, c->d.kbB.as<double>(), c->ld_w, st));
  WGW_CK(launch_sphere_to_rb(np, tmp.as<double>(), 2L * c->wfc.n, nullptr, c->wfc.map(), 1, anti.as<double>(), c->ld_w, st));
  WGW_TRY(nrm.ensure(sizeof(double) * 2 * np));
  WGW_CK(launch_norm2<double>(np, c->wfc.nrb(), c->d.kbB.as<double>(), c->ld_w, nrm.as<double>(), st));
  WGW_CK(launch_norm2<double>(np, c->wfc.nrb(), anti.as<double>(), c->ld_w, nrm.as<double>() + np, st));
  std::vector<double> h(2 * np);
  WGW_CK(cudaMemcpyAsync(h.data(), nrm.p, sizeof(double) * 2 * np, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  for (int p = 0; p < np; ++p)
    if (h[np + p] > 1e-24 * std::max(1.0, h[p])) return fail(WGW_ERR_ARG, "KB projector not real in r");
  WGW_TRY(c->f.kbB.ensure(sizeof(float) * (size_t)np * c->ld_w));
  WGW_CK((launch_copy_cast<double, float>(np, (int)c->ld_w, c->d.kbB.as<double>(), c->ld_w, c->f.kbB.as<float>(), c->ld_w, nullptr, st)));
  std::vector<double> dd(d_proj, d_proj + np);
  std::vector<float> df(np);
  for (int p = 0; p < np; ++p) df[p] = (float)dd[p];
  WGW_TRY(upload(c->d.kbD, dd));
  WGW_TRY(upload(c->f.kbD, df));
  WGW_CK(cudaStreamSynchronize(st));
  return WGW_OK;
}

int wgw_setup(wgw_ctx** out, double L, double ecut, int grid, const double* vloc_G, int n_proj,
              const double* beta_G, const double* d_proj, const double* psi_v, const double* e_v,
              int n_v, const wgw_options* opt) {
  g_last_error.clear();
  if (!out) return fail(WGW_ERR_ARG, "null output pointer");
  *out = nullptr;
  if (!(L > 0) || !(ecut > 0) || grid < 4 || n_v < 1 || !vloc_G || !psi_v || !e_v)
    return fail(WGW_ERR_ARG, "invalid L, ecut, grid, n_v or null input");
  if (n_proj < 0 || (n_proj > 0 && (!beta_G || !d_proj))) return fail(WGW_ERR_ARG, "bad Kleinman-Bylander projectors");
  wgw_options o;
  wgw_default_options(&o);
  if (opt) o = *opt;
  WGW_TRY(check_options(o));
  wgw_ctx* c = new wgw_ctx();
  c->L = L; c->ecut = ecut; c->N = grid; c->n_v = n_v; c->n_proj = n_proj; c->omega_cell = L * L * L; c->opt = o;
  int s = setup_impl(c, vloc_G, psi_v, e_v);
  if (s == WGW_OK && n_proj > 0) s = setup_kb(c, beta_G, d_proj);
  if (s != WGW_OK) { delete c; return s; }
  *out = c;
  return WGW_OK;
}

int wgw_sphere_size(const wgw_ctx* c, int which, int* n) {
  if (!c || !n || (which != WGW_SPHERE_WFC && which != WGW_SPHERE_RHO)) return fail(WGW_ERR_ARG, "bad argument");
  *n = which == WGW_SPHERE_WFC ? c->wfc.n : c->rho.n;
  return WGW_OK;
}

int wgw_get_gvectors(const wgw_ctx* c, int which, int32_t* miller) {
  if (!c || !miller || (which != WGW_SPHERE_WFC && which != WGW_SPHERE_RHO)) return fail(WGW_ERR_ARG, "bad argument");
  const HostSphere& s = which == WGW_SPHERE_WFC ? c->wfc : c->rho;
  for (int i = 0; i < 3 * s.n; ++i) miller[i] = s.miller[i];
  return WGW_OK;
}

int wgw_apply_chi0_dev(wgw_ctx* c, const double* dV_dev, int n_pert, const double* omega, int n_omega,
                       double* drho_dev, void* stream, wgw_stats* st) {
  g_last_error.clear();
  if (!c) return fail(WGW_ERR_ARG, "null context");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  return apply_core(c, dV_dev, n_pert, omega, n_omega, drho_dev, false, (cudaStream_t)stream, st);
}

int wgw_apply_chibar0_dev(wgw_ctx* c, const double* phi_dev, int n_pert, const double* omega,
                          int n_omega, double* out_dev, void* stream, wgw_stats* st) {
  g_last_error.clear();
  if (!c) return fail(WGW_ERR_ARG, "null context");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  return apply_core(c, phi_dev, n_pert, omega, n_omega, out_dev, true, (cudaStream_t)stream, st);
}

static int apply_host(wgw_ctx* c, const double* dV, int n_pert, const double* omega, int n_omega,
                      double* drho, bool sym, wgw_stats* st) {
  g_last_error.clear();
  if (!c) return fail(WGW_ERR_ARG, "null context");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if (n_pert <= 0) return n_pert == 0 ? WGW_OK : fail(WGW_ERR_ARG, "n_pert < 0");
  if (n_omega < 1) return fail(WGW_ERR_ARG, "n_omega < 1");
  if (!dV || !drho) return fail(WGW_ERR_ARG, "null dV or drho");
  const size_t in_b = sizeof(double) * 2 * (size_t)c->rho.n * n_pert;
  const size_t out_b = in_b * n_omega;
  WGW_TRY(c->dvin.ensure(in_b + out_b));
  double* din = c->dvin.as<double>();
  double* dout = din + 2 * (size_t)c->rho.n * n_pert;
  WGW_CK(cudaMemcpyAsync(din, dV, in_b, cudaMemcpyHostToDevice, c->stream));
  const int s = apply_core(c, din, n_pert, omega, n_omega, dout, sym, c->stream, st);
  if (s != WGW_OK && s != WGW_ERR_NOCONV) return s;
  WGW_CK(cudaMemcpyAsync(drho, dout, out_b, cudaMemcpyDeviceToHost, c->stream));
  WGW_CK(cudaStreamSynchronize(c->stream));
  return s;
}

int wgw_apply_chi0(wgw_ctx* c, const double* dV, int n_pert, const double* omega, int n_omega,
                   double* drho, wgw_stats* st) {
  return apply_host(c, dV, n_pert, omega, n_omega, drho, false, st);
}

int wgw_apply_chibar0(wgw_ctx* c, const double* phi, int n_pert, const double* omega, int n_omega,
                      double* out, wgw_stats* st) {
  return apply_host(c, phi, n_pert, omega, n_omega, out, true, st);
}

int wgw_apply_channels(wgw_ctx* const* ctxs, int n_ctx, int symmetrized, const double* dV, int n_pert,
                       const double* omega, int n_omega, double* out, wgw_stats* st) {
  g_last_error.clear();
  if (!ctxs || n_ctx < 1 || n_ctx > 8) return fail(WGW_ERR_ARG, "need 1..8 contexts");
  for (int k = 0; k < n_ctx; ++k) {
    const wgw_ctx* c = ctxs[k];
    if (!c) return fail(WGW_ERR_ARG, "null context");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == c) return fail(WGW_ERR_ARG, "a context is listed twice");
    if (c->N != ctxs[0]->N || c->L != ctxs[0]->L || c->ecut != ctxs[0]->ecut)
      return fail(WGW_ERR_ARG, "the channels differ in cell, cutoff or grid");
  }
  if (n_pert <= 0) return n_pert == 0 ? WGW_OK : fail(WGW_ERR_ARG, "n_pert < 0");
  if (n_omega < 1 || !omega || !dV || !out) return fail(WGW_ERR_ARG, "need dV, out and n_omega >= 1 frequencies");
  const size_t n_out = 2 * (size_t)ctxs[0]->rho.n * n_pert * n_omega;
  // Every channel on its own context (own stream and buffers) from its own host thread, so that
  // the channels overlap on the GPU; the sum is taken in channel order.
  std::vector<std::vector<double>> part(n_ctx);
  std::vector<int> status(n_ctx, WGW_OK);
  std::vector<std::string> err(n_ctx);
  std::vector<wgw_stats> sts(n_ctx);
  std::vector<std::thread> th;
  for (int k = 0; k < n_ctx; ++k) {
    part[k].assign(n_out, 0.0);
    th.emplace_back([&, k] {
      if (cudaSetDevice(ctxs[k]->device) != cudaSuccess) { status[k] = WGW_ERR_CUDA; err[k] = "cudaSetDevice"; return; }
      status[k] = apply_host(ctxs[k], dV, n_pert, omega, n_omega, part[k].data(), symmetrized != 0, &sts[k]);
      err[k] = g_last_error;
    });
  }
  for (std::thread& t : th) t.join();
  for (int k = 0; k < n_ctx; ++k)
    if (status[k] != WGW_OK && status[k] != WGW_ERR_NOCONV) return fail(status[k], err[k].c_str());
  for (size_t i = 0; i < n_out; ++i) {
    double acc = 0.0;
    for (int k = 0; k < n_ctx; ++k) acc += part[k][i];
    out[i] = acc;
  }
  int result = WGW_OK;
  wgw_stats tot{};
  for (int k = 0; k < n_ctx; ++k) {
    tot.n_systems += sts[k].n_systems;
    tot.n_converged += sts[k].n_converged;
    tot.max_iters = std::max(tot.max_iters, sts[k].max_iters);
    tot.refinements = std::max(tot.refinements, sts[k].refinements);
    tot.max_rel_residual = std::max(tot.max_rel_residual, sts[k].max_rel_residual);
    if (status[k] == WGW_ERR_NOCONV) result = fail(WGW_ERR_NOCONV, err[k].c_str());
  }
  if (st) *st = tot;
  return result;
}

int wgw_profile_enable(wgw_ctx* c, int on) {
  if (!c) return fail(WGW_ERR_ARG, "null context");
  c->prof.reset();
  c->prof.on = on != 0;
  return WGW_OK;
}

int wgw_profile_classes(wgw_ctx* c, unsigned mask) {
  if (!c) return fail(WGW_ERR_ARG, "null context");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->prof.mask = mask;
  return WGW_OK;
}

int wgw_profile_read(wgw_ctx* c, int kind, double* ms, long* launches, double* bytes, double* flops) {
  if (!c || kind < 0 || kind >= kProfKinds) return fail(WGW_ERR_ARG, "bad profile kind");
  c->prof.flush();
  if (ms) *ms = c->prof.ms[kind];
  if (launches) *launches = c->prof.n[kind];
  if (bytes) *bytes = c->prof.bytes[kind];
  if (flops) *flops = c->prof.flops[kind];
  return WGW_OK;
}

const char* wgw_profile_kind_name(int kind) {
  return (kind >= 0 && kind < kProfKinds) ? kProfNames[kind] : "";
}

int wgw_system_info(const wgw_ctx* c, int n, int* iters, double* rel_residual, int* converged) {
  if (!c || n < 0) return fail(WGW_ERR_ARG, "bad argument");
  const int m = std::min<int>(n, (int)c->last_iters.size());
  for (int s = 0; s < m; ++s) {
    if (iters) iters[s] = c->last_iters[s];
    if (rel_residual) rel_residual[s] = c->last_relres[s];
    if (converged) converged[s] = c->last_conv[s];
  }
  return m;
}

int wgw_sample_solutions(wgw_ctx* c, int n, const int* systems) {
  g_last_error.clear();
  if (!c || n < 0 || (n > 0 && !systems)) return fail(WGW_ERR_ARG, "bad argument");
  for (int k = 0; k < n; ++k)
    if (systems[k] < 0) return fail(WGW_ERR_ARG, "negative system index");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  c->sample_sys.assign(systems, systems + n);
  c->sample_out.assign((size_t)n * 2 * c->wfc.n, 0.0);
  return WGW_OK;
}

int wgw_read_samples(wgw_ctx* c, int n, double* dpsi) {
  g_last_error.clear();
  if (!c || n < 0 || (n > 0 && !dpsi)) return fail(WGW_ERR_ARG, "bad argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if ((size_t)n > c->sample_sys.size()) return fail(WGW_ERR_ARG, "more samples requested than selected");
  std::copy(c->sample_out.begin(), c->sample_out.begin() + (size_t)n * 2 * c->wfc.n, dpsi);
  return WGW_OK;
}

int wgw_pdep_davidson(wgw_ctx* c, int n_pdep, const double* x0, double* eig, double* basis, wgw_stats* st) {
  g_last_error.clear();
  if (!c || n_pdep < 1 || !eig) return fail(WGW_ERR_ARG, "need a context, n_pdep >= 1 and eig");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if (n_pdep > c->rho.nrb() / 2) return fail(WGW_ERR_ARG, "n_pdep too large for the density sphere");
  return davidson_impl(c, n_pdep, x0, eig, basis, st);
}

int wgw_pdep_davidson_channels(wgw_ctx* const* ctxs, int n_ctx, int n_pdep, const double* x0, double* eig,
                               double* basis, wgw_stats* st) {
  g_last_error.clear();
  if (!ctxs || n_ctx < 1 || n_ctx > 8 || n_pdep < 1 || !eig)
    return fail(WGW_ERR_ARG, "need 1..8 contexts, n_pdep >= 1 and eig");
  for (int k = 0; k < n_ctx; ++k) {
    if (!ctxs[k]) return fail(WGW_ERR_ARG, "null context");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return fail(WGW_ERR_ARG, "a context is listed twice");
    if (ctxs[k]->N != ctxs[0]->N || ctxs[k]->L != ctxs[0]->L || ctxs[k]->ecut != ctxs[0]->ecut)
      return fail(WGW_ERR_ARG, "the channels differ in cell, cutoff or grid");
  }
  wgw_ctx* c = ctxs[0];
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if (n_pdep > c->rho.nrb() / 2) return fail(WGW_ERR_ARG, "n_pdep too large for the density sphere");
  const std::vector<wgw_ctx*> chans(ctxs + 1, ctxs + n_ctx);
  return davidson_impl(c, n_pdep, x0, eig, basis, st, chans);
}

int wgw_apply_h_dev(wgw_ctx* c, const double* psi_dev, int n_psi, double* out_dev, int fp32, void* stream) {
  g_last_error.clear();
  if (!c || n_psi < 0 || (n_psi > 0 && (!psi_dev || !out_dev))) return fail(WGW_ERR_ARG, "bad argument");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  if (n_psi == 0) return WGW_OK;
  if (fp32 && c->opt.precision != WGW_MIXED)
    return fail(WGW_ERR_ARG, "the FP32 H needs a mixed-precision context (it holds the FP32 copies)");
  cudaStream_t st = (cudaStream_t)stream;
  set_ff(c);
  WGW_TRY(ensure_work(c, n_psi, 1));
  const int n = c->wfc.nrb();
  const long ld = c->ld_w;
  double* P = c->d.P.as<double>();
  double* Q = c->d.Q.as<double>();
  WGW_CK(cudaMemsetAsync(P, 0, sizeof(double) * (size_t)n_psi * ld, st));
  WGW_CK(launch_sphere_to_rb(n_psi, psi_dev, 2L * c->wfc.n, nullptr, c->wfc.map(), 0, P, ld, st));
  if (fp32) {
    WGW_CK(cudaMemsetAsync(c->f.shift.p, 0, sizeof(float) * n_psi, st));
    WGW_CK((launch_copy_cast<double, float>(n_psi, n, P, ld, c->f.P.as<float>(), ld, nullptr, st)));
    WGW_TRY(apply_A<float>(c, c->f, c->f.P.as<float>(), c->f.Q.as<float>(), n_psi, nullptr, nullptr, st, false));
    WGW_CK((launch_copy_cast<float, double>(n_psi, n, c->f.Q.as<float>(), ld, Q, ld, nullptr, st)));
  } else {
    WGW_CK(cudaMemsetAsync(c->d.shift.p, 0, sizeof(double) * n_psi, st));
    WGW_TRY(apply_A<double>(c, c->d, P, Q, n_psi, nullptr, nullptr, st, false));
  }
  WGW_CK(launch_rb_to_sphere(n_psi, Q, ld, nullptr, nullptr, c->wfc.map(), out_dev, 2L * c->wfc.n, st));
  return WGW_OK;
}

static int sigma_x_impl(wgw_ctx* c, const int* states, int n_states, double* sigma_x) {
  cudaStream_t st = c->stream;
  set_ff(c);
  const int N = c->N, n_v = c->n_v;
  const HostSphere& rs = c->rho;
  const long ldr = c->ld_r;
  const int nr = rs.nrb();
  // v^1/2 per real-basis element of the density sphere (0 at G = 0).
  std::vector<double> vsh(nr, 0.0);
  for (int j = 1; j <= rs.n_pairs; ++j) vsh[2 * j - 1] = vsh[2 * j] = rs.vsqrt[rs.pos[j]];
  DevBuf vs, out, nrm;
  WGW_TRY(vs.ensure(sizeof(double) * nr));
  WGW_CK(cudaMemcpyAsync(vs.p, vsh.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st));
  // Pair densities u_i u_j of every listed i with every occupied j (real in r at Gamma), in
  // batches of about 512: products in real space and the x transform in the x-line kernel,
  // then the plane transforms onto the density sphere; |v^1/2 n_ij|^2 summed over G.
  const int per = std::max(1, std::min(n_states, 512 / std::max(1, n_v)));
  std::vector<double> acc(n_states, 0.0);
  for (int q0 = 0; q0 < n_states; q0 += per) {
    const int nq = std::min(per, n_states - q0), n_sys = nq * n_v;
    WGW_TRY(ensure_work(c, n_sys, 1));
    std::vector<int> ai(n_sys), bi(n_sys);
    for (int q = 0; q < nq; ++q)
      for (int j = 0; j < n_v; ++j) { ai[q * n_v + j] = states[q0 + q]; bi[q * n_v + j] = j; }
    WGW_CK(cudaMemcpyAsync(c->a_idx.p, ai.data(), sizeof(int) * n_sys, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(c->b_idx.p, bi.data(), sizeof(int) * n_sys, cudaMemcpyHostToDevice, st));
    const int NPr = 2 * rs.m + 1, pairs = (n_sys + 1) / 2;
    WGW_TRY(c->Trho.ensure(sizeof(cplx<double>) * (size_t)pairs * NPr * N * N));
    WGW_TRY(out.ensure(sizeof(double) * (size_t)n_sys * ldr));
    WGW_TRY(nrm.ensure(sizeof(double) * n_sys));
    FftCtx<double> f = c->d.fft(c->plan);
    XArgs<double> a{};
    a.mode = XM_FROM_REAL; a.A = c->d.psi_r_fft(); a.lda = c->grid3; a.a_index = c->a_idx.as<int>();
    a.Bm = c->d.psi_r_fft(); a.ldb = c->grid3; a.b_index = c->b_idx.as<int>(); a.n_sys = n_sys;
    WGW_CK(launch_xline<double>(rs.m, f, c->Trho.as<cplx<double>>(), a, nullptr, st));
    Epi<double> e{};
    e.out = out.as<double>(); e.ldo = ldr; e.vcoef = 1.0; e.n_sys = n_sys;
    WGW_CK(launch_plane_r2g<double>(rs.tab(), rs.npt_max, f, c->Trho.as<cplx<double>>(), e, st));
    dim3 g(std::max(1, std::min(64, (nr + 255) / 256)), std::min(n_sys, 65535));
    k_scale_rows<<<g, 256, 0, st>>>(nr, n_sys, out.as<double>(), ldr, vs.as<double>(), out.as<double>(), ldr);
    WGW_CK(cudaGetLastError());
    WGW_CK(launch_norm2<double>(n_sys, nr, out.as<double>(), ldr, nrm.as<double>(), st));
    std::vector<double> h(n_sys);
    WGW_CK(cudaMemcpyAsync(h.data(), nrm.p, sizeof(double) * n_sys, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    for (int q = 0; q < nq; ++q)
      for (int j = 0; j < n_v; ++j) acc[q0 + q] += h[q * n_v + j];
  }
  for (int k = 0; k < n_states; ++k) sigma_x[k] = -acc[k] / c->omega_cell;
  return WGW_OK;
}

int wgw_sigma_x(wgw_ctx* c, const int* states, int n_states, double* sigma_x) {
  g_last_error.clear();
  if (!c || !states || n_states < 1 || !sigma_x) return fail(WGW_ERR_ARG, "need a context, states and output");
  for (int k = 0; k < n_states; ++k)
    if (states[k] < 0 || states[k] >= c->n_v) return fail(WGW_ERR_ARG, "state index outside 0..n_v-1");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  return sigma_x_impl(c, states, n_states, sigma_x);
}

int wgw_autotune_info(const wgw_ctx* c, int* tc_split, int* splits, double* ms, int n_max, int* fused_h,
                      double* h_ms) {
  if (!c || n_max < 0) {
    fail(WGW_ERR_ARG, "bad argument");
    return -WGW_ERR_ARG;
  }
  if (fused_h) *fused_h = c->h_choice;
  if (h_ms) { h_ms[0] = c->h_ms[0]; h_ms[1] = c->h_ms[1]; }
  if (tc_split) *tc_split = c->tc_split;
  const int m = std::min<int>(n_max, (int)c->tc_tune.size());
  for (int k = 0; k < m; ++k) {
    if (splits) splits[k] = c->tc_tune[k].first;
    if (ms) ms[k] = c->tc_tune[k].second;
  }
  return m;
}

int wgw_autotune_fft(const wgw_ctx* c, int* choice, double* ms) {
  if (!c) return fail(WGW_ERR_ARG, "null context");
  const FftKern k = fft_choice(c);
  const int ch[3] = {k.g2r, k.xline, k.r2g};
  for (int s = 0; s < 3; ++s) {
    if (choice) choice[s] = ch[s];
    for (int q = 0; q < kFftChoices; ++q)
      if (ms) ms[3 * s + q] = c->fft_ms[s][q];
  }
  return WGW_OK;
}

int wgw_autotune_chunk(const wgw_ctx* c, int* chunk_pairs, int* candidates, double* ms, int n_max) {
  if (!c || n_max < 0) {
    fail(WGW_ERR_ARG, "bad argument");
    return -WGW_ERR_ARG;
  }
  if (chunk_pairs) *chunk_pairs = c->opt.h_chunk_pairs >= 0 ? c->opt.h_chunk_pairs : (c->chunk_tuned ? c->h_chunk : -1);
  const int m = std::min<int>(n_max, (int)c->chunk_ms.size());
  for (int k = 0; k < m; ++k) {
    if (candidates) candidates[k] = c->chunk_ms[k].first;
    if (ms) ms[k] = c->chunk_ms[k].second;
  }
  return m;
}

int wgw_selftest_wait_timeout(int* timed_out) {
  g_last_error.clear();
  if (!timed_out) return fail(WGW_ERR_ARG, "null argument");
  DevBuf flag;
  WGW_TRY(flag.ensure(sizeof(int)));
  WGW_CK(cudaMemset(flag.p, 0, sizeof(int)));
  WGW_CK(tc_wait_selftest(flag.as<int>(), nullptr));
  WGW_CK(cudaMemcpy(timed_out, flag.p, sizeof(int), cudaMemcpyDeviceToHost));
  return WGW_OK;
}

int wgw_dyson(int n, int n_omega, const double* chi0bar, double* chibar) {
  g_last_error.clear();
  if (n < 1 || n > 4096 || n_omega < 0) return fail(WGW_ERR_ARG, "need 1 <= n <= 4096 and n_omega >= 0");
  if (n_omega == 0) return WGW_OK;
  if (!chi0bar || !chibar) return fail(WGW_ERR_ARG, "null argument");
  const size_t bytes = sizeof(double) * (size_t)n * n * n_omega;
  cudaStream_t st = cudaStreamPerThread;
  DevBuf a, x, m, info;
  WGW_TRY(a.ensure(bytes));
  WGW_TRY(x.ensure(bytes));
  WGW_TRY(m.ensure(bytes));
  WGW_TRY(info.ensure(sizeof(int) * n_omega));
  WGW_CK(cudaMemcpyAsync(a.p, chi0bar, bytes, cudaMemcpyHostToDevice, st));
  WGW_CK(launch_dyson(n, n_omega, a.as<double>(), x.as<double>(), m.as<double>(), info.as<int>(), st));
  std::vector<int> flags(n_omega);
  WGW_CK(cudaMemcpyAsync(chibar, x.p, bytes, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaMemcpyAsync(flags.data(), info.p, sizeof(int) * n_omega, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  for (int k = 0; k < n_omega; ++k)
    if (flags[k]) return fail(WGW_ERR_ARG, "1 - chi0bar is singular at one of the frequencies");
  return WGW_OK;
}

int wgw_lanczos(wgw_ctx* c, const double* phi, int n_pdep, int n_steps, const double* omega, int n_omega,
                double* alpha, double* beta, double* chi0_pdep, wgw_stats* st) {
  g_last_error.clear();
  if (!c || !phi || n_pdep < 1 || n_steps < 1 || n_steps > 255 || n_omega < 0 || (n_omega > 0 && !omega))
    return fail(WGW_ERR_ARG, "need a context, phi, n_pdep >= 1, 1 <= n_steps <= 255, n_omega >= 0");
  for (int k = 0; k < n_omega; ++k)
    if (!(omega[k] >= 0.0)) return fail(WGW_ERR_ARG, "imaginary frequencies must be >= 0");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  return lanczos_impl(c, phi, n_pdep, n_steps, omega, n_omega, alpha, beta, chi0_pdep, st);
}

int wgw_g0_lanczos(wgw_ctx* c, const double* phi, int n_pdep, const int* states, int n_states, int n_steps,
                   const double* z, int n_z, double* alpha, double* beta, double* d, double* residues,
                   double* g0, wgw_stats* st) {
  g_last_error.clear();
  if (!c || !phi || n_pdep < 1 || !states || n_states < 1 || n_steps < 1 || n_steps > 255 || n_z < 0 ||
      (n_z > 0 && !z))
    return fail(WGW_ERR_ARG, "need a context, phi, n_pdep >= 1, states, n_states >= 1, 1 <= n_steps <= 255, n_z >= 0");
  for (int i = 0; i < n_states; ++i)
    if (states[i] < 0 || states[i] >= c->n_v) return fail(WGW_ERR_ARG, "state index outside 0..n_v-1");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  const LzG0 g{states, n_states, z, n_z, d, residues, g0};
  return lanczos_impl(c, phi, n_pdep, n_steps, nullptr, 0, alpha, beta, nullptr, st, &g);
}

int wgw_isr(wgw_ctx* c, const double* phi, int n_pdep, const int* states, int n_states, int n_steps,
            const double* omega, int n_omega, const double* lam, const double* nodes, const double* weights,
            int n_nodes, double* isr, wgw_stats* st) {
  g_last_error.clear();
  if (!c || !phi || n_pdep < 1 || !states || n_states < 1 || n_steps < 1 || n_steps > 255 || n_omega < 1 ||
      !omega || n_nodes < 1 || !lam || !nodes || !weights || !isr)
    return fail(WGW_ERR_ARG, "need a context, phi, states, 1 <= n_steps <= 255, frequencies, Lambda and nodes");
  for (int i = 0; i < n_states; ++i)
    if (states[i] < 0 || states[i] >= c->n_v) return fail(WGW_ERR_ARG, "state index outside 0..n_v-1");
  for (int k = 0; k < n_nodes; ++k)
    if (!(nodes[k] >= 0.0)) return fail(WGW_ERR_ARG, "quadrature nodes must be >= 0");
  std::vector<double> z;
  z.reserve(4 * (size_t)n_omega * n_nodes);
  for (int j = 0; j < n_omega; ++j)
    for (int k = 0; k < n_nodes; ++k) {
      z.push_back(omega[j]); z.push_back(nodes[k]);
      z.push_back(omega[j]); z.push_back(-nodes[k]);
    }
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  LzG0 g{states, n_states, z.data(), 2 * n_omega * n_nodes, nullptr, nullptr, nullptr};
  g.lam = lam; g.weights = weights; g.n_omega = n_omega; g.n_nodes = n_nodes; g.isr = isr;
  return lanczos_impl(c, phi, n_pdep, n_steps, nullptr, 0, nullptr, nullptr, nullptr, st, &g);
}

// ---------------------------------------------------------------- self-energy at real frequencies
// chi0bar(z) and Lambda(z) = (1 - chi0bar(z))^-1 chi0bar(z) in the basis at the n_z complex
// frequencies z_host (interleaved) from kept chi0 chains; device outputs chi and lam, n_z x
// n_pdep^2 complex each.
static int lambda_z(wgw_ctx* c, const LzKeep& kc, int npd, int n_steps, const double* z_host, int n_z, DevBuf& chi,
                    DevBuf& lam) {
  cudaStream_t st = c->stream;
  const size_t mat = 2 * (size_t)npd * npd;
  DevBuf zd, M, info;
  WGW_TRY(zd.ensure(sizeof(double) * 2 * n_z));
  WGW_TRY(chi.ensure(sizeof(double) * mat * n_z));
  WGW_TRY(lam.ensure(sizeof(double) * mat * n_z));
  WGW_TRY(M.ensure(sizeof(double) * mat * n_z));
  WGW_TRY(info.ensure(sizeof(int) * n_z));
  WGW_CK(cudaMemcpyAsync(zd.p, z_host, sizeof(double) * 2 * n_z, cudaMemcpyHostToDevice, st));
  WGW_CK(launch_chi_z(npd, c->n_v, n_steps, n_z, kc.W.as<double>(), kc.d.as<double>(), c->e_v_d.as<double>(),
                      zd.as<double>(), c->opt.f_s / c->omega_cell, chi.as<double>(), st));
  WGW_CK(launch_dyson_z(npd, n_z, chi.as<double>(), lam.as<double>(), M.as<double>(), info.as<int>(), st));
  std::vector<int> flags(n_z);
  WGW_CK(cudaMemcpyAsync(flags.data(), info.p, sizeof(int) * n_z, cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  for (int k = 0; k < n_z; ++k)
    if (flags[k]) return fail(WGW_ERR_ARG, "1 - chi0bar is singular at one of the frequencies");
  return WGW_OK;
}

// What the self-energy of a set of states needs, computed once: the chi0 chains of the basis
// (for Lambda at any frequency), the G0 chains of the states with the overlaps <psi_j|psi_i phi~_m>,
// Lambda at the quadrature nodes, and Sigma_X.
struct SigmaCtx {
  int npd = 0, ns = 0;
  wgw_sigma_params prm{};
  LzKeep chi, g0;
  DevBuf lam_nodes, nodes, wts;
  std::vector<double> sx;
};

static int sigma_check(const wgw_ctx* c, const double* phi, int npd, const int* states, int ns,
                       const wgw_sigma_params* p) {
  if (!c || !phi || npd < 1 || !states || ns < 1 || !p)
    return fail(WGW_ERR_ARG, "need a context, phi, n_pdep >= 1, states and parameters");
  if (p->n_steps_chi < 1 || p->n_steps_chi > 255 || p->n_steps_g0 < 1 || p->n_steps_g0 > 255)
    return fail(WGW_ERR_ARG, "chain lengths must be within 1..255");
  if (p->n_nodes < 1 || !p->nodes || !p->weights) return fail(WGW_ERR_ARG, "need quadrature nodes and weights");
  for (int k = 0; k < p->n_nodes; ++k)
    if (!(p->nodes[k] >= 0.0) || !std::isfinite(p->nodes[k]) || !std::isfinite(p->weights[k]))
      return fail(WGW_ERR_ARG, "quadrature nodes must be finite and >= 0, weights finite");
  if (!(p->eta >= 0.0) || !std::isfinite(p->eta)) return fail(WGW_ERR_ARG, "eta must be finite and >= 0");
  for (int k = 0; k < ns; ++k)
    if (states[k] < 0 || states[k] >= c->n_v) return fail(WGW_ERR_ARG, "state index outside 0..n_v-1");
  for (int v = 0; v < c->n_v; ++v)
    if (!(c->e_v[v] <= p->e_fermi)) return fail(WGW_ERR_ARG, "e_fermi lies below an occupied energy");
  return WGW_OK;
}

static int sigma_prepare(wgw_ctx* c, const double* phi, int npd, const int* states, int ns, const wgw_sigma_params& p,
                         SigmaCtx& S) {
  S.npd = npd;
  S.ns = ns;
  S.prm = p;
  WGW_TRY(lanczos_impl(c, phi, npd, p.n_steps_chi, nullptr, 0, nullptr, nullptr, nullptr, nullptr, nullptr, &S.chi));
  const LzG0 g{states, ns, nullptr, 0, nullptr, nullptr, nullptr};
  WGW_TRY(lanczos_impl(c, phi, npd, p.n_steps_g0, nullptr, 0, nullptr, nullptr, nullptr, nullptr, &g, &S.g0));
  std::vector<double> zn(2 * (size_t)p.n_nodes);
  for (int k = 0; k < p.n_nodes; ++k) zn[2 * k + 1] = p.nodes[k];
  DevBuf chi;
  WGW_TRY(lambda_z(c, S.chi, npd, p.n_steps_chi, zn.data(), p.n_nodes, chi, S.lam_nodes));
  WGW_TRY(S.nodes.ensure(sizeof(double) * p.n_nodes));
  WGW_TRY(S.wts.ensure(sizeof(double) * p.n_nodes));
  WGW_CK(cudaMemcpyAsync(S.nodes.p, p.nodes, sizeof(double) * p.n_nodes, cudaMemcpyHostToDevice, c->stream));
  WGW_CK(cudaMemcpyAsync(S.wts.p, p.weights, sizeof(double) * p.n_nodes, cudaMemcpyHostToDevice, c->stream));
  S.sx.assign(ns, 0.0);
  WGW_TRY(sigma_x_impl(c, states, ns, S.sx.data()));
  WGW_CK(cudaStreamSynchronize(c->stream));
  return WGW_OK;
}

// I^SR (real) and R (complex, interleaved) at evaluation points p = (listed state pi[p], real
// frequency pw[p] <= e_fermi).  R sums, in the order of j, the occupied states above w.
static int sigma_eval(wgw_ctx* c, SigmaCtx& S, const std::vector<int>& pi, const std::vector<double>& pw,
                      std::vector<double>& isr, std::vector<double>& res) {
  cudaStream_t st = c->stream;
  const int np = (int)pi.size(), npd = S.npd;
  isr.assign(np, 0.0);
  res.assign(2 * (size_t)np, 0.0);
  if (np == 0) return WGW_OK;
  {
    DevBuf dpi, dpw, dout;
    WGW_TRY(dpi.ensure(sizeof(int) * np));
    WGW_TRY(dpw.ensure(sizeof(double) * np));
    WGW_TRY(dout.ensure(sizeof(double) * np));
    WGW_CK(cudaMemcpyAsync(dpi.p, pi.data(), sizeof(int) * np, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(dpw.p, pw.data(), sizeof(double) * np, cudaMemcpyHostToDevice, st));
    WGW_CK(launch_isr_points(npd, S.ns, S.prm.n_steps_g0, S.prm.n_nodes, np, S.g0.W.as<double>(), S.g0.d.as<double>(),
                             dpi.as<int>(), dpw.as<double>(), S.lam_nodes.as<double>(), S.nodes.as<double>(),
                             S.wts.as<double>(), 1.0 / c->omega_cell, dout.as<double>(), st));
    WGW_CK(cudaMemcpyAsync(isr.data(), dout.p, sizeof(double) * np, cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
  }
  // Residue term: f = -1 for every occupied j with e_j > w (w <= e_fermi: no empty state enters).
  std::vector<int> es, ej, ep;
  std::vector<double> ef, ez;
  for (int p = 0; p < np; ++p)
    for (int j = 0; j < c->n_v; ++j)
      if (c->e_v[j] > pw[p]) {
        es.push_back(pi[p]); ej.push_back(j); ep.push_back(p); ef.push_back(-1.0);
        ez.push_back(c->e_v[j] - pw[p]); ez.push_back(S.prm.eta);
      }
  // Entries per round: chi0bar, Lambda and the elimination work of one entry take 3 x 16 n_pdep^2
  // bytes; at most 512 entries and about 256 MB per round.
  const int n_e = (int)es.size();
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(512, ((size_t)256 << 20) / (48 * (size_t)npd * npd)));
  DevBuf chi, lam, des, dej, def, dout;
  for (int e0 = 0; e0 < n_e; e0 += chunk) {
    const int ne = std::min(chunk, n_e - e0);
    WGW_TRY(lambda_z(c, S.chi, npd, S.prm.n_steps_chi, ez.data() + 2 * (size_t)e0, ne, chi, lam));
    WGW_TRY(des.ensure(sizeof(int) * ne));
    WGW_TRY(dej.ensure(sizeof(int) * ne));
    WGW_TRY(def.ensure(sizeof(double) * ne));
    WGW_TRY(dout.ensure(sizeof(double) * 2 * ne));
    WGW_CK(cudaMemcpyAsync(des.p, es.data() + e0, sizeof(int) * ne, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(dej.p, ej.data() + e0, sizeof(int) * ne, cudaMemcpyHostToDevice, st));
    WGW_CK(cudaMemcpyAsync(def.p, ef.data() + e0, sizeof(double) * ne, cudaMemcpyHostToDevice, st));
    WGW_CK(launch_residue_entries(npd, ne, lam.as<double>(), S.g0.Y.as<double>(), S.g0.ys, des.as<int>(),
                                  dej.as<int>(), def.as<double>(), dout.as<double>(), st));
    std::vector<double> h(2 * (size_t)ne);
    WGW_CK(cudaMemcpyAsync(h.data(), dout.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    WGW_CK(cudaStreamSynchronize(st));
    for (int e = 0; e < ne; ++e) {
      res[2 * (size_t)ep[e0 + e]] += h[2 * e] / c->omega_cell;
      res[2 * (size_t)ep[e0 + e] + 1] += h[2 * e + 1] / c->omega_cell;
    }
  }
  return WGW_OK;
}

static void sigma_stats(const wgw_ctx* c, const SigmaCtx& S, wgw_stats* st) {
  if (!st) return;
  *st = wgw_stats{};
  st->n_systems = S.npd * (c->n_v + S.ns);   // chains
  st->n_converged = st->n_systems;
  st->max_iters = std::max(S.prm.n_steps_chi, S.prm.n_steps_g0);
}

int wgw_lanczos_z(wgw_ctx* c, const double* phi, int n_pdep, int n_steps, const double* z, int n_z, double* chi0_z,
                  double* lam_z, wgw_stats* st) {
  g_last_error.clear();
  if (!c || !phi || n_pdep < 1 || n_steps < 1 || n_steps > 255 || n_z < 1 || !z)
    return fail(WGW_ERR_ARG, "need a context, phi, n_pdep >= 1, 1 <= n_steps <= 255 and n_z >= 1 frequencies");
  for (int k = 0; k < 2 * n_z; ++k)
    if (!std::isfinite(z[k])) return fail(WGW_ERR_ARG, "frequencies must be finite");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  LzKeep kc;
  WGW_TRY(lanczos_impl(c, phi, n_pdep, n_steps, nullptr, 0, nullptr, nullptr, nullptr, st, nullptr, &kc));
  DevBuf chi, lam;
  const int rc = lambda_z(c, kc, n_pdep, n_steps, z, n_z, chi, lam);
  if (rc != WGW_OK && rc != WGW_ERR_ARG) return rc;
  const size_t bytes = sizeof(double) * 2 * (size_t)n_pdep * n_pdep * n_z;
  if (chi0_z) WGW_CK(cudaMemcpyAsync(chi0_z, chi.p, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (lam_z && rc == WGW_OK) WGW_CK(cudaMemcpyAsync(lam_z, lam.p, bytes, cudaMemcpyDeviceToHost, c->stream));
  WGW_CK(cudaStreamSynchronize(c->stream));
  return rc;
}

int wgw_sigma(wgw_ctx* c, const double* phi, int n_pdep, const int* states, int n_states,
              const wgw_sigma_params* prm, const double* omega, int n_omega, double* sigma_x, double* isr,
              double* res, wgw_stats* st) {
  g_last_error.clear();
  WGW_TRY(sigma_check(c, phi, n_pdep, states, n_states, prm));
  if (n_omega < 0 || (n_omega > 0 && !omega)) return fail(WGW_ERR_ARG, "need n_omega >= 0 frequencies");
  for (int j = 0; j < n_omega; ++j)
    if (!std::isfinite(omega[j]) || !(omega[j] <= prm->e_fermi))
      return fail(WGW_ERR_ARG, "frequencies must be finite and <= e_fermi (the context holds no empty states)");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  SigmaCtx S;
  WGW_TRY(sigma_prepare(c, phi, n_pdep, states, n_states, *prm, S));
  if (sigma_x) std::copy(S.sx.begin(), S.sx.end(), sigma_x);
  std::vector<int> pi;
  std::vector<double> pw, hi, hr;
  for (int i = 0; i < n_states; ++i)
    for (int j = 0; j < n_omega; ++j) { pi.push_back(i); pw.push_back(omega[j]); }
  WGW_TRY(sigma_eval(c, S, pi, pw, hi, hr));
  if (isr) std::copy(hi.begin(), hi.end(), isr);
  if (res) std::copy(hr.begin(), hr.end(), res);
  sigma_stats(c, S, st);
  return WGW_OK;
}

int wgw_qp(wgw_ctx* c, const double* phi, int n_pdep, const int* states, int n_states,
           const wgw_sigma_params* prm, const double* v_xc, double tol, int max_iter, double* e_qp,
           double* sigma_qp, int* iters, wgw_stats* st) {
  g_last_error.clear();
  WGW_TRY(sigma_check(c, phi, n_pdep, states, n_states, prm));
  if (!e_qp || !(tol > 0.0) || max_iter < 1) return fail(WGW_ERR_ARG, "need e_qp, tol > 0 and max_iter >= 1");
  for (int i = 0; i < n_states; ++i)
    if (!(c->e_v[states[i]] + 0.01 <= prm->e_fermi))
      return fail(WGW_ERR_ARG, "the secant's second start point e_i + 0.01 lies above e_fermi");
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  SigmaCtx S;
  WGW_TRY(sigma_prepare(c, phi, n_pdep, states, n_states, *prm, S));
  const int ns = n_states;
  // Secant per state on F(E) = e_i + Re Sigma_i(E) - v_xc - E from e_i and e_i + 0.01; the
  // states still iterating are evaluated together.
  std::vector<double> x0(ns), x1(ns), f0(ns), f1(ns), sig(2 * (size_t)ns, 0.0);
  std::vector<int> done(ns, 0), it(ns, 0);
  auto F = [&](const std::vector<int>& who, const std::vector<double>& E, std::vector<double>& out,
               std::vector<double>& sg) -> int {
    std::vector<double> hi, hr;
    WGW_TRY(sigma_eval(c, S, who, E, hi, hr));
    out.resize(who.size());
    sg.resize(2 * who.size());
    for (size_t q = 0; q < who.size(); ++q) {
      const int i = who[q];
      const double re = S.sx[i] + hi[q] + hr[2 * q];
      sg[2 * q] = re;
      sg[2 * q + 1] = hr[2 * q + 1];
      out[q] = c->e_v[states[i]] + re - (v_xc ? v_xc[i] : 0.0) - E[q];
    }
    return WGW_OK;
  };
  {
    std::vector<int> who;
    std::vector<double> E, out, sg;
    for (int i = 0; i < ns; ++i) {
      x0[i] = c->e_v[states[i]];
      x1[i] = x0[i] + 0.01;
      who.push_back(i); E.push_back(x0[i]);
      who.push_back(i); E.push_back(x1[i]);
    }
    WGW_TRY(F(who, E, out, sg));
    for (int i = 0; i < ns; ++i) { f0[i] = out[2 * i]; f1[i] = out[2 * i + 1]; }
  }
  int status = WGW_OK;
  for (int step = 0; step < max_iter; ++step) {
    std::vector<int> who;
    std::vector<double> E, out, sg;
    for (int i = 0; i < ns; ++i) {
      if (done[i]) continue;
      if (f1[i] == f0[i]) { done[i] = -1; continue; }   // stalled
      const double x2 = x1[i] - f1[i] * (x1[i] - x0[i]) / (f1[i] - f0[i]);
      if (!std::isfinite(x2) || !(x2 <= prm->e_fermi))
        return fail(WGW_ERR_ARG, "a secant iterate rose above e_fermi (the context holds no empty states)");
      who.push_back(i);
      E.push_back(x2);
    }
    if (who.empty()) break;
    WGW_TRY(F(who, E, out, sg));
    for (size_t q = 0; q < who.size(); ++q) {
      const int i = who[q];
      x0[i] = x1[i]; f0[i] = f1[i];
      x1[i] = E[q]; f1[i] = out[q];
      sig[2 * i] = sg[2 * q];
      sig[2 * i + 1] = sg[2 * q + 1];
      ++it[i];
      if (std::fabs(x1[i] - x0[i]) <= tol * std::max(1.0, std::fabs(x1[i]))) done[i] = 1;
    }
  }
  for (int i = 0; i < ns; ++i) {
    e_qp[i] = x1[i];
    if (sigma_qp) { sigma_qp[2 * i] = sig[2 * i]; sigma_qp[2 * i + 1] = sig[2 * i + 1]; }
    if (iters) iters[i] = it[i];
    if (done[i] != 1) status = WGW_ERR_NOCONV;
  }
  sigma_stats(c, S, st);
  return status == WGW_OK ? WGW_OK : fail(status, "the secant did not converge for some states");
}

int wgw_symm_eig_dev(int n, double* A_dev, double* w_dev, double* Z_dev, void* stream) {
  g_last_error.clear();
  if (n < 1 || n > 2048 || !A_dev || !w_dev || !Z_dev) return fail(WGW_ERR_ARG, "need 1 <= n <= 2048 and buffers");
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf wk, info;
  WGW_TRY(wk.ensure(sizeof(double) * syev_work_elems(n)));
  WGW_TRY(info.ensure(sizeof(int)));
  WGW_CK(launch_syev(n, A_dev, n, w_dev, Z_dev, n, wk.as<double>(), info.as<int>(), st));
  int h = 0;
  WGW_CK(cudaMemcpyAsync(&h, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  WGW_CK(cudaStreamSynchronize(st));
  return h == 0 ? WGW_OK : fail(WGW_ERR_NOCONV, "dense eigensolver did not converge");
}


// ---------------------------------------------------------------- serving: request queue
// Requests are checked and copied in by wgw_submit and executed by one worker thread per
// context on the context's stream.  The worker takes the head request when the least memory it
// can run in fits 80 % of the free device memory (plus the work buffers the context holds), and
// merges every queued request of the same kind and frequency set that keeps the whole batch
// resident in that budget into one batched apply, then scatters the results back; requests to
// different contexts run on different streams and overlap on the GPU.
static double batch_bytes(const wgw_ctx* c, int n_real, bool whole) {
  double per_sys = 0, per_pert = 0;
  solve_bytes(c, &per_sys, &per_pert);
  const int n_pert = (n_real + 1) / 2;
  const double io = 8.0 * (2.0 * c->rho.n * n_pert * 2 + (double)n_real * c->ld_r * 3);
  const int resident = whole ? n_real : 1;
  return resident * (per_sys * c->n_v + per_pert) + io;
}

// Slots of the engine: 60 % of the free device memory (plus the context's work buffers) at the
// bytes one batched-solve system needs, at most 16384 (the option max_batch_systems caps it too).
static int engine_capacity(wgw_ctx* c) {
  double per_sys = 0, per_pert = 0;
  solve_bytes(c, &per_sys, &per_pert);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  const double budget = 0.6 * ((double)free_b + held_work_bytes(c));
  int cap = (int)std::min(16384.0, budget / (per_sys + 2.0 * per_pert / std::max(1, c->n_v)));
  if (c->opt.max_batch_systems > 0) cap = std::min(cap, c->opt.max_batch_systems);
  return cap;
}

// Runs the engine until no live request is left and the queue's head is not one it takes.
// Returns false (nothing taken) when the engine's buffers cannot be set up.
static bool run_engine(wgw_ctx* c, int cap) {
  std::lock_guard<std::recursive_mutex> ctx_lock(c->mu);
  set_ff(c);
  Engine E;
  E.c = c;
  E.st = c->stream;
  const int n_v = c->n_v;
  int rc;
  {
    // Contexts of one process share the device memory: sizing the engine from the free memory
    // and allocating it is one step, so that two contexts never size from the same reading.
    static std::mutex hbm_mu;
    std::lock_guard<std::mutex> adm(hbm_mu);
    cap = std::min(cap, engine_capacity(c));
    if (cap < 2 * n_v) return false;
    rc = E.init(cap, 2 * (cap / n_v) + 2);
  }
  auto fail_all = [&](int status) {
    std::lock_guard<std::mutex> lk(c->qmu);
    const auto now = std::chrono::steady_clock::now();
    for (auto& kv : E.live) c->sq.finish_one(kv.second.rq, status, kv.second.t_admit, now, kv.second.peers, 0, g_last_error);
    E.live.clear();
  };
  if (rc != WGW_OK) return false;   // nothing admitted yet: the head is left to the batched path
  for (;;) {
    // Admission into the free slots, in queue order.
    for (;;) {
      serve::Request rq;
      bool got;
      {
        std::lock_guard<std::mutex> lk(c->qmu);
        got = c->sq.take_head_if([&](const serve::Request& h) {
          const int worst = 2 * h.n_pert;
          if (!engine_eligible(h) || worst * n_v > (int)E.free_slots.size()) return false;
          int room = 0, best = 0;
          for (int k = 0; k < E.pcap; ++k) { room = E.pool_used[k] ? 0 : room + 1; best = std::max(best, room); }
          return best >= worst;
        }, &rq);
      }
      if (!got) break;
      const uint64_t t = rq.ticket;
      const auto t0 = std::chrono::steady_clock::now();
      serve::Request keep = rq;
      rc = E.admit(std::move(rq));
      if (rc != WGW_OK) {
        std::lock_guard<std::mutex> lk(c->qmu);
        c->sq.finish_one(keep, rc, t0, std::chrono::steady_clock::now(), 1, 0, g_last_error);
        (void)t;
        break;
      }
    }
    if (rc != WGW_OK && rc != WGW_ERR_STATE) { fail_all(rc); break; }
    rc = WGW_OK;
    // Cancelled live requests leave at once.
    std::vector<uint64_t> gone;
    {
      std::lock_guard<std::mutex> lk(c->qmu);
      for (auto& kv : E.live)
        if (c->sq.cancelled(kv.first)) gone.push_back(kv.first);
    }
    for (uint64_t t : gone) {
      EngReq& er = E.live.at(t);
      E.release(er);
      std::lock_guard<std::mutex> lk(c->qmu);
      c->sq.finish_one(er.rq, WGW_ERR_CANCELLED, er.t_admit, std::chrono::steady_clock::now(), er.peers,
                       (int)er.slots.size());
      E.live.erase(t);
    }
    if (!gone.empty()) c->qcv.notify_all();
    if (E.live.empty()) break;
    rc = E.start_inner();
    if (rc == WGW_OK) rc = E.window();
    if (rc != WGW_OK) { fail_all(rc); break; }
    // Requests whose systems are all done.
    std::vector<uint64_t> ready;
    for (auto& kv : E.live)
      if (kv.second.n_done == (int)kv.second.slots.size()) ready.push_back(kv.first);
    for (uint64_t t : ready) {
      EngReq& er = E.live.at(t);
      rc = E.finish(er);
      E.release(er);
      const int status = rc != WGW_OK ? rc : (er.n_conv == (int)er.slots.size() ? WGW_OK : WGW_ERR_NOCONV);
      {
        std::lock_guard<std::mutex> lk(c->qmu);
        c->sq.finish_one(er.rq, status, er.t_admit, std::chrono::steady_clock::now(), er.peers, (int)er.slots.size(),
                         g_last_error);
      }
      E.live.erase(t);
      if (rc != WGW_OK) break;
    }
    if (!ready.empty()) c->qcv.notify_all();
    if (rc != WGW_OK) { fail_all(rc); break; }
  }
  c->qcv.notify_all();
  return true;
}

// A served Davidson request (Sec. 3, Sec. 4.2) on its own host thread and stream: the Davidson
// iteration of davidson_impl, whose chibar0 block applications are submitted to the queue as
// chibar0 requests (so that they are batched with everything else the context serves) and waited
// for; the Rayleigh-Ritz work runs on the helper's stream.  Outputs: eigenvalues then the basis.
static void pdep_helper(wgw_ctx* c, serve::Request rq) {
  cudaSetDevice(c->device);
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t hs = nullptr;
  int rc = cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking) == cudaSuccess ? WGW_OK : WGW_ERR_CUDA;
  const int n_rho = c->rho.n, npd = rq.n_pert;
  int n_apply = 0;
  wgw_stats st{};
  DevBuf cin, cout;
  auto ext = [&](const double* in, int nb, double* out, wgw_stats* acc) -> int {
    {
      std::lock_guard<std::mutex> lk(c->qmu);
      if (c->sq.cancelled(rq.ticket)) return fail(WGW_ERR_CANCELLED, "request cancelled");
    }
    WGW_TRY(cin.ensure(sizeof(double) * 2 * (size_t)n_rho * nb));
    WGW_TRY(cout.ensure(sizeof(double) * 2 * (size_t)n_rho * nb));
    WGW_CK(launch_rb_to_sphere(nb, in, c->ld_r, nullptr, nullptr, c->rho.map(), cin.as<double>(), 2L * n_rho, hs));
    serve::Request r;
    r.kind = WGW_REQ_CHIBAR0;
    r.n_pert = nb;
    r.dV.resize(2 * (size_t)n_rho * nb);
    r.omega = {0.0};
    std::vector<double> o(2 * (size_t)n_rho * nb, 0.0);
    r.out = o.data();
    WGW_CK(cudaMemcpyAsync(r.dV.data(), cin.p, sizeof(double) * r.dV.size(), cudaMemcpyDeviceToHost, hs));
    WGW_CK(cudaStreamSynchronize(hs));
    r.t_submit = std::chrono::steady_clock::now();
    uint64_t t;
    {
      std::lock_guard<std::mutex> lk(c->qmu);
      t = c->sq.push(std::move(r));
    }
    c->qcv.notify_all();
    serve::Done d;
    {
      std::unique_lock<std::mutex> lk(c->qmu);
      c->qcv.wait(lk, [&] { return c->sq.state(t) == serve::Queue::kDone; });
      c->sq.take_done(t, &d);
    }
    if (d.status != WGW_OK && d.status != WGW_ERR_NOCONV) return fail(d.status, "served chibar0 block: " + d.msg);
    WGW_CK(cudaMemcpyAsync(cout.p, o.data(), sizeof(double) * o.size(), cudaMemcpyHostToDevice, hs));
    WGW_CK(cudaMemsetAsync(out, 0, sizeof(double) * (size_t)nb * c->ld_r, hs));
    WGW_CK(launch_sphere_to_rb(nb, cout.as<double>(), 2L * n_rho, nullptr, c->rho.map(), 0, out, c->ld_r, hs));
    WGW_CK(cudaStreamSynchronize(hs));   // o leaves scope
    acc->n_systems += d.batch_systems;
    ++n_apply;
    return WGW_OK;
  };
  if (rc == WGW_OK)
    rc = davidson_impl(c, npd, rq.dV.empty() ? nullptr : rq.dV.data(), rq.out, rq.out + npd, &st, {}, ext, hs);
  cin.release();
  cout.release();
  if (hs) cudaStreamDestroy(hs);
  {
    std::lock_guard<std::mutex> lk(c->qmu);
    c->sq.finish_one(rq, rc, t_start, std::chrono::steady_clock::now(), n_apply, st.n_systems, g_last_error);
    c->pdep_active--;
  }
  c->qcv.notify_all();
}

static void serve_loop(wgw_ctx* c) {
  cudaSetDevice(c->device);
  for (;;) {
    std::vector<serve::Request> batch;
    int eng_cap = 0;
    {
      std::unique_lock<std::mutex> lk(c->qmu);
      c->qcv.wait(lk, [&] { return (c->stop && c->pdep_active == 0) || !c->sq.empty(); });
      if (c->sq.empty()) return;
      const serve::Request* h = c->sq.head();
      if (h->kind == WGW_REQ_PDEP) {
        serve::Request rq;
        c->sq.take_head_if([](const serve::Request&) { return true; }, &rq);
        c->pdep_active++;
        c->pdep_threads.emplace_back(pdep_helper, c, std::move(rq));
        continue;
      }
      if (c->opt.precision == WGW_MIXED && engine_eligible(*h)) {
        lk.unlock();
        eng_cap = engine_capacity(c);
        lk.lock();
        h = c->sq.head();
        if (!h || !engine_eligible(*h) || 2 * h->n_pert * c->n_v > eng_cap) eng_cap = 0;
      }
    }
    if (eng_cap > 0 && run_engine(c, eng_cap)) continue;
    {
      std::unique_lock<std::mutex> lk(c->qmu);
      if (c->sq.empty()) continue;
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
      }
      const double budget = 0.8 * ((double)free_b + held_work_bytes(c));
      std::vector<std::pair<uint64_t, serve::Done>> rejected;
      batch = c->sq.take_batch(budget, [&](int n_real, bool whole) { return batch_bytes(c, n_real, whole); },
                               false, &rejected);
      if (!rejected.empty()) c->qcv.notify_all();
      if (batch.empty()) continue;
    }
    const auto t_start = std::chrono::steady_clock::now();
    const int n_rho = c->rho.n, n_om = (int)batch[0].omega.size();
    int n_tot = 0;
    for (auto& r : batch) n_tot += r.n_pert;
    std::vector<double> dv((size_t)2 * n_rho * n_tot), out((size_t)2 * n_rho * n_tot * n_om);
    int off = 0;
    for (auto& r : batch) {
      std::copy(r.dV.begin(), r.dV.end(), dv.begin() + (size_t)2 * n_rho * off);
      off += r.n_pert;
    }
    wgw_stats stt{};
    const int status = apply_host(c, dv.data(), n_tot, batch[0].omega.data(), n_om, out.data(),
                                  batch[0].kind == WGW_REQ_CHIBAR0, &stt);
    {
      std::lock_guard<std::mutex> lk(c->qmu);
      off = 0;
      for (auto& r : batch) {
        if ((status == WGW_OK || status == WGW_ERR_NOCONV) && !c->sq.cancelled(r.ticket))
          for (int k = 0; k < n_om; ++k)
            std::copy(out.begin() + (size_t)2 * n_rho * ((size_t)k * n_tot + off),
                      out.begin() + (size_t)2 * n_rho * ((size_t)k * n_tot + off + r.n_pert),
                      r.out + (size_t)2 * n_rho * ((size_t)k * r.n_pert));
        off += r.n_pert;
      }
      c->sq.finish(batch, status, t_start, std::chrono::steady_clock::now(), stt.n_systems, g_last_error);
    }
    c->qcv.notify_all();
  }
}

int wgw_submit(wgw_ctx* c, const wgw_request* req, uint64_t* ticket) {
  g_last_error.clear();
  if (!c || !req || !ticket) return fail(WGW_ERR_ARG, "null argument");
  std::string why;
  if (serve::validate(req->kind, req->dV, req->n_pert, req->omega, req->n_omega, req->out, c->rho.n, &why) !=
      serve::kOk)
    return fail(WGW_ERR_ARG, why);
  serve::Request r;
  r.kind = req->kind;
  r.n_pert = req->n_pert;
  if (req->kind == WGW_REQ_PDEP) {
    if (req->n_pert > c->rho.nrb() / 2 || c->opt.dav_factor * req->n_pert > 2048)
      return fail(WGW_ERR_ARG, "n_pdep too large for the density sphere or the Davidson subspace");
    if (req->dV) r.dV.assign(req->dV, req->dV + (size_t)2 * c->rho.n * req->n_pert);
  } else {
    r.dV.assign(req->dV, req->dV + (size_t)2 * c->rho.n * req->n_pert);
    r.omega.assign(req->omega, req->omega + req->n_omega);
  }
  r.out = req->out;
  r.t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(c->qmu);
    if (c->stop) return fail(WGW_ERR_STATE, "context is shutting down");
    *ticket = c->sq.push(std::move(r));
    if (!c->worker.joinable()) c->worker = std::thread(serve_loop, c);
  }
  c->qcv.notify_all();
  return WGW_OK;
}

static void fill_result(const serve::Done& d, wgw_result* res) {
  // The failure of a served request is reported by wgw_last_error on the thread that collects it.
  if (d.status != WGW_OK) g_last_error = d.msg;
  if (!res) return;
  res->status = d.status;
  res->latency_s = d.latency_s;
  res->queue_s = d.queue_s;
  res->batch_requests = d.batch_requests;
  res->batch_systems = d.batch_systems;
}

int wgw_poll(wgw_ctx* c, uint64_t ticket, int* done, wgw_result* res) {
  g_last_error.clear();
  if (!c || !done) return fail(WGW_ERR_ARG, "null argument");
  std::lock_guard<std::mutex> lk(c->qmu);
  serve::Done d;
  if (c->sq.take_done(ticket, &d)) {
    *done = 1;
    fill_result(d, res);
    return WGW_OK;
  }
  if (c->sq.state(ticket) != serve::Queue::kUnknown) {
    *done = 0;
    return WGW_OK;
  }
  return fail(WGW_ERR_ARG, "unknown or already released ticket");
}

int wgw_wait(wgw_ctx* c, uint64_t ticket, wgw_result* res) {
  g_last_error.clear();
  if (!c) return fail(WGW_ERR_ARG, "null argument");
  std::unique_lock<std::mutex> lk(c->qmu);
  if (c->sq.state(ticket) == serve::Queue::kUnknown) return fail(WGW_ERR_ARG, "unknown or already released ticket");
  c->qcv.wait(lk, [&] { return c->sq.state(ticket) == serve::Queue::kDone; });
  serve::Done d;
  c->sq.take_done(ticket, &d);
  fill_result(d, res);
  return WGW_OK;
}

int wgw_cancel(wgw_ctx* c, uint64_t ticket) {
  g_last_error.clear();
  if (!c) return fail(WGW_ERR_ARG, "null argument");
  int rc;
  {
    std::lock_guard<std::mutex> lk(c->qmu);
    rc = c->sq.cancel(ticket);
  }
  c->qcv.notify_all();
  return rc == serve::kOk ? WGW_OK : fail(WGW_ERR_ARG, "unknown or already finished ticket");
}

void wgw_destroy(wgw_ctx* c) { delete c; }

const char* wgw_status_string(int s) {
  switch (s) {
    case WGW_OK: return "ok";
    case WGW_ERR_ARG: return "invalid argument";
    case WGW_ERR_NOMEM: return "device allocation failed";
    case WGW_ERR_NOCONV: return "Sternheimer solve did not converge";
    case WGW_ERR_CUDA: return "CUDA error";
    case WGW_ERR_TIMEOUT: return "bounded device wait timed out";
    case WGW_ERR_STATE: return "invalid state";
    case WGW_ERR_CANCELLED: return "request cancelled";
    default: return "unknown status";
  }
}

const char* wgw_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
