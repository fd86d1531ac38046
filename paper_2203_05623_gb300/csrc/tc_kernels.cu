// P_c = 1 - Psi Psi^T on the 5th-generation tensor cores (tcgen05, sm_103a), FP32 in and out.
//
// Phase 1  C^T[j][v] = sum_k Y[k][s_j] Psi[k][v]      D = 128 systems x N states (split over K)
// Reduce   sum of the K-block partials in a fixed order
// Phase 2  Y[k][s_j] = beta Y + alpha sum_v Psi[k][v] C^T[j][v]   D = 128 rows x 128 systems
//
// Both phases are TF32 MMAs with FP32 accumulation in tensor memory.  Every FP32 operand x is
// split as x = hi + lo with hi the nearest TF32 value and lo the nearest TF32 value of x - hi
// (|x - hi - lo| <= 2^-22 |x|), and each product is formed as hi*hi + hi*lo + lo*hi ("3xTF32"),
// which leaves the lo*lo term and the split error, both ~2^-22 relative: close to FP32.  Operands are staged by the CTA's threads in the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices, adjacent in K at
// 128 bytes (leading byte offset) and adjacent in M/N at 1024 bytes (stride byte offset) for
// K chunks of 32 elements.  One thread issues the MMAs and commits them to an mbarrier; every
// wait on that mbarrier is bounded and reports a timeout through the caller's error flag.
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace wgw {


namespace tc {

constexpr int kThreads = 128;    // 4 warps: warp w reads TMEM lanes 32w..32w+31
constexpr int kKC = 32;          // K elements per staged chunk (8 core matrices of 4 TF32)
constexpr int kRowsA = 128;      // M of every MMA
constexpr uint32_t kCoreBytes = 128;
constexpr uint32_t kLbo = kCoreBytes;             // K-adjacent core matrices
constexpr uint32_t kSbo = (kKC / 4) * kCoreBytes; // M/N-adjacent core matrices (8 rows)
constexpr unsigned long long kWaitNs = 1000000000ull;   // bound of every mbarrier wait: 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (tcgen05 format, no swizzle, relative leading offset).
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((kLbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((kSbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1u) << 46;   // descriptor version of tcgen05
  return d;                               // base offset 0, swizzle mode 0 (none)
}

// Instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait (about one second of wall time) for the completion of phase `parity`; false,
// with *err set, on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int* err) {
  if (mbar_test(mbar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(mbar, parity))
    if (global_ns() - t0 > kWaitNs) {
      atomicExch(err, 1);
      return false;
    }
  return true;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warp-wide: allocate `ncols` (power of 2, >= 32) TMEM columns, address written to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row r, k) of a staged [rows x 32] K-major tile.
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return static_cast<uint32_t>(((r >> 3) * (kKC / 4) + (k >> 2)) * kCoreBytes + (r & 7) * 16 + (k & 3) * 4);
}

// Nearest TF32 value (10 explicit mantissa bits; ties away from zero), so that the tensor
// core, which ignores the low 13 bits of each operand, sees it exactly.
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// x = hi + lo + O(2^-22 |x|) with hi, lo both TF32: |x - hi| <= 2^-11 |x| and lo = round(x - hi).
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}

// Store 4 K-consecutive values of row r (k multiple of 4) as hi and lo parts.
__device__ __forceinline__ void put4(unsigned char* hi, unsigned char* lo, int r, int k, float4 v) {
  float4 h, l;
  split_tf32(v.x, h.x, l.x);
  split_tf32(v.y, h.y, l.y);
  split_tf32(v.z, h.z, l.z);
  split_tf32(v.w, h.w, l.w);
  const uint32_t o = tile_off(r, k);
  *reinterpret_cast<float4*>(hi + o) = h;
  *reinterpret_cast<float4*>(lo + o) = l;
}

__device__ __forceinline__ void put1(unsigned char* hi, unsigned char* lo, int r, int k, float v) {
  float h, l;
  split_tf32(v, h, l);
  const uint32_t o = tile_off(r, k);
  *reinterpret_cast<float*>(hi + o) = h;
  *reinterpret_cast<float*>(lo + o) = l;
}

// 4 consecutive floats of a row at [k, k + 4) with zeros at and beyond k_hi.
__device__ __forceinline__ float4 load4(const float* row, int k, int k_hi) {
  if (k + 4 <= k_hi) return *reinterpret_cast<const float4*>(row + k);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (k + 0 < k_hi) v.x = row[k + 0];
  if (k + 1 < k_hi) v.y = row[k + 1];
  if (k + 2 < k_hi) v.z = row[k + 2];
  if (k + 3 < k_hi) v.w = row[k + 3];
  return v;
}

// Issue the 4 K-steps (K = 8 each) x 3 split products of one staged chunk.
__device__ __forceinline__ void issue_chunk(uint32_t tmem_d, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                            uint32_t b_lo, uint32_t idesc, bool first) {
#pragma unroll
  for (int s = 0; s < kKC / 8; ++s) {
    const uint32_t off = s * 2 * kCoreBytes;
    mma_tf32(tmem_d, mat_desc(a_hi + off), mat_desc(b_hi + off), idesc, (first && s == 0) ? 0u : 1u);
    mma_tf32(tmem_d, mat_desc(a_hi + off), mat_desc(b_lo + off), idesc, 1u);
    mma_tf32(tmem_d, mat_desc(a_lo + off), mat_desc(b_hi + off), idesc, 1u);
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared through the TMA engine, completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

constexpr uint32_t kTile = kRowsA * kKC * 4;   // bytes of one 128 x 32 TF32 part (16 KB)

// Operand tiles of a constant matrix, split and laid out once:
//  tiles1 (phase-1 B): chunk kc of 32 k, part (hi, lo), Nn rows v: ((kc * 2 + part) * Nn * 128) + tile_off(v, k % 32)
//  tiles2 (phase-2 A): row tile rt of 128 k, state chunk vc, part: ((rt * nvc + vc) * 2 + part) * kTile + tile_off(k % 128, v % 32)
__global__ void k_tc_tile_psi(const float* __restrict__ Psi, long ldp, int n, int nv, int Nn, int nkc, int nrt,
                              int nvc, unsigned char* __restrict__ t1, unsigned char* __restrict__ t2) {
  const long total = static_cast<long>(nkc) * kKC * Nn;
  for (long e = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long>(gridDim.x) * blockDim.x) {
    const int v = static_cast<int>(e % Nn);
    const int k = static_cast<int>(e / Nn);
    const float x = (v < nv && k < n) ? Psi[static_cast<size_t>(v) * ldp + k] : 0.f;
    float hi, lo;
    split_tf32(x, hi, lo);
    const int kc = k / kKC, kk = k % kKC;
    const size_t b1 = static_cast<size_t>(kc) * 2 * Nn * 128;
    *reinterpret_cast<float*>(t1 + b1 + tile_off(v, kk)) = hi;
    *reinterpret_cast<float*>(t1 + b1 + static_cast<size_t>(Nn) * 128 + tile_off(v, kk)) = lo;
    if (k < nrt * kRowsA && v < nvc * kKC) {
      const int rt = k / kRowsA, r = k % kRowsA, vc = v / kKC, vv = v % kKC;
      const size_t b2 = (static_cast<size_t>(rt) * nvc + vc) * 2 * kTile;
      *reinterpret_cast<float*>(t2 + b2 + tile_off(r, vv)) = hi;
      *reinterpret_cast<float*>(t2 + b2 + kTile + tile_off(r, vv)) = lo;
    }
  }
}

// Phase 1.  Grid (ceil(n_list / 128), n_kb); CTA (jt, kb) owns K chunks [kb * kcpb, ...).
// A (128 systems x 32 k) is staged by the threads (split on the fly, next chunk prefetched
// into registers while the current MMAs run); B (Nn states x 32 k) arrives by bulk copy
// from tiles1.  Two shared-memory stages.  Cpart[kb][j][v] (row length ldc).
__global__ void __launch_bounds__(kThreads) k_tc_pc1(const unsigned char* __restrict__ t1, const float* __restrict__ Y,
                                                     long ldy, int n, int nv, int n_list,
                                                     const int* __restrict__ list, int kcpb, int Nn, int ldc,
                                                     float* __restrict__ Cpart, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * kRowsA, kb = blockIdx.y;
  const int nkc = (n + kKC - 1) / kKC;
  const int kc_lo = kb * kcpb, kc_hi = min(nkc, kc_lo + kcpb);
  const uint32_t b_bytes = 2u * Nn * 128;
  const uint32_t stage_bytes = 2 * kTile + b_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes);   // full[2], mma[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
  uint32_t ncols = 32;
  while (ncols < static_cast<uint32_t>(Nn)) ncols <<= 1;
  if (warp == 0) tmem_alloc(tslot, ncols);
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(smem_u32(bars + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_tf32(kRowsA, Nn);
  // This thread's 8 A rows (systems) and its 16-byte column within a chunk.
  const int rr = tid & 7, kq = (tid >> 3) & 7, mg0 = tid >> 6;
  const float* rowp[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int j = j0 + (mg0 + 2 * i) * 8 + rr;
    const int sj = j < n_list ? (list ? list[j] : j) : -1;
    rowp[i] = sj >= 0 ? Y + static_cast<size_t>(sj) * ldy : nullptr;
  }
  float4 pre[8];
  auto load_a = [&](int kc) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      pre[i] = rowp[i] ? load4(rowp[i], kc * kKC + kq * 4, n) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto stage_in = [&](int kc, int st) {
    unsigned char* base = smem + st * stage_bytes;
#pragma unroll
    for (int i = 0; i < 8; ++i) put4(base, base + kTile, (mg0 + 2 * i) * 8 + rr, kq * 4, pre[i]);
    if (tid == 0) {
      const uint32_t fb = smem_u32(bars + st);
      mbar_expect_tx(fb, b_bytes);
      bulk_g2s(smem_u32(base + 2 * kTile), t1 + static_cast<size_t>(kc) * b_bytes, b_bytes, fb);
    }
  };
  bool ok = true;
  const int nc = kc_hi - kc_lo;
  if (nc > 0) {
    load_a(kc_lo);
    stage_in(kc_lo, 0);
    fence_async_smem();
    __syncthreads();
  }
  for (int c = 0; c < nc; ++c) {
    const int st = c & 1;
    if (tid == 0) {
      ok = ok && mbar_wait(smem_u32(bars + st), (c >> 1) & 1, err);   // B of chunk c landed
      if (ok) {
        fence_after();
        unsigned char* base = smem + st * stage_bytes;
        issue_chunk(tmem, smem_u32(base), smem_u32(base + kTile), smem_u32(base + 2 * kTile),
                    smem_u32(base + 2 * kTile + Nn * 128), idesc, c == 0);
        mma_commit(smem_u32(bars + 2 + st));
      }
    }
    if (c + 1 < nc) {
      load_a(kc_lo + c + 1);                 // global loads in flight while the MMAs run
      const int s1 = (c + 1) & 1;
      if (c >= 1) {                          // stage s1 was read by the MMAs of chunk c - 1
        const bool w = mbar_wait(smem_u32(bars + 2 + s1), ((c - 1) >> 1) & 1, err);
        ok = ok && w;
      }
      ok = __syncthreads_and(ok) != 0;
      if (!ok) break;
      stage_in(kc_lo + c + 1, s1);
      fence_async_smem();
      __syncthreads();
    }
  }
  if (nc > 0) {
    const bool w = ok && mbar_wait(smem_u32(bars + 2 + ((nc - 1) & 1)), ((nc - 1) >> 1) & 1, err);
    ok = __syncthreads_and(w) != 0;
  }
  fence_after();
  const int j = j0 + warp * 32 + lane;
  float* out = Cpart + (static_cast<size_t>(kb) * n_list + (j < n_list ? j : 0)) * ldc;
  for (int c0 = 0; c0 < ldc; c0 += 16) {
    float v[16];
    if (ok && nc > 0 && c0 < Nn) {
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
    if (j < n_list) {
#pragma unroll
      for (int i = 0; i < 16; i += 4) {
        float4 w = make_float4(c0 + i < nv ? v[i] : 0.f, c0 + i + 1 < nv ? v[i + 1] : 0.f,
                               c0 + i + 2 < nv ? v[i + 2] : 0.f, c0 + i + 3 < nv ? v[i + 3] : 0.f);
        *reinterpret_cast<float4*>(out + c0 + i) = w;
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// C^T[j][v] = scale[v] sum_kb Cpart[kb][j][v] (fixed order; scale null = 1), written split and
// tiled for phase 2: ((jt * nvc + vc) * 2 + part) * kTile + tile_off(j % 128, v % 32); zero outside
// n_list x nv.
__global__ void k_tc_reduce(const float* __restrict__ Cpart, int n_list, int ldc, int n_kb, int nv, int njt,
                            int nvc, const float* __restrict__ scale, unsigned char* __restrict__ ct) {
  const long total = static_cast<long>(njt) * kRowsA * nvc * kKC;
  const size_t slice = static_cast<size_t>(n_list) * ldc;
  for (long e = blockIdx.x * static_cast<long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long>(gridDim.x) * blockDim.x) {
    const int v = static_cast<int>(e % (nvc * kKC));
    const int j = static_cast<int>(e / (nvc * kKC));
    float sum = 0.f;
    if (j < n_list && v < nv) {
      const size_t o = static_cast<size_t>(j) * ldc + v;
      float s0 = Cpart[o], s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int kb = 1;
      for (; kb + 3 < n_kb; kb += 4) {
        s1 += Cpart[static_cast<size_t>(kb) * slice + o];
        s2 += Cpart[static_cast<size_t>(kb + 1) * slice + o];
        s3 += Cpart[static_cast<size_t>(kb + 2) * slice + o];
        s0 += Cpart[static_cast<size_t>(kb + 3) * slice + o];
      }
      for (; kb < n_kb; ++kb) s1 += Cpart[static_cast<size_t>(kb) * slice + o];
      sum = (s0 + s1) + (s2 + s3);
      if (scale) sum *= scale[v];
    }
    float hi, lo;
    split_tf32(sum, hi, lo);
    const int jt = j / kRowsA, vc = v / kKC;
    const size_t b = (static_cast<size_t>(jt) * nvc + vc) * 2 * kTile;
    *reinterpret_cast<float*>(ct + b + tile_off(j % kRowsA, v % kKC)) = hi;
    *reinterpret_cast<float*>(ct + b + kTile + tile_off(j % kRowsA, v % kKC)) = lo;
  }
}

// Phase 2.  Grid (ceil(n / 128), ceil(n_list / 128)).  D = rows rt x systems jt, K = states in
// chunks of 32; A from tiles2 and B from the reduced C^T tiles, both by bulk copy into one
// 64 KB stage (several CTAs per SM), chunk after chunk.
constexpr int kThreads2 = 256;   // phase 2: warp w reads TMEM lanes 32 (w % 4); warps 4-7 take columns 64-127

__global__ void __launch_bounds__(kThreads2, 2) k_tc_pc2(const unsigned char* __restrict__ t2,
                                                      const unsigned char* __restrict__ ct, float* __restrict__ Y,
                                                      long ldy, int n, int nvc, int n_list,
                                                      const int* __restrict__ list, float alpha, float beta,
                                                      const int* __restrict__ active, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rt = blockIdx.x, jt = blockIdx.y;
  const int r0 = rt * kRowsA, j0 = jt * kRowsA;
  constexpr uint32_t stage_bytes = 4 * kTile;   // A hi, A lo, B hi, B lo
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + stage_bytes);   // full, mma
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  int* sys = reinterpret_cast<int*>(tslot + 2);                       // 128 target systems (-1: skip)
  int any = 0;
  for (int t = tid; t < kRowsA; t += kThreads2) {
    const int j = j0 + t;
    int sx = -1;
    if (j < n_list) {
      sx = list ? list[j] : j;
      if (sx >= 0 && active && !active[sx]) sx = -1;
    }
    sys[t] = sx;
    any |= sx >= 0;
  }
  if (!__syncthreads_or(any)) return;   // every system of the tile has finished
  constexpr uint32_t ncols = kRowsA;
  if (warp == 0) tmem_alloc(tslot, ncols);
  if (tid == 0) {
    mbar_init(smem_u32(bars), 1);
    mbar_init(smem_u32(bars + 1), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_tf32(kRowsA, kRowsA);
  bool ok = true;
  if (tid == 0) {
    for (int vc = 0; vc < nvc && ok; ++vc) {
      if (vc > 0) ok = mbar_wait(smem_u32(bars + 1), (vc - 1) & 1, err);   // previous MMAs read the stage
      if (!ok) break;
      const uint32_t fb = smem_u32(bars);
      mbar_expect_tx(fb, 4 * kTile);
      bulk_g2s(smem_u32(smem), t2 + (static_cast<size_t>(rt) * nvc + vc) * 2 * kTile, 2 * kTile, fb);
      bulk_g2s(smem_u32(smem + 2 * kTile), ct + (static_cast<size_t>(jt) * nvc + vc) * 2 * kTile, 2 * kTile, fb);
      ok = mbar_wait(fb, vc & 1, err);
      if (!ok) break;
      fence_after();
      issue_chunk(tmem, smem_u32(smem), smem_u32(smem + kTile), smem_u32(smem + 2 * kTile),
                  smem_u32(smem + 3 * kTile), idesc, vc == 0);
      mma_commit(smem_u32(bars + 1));
    }
  }
  ok = __syncthreads_and(ok) != 0;
  if (ok && nvc > 0) {
    const bool w = mbar_wait(smem_u32(bars + 1), (nvc - 1) & 1, err);
    ok = __syncthreads_and(w) != 0;
  }
  fence_after();
  const int quad = warp & 3, half = warp >> 2;
  const int k = r0 + quad * 32 + lane;   // this thread's row; columns [64 half, 64 half + 64)
  // The TMEM loads are warp-collective: every lane executes the same sequence, and only the
  // global accesses depend on the lane's row (rows past n take part without storing).
  const bool row_ok = k < n;
  if (ok && nvc > 0) {
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32) {
      float old[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int sx = sys[half * 64 + c0 + i];
        old[i] = (row_ok && sx >= 0 && beta != 0.f) ? Y[static_cast<size_t>(sx) * ldy + k] : 0.f;
      }
#pragma unroll
      for (int c1 = 0; c1 < 32; c1 += 16) {
        float v[16];
        tmem_ld16(tmem + (static_cast<uint32_t>(quad * 32) << 16) + half * 64 + c0 + c1, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int sx = sys[half * 64 + c0 + c1 + i];
          if (row_ok && sx >= 0) Y[static_cast<size_t>(sx) * ldy + k] = beta * old[c1 + i] + alpha * v[i];
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// Self-test of the bounded wait: one thread waits on a fresh mbarrier that nothing arrives on;
// after about one second the wait gives up, sets *err and the kernel returns normally.
__global__ void k_tc_wait_selftest(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(smem_u32(&bar), 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_wait(smem_u32(&bar), 0, err);
}

}  // namespace tc

namespace {
struct TcGeom {
  int Nn, ldc, nkc, nrt, nvc, njt, n_kb, kcpb;
};
TcGeom tc_geom(int n, int n_sys, int nv, int split = kTcSplitDefault) {
  TcGeom g;
  g.Nn = (nv + 15) / 16 * 16;
  g.ldc = (nv + 31) / 32 * 32;
  g.nkc = (n + tc::kKC - 1) / tc::kKC;
  g.nrt = (n + tc::kRowsA - 1) / tc::kRowsA;
  g.nvc = g.ldc / tc::kKC;
  g.njt = (n_sys + tc::kRowsA - 1) / tc::kRowsA;
  // About `split` phase-1 CTAs per SM (two resident at a time), each with at least 4 chunks of K
  // and at most kMaxChunksPerBlock: the MMAs accumulate in FP32 inside tensor memory, and over
  // long K runs (15k terms on 30k-element vectors) that sum lost enough accuracy to stall the
  // FP32 inner solves near 1e-5 (three refinements and up to 6x the iterations on the 96^3
  // model); blocks of at most 2048 terms, summed in a fixed order by the reduce, keep the
  // projection FP32-accurate.
  constexpr int kMaxChunksPerBlock = 64;
  int kb = (split * 152 + g.njt - 1) / g.njt;
  kb = std::max(1, std::min(kb, std::max(1, g.nkc / 4)));
  kb = std::max(kb, (g.nkc + kMaxChunksPerBlock - 1) / kMaxChunksPerBlock);
  g.kcpb = (g.nkc + kb - 1) / kb;
  g.n_kb = (g.nkc + g.kcpb - 1) / g.kcpb;
  return g;
}
}  // namespace

size_t tc_psi_tile_bytes(int n, int nv) {
  const TcGeom g = tc_geom(n, 1, nv);
  return static_cast<size_t>(g.nkc) * 2 * g.Nn * 128 + static_cast<size_t>(g.nrt) * g.nvc * 2 * tc::kTile;
}

cudaError_t launch_tc_tile_psi(const float* Psi, long ldp, int n, int nv, unsigned char* tiles, cudaStream_t st) {
  const TcGeom g = tc_geom(n, 1, nv);
  unsigned char* t1 = tiles;
  unsigned char* t2 = tiles + static_cast<size_t>(g.nkc) * 2 * g.Nn * 128;
  cudaError_t e = cudaMemsetAsync(tiles, 0, tc_psi_tile_bytes(n, nv), st);
  if (e != cudaSuccess) return e;
  const long total = static_cast<long>(g.nkc) * tc::kKC * g.Nn;
  tc::k_tc_tile_psi<<<static_cast<int>(std::min<long>((total + 255) / 256, 8192)), 256, 0, st>>>(
      Psi, ldp, n, nv, g.Nn, g.nkc, g.nrt, g.nvc, t1, t2);
  return cudaGetLastError();
}

size_t tc_pc_work_elems(int n, int n_sys, int nv) {
  // Cpart floats, then the split C^T tiles (bytes / 4); room for every split the tuner tries.
  size_t most = 0;
  for (int split = 1; split <= kTcSplitMax; ++split) {
    const TcGeom g = tc_geom(n, n_sys, nv, split);
    most = std::max(most, static_cast<size_t>(g.n_kb) * n_sys * g.ldc +
                              static_cast<size_t>(g.njt) * g.nvc * 2 * tc::kTile / 4);
  }
  return most;
}

bool tc_pc_supported(int nv) { return nv >= 1 && nv <= 256; }

// Yout[s] = beta Yout[s] + alpha M diag(scale) M^T Yin[s] for the systems of a list, M (n x nv) given
// as operand tiles (launch_tc_tile_psi): phase 1 reads Yin, phase 2 updates Yout (which may be Yin).
static cudaError_t launch_tc_pair(const float* Yin, float* Yout, long ldy, int n_sys, const int* list,
                                  const unsigned char* tiles, int n, int nv, const float* scale, float alpha, float beta,
                                  const int* active, float* work, cudaStream_t st, int* err, int split) {
  if (n_sys == 0 || nv == 0) return cudaSuccess;
  if (!tc_pc_supported(nv) || !err || split < 1 || split > kTcSplitMax) return cudaErrorInvalidValue;
  const TcGeom g = tc_geom(n, n_sys, nv, split);
  const unsigned char* t1 = tiles;
  const unsigned char* t2 = tiles + static_cast<size_t>(g.nkc) * 2 * g.Nn * 128;
  float* Cpart = work;
  unsigned char* ct = reinterpret_cast<unsigned char*>(work + static_cast<size_t>(g.n_kb) * n_sys * g.ldc);
  const size_t smem1 = 2u * (2u * tc::kTile + 2u * g.Nn * 128) + 64;
  cudaError_t e = ensure_smem_limit((const void*)tc::k_tc_pc1, smem1);
  if (e != cudaSuccess) return e;
  tc::k_tc_pc1<<<dim3(g.njt, g.n_kb), tc::kThreads, smem1, st>>>(t1, Yin, ldy, n, nv, n_sys, list, g.kcpb, g.Nn,
                                                                 g.ldc, Cpart, err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long total = static_cast<long>(g.njt) * tc::kRowsA * g.nvc * tc::kKC;
  tc::k_tc_reduce<<<static_cast<int>(std::min<long>((total + 255) / 256, 8192)), 256, 0, st>>>(
      Cpart, n_sys, g.ldc, g.n_kb, nv, g.njt, g.nvc, scale, ct);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem2 = 4u * tc::kTile + 64 + tc::kRowsA * sizeof(int);
  e = ensure_smem_limit((const void*)tc::k_tc_pc2, smem2);
  if (e != cudaSuccess) return e;
  tc::k_tc_pc2<<<dim3(g.nrt, g.njt), tc::kThreads2, smem2, st>>>(t2, ct, Yout, ldy, n, g.nvc, n_sys, list, alpha,
                                                                beta, active, err);
  return cudaGetLastError();
}

cudaError_t launch_pc_tc(float* Y, long ldy, int n_sys, const int* list, const unsigned char* tiles, int n, int nv,
                         const int* active, float* work, cudaStream_t st, int* err, int split) {
  return launch_tc_pair(Y, Y, ldy, n_sys, list, tiles, n, nv, nullptr, -1.f, 1.f, active, work, st, err, split);
}

cudaError_t launch_kb_tc(float* Q, const float* P, long ld, int n_sys, const int* list, const unsigned char* tiles,
                         int n, int n_proj, const float* D, const int* active, float* work, cudaStream_t st, int* err,
                         int split) {
  return launch_tc_pair(P, Q, ld, n_sys, list, tiles, n, n_proj, D, 1.f, 1.f, active, work, st, err, split);
}

cudaError_t tc_wait_selftest(int* dev_flag, cudaStream_t st) {
  tc::k_tc_wait_selftest<<<1, 32, 0, st>>>(dev_flag);
  return cudaGetLastError();
}

cudaError_t tc_error_read_and_clear(int* flag, int* dev_flag, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(flag, dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (*flag) e = cudaMemsetAsync(dev_flag, 0, sizeof(int), st);
  return e;
}

}  // namespace wgw
