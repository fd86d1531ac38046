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
// wait on that mbarrier is bounded and reports a timeout through g_tc_error.
#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace wgw {

__device__ int g_tc_error = 0;

namespace tc {

constexpr int kThreads = 128;    // 4 warps: warp w reads TMEM lanes 32w..32w+31
constexpr int kKC = 32;          // K elements per staged chunk (8 core matrices of 4 TF32)
constexpr int kRowsA = 128;      // M of every MMA
constexpr uint32_t kCoreBytes = 128;
constexpr uint32_t kLbo = kCoreBytes;             // K-adjacent core matrices
constexpr uint32_t kSbo = (kKC / 4) * kCoreBytes; // M/N-adjacent core matrices (8 rows)
constexpr long kWaitLimit = 1L << 26;

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

// Bounded wait for the completion of phase `parity`; false (and g_tc_error set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (long i = 0; i < kWaitLimit; ++i)
    if (mbar_test(mbar, parity)) return true;
  atomicExch(&g_tc_error, 1);
  return false;
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

// Phase 1.  Grid (ceil(n_list / 128), n_kb).  Cpart[kb][j][v] (row length ldc) for j < n_list,
// v < ldc (zero for v >= nv).  N = states padded to 16 (<= 256).
__global__ void __launch_bounds__(kThreads) k_tc_pc1(const float* __restrict__ Psi, long ldp,
                                                     const float* __restrict__ Y, long ldy, int n, int nv,
                                                     int n_list, const int* __restrict__ list, int kblk, int N,
                                                     int ldc, float* __restrict__ Cpart) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j0 = blockIdx.x * kRowsA, kb = blockIdx.y;
  const int k_lo = kb * kblk, k_hi = min(n, k_lo + kblk);
  const uint32_t a_bytes = kRowsA * kKC * 4, b_bytes = static_cast<uint32_t>(N) * kKC * 4;
  unsigned char* a_hi = smem;
  unsigned char* a_lo = a_hi + a_bytes;
  unsigned char* b_hi = a_lo + a_bytes;
  unsigned char* b_lo = b_hi + b_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + b_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  uint32_t ncols = 32;
  while (ncols < static_cast<uint32_t>(N)) ncols <<= 1;
  if (warp == 0) tmem_alloc(tslot, ncols);
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_tf32(kRowsA, N);
  // A rows: systems j0 + r (r < 128); thread -> (rr, kq, half) with 8 rows per pass.
  const int rr = tid & 7, kq = (tid >> 3) & 7, mg0 = tid >> 6;
  uint32_t parity = 0;
  bool ok = true;
  int chunk = 0;
  for (int k0 = k_lo; k0 < k_hi; k0 += kKC, ++chunk) {
    if (chunk > 0) {
      const bool w = mbar_wait(smem_u32(mbar), parity);
      parity ^= 1u;
      ok = __syncthreads_and(w) != 0;
      if (!ok) break;
    }
    for (int mg = mg0; mg < kRowsA / 8; mg += 2) {
      const int r = mg * 8 + rr, j = j0 + r;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < n_list) {
        const int s = list ? list[j] : j;
        v = load4(Y + static_cast<size_t>(s) * ldy, k0 + kq * 4, k_hi);
      }
      put4(a_hi, a_lo, r, kq * 4, v);
    }
    for (int mg = mg0; mg < N / 8; mg += 2) {
      const int r = mg * 8 + rr;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < nv) v = load4(Psi + static_cast<size_t>(r) * ldp, k0 + kq * 4, k_hi);
      put4(b_hi, b_lo, r, kq * 4, v);
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      issue_chunk(tmem, smem_u32(a_hi), smem_u32(a_lo), smem_u32(b_hi), smem_u32(b_lo), idesc, chunk == 0);
      mma_commit(smem_u32(mbar));
    }
  }
  if (ok && chunk > 0) {
    const bool w = mbar_wait(smem_u32(mbar), parity);
    ok = __syncthreads_and(w) != 0;
  }
  fence_after();
  // Epilogue: lane (32 warp + lane) = system j0 + that; columns = states.
  const int j = j0 + warp * 32 + lane;
  float* out = Cpart + (static_cast<size_t>(kb) * n_list + (j < n_list ? j : 0)) * ldc;
  for (int c0 = 0; c0 < ldc; c0 += 16) {
    float v[16];
    if (ok && chunk > 0 && c0 < N) {
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

// C^T[j][v] = sum_kb Cpart[kb][j][v], fixed order (in place into slice 0).
__global__ void k_tc_reduce(float* __restrict__ Cpart, size_t slice, int n_kb) {
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < slice;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    float s = Cpart[e];
    for (int kb = 1; kb < n_kb; ++kb) s += Cpart[static_cast<size_t>(kb) * slice + e];
    Cpart[e] = s;
  }
}

// Phase 2.  Grid (ceil(n / 128), ceil(n_list / 128)).  D = rows k0..k0+127 x systems j0..j0+127,
// K = states in chunks of 32 (Ct row length ldc, a multiple of 32).
__global__ void __launch_bounds__(kThreads) k_tc_pc2(const float* __restrict__ Psi, long ldp, float* __restrict__ Y,
                                                     long ldy, int n, int nv, int n_list,
                                                     const int* __restrict__ list, const float* __restrict__ Ct,
                                                     int ldc, float alpha, float beta,
                                                     const int* __restrict__ active) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = blockIdx.x * kRowsA, j0 = blockIdx.y * kRowsA;
  const uint32_t t_bytes = kRowsA * kKC * 4;
  unsigned char* a_hi = smem;
  unsigned char* a_lo = a_hi + t_bytes;
  unsigned char* b_hi = a_lo + t_bytes;
  unsigned char* b_lo = b_hi + t_bytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + t_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  if (active) {   // skip tiles whose systems are all finished
    int any = 0;
    for (int t = tid; t < kRowsA && j0 + t < n_list; t += kThreads) any |= active[list ? list[j0 + t] : j0 + t];
    if (!__syncthreads_or(any)) return;
  }
  const uint32_t ncols = kRowsA;
  if (warp == 0) tmem_alloc(tslot, ncols);
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_tf32(kRowsA, kRowsA);
  uint32_t parity = 0;
  bool ok = true;
  int chunk = 0;
  for (int v0 = 0; v0 < nv; v0 += kKC, ++chunk) {
    if (chunk > 0) {
      const bool w = mbar_wait(smem_u32(mbar), parity);
      parity ^= 1u;
      ok = __syncthreads_and(w) != 0;
      if (!ok) break;
    }
    // A: rows k (M) x states (K) from Psi[v][k]: thread -> state vv = tid & 31, rows in quads.
    {
      const int vv = tid & 31, v = v0 + vv;
      const float* col = Psi + static_cast<size_t>(v < nv ? v : 0) * ldp;
      for (int q = tid >> 5; q < kRowsA / 4; q += kThreads / 32) {
        const int r = q * 4, k = r0 + r;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v < nv) x = load4(col, k, n);
        put1(a_hi, a_lo, r + 0, vv, x.x);
        put1(a_hi, a_lo, r + 1, vv, x.y);
        put1(a_hi, a_lo, r + 2, vv, x.z);
        put1(a_hi, a_lo, r + 3, vv, x.w);
      }
    }
    // B: systems j (N) x states (K) from Ct[j][v] (row length ldc >= v0 + 32).
    {
      const int rr = tid & 7, kq = (tid >> 3) & 7, mg0 = tid >> 6;
      for (int mg = mg0; mg < kRowsA / 8; mg += 2) {
        const int r = mg * 8 + rr, j = j0 + r;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < n_list) x = *reinterpret_cast<const float4*>(Ct + static_cast<size_t>(j) * ldc + v0 + kq * 4);
        put4(b_hi, b_lo, r, kq * 4, x);
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      issue_chunk(tmem, smem_u32(a_hi), smem_u32(a_lo), smem_u32(b_hi), smem_u32(b_lo), idesc, chunk == 0);
      mma_commit(smem_u32(mbar));
    }
  }
  if (ok && chunk > 0) {
    const bool w = mbar_wait(smem_u32(mbar), parity);
    ok = __syncthreads_and(w) != 0;
  }
  fence_after();
  const int k = r0 + warp * 32 + lane;   // this thread's row
  if (ok && chunk > 0) {
    for (int c0 = 0; c0 < kRowsA; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int j = j0 + c0 + i;
        if (j >= n_list || k >= n) continue;
        const int s = list ? list[j] : j;
        if (active && !active[s]) continue;
        float* y = Y + static_cast<size_t>(s) * ldy + k;
        *y = (beta != 0.f ? beta * *y : 0.f) + alpha * v[i];
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace tc

size_t tc_pc_work_elems(int n, int n_sys, int nv) {
  const int ldc = (nv + 31) / 32 * 32;
  return static_cast<size_t>(pc_kblocks(n, n_sys)) * n_sys * ldc;
}

bool tc_pc_supported(int nv) { return nv >= 1 && nv <= 256; }

cudaError_t launch_pc_tc(float* Y, long ldy, int n_sys, const int* list, const float* Psi, long ldp, int n, int nv,
                         const int* active, float* work, cudaStream_t st) {
  if (n_sys == 0 || nv == 0) return cudaSuccess;
  if (!tc_pc_supported(nv)) return cudaErrorInvalidValue;
  const int n_kb = pc_kblocks(n, n_sys);
  const int kblk = ((n + n_kb - 1) / n_kb + tc::kKC - 1) / tc::kKC * tc::kKC;
  const int N = (nv + 15) / 16 * 16;
  const int ldc = (nv + 31) / 32 * 32;
  const size_t smem1 = 2u * (tc::kRowsA + N) * tc::kKC * 4 + 16;
  cudaError_t e1 = cudaFuncSetAttribute(tc::k_tc_pc1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(2u * (tc::kRowsA + 256) * tc::kKC * 4 + 16));
  if (e1 != cudaSuccess) return e1;
  dim3 g1((n_sys + tc::kRowsA - 1) / tc::kRowsA, n_kb);
  tc::k_tc_pc1<<<g1, tc::kThreads, smem1, st>>>(Psi, ldp, Y, ldy, n, nv, n_sys, list, kblk, N, ldc, work);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const size_t slice = static_cast<size_t>(n_sys) * ldc;
  if (n_kb > 1) {
    tc::k_tc_reduce<<<static_cast<int>(std::min<size_t>((slice + 255) / 256, 4096)), 256, 0, st>>>(work, slice, n_kb);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  const size_t smem2 = 4u * tc::kRowsA * tc::kKC * 4 + 16;
  cudaError_t e2 = cudaFuncSetAttribute(tc::k_tc_pc2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        static_cast<int>(smem2));
  if (e2 != cudaSuccess) return e2;
  dim3 g2((n + tc::kRowsA - 1) / tc::kRowsA, (n_sys + tc::kRowsA - 1) / tc::kRowsA);
  tc::k_tc_pc2<<<g2, tc::kThreads, smem2, st>>>(Psi, ldp, Y, ldy, n, nv, n_sys, list, work, ldc, -1.f, 1.f, active);
  return cudaGetLastError();
}

cudaError_t tc_error_read_and_clear(int* flag, cudaStream_t st) {
  cudaError_t e = cudaMemcpyFromSymbolAsync(flag, g_tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (*flag) {
    const int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  }
  return e;
}

}  // namespace wgw
