// Shared device/host helpers for the wgw kernels.
//
// Kernel bodies in this library are written as __host__ __device__ functions
// that take an explicit thread context (thread index, thread count, block
// index).  The __global__ wrappers in the .cu files pass the CUDA built-ins;
// the same bodies can be stepped through on the host with one "thread" per
// block to check index arithmetic (a test harness, never a fallback path).
#pragma once

#include <cstdint>
#include <cstddef>

#include <cuda_runtime.h>

#if defined(__CUDACC__)
#define WGW_HD __host__ __device__ __forceinline__
#else
#define WGW_HD inline
#endif

#if defined(__CUDA_ARCH__)
#define WGW_SYNC() __syncthreads()
#else
#define WGW_SYNC() ((void)0)
#endif

namespace wgw {

constexpr double kInvSqrt2 = 0.70710678118654752440;
constexpr double kSqrt2 = 1.41421356237309504880;

template <typename T>
struct cplx {
  T re, im;
};

template <typename T>
WGW_HD cplx<T> mk(T r, T i) { cplx<T> c; c.re = r; c.im = i; return c; }
template <typename T>
WGW_HD cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk<T>(a.re + b.re, a.im + b.im); }
template <typename T>
WGW_HD cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk<T>(a.re - b.re, a.im - b.im); }
template <typename T>
WGW_HD cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return mk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
WGW_HD cplx<T> cscale(cplx<T> a, T s) { return mk<T>(a.re * s, a.im * s); }
// Multiply by sign * i.
template <typename T>
WGW_HD cplx<T> mul_i(cplx<T> a, int sign) {
  return sign > 0 ? mk<T>(-a.im, a.re) : mk<T>(a.im, -a.re);
}

// Thread context of a kernel body.
struct Thr {
  int tid;       // thread index within the block
  int nth;       // threads per block
};

// Mixed-radix plan of one FFT length: N = prod radix[0..nst-1], radices in {2,3,4,5,8}.
struct FftPlan {
  int n;
  int nst;
  int radix[6];
};

// Sphere <-> grid tables of one plane-wave sphere, built on the host.
//
// The sphere is split into planes of constant h (Miller index along x),
// h = -m..m, plane index hi = h + m.  plane_off[hi]..plane_off[hi+1] index
// `ent`, one entry per sphere point of the plane:
//   ent.x = (k mod N) | (l mod N) << 8 | neg << 16,
//   ent.y = j, the real-basis pair index (0 for G = 0, j >= 1 otherwise);
// neg = 1 when the point is the mirror -G_j of the positive member G_j.
// For h > 0 the plane's entries are all positive members and plane -h lists
// their mirrors in the same order.  Plane 0 lists G = 0 first, then its
// positive members, then their mirrors in the same order.
struct SphereTab {
  int m;            // max |h|, |k|, |l| over the sphere
  int n_pairs;      // number of positive members (real-basis length = 2 n_pairs + 1)
  const int* plane_off;   // 2m+2 entries
  const int2* ent;        // plane_off[2m+1] entries
  const double* g2;       // 0.5 |G|^2 per real-basis element (length 2 n_pairs + 1)
};

}  // namespace wgw
