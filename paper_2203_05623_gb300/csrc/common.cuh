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
#include <cmath>

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

// ---------------------------------------------------------------- float-float arithmetic
// A value held as the unevaluated sum hi + lo of two floats, |lo| a few ulp(hi) at most: about 48
// significant bits computed on the FP32 pipes only.  On GB300 the FP64 rate is 1/64 of the
// FP32 rate, so FFT passes that need more than FP32 accuracy run in this format instead of
// FP64.  The operations are the error-free transformations TwoSum (Knuth), Fast2Sum (Dekker)
// and the FMA TwoProduct, combined as in the double-double literature (Dekker 1971; Hida, Li
// and Bailey 2001); additions use the "sloppy" form, whose error is bounded by about 2^-47
// (|a| + |b|), enough for norm-wise stable sums such as FFT butterflies.
// Every primitive below must be evaluated exactly as written: on the device through the
// round-to-nearest intrinsics (never contracted into FMAs), on the host through volatile
// temporaries.
#if defined(__CUDA_ARCH__)
WGW_HD float ffa(float a, float b) { return __fadd_rn(a, b); }
WGW_HD float ffs(float a, float b) { return __fsub_rn(a, b); }
WGW_HD float ffm(float a, float b) { return __fmul_rn(a, b); }
WGW_HD float fff(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
inline float ffa(float a, float b) { volatile float r = a + b; return r; }
inline float ffs(float a, float b) { volatile float r = a - b; return r; }
inline float ffm(float a, float b) { volatile float r = a * b; return r; }
inline float fff(float a, float b, float c) { return std::fmaf(a, b, c); }
#endif

struct alignas(8) ff {
  float hi, lo;
  ff() = default;
  WGW_HD constexpr ff(float h, float l) : hi(h), lo(l) {}
  // Nearest float to d, and the nearest float to the remainder.
  WGW_HD constexpr explicit ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  WGW_HD constexpr explicit ff(int i) : hi((float)i), lo((float)((double)i - (double)(float)i)) {}
  WGW_HD explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (any a, b).
WGW_HD ff two_sum(float a, float b) {
  const float s = ffa(a, b), bb = ffs(s, a);
  return ff(s, ffa(ffs(a, ffs(s, bb)), ffs(b, bb)));
}
// s + e = a + b exactly when the exponent of a is not below that of b.
WGW_HD ff fast_two_sum(float a, float b) {
  const float s = ffa(a, b);
  return ff(s, ffs(b, ffs(s, a)));
}
// The sum is left unnormalised: hi is the rounded sum of the leading parts and lo collects its
// exact rounding error and the low parts (|lo| stays a few ulps of hi).  Every later operation is
// exact in the leading parts (TwoSum) or renormalises (the product), so skipping the final
// Fast2Sum costs no accuracy and saves a quarter of the additions' instructions.
WGW_HD ff operator+(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return ff(s.hi, ffa(s.lo, ffa(a.lo, b.lo)));
}
WGW_HD ff operator-(ff a) { return ff(-a.hi, -a.lo); }
WGW_HD ff operator-(ff a, ff b) { return a + (-b); }
// The product is left unnormalised too (|lo| is within a few ulp(hi)); its error is about 2^-46
// of |a b| plus the norm-wise error the unnormalised operands carry.
WGW_HD ff operator*(ff a, ff b) {
  const float p = ffm(a.hi, b.hi);
  float e = fff(a.hi, b.hi, -p);            // exact low part of a.hi * b.hi
  e = fff(a.hi, b.lo, fff(a.lo, b.hi, e));
  return ff(p, e);
}
// a b + c d: both leading products with their exact low parts, one TwoSum (unnormalised, as the
// sum); 16 FP32 operations instead of the 22 of two products and a sum.
WGW_HD ff ff_dot2(ff a, ff b, ff c, ff d) {
  const float p = ffm(a.hi, b.hi), q = ffm(c.hi, d.hi);
  float e = fff(a.hi, b.hi, -p);
  float f = fff(c.hi, d.hi, -q);
  e = fff(a.hi, b.lo, fff(a.lo, b.hi, e));
  f = fff(c.hi, d.lo, fff(c.lo, d.hi, f));
  const ff s = two_sum(p, q);
  return ff(s.hi, ffa(s.lo, ffa(e, f)));
}
WGW_HD ff& operator+=(ff& a, ff b) { a = a + b; return a; }
WGW_HD ff& operator*=(ff& a, ff b) { a = a * b; return a; }

// acc += a * b.  The float-float form keeps the running sum unnormalised (acc.hi holds the
// rounded sum of the leading products, acc.lo collects their exact rounding errors and the low
// parts), which is accurate to about 2^-47 of the magnitudes summed for sums of thousands of
// terms; convert with double(acc).
WGW_HD void mac(float& acc, float a, float b) { acc += a * b; }
WGW_HD void mac(double& acc, double a, double b) { acc += a * b; }
WGW_HD void mac(ff& acc, ff a, ff b) {
  const float p = ffm(a.hi, b.hi);
  float e = fff(a.hi, b.hi, -p);
  e = fff(a.hi, b.lo, fff(a.lo, b.hi, e));
  const ff s = two_sum(acc.hi, p);
  acc.hi = s.hi;
  acc.lo = ffa(acc.lo, ffa(s.lo, e));
}

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
template <>
WGW_HD cplx<ff> cmul<ff>(cplx<ff> a, cplx<ff> b) {
  return mk<ff>(ff_dot2(a.re, b.re, -a.im, b.im), ff_dot2(a.re, b.im, a.im, b.re));
}
template <typename T>
WGW_HD cplx<T> cscale(cplx<T> a, T s) { return mk<T>(a.re * s, a.im * s); }
// Multiply by sign * i.
template <typename T>
WGW_HD cplx<T> mul_i(cplx<T> a, int sign) {
  return sign > 0 ? mk<T>(-a.im, a.re) : mk<T>(a.im, -a.re);
}

// Complex sum, difference and real scaling with a packing choice P: P = false is the scalar
// form; P = true on FP32 values computes each as one f32x2 instruction (sm_100 and later) instead
// of two scalar ones, with the same round-to-nearest result per component.  The FFT butterflies
// are mostly such operations; kernels pick P where it measured faster.
#ifndef WGW_F32X2
#define WGW_F32X2 1
#endif
template <bool P, typename T>
WGW_HD cplx<T> cadd(cplx<T> a, cplx<T> b) { return a + b; }
template <bool P, typename T>
WGW_HD cplx<T> csub(cplx<T> a, cplx<T> b) { return a - b; }
template <bool P, typename T>
WGW_HD cplx<T> cscl(cplx<T> a, T s) { return cscale(a, s); }
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && WGW_F32X2
__device__ __forceinline__ unsigned long long pk_f32x2(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ cplx<float> upk_f32x2(unsigned long long r) {
  cplx<float> c;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(c.re), "=f"(c.im) : "l"(r));
  return c;
}
template <>
__device__ __forceinline__ cplx<float> cadd<true, float>(cplx<float> a, cplx<float> b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk_f32x2(a.re, a.im)), "l"(pk_f32x2(b.re, b.im)));
  return upk_f32x2(r);
}
template <>
__device__ __forceinline__ cplx<float> csub<true, float>(cplx<float> a, cplx<float> b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk_f32x2(a.re, a.im)), "l"(pk_f32x2(b.re, b.im)));
  return upk_f32x2(r);
}
template <>
__device__ __forceinline__ cplx<float> cscl<true, float>(cplx<float> a, float s) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk_f32x2(a.re, a.im)), "l"(pk_f32x2(s, s)));
  return upk_f32x2(r);
}
#endif

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
  const float* g2f;       // the same rounded to FP32 (for the FP32 kernels)
};

}  // namespace wgw
