// Device helpers shared by the lane-group solve kernels (complex arithmetic
// on a small struct, precision-generic math, loads and stores of interleaved
// complex arrays, the lane mask of a group).  Internal to libhpt.
#pragma once

#include <math.h>
#include <stdint.h>

namespace hpt {
namespace {

template <typename T>
struct cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> csub_mul(cx<T> acc, cx<T> a, cx<T> b) {  // acc - a b
  return mk<T>(acc.x - (a.x * b.x - a.y * b.y), acc.y - (a.x * b.y + a.y * b.x));
}
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) {
  return mk<T>(a.x * s, a.y * s);
}
template <typename T>
__device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
  const T d = b.x * b.x + b.y * b.y;
  return mk<T>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
template <typename T>
__device__ __forceinline__ cx<T> cmul_conj_scale(cx<T> a, cx<T> b, T r) {   // a conj(b) r
  return mk<T>((a.x * b.x + a.y * b.y) * r, (a.y * b.x - a.x * b.y) * r);
}
template <typename T>
__device__ __forceinline__ T abs2(cx<T> a) {
  return a.x * a.x + a.y * a.y;
}
template <typename T>
__device__ __forceinline__ bool finite(cx<T> a) {
  return isfinite(a.x) && isfinite(a.y);
}
template <typename T, int G>
__device__ __forceinline__ cx<T> shfl(cx<T> v, int src) {
  return mk<T>(__shfl_sync(0xffffffffu, v.x, src, G), __shfl_sync(0xffffffffu, v.y, src, G));
}

__device__ __forceinline__ float t_hypot(float a, float b) { return hypotf(a, b); }
__device__ __forceinline__ double t_hypot(double a, double b) { return hypot(a, b); }
__device__ __forceinline__ float t_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double t_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float t_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double t_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float t_sqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double t_sqrt(double a) { return sqrt(a); }
// Reciprocal on the elimination's critical path: the approximate MUFU
// reciprocal (at most 1 ulp off) for FP32, whose solves the Newton corrector
// refines anyway; a correctly rounded one for FP64.
__device__ __forceinline__ float t_rcp(float a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ double t_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float t_abs(float a) { return fabsf(a); }
__device__ __forceinline__ double t_abs(double a) { return fabs(a); }
// 2^-e for m in [2^(e-1), 2^e): an exact power-of-two scale bringing m to
// [1/2, 1), read off the exponent field (1 for zero, subnormal, inf, NaN).
__device__ __forceinline__ float pow2_inv(float m) {
  const unsigned b = (__float_as_uint(m) >> 23) & 0xffu;
  return (b == 0u || b == 0xffu) ? 1.f : __uint_as_float((253u - min(b, 252u)) << 23);
}
__device__ __forceinline__ double pow2_inv(double m) {
  const unsigned long long b = ((unsigned long long)__double_as_longlong(m) >> 52) & 0x7ffull;
  return (b == 0ull || b == 0x7ffull) ? 1.0
                                      : __longlong_as_double((long long)((2045ull - min(b, 2044ull)) << 52));
}
template <typename T>
__device__ __forceinline__ T cabs_t(cx<T> a) {
  return t_hypot(a.x, a.y);
}
template <typename T>
__device__ __forceinline__ T cmag(cx<T> a) {   // max(|re|, |im|): a cheap magnitude for scaling
  return t_max(t_abs(a.x), t_abs(a.y));
}


template <typename T>
struct cplx_t;
template <>
struct cplx_t<double> {
  typedef double2 type;
};
template <>
struct cplx_t<float> {
  typedef float2 type;
};
template <typename T>
__device__ __forceinline__ cx<T> ld(const void* base, size_t idx) {
  const typename cplx_t<T>::type v = ((const typename cplx_t<T>::type*)base)[idx];
  return mk<T>(v.x, v.y);
}
template <typename T>
__device__ __forceinline__ void st(void* base, size_t idx, cx<T> v) {
  typename cplx_t<T>::type w;
  w.x = v.x;
  w.y = v.y;
  ((typename cplx_t<T>::type*)base)[idx] = w;
}

// Complex FP32 values as packed pairs (re in the low, im in the high half)
// for the paired FP32 instructions of this architecture: one instruction
// rounds each half exactly as the scalar operation would.
__device__ __forceinline__ uint64_t pk2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 upk2(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ uint64_t fma_x2(uint64_t a, uint64_t b, uint64_t c) {   // a * b + c
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t mul_x2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Lanes of the calling thread's G-lane group within its warp.
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  return (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
}

}  // namespace
}  // namespace hpt
