// Two FP32 lanes in one value, for kernels that update two lattice nodes per
// thread.  Arithmetic maps to Blackwell's packed FP32x2 instructions (one
// instruction computes both lanes); per-lane operations (reciprocal,
// inverse square root, selects) act on each lane.  The collision templates
// are written against this small interface and also compile for scalar
// float / double (one node per thread).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace lbmk {

struct F2 {
  float2 v;
  __host__ __device__ __forceinline__ F2() {}
  __host__ __device__ __forceinline__ F2(float2 a) : v(a) {}
  __host__ __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  template <typename S>
  __host__ __device__ __forceinline__ explicit F2(S s) : v(make_float2((float)s, (float)s)) {}
};

__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }

// a * b + c, fused
__device__ __forceinline__ F2 fma_(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__host__ __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }

// per-lane flags
struct M2 {
  bool x, y;
};
template <typename R>
struct MaskOf { using type = bool; };
template <>
struct MaskOf<F2> { using type = M2; };

__device__ __forceinline__ bool gt_(double a, double b) { return a > b; }
__device__ __forceinline__ bool gt_(float a, float b) { return a > b; }
__device__ __forceinline__ M2 gt_(F2 a, F2 b) { return M2{a.v.x > b.v.x, a.v.y > b.v.y}; }
__device__ __forceinline__ bool any_(bool m) { return m; }
__device__ __forceinline__ bool any_(M2 m) { return m.x || m.y; }

template <typename R>
__device__ __forceinline__ R select_(bool m, R a, R b) { return m ? a : b; }
__device__ __forceinline__ F2 select_(M2 m, F2 a, F2 b) { return F2(m.x ? a.v.x : b.v.x, m.y ? a.v.y : b.v.y); }

__device__ __forceinline__ F2 rcp_(F2 x) { return F2(__fdividef(1.0f, x.v.x), __fdividef(1.0f, x.v.y)); }
__device__ __forceinline__ F2 rsqrt_(F2 x) { return F2(rsqrtf(x.v.x), rsqrtf(x.v.y)); }
__device__ __forceinline__ F2 sat_(F2 x) { return F2(__saturatef(x.v.x), __saturatef(x.v.y)); }
__device__ __forceinline__ F2 exact_div_(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }

}  // namespace lbmk
