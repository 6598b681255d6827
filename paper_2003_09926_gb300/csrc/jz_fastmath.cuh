// jz_fastmath.cuh -- elementary-function choices of the FP32 and FP64
// arithmetic, shared by the fused stage kernels and the boundary pass.
#pragma once

#include <cmath>

namespace jz {
namespace stg {

// Elementary functions.  FP32 arithmetic uses the hardware approximations
// (sqrt.approx, rcp.approx, ex2/lg2.approx: a few ulp, far below the FP32
// error of the scheme itself); FP64 arithmetic keeps IEEE operations.
template <typename R> struct Fn;
template <> struct Fn<float> {
  static __device__ __forceinline__ float sqrt_(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
  }
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
  // a product that is never fused into a later addition
  static __device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
  // x^e = 2^(e log2 x) for x > 0 (no library call inside the flux code)
  static __device__ __forceinline__ float powp(float x, float e) {
    float l, y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    l *= e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(l));
    return y;
  }
  // J^(-2/3) = 2^(-2/3 log2 J), J > 0
  static __device__ __forceinline__ float jm23(float J) {
    float l, y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(J));
    l *= -2.0f / 3.0f;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(l));
    return y;
  }
};
template <> struct Fn<double> {
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double div(double a, double b) { return a / b; }
  static __device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double powp(double x, double e) { return pow(x, e); }
  static __device__ __forceinline__ double jm23(double J) {
    const double cb = cbrt(J);
    return 1.0 / (cb * cb);
  }
};

}  // namespace stg
}  // namespace jz
