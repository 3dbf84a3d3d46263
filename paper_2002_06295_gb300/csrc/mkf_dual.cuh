// mkf_dual.cuh -- forward-mode dual number (value, derivative) in FP32, with
// the scalar-dispatch overloads used by the templated Kalman arithmetic.  The
// fit adjoint uses it for the derivatives of the propagation Jacobian with
// respect to the start state and the surface position (second derivatives of
// the propagator), and for the derivatives of the multiple-scattering width.
#pragma once
#include "mkf_device.cuh"

namespace mkf {

struct DF {
  float v, d;
  __device__ __forceinline__ DF() {}
  __device__ __forceinline__ DF(float x) : v(x), d(0.0f) {}
  __device__ __forceinline__ DF(double x) : v((float)x), d(0.0f) {}
  __device__ __forceinline__ DF(float a, float b) : v(a), d(b) {}
};

__device__ __forceinline__ DF operator+(DF a, DF b) { return DF(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return DF(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.v, -a.d); }
__device__ __forceinline__ DF operator*(DF a, DF b) { return DF(a.v * b.v, fmaf(a.d, b.v, a.v * b.d)); }
__device__ __forceinline__ DF operator/(DF a, DF b) {
  const float q = a.v / b.v;
  return DF(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ DF& operator+=(DF& a, DF b) {
  a = a + b;
  return a;
}
__device__ __forceinline__ DF& operator-=(DF& a, DF b) {
  a = a - b;
  return a;
}

__device__ __forceinline__ float vv(DF x) { return x.v; }
__device__ __forceinline__ DF mfma(DF a, DF b, DF c) { return DF(fmaf(a.v, b.v, c.v), fmaf(a.d, b.v, fmaf(a.v, b.d, c.d))); }
__device__ __forceinline__ void msincos(DF x, DF* s, DF* c) {
  float sv, cv;
  sincosf(x.v, &sv, &cv);
  *s = DF(sv, cv * x.d);
  *c = DF(cv, -sv * x.d);
}
__device__ __forceinline__ DF msqrt(DF x) {
  const float r = sqrtf(x.v);
  return DF(r, x.d / (2.0f * r));
}
__device__ __forceinline__ DF mrsqrt(DF x) {
  const float r = rsqrtf(x.v);
  return DF(r, -0.5f * r * r * r * x.d);
}
__device__ __forceinline__ DF matan(DF x) { return DF(atanf(x.v), x.d / fmaf(x.v, x.v, 1.0f)); }
__device__ __forceinline__ DF mlog(DF x) { return DF(logf(x.v), x.d / x.v); }
__device__ __forceinline__ DF mabs(DF x) { return x.v < 0.0f ? -x : x; }
__device__ __forceinline__ DF mrint(DF x) { return DF(rintf(x.v), 0.0f); }
__device__ __forceinline__ DF mcopysign(DF a, DF b) { return (a.v < 0.0f) != (b.v < 0.0f) ? -a : a; }

}  // namespace mkf
