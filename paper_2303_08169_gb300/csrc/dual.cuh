// dual.cuh - tangent (forward-mode) numbers for the second-order adjoint.
//
// The force term of the SAM loss (Eq. 3 with L_F = c sum_i |F_i - F*_i|^2,
// F = -dE/dr, Eq. 1) has the weight gradient
//     dL_F/dw = -d/dw (v . dE/dr),   v = 2 c (F - F*)   (held fixed),
// the derivative along v of the weight adjoint.  The FP32 pass kernels are
// templated on their scalar type; instantiated with Dual, every quantity x
// carries its value and its tangent x' = d x / d h along r + h v, so one pass
// sequence returns the weight adjoint and its exact derivative along v (the
// "R-operator" applied to the hand-written adjoint).  Weights are plain
// floats (tangent zero).
#pragma once
#include <cuda_runtime.h>

#define AL_DEV __device__ __forceinline__

namespace al {

// the float versions stay visible beside the Dual overloads declared here
using ::fmaf;
using ::sqrtf;

// float versions of the intrinsics used by the templated helpers
AL_DEV float fexp(float a) { return __expf(a); }
AL_DEV float frcp(float a) { return __frcp_rn(a); }
AL_DEV void fsincospi(float a, float* s, float* c) { sincospif(a, s, c); }
AL_DEV float shfl_xor(unsigned mask, float a, int o) { return __shfl_xor_sync(mask, a, o); }

struct Dual {
  float v;   // value
  float t;   // tangent
  Dual() = default;
  AL_DEV constexpr Dual(float a) : v(a), t(0.0f) {}
  AL_DEV constexpr Dual(float a, float b) : v(a), t(b) {}
};

AL_DEV Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.t + b.t}; }
AL_DEV Dual operator+(Dual a, float b) { return {a.v + b, a.t}; }
AL_DEV Dual operator+(float a, Dual b) { return {a + b.v, b.t}; }
AL_DEV Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.t - b.t}; }
AL_DEV Dual operator-(Dual a, float b) { return {a.v - b, a.t}; }
AL_DEV Dual operator-(float a, Dual b) { return {a - b.v, -b.t}; }
AL_DEV Dual operator-(Dual a) { return {-a.v, -a.t}; }
AL_DEV Dual operator*(Dual a, Dual b) { return {a.v * b.v, fmaf(a.t, b.v, a.v * b.t)}; }
AL_DEV Dual operator*(Dual a, float b) { return {a.v * b, a.t * b}; }
AL_DEV Dual operator*(float a, Dual b) { return {a * b.v, a * b.t}; }
AL_DEV Dual operator/(Dual a, Dual b) {
  const float q = a.v / b.v;
  return {q, (a.t - q * b.t) / b.v};
}
AL_DEV Dual operator/(Dual a, float b) { return {a.v / b, a.t / b}; }
AL_DEV Dual operator/(float a, Dual b) {
  const float q = a / b.v;
  return {q, -q * b.t / b.v};
}
AL_DEV Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
AL_DEV Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
AL_DEV Dual& operator*=(Dual& a, Dual b) { return a = a * b; }
AL_DEV bool operator>=(Dual a, float b) { return a.v >= b; }

AL_DEV Dual fmaf(Dual a, Dual b, Dual c) { return {fmaf(a.v, b.v, c.v), fmaf(a.t, b.v, fmaf(a.v, b.t, c.t))}; }
AL_DEV Dual fmaf(Dual a, float b, Dual c) { return {fmaf(a.v, b, c.v), fmaf(a.t, b, c.t)}; }
AL_DEV Dual fmaf(float a, Dual b, Dual c) { return {fmaf(a, b.v, c.v), fmaf(a, b.t, c.t)}; }
AL_DEV Dual sqrtf(Dual a) {
  const float s = ::sqrtf(a.v);
  return {s, 0.5f * a.t / s};
}
AL_DEV Dual fexp(Dual a) {
  const float e = __expf(a.v);
  return {e, e * a.t};
}
AL_DEV Dual frcp(Dual a) {
  const float r = __frcp_rn(a.v);
  return {r, -r * r * a.t};
}
// (sin pi a, cos pi a)
AL_DEV void fsincospi(Dual a, Dual* s, Dual* c) {
  float sv, cv;
  sincospif(a.v, &sv, &cv);
  const float k = 3.14159265358979323846f * a.t;
  *s = Dual(sv, cv * k);
  *c = Dual(cv, -sv * k);
}
AL_DEV Dual shfl_xor(unsigned mask, Dual a, int o) {
  return {__shfl_xor_sync(mask, a.v, o), __shfl_xor_sync(mask, a.t, o)};
}

// value and tangent parts of a float or Dual
AL_DEV float val(float a) { return a; }
AL_DEV float val(Dual a) { return a.v; }
AL_DEV float tan_part(float) { return 0.0f; }
AL_DEV float tan_part(Dual a) { return a.t; }

template <class T> struct is_dual { static constexpr bool value = false; };
template <> struct is_dual<Dual> { static constexpr bool value = true; };

// non-deduced context for template arguments
template <class X> struct nodeduce { using type = X; };

}  // namespace al
