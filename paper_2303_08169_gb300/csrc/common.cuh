// common.cuh - shared device helpers for the Allegro GB300 kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "dual.cuh"

namespace al {

constexpr float kSqrt3 = 1.7320508075688772f;
constexpr float kSqrt5 = 2.2360679774997896f;
constexpr float kSqrt15 = 3.8729833462074170f;
constexpr float kPi = 3.14159265358979323846f;

// Image vector packed in one int32: (n_x + 2) * 25 + (n_y + 2) * 5 + (n_z + 2),
// |n_a| <= 2.  The same code orders pairs inside a CSR row.
AL_DEV int img_code(int nx, int ny, int nz) { return (nx + 2) * 25 + (ny + 2) * 5 + (nz + 2); }
AL_DEV void img_decode(int c, int& nx, int& ny, int& nz) {
  nx = c / 25 - 2;
  ny = (c / 5) % 5 - 2;
  nz = c % 5 - 2;
}
AL_DEV int img_code_neg(int c) {
  int nx, ny, nz;
  img_decode(c, nx, ny, nz);
  return img_code(-nx, -ny, -nz);
}

// Box description (orthorhombic), FP64.
struct Box {
  double L[3];
};

// Pair separation Delta = (w_j - w_i) + n L with every operation rounded in
// FP64 (no contraction), the same arithmetic that decides pair membership.
AL_DEV void pair_delta(const double* __restrict__ w, int i, int j, int code, const Box& box,
                       double d[3]) {
  int n[3];
  img_decode(code, n[0], n[1], n[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    d[a] = __dadd_rn(__dsub_rn(w[3 * j + a], w[3 * i + a]), (double)n[a] * box.L[a]);
}

// Real spherical harmonics in component normalisation (sum_m Y_lm^2 = 2l+1),
// index l*l + m + l, for a unit vector (x, y, z):
//   Y_0 = 1; Y_1 = sqrt3 (y, z, x);
//   Y_2 = (sqrt15 xy, sqrt15 yz, sqrt5/2 (3z^2 - 1), sqrt15 xz, sqrt15/2 (x^2 - y^2)).
// (T is float, or Dual for the tangent passes of the second-order adjoint.)
template <int LMAX, class T>
AL_DEV void sph_harm(T x, T y, T z, T* Y) {
  Y[0] = 1.0f;
  if (LMAX >= 1) {
    Y[1] = kSqrt3 * y;
    Y[2] = kSqrt3 * z;
    Y[3] = kSqrt3 * x;
  }
  if (LMAX >= 2) {
    Y[4] = kSqrt15 * x * y;
    Y[5] = kSqrt15 * y * z;
    Y[6] = 0.5f * kSqrt5 * (3.0f * z * z - 1.0f);
    Y[7] = kSqrt15 * x * z;
    Y[8] = 0.5f * kSqrt15 * (x * x - y * y);
  }
}

// g_u = sum_lm dY[lm] * dY_lm/du (gradient of the polynomial forms w.r.t. the
// unit-vector components, before projection onto the sphere's tangent).
template <int LMAX, class T>
AL_DEV void sph_harm_vjp(T x, T y, T z, const T* dY, T g[3]) {
  g[0] = g[1] = g[2] = T(0.0f);
  if (LMAX >= 1) {
    g[1] += kSqrt3 * dY[1];
    g[2] += kSqrt3 * dY[2];
    g[0] += kSqrt3 * dY[3];
  }
  if (LMAX >= 2) {
    g[0] += kSqrt15 * (y * dY[4] + z * dY[7] + x * dY[8]);
    g[1] += kSqrt15 * (x * dY[4] + z * dY[5] - y * dY[8]);
    g[2] += kSqrt15 * (y * dY[5] + x * dY[7]) + 3.0f * kSqrt5 * z * dY[6];
  }
}

// Bessel radial basis B_n(d) = sqrt(2/rc) sin(n pi d / rc) / d, n = 1..NB, and
// dB_n/dd, through the angle-addition recurrence from sincospi(d/rc).
template <int NB, class T>
AL_DEV void bessel(T d, float rc, T* B, typename nodeduce<T>::type* dB) {
  const float c = sqrtf(2.0f / rc);
  const T t = d / rc;
  T s1, c1;
  fsincospi(t, &s1, &c1);
  T sn = s1, cn = c1;
  const T inv_d = 1.0f / d;
#pragma unroll
  for (int n = 1; n <= NB; ++n) {
    B[n - 1] = c * sn * inv_d;
    if (dB) dB[n - 1] = c * ((float)n * kPi / rc * cn - sn * inv_d) * inv_d;
    const T s2 = sn * c1 + cn * s1;
    const T c2 = cn * c1 - sn * s1;
    sn = s2;
    cn = c2;
  }
}

// Polynomial envelope (p = 6): u(x) = 1 - 28 x^6 + 48 x^7 - 21 x^8, x = d/rc,
// and du/dd = (-168 x^5 + 336 x^6 - 168 x^7) / rc.
// (zero at and beyond r_c, where a pair contributes nothing: C^2 continuous)
template <class T>
AL_DEV void envelope(T d, float rc, T& u, T& du) {
  if (d >= rc) {
    u = T(0.0f);
    du = T(0.0f);
    return;
  }
  const T x = d / rc;
  const T x2 = x * x, x5 = x2 * x2 * x, x6 = x5 * x;
  u = 1.0f + x6 * (-28.0f + x * (48.0f - 21.0f * x));
  du = x5 * (-168.0f + x * (336.0f - 168.0f * x)) / rc;
}

template <class T>
AL_DEV T sigmoidf_(T z) { return frcp(1.0f + fexp(-z)); }
template <class T>
AL_DEV T silu(T z) { return z * sigmoidf_(z); }
// d silu / dz = s (1 + z (1 - s)), s = sigmoid(z)
template <class T>
AL_DEV T silu_grad(T z) {
  const T s = sigmoidf_(z);
  return s * (1.0f + z * (1.0f - s));
}

}  // namespace al
