// Shared device helpers of the CUDA path: complex arithmetic on float2/double2
// and the device views of the symbolic plan and of the operator coefficients.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"

namespace fdfd {

template <typename T> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

__device__ __forceinline__ float2 cmk(float r, float i) { return make_float2(r, i); }
__device__ __forceinline__ double2 cmk(double r, double i) { return make_double2(r, i); }

template <typename T> __device__ __forceinline__ T czero() {
  T z; z.x = 0; z.y = 0; return z;
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { a.x += b.x; a.y += b.y; return a; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  T c;
  c.x = a.x * b.x - a.y * b.y;
  c.y = a.x * b.y + a.y * b.x;
  return c;
}
// c + a*b
template <typename T> __device__ __forceinline__ T cfma(T a, T b, T c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
// c - a*b
template <typename T> __device__ __forceinline__ T cfms(T a, T b, T c) {
  c.x = fma(-a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
template <typename T> __device__ __forceinline__ T cconj(T a) { a.y = -a.y; return a; }
template <typename T> __device__ __forceinline__ typename RealOf<T>::type cabs2(T a) {
  return a.x * a.x + a.y * a.y;
}
template <typename T> __device__ __forceinline__ T cscale(T a, typename RealOf<T>::type s) {
  a.x *= s; a.y *= s; return a;
}
// 1 / (a + ib) by Smith's algorithm (R. L. Smith, CACM 5(8), 1962): scale by the
// larger component first so that neither the square nor the quotient overflows.
template <typename T> __device__ __forceinline__ T crcp(T z) {
  using R = typename RealOf<T>::type;
  T r;
  if (fabs(z.x) >= fabs(z.y)) {
    R q = z.y / z.x;
    R d = z.x + z.y * q;
    r.x = R(1) / d;
    r.y = -q / d;
  } else {
    R q = z.x / z.y;
    R d = z.x * q + z.y;
    r.x = q / d;
    r.y = R(-1) / d;
  }
  return r;
}
template <typename T> __device__ __forceinline__ T cfrom(double2 v) {
  T r; r.x = (typename RealOf<T>::type)v.x; r.y = (typename RealOf<T>::type)v.y; return r;
}
template <typename T> __device__ __forceinline__ double2 cto64(T v) {
  return make_double2((double)v.x, (double)v.y);
}

// Device view of the symbolic plan (all arrays are read-only device memory).
struct DevPlan {
  const FrontDesc* fronts;
  const int* children;
  const int* idx;
  const int* inv;
  const int* orig_ptr;
  const int* orig_col;
  const int* orig_code;
  int nx, ny;
};

// Stencil coefficients per wavelength (FP64), see assembly.cu.
struct DevCoef {
  const double2* cxm;    // [n_omega][nx]  A[(i,j),(i-1,j)]
  const double2* cxp;    // [n_omega][nx]  A[(i,j),(i+1,j)]
  const double2* cym;    // [n_omega][ny]  A[(i,j),(i,j-1)]
  const double2* cyp;    // [n_omega][ny]  A[(i,j),(i,j+1)]
  const double* k0dx2;   // [n_omega]      (k0 dx)^2
  const double* eps;     // [nx*ny]        relative permittivity
  const double2* sxc;    // [n_omega][nx]  stretch s_x at cell centres
  const double2* syc;    // [n_omega][ny]  stretch s_y at cell centres
  int nx, ny;
};

// D[cell] = s_x(i + 1/2) s_y(j + 1/2): the diagonal for which D A is complex
// symmetric (discrete reciprocity: the coupling of two neighbours becomes
// -s_y / s_x' (or -s_x / s_y') on both sides of the diagonal).
__device__ __forceinline__ double2 sym_scale(const DevCoef& c, int w, int cell) {
  const int i = cell / c.ny, j = cell - i * c.ny;
  const double2 a = c.sxc[(size_t)w * c.nx + i], b = c.syc[(size_t)w * c.ny + j];
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Value of the stencil entry with code = cell*5 + direction at wavelength w.
__device__ __forceinline__ double2 stencil_entry(const DevCoef& c, int w, int code) {
  int cell = code / 5, dir = code - cell * 5;
  int i = cell / c.ny, j = cell - i * c.ny;
  const double2 xm = c.cxm[(size_t)w * c.nx + i], xp = c.cxp[(size_t)w * c.nx + i];
  const double2 ym = c.cym[(size_t)w * c.ny + j], yp = c.cyp[(size_t)w * c.ny + j];
  switch (dir) {
    case DIR_XM: return xm;
    case DIR_XP: return xp;
    case DIR_YM: return ym;
    case DIR_YP: return yp;
    default: {
      double2 d;
      d.x = -(xm.x + xp.x + ym.x + yp.x) - c.k0dx2[w] * c.eps[cell];
      d.y = -(xm.y + xp.y + ym.y + yp.y);
      return d;
    }
  }
}

}  // namespace fdfd
