// pma_device.cuh -- device helpers of the DDPMA sweep: math traits, the
// monitor densities and index helpers.  Included by the kernel TUs only.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pma_internal.h"

namespace pma {

// ---------------------------------------------------------------- math
// FP32 uses the SFU approximations (ex2/lg2/sin), FP64 the accurate library
// functions.
template <typename T>
struct Fm;

template <>
struct Fm<float> {
  __device__ __forceinline__ static float ex(float x) { return __expf(x); }
  __device__ __forceinline__ static float ln(float x) { return __logf(x); }
  __device__ __forceinline__ static float sinpi(float x) { return sinpif(x); }
  __device__ __forceinline__ static float cospi(float x) { return cospif(x); }
  __device__ __forceinline__ static float sq(float x) { return sqrtf(x); }
  __device__ __forceinline__ static float at2(float y, float x) { return atan2f(y, x); }
  __device__ __forceinline__ static float cs(float x) { return cosf(x); }
  __device__ __forceinline__ static float sn(float x) { return sinf(x); }
  __device__ __forceinline__ static float pw(float x, float y) { return __powf(x, y); }
};

template <>
struct Fm<double> {
  __device__ __forceinline__ static double ex(double x) { return exp(x); }
  __device__ __forceinline__ static double ln(double x) { return log(x); }
  __device__ __forceinline__ static double sinpi(double x) { return ::sinpi(x); }
  __device__ __forceinline__ static double cospi(double x) { return ::cospi(x); }
  __device__ __forceinline__ static double sq(double x) { return sqrt(x); }
  __device__ __forceinline__ static double at2(double y, double x) { return atan2(y, x); }
  __device__ __forceinline__ static double cs(double x) { return cos(x); }
  __device__ __forceinline__ static double sn(double x) { return sin(x); }
  __device__ __forceinline__ static double pw(double x, double y) { return pow(x, y); }
};

// ---------------------------------------------------------------- monitor
// Parameters of one problem's density converted to the sweep precision,
// staged in shared memory once per tile.
template <typename T>
struct MonT {
  int kind, nterms, dim, pad;
  T base, p0;
  struct Term {
    int type, axis, along, pad;
    T amp, width, r2, a, k2;  // k2 = 2k: sin(2 pi k s) = sinpi(k2 s)
    T c[3];
  } t[kMaxTerms];
};

template <typename T>
__device__ __forceinline__ void mon_load(MonT<T>& m, const MonDev& d, int dim) {
  m.kind = d.kind;
  m.nterms = d.nterms;
  m.dim = dim;
  m.base = (T)d.base;
  m.p0 = (T)d.p0;
  for (int i = 0; i < kMaxTerms; ++i) {
    m.t[i].type = d.t[i].type;
    m.t[i].axis = d.t[i].axis;
    m.t[i].along = d.t[i].along;
    m.t[i].amp = (T)d.t[i].amp;
    m.t[i].width = (T)d.t[i].width;
    m.t[i].r2 = (T)d.t[i].r2;
    m.t[i].a = (T)d.t[i].a;
    m.t[i].k2 = (T)(2.0 * d.t[i].k);
    for (int a = 0; a < 3; ++a) m.t[i].c[a] = (T)d.t[i].c[a];
  }
}

// sech^2(z) = 4 e^{-2|z|} / (1 + e^{-2|z|})^2, overflow-free.
template <typename T>
__device__ __forceinline__ T sech2(T z) {
  T e = Fm<T>::ex(-2 * fabs(z));
  T d = 1 + e;
  return 4 * e / (d * d);
}

template <typename T>
__device__ __forceinline__ T term_value(const typename MonT<T>::Term& t, int dim, const T* x) {
  T q = 0;
  switch (t.type) {
    case PMA_TERM_BUMP:
      for (int a = 0; a < 3; ++a)
        if (a < dim) {
          T d = x[a] - t.c[a];
          q = fma(d, d, q);
        }
      return t.amp * Fm<T>::ex(-t.width * q);
    case PMA_TERM_RING: {
      for (int a = 0; a < 3; ++a)
        if (a < dim) {
          T d = x[a] - t.c[a];
          q = fma(d, d, q);
        }
      T s = q - t.r2;
      return t.amp * Fm<T>::ex(-t.width * s * s);
    }
    case PMA_TERM_SINE: {
      T s = x[t.axis] - t.c[t.axis] - t.a * Fm<T>::sinpi(t.k2 * x[t.along]);
      return t.amp * Fm<T>::ex(-t.width * s * s);
    }
    case PMA_TERM_BUMP1: {
      T s = x[t.axis] - t.c[t.axis];
      return t.amp * Fm<T>::ex(-t.width * s * s);
    }
  }
  return T(0);
}

// rho = sqrt(1 + |grad u|^2) for the test functions of Sect. 4.
template <typename T>
__device__ T arclen_rho(const MonT<T>& m, const T* x) {
  T g0 = 0, g1 = 0, g2 = 0;
  switch (m.kind) {
    case PMA_MON_ARCLEN_BURGERS: {
      T eps = m.p0;
      T s = (x[0] + x[1] - 1) / (2 * eps);
      T d = -T(0.25) * sech2<T>(T(0.5) * s) / (2 * eps);
      g0 = d;
      g1 = d;
      break;
    }
    case PMA_MON_ARCLEN_SPIRAL: {
      T dx = x[0] - T(0.7), dy = x[1] - T(0.5);
      T r2 = dx * dx + dy * dy;
      T phi = Fm<T>::at2(dy, dx) - 20 * r2;
      T cp = Fm<T>::cs(phi), s2 = Fm<T>::sn(2 * phi);
      T q = 100 * r2 * cp * cp;
      T gqx = 100 * (2 * cp * cp * dx - s2 * (-dy - 40 * r2 * dx));
      T gqy = 100 * (2 * cp * cp * dy - s2 * (dx - 40 * r2 * dy));
      T f = -9 / ((1 + q) * (1 + q));
      g0 = f * gqx;
      g1 = f * gqy;
      break;
    }
    case PMA_MON_ARCLEN_TANH_SPHERE: {
      T r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
      T f = 200 * sech2<T>(100 * (r2 - T(0.125)));
      g0 = f * x[0];
      g1 = f * x[1];
      g2 = f * x[2];
      break;
    }
    case PMA_MON_ARCLEN_NINE_SPHERES: {
      for (int k = 0; k < 9; ++k) {
        T cx = (k == 0) ? T(0) : ((k == 1 || k == 2 || k == 5 || k == 6) ? T(0.5) : T(-0.5));
        T cy = (k == 0) ? T(0) : ((k & 1) ? T(0.5) : T(-0.5));
        T cz = (k == 0) ? T(0) : (k <= 4 ? T(0.5) : T(-0.5));
        T ex = x[0] - cx, ey = x[1] - cy, ez = x[2] - cz;
        T f = 100 * sech2<T>(50 * (ex * ex + ey * ey + ez * ez - T(0.1875)));
        g0 += f * ex;
        g1 += f * ey;
        g2 += f * ez;
      }
      break;
    }
  }
  return Fm<T>::sq(1 + g0 * g0 + g1 * g1 + g2 * g2);
}

template <typename T>
__device__ __forceinline__ T rho_at(const MonT<T>& m, const T* x) {
  if (m.kind == PMA_MON_SUM) {
    T r = m.base;
    for (int i = 0; i < kMaxTerms; ++i)
      if (i < m.nterms) r += term_value<T>(m.t[i], m.dim, x);
    return r;
  }
  if (m.kind == PMA_MON_PRODUCT) {
    T r = 1;
    for (int i = 0; i < kMaxTerms; ++i)
      if (i < m.nterms) r *= m.base + term_value<T>(m.t[i], m.dim, x);
    return r;
  }
  return arclen_rho<T>(m, x);
}

// ---------------------------------------------------------------- indices
// Mirror ghost across a Neumann face (index -1 -> 1, n -> n-2), clamp
// across a transmission face or beyond the subdomain (those values are
// never used by an updated node).
__device__ __forceinline__ int reflect_clamp(int i, int n, bool phys_lo, bool phys_hi) {
  if (i < 0) i = phys_lo ? -i : 0;
  if (i >= n) i = phys_hi ? 2 * (n - 1) - i : n - 1;
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Transmission (Dirichlet) node: on a face of the subdomain that is not a
// face of Omega_c.
__device__ __forceinline__ bool is_dir(int faces, int dim, int i, int j, int l, int n0, int n1,
                                       int n2) {
  bool d = (i == 0 && !(faces & 1)) || (i == n0 - 1 && !(faces & 2));
  if (dim > 1) d = d || (j == 0 && !(faces & 4)) || (j == n1 - 1 && !(faces & 8));
  if (dim > 2) d = d || (l == 0 && !(faces & 16)) || (l == n2 - 1 && !(faces & 32));
  return d;
}

__device__ __forceinline__ double trap_w(int gi, int N, double h) {
  return (gi == 0 || gi == N - 1) ? 0.5 * h : h;
}

// Owner block index along one axis for global index g, starting from k.
__device__ __forceinline__ int owner_k(const int* b, int parts, int g, int k) {
  while (k > 0 && g < b[k]) --k;
  while (k < parts - 1 && g >= b[k + 1]) ++k;
  return k;
}

}  // namespace pma
