// pma_device.cuh -- device helpers of the DDPMA sweep: math traits, the
// monitor densities and index helpers.  Included by the kernel TUs only.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pma_internal.h"

namespace pma {

// ---------------------------------------------------------------- math
// FP32 uses the SFU (ex2/lg2 approximations), FP64 the accurate library
// functions.  exw(q) = exp(-width * q) with the term width as stored in
// MonT<T> (pre-scaled by log2(e) for FP32).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <typename T>
struct Fm;

template <>
struct Fm<float> {
  static constexpr float kLog2e = 1.4426950408889634f;
  static constexpr float kLn2 = 0.6931471805599453f;
  __device__ __forceinline__ static float exw(float negwq) { return ex2_approx(negwq); }
  __device__ __forceinline__ static float ex(float x) { return ex2_approx(x * kLog2e); }
  __device__ __forceinline__ static float ln(float x) { return lg2_approx(x) * kLn2; }
  __device__ __forceinline__ static float sinpi(float x) { return sinpif(x); }
  __device__ __forceinline__ static float sq(float x) { return sqrtf(x); }
  __device__ __forceinline__ static float at2(float y, float x) { return atan2f(y, x); }
  __device__ __forceinline__ static float cs(float x) { return cosf(x); }
  __device__ __forceinline__ static float sn(float x) { return sinf(x); }
  __device__ __forceinline__ static float pw(float x, float y) { return ex2_approx(y * lg2_approx(x)); }
};

template <>
struct Fm<double> {
  __device__ __forceinline__ static double exw(double negwq) { return exp(negwq); }
  __device__ __forceinline__ static double ex(double x) { return exp(x); }
  __device__ __forceinline__ static double ln(double x) { return log(x); }
  __device__ __forceinline__ static double sinpi(double x) { return ::sinpi(x); }
  __device__ __forceinline__ static double sq(double x) { return sqrt(x); }
  __device__ __forceinline__ static double at2(double y, double x) { return atan2(y, x); }
  __device__ __forceinline__ static double cs(double x) { return cos(x); }
  __device__ __forceinline__ static double sn(double x) { return sin(x); }
  __device__ __forceinline__ static double pw(double x, double y) { return pow(x, y); }
};

// ---------------------------------------------------------------- monitor
// sech^2(z) = 4 e^{-2|z|} / (1 + e^{-2|z|})^2, overflow-free.
template <typename T>
__device__ __forceinline__ T sech2(T z) {
  T e = Fm<T>::ex(-2 * fabs(z));
  T d = 1 + e;
  return 4 * e / (d * d);
}

template <typename T>
__device__ __forceinline__ T term_value(const typename MonT<T>::Term& t, int dim, T x0, T x1,
                                        T x2) {
  switch (t.type) {
    case PMA_TERM_BUMP: {
      T d0 = x0 - t.c[0], d1 = x1 - t.c[1];
      T q = fma(d0, d0, d1 * d1);
      if (dim > 2) {
        T d2 = x2 - t.c[2];
        q = fma(d2, d2, q);
      }
      return t.amp * Fm<T>::exw(-t.width * q);
    }
    case PMA_TERM_RING: {
      T d0 = x0 - t.c[0], d1 = x1 - t.c[1];
      T q = fma(d0, d0, d1 * d1);
      if (dim > 2) {
        T d2 = x2 - t.c[2];
        q = fma(d2, d2, q);
      }
      T s = q - t.r2;
      return t.amp * Fm<T>::exw(-t.width * s * s);
    }
    case PMA_TERM_SINE: {
      const T xa = t.axis == 0 ? x0 : (t.axis == 1 ? x1 : x2);
      const T xb = t.along == 0 ? x0 : (t.along == 1 ? x1 : x2);
      T s = xa - t.c[t.axis] - t.a * Fm<T>::sinpi(t.k2 * xb);
      return t.amp * Fm<T>::exw(-t.width * s * s);
    }
    case PMA_TERM_BUMP1: {
      const T xa = t.axis == 0 ? x0 : (t.axis == 1 ? x1 : x2);
      T s = xa - t.c[t.axis];
      return t.amp * Fm<T>::exw(-t.width * s * s);
    }
  }
  return T(0);
}

// rho = sqrt(1 + |grad u|^2) for the test functions of Sect. 4.
template <typename T>
__device__ T arclen_rho(const MonT<T>& m, T x0, T x1, T x2) {
  T g0 = 0, g1 = 0, g2 = 0;
  switch (m.kind) {
    case PMA_MON_ARCLEN_BURGERS: {
      T eps = m.p0;
      T s = (x0 + x1 - 1) / (2 * eps);
      T d = -T(0.25) * sech2<T>(T(0.5) * s) / (2 * eps);
      g0 = d;
      g1 = d;
      break;
    }
    case PMA_MON_ARCLEN_SPIRAL: {
      T dx = x0 - T(0.7), dy = x1 - T(0.5);
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
      T r2 = x0 * x0 + x1 * x1 + x2 * x2;
      T f = 200 * sech2<T>(100 * (r2 - T(0.125)));
      g0 = f * x0;
      g1 = f * x1;
      g2 = f * x2;
      break;
    }
    case PMA_MON_ARCLEN_NINE_SPHERES: {
      for (int k = 0; k < 9; ++k) {
        T cx = (k == 0) ? T(0) : ((k == 1 || k == 2 || k == 5 || k == 6) ? T(0.5) : T(-0.5));
        T cy = (k == 0) ? T(0) : ((k & 1) ? T(0.5) : T(-0.5));
        T cz = (k == 0) ? T(0) : (k <= 4 ? T(0.5) : T(-0.5));
        T ex = x0 - cx, ey = x1 - cy, ez = x2 - cz;
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

// Tabulated density: multilinear interpolation, the point clamped to the
// table's box per axis (cell index at most tn - 2), corners combined with
// product weights in axis order.
template <typename T>
__device__ T table_rho(const MonT<T>& m, T x0, T x1, T x2) {
  const T xs[3] = {x0, x1, x2};
  int base = 0, stride = 1;
  int st[3];
  T f[3];
  for (int a = 0; a < 3; ++a) {
    st[a] = stride;
    f[a] = T(0);
    if (a < m.dim) {
      T s = (xs[a] - m.tlo[a]) * m.tsc[a];
      s = fmin(fmax(s, T(0)), (T)(m.tn[a] - 1));
      int k = (int)floor(s);
      k = k > m.tn[a] - 2 ? m.tn[a] - 2 : k;
      f[a] = s - (T)k;
      base += k * stride;
    }
    stride *= m.tn[a];
  }
  T r = T(0);
  for (int corner = 0; corner < (1 << m.dim); ++corner) {
    T w = T(1);
    int idx = base;
    for (int a = 0; a < m.dim; ++a) {
      const int up = (corner >> a) & 1;
      w *= up ? f[a] : T(1) - f[a];
      idx += up * st[a];
    }
    r = fma(w, __ldg(m.table + idx), r);
  }
  return r;
}

template <typename T>
__device__ __forceinline__ T rho_at(const MonT<T>& m, T x0, T x1, T x2) {
  if (m.kind == PMA_MON_TABLE) return table_rho<T>(m, x0, x1, x2);
  if (m.kind == PMA_MON_SUM) {
    T r = m.base;
    for (int i = 0; i < kMaxTerms; ++i)
      if (i < m.nterms) r += term_value<T>(m.t[i], m.dim, x0, x1, x2);
    return r;
  }
  if (m.kind == PMA_MON_PRODUCT) {
    T r = 1;
    for (int i = 0; i < kMaxTerms; ++i)
      if (i < m.nterms) r *= m.base + term_value<T>(m.t[i], m.dim, x0, x1, x2);
    return r;
  }
  return arclen_rho<T>(m, x0, x1, x2);
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

// Owner block index along one axis for global index g, starting from k.
__device__ __forceinline__ int owner_k(const int* b, int parts, int g, int k) {
  while (k > 0 && g < b[k]) --k;
  while (k < parts - 1 && g >= b[k + 1]) ++k;
  return k;
}

// Global stores that the compiler need not treat as aliasing shared memory
// (a store through a generic pointer would force every shared-memory value
// to be reloaded after it).
__device__ __forceinline__ void st_global(float* p, float v) {
  asm volatile("st.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}
__device__ __forceinline__ void st_global(double* p, double v) {
  asm volatile("st.global.f64 [%0], %1;" ::"l"(p), "d"(v));
}

// Asynchronous 16-byte global -> shared copies (completion: cp_async_wait
// by the issuing thread, then a barrier for the others).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Tensor-memory-access (TMA) copies into shared memory, completed on an
// mbarrier: the issuing thread announces the bytes (expect_tx) and issues
// the copy; every thread then waits on the barrier's phase.
__device__ __forceinline__ unsigned int smem_u32(const void* p) {
  return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Orders this thread's (and, after a barrier, the block's) earlier generic
// shared-memory accesses before later asynchronous-proxy writes.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned int bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 2D tiled copy of the box at (x, y) (x a multiple of 16 bytes of elements;
// coordinates outside the tensor read zeros).
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// 3D tiled copy of the box at (x, y, z) (x as for the 2D copy).
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// Wait until the barrier's phase with parity `phase` has completed, for at
// most about a second of SM clock; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int phase) {
  const unsigned int a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    unsigned int ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(phase)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

// Thread-block clusters: rank, size, barrier (release / acquire), and loads
// from another CTA's shared memory through the shared::cluster window.
__device__ __forceinline__ unsigned int cluster_rank() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned int cluster_size() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of `p` (this CTA's shared memory) in the CTA of cluster rank `rank`.
__device__ __forceinline__ unsigned int dsmem_map(const void* p, unsigned int rank) {
  const unsigned int a = (unsigned int)__cvta_generic_to_shared(p);
  unsigned int d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(rank));
  return d;
}
__device__ __forceinline__ float dsmem_ld(unsigned int a, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ double dsmem_ld(unsigned int a, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ int dsmem_ld(unsigned int a, int) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

// Cooperative copy of a 16-byte-aligned struct into shared memory.
template <int NT>
__device__ __forceinline__ void coop_copy(void* dst, const void* src, int bytes, int first) {
  const int4* s = (const int4*)src;
  int4* d = (int4*)dst;
  const int n = bytes / 16;
  for (int i = threadIdx.x - first; i >= 0 && i < n; i += NT) d[i] = __ldcg(s + i);
}

}  // namespace pma
