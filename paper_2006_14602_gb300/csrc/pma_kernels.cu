// pma_kernels.cu -- sm_103a kernels of the DDPMA hot path.
//
// One launch of k_sweep advances every problem of one class (2D/3D x
// FP32/FP64) by one forward-Euler step (Sect. 4.4) of the parallel DD method
// (Sect. 3, Eq. transmission_condition3).  Per tile of one subdomain it
//   * stages the tile plus a one-node halo of v^n in shared memory, with the
//     Neumann mirror ghost of Eq. (nbd) on faces of Omega_c,
//   * forms grad_h and D_h^2 of Psi = |xi|^2/2 + v (Eqs. pmae1d/pmae2d),
//     evaluates rho at the mesh point x = grad_h Psi and the right-hand side
//     G = log(rho det D_h^2 Psi) of Eq. (pmae),
//   * writes v^{n+1} = v^n + dt (G - c) at updated nodes and the owner's v^n
//     at transmission nodes,
//   * reduces theta = sum w rho det (owned nodes), max/min G, min det and the
//     L2-increment pieces into one 64-byte record per tile.
// The last tile of a problem to finish folds the records in a fixed order
// (bitwise reproducible, independent of scheduling), derives the
// normalisation c^n = log(theta^n/|Omega_c|), the residual, the stop test of
// Eq. (dd_stop_criterion) / Algorithm 1 and advances the problem's scalars.
//
// The update uses c of the previous step (c is uniform in space, so it only
// offsets v by a constant S that is tracked per problem; transmission nodes,
// copied one step earlier, carry the previous offset and are corrected by
// `corr` when read).  The mesh x = grad_h Psi is therefore unaffected.
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "pma_device.cuh"
#include "pma_internal.h"

namespace pma {

// ---------------------------------------------------------------- tile header
template <typename T>
struct TileHdr {
  int sub, x0, y0, z0;
  int prob, phase, parity, faces;
  int n[3], g0[3], clo[3], chi[3], N[3], k[3], parts[3];
  int dim, rhs, normalize, stop_norm, sub_base, tile_begin, tile_end, ntiles;
  T dt, c_lag, corr, scale_root;
  T inv2h[3], invh2[3], inv4hh[3], lo[3], h[3];
  double hd[3];
  const T* src;
  T* dst;
  const double* psi0;
};

template <typename T>
__device__ void load_header(const LaunchArgs& a, int t, TileHdr<T>& H, MonT<T>& M) {
  const WorkItem w = a.work[t];
  const SubDesc& sd = a.subs[w.sub];
  const int p = sd.prob;
  const ProbDesc& pd = a.probs[p];
  const ProbState& ps = a.st[p];
  H.sub = w.sub;
  H.x0 = w.x0;
  H.y0 = w.y0;
  H.z0 = w.z0;
  H.prob = p;
  H.phase = *((volatile const int*)&ps.phase);
  H.parity = ps.parity;
  H.faces = sd.faces;
  H.dim = pd.dim;
  for (int q = 0; q < 3; ++q) {
    H.n[q] = sd.n[q];
    H.g0[q] = sd.g0[q];
    H.clo[q] = sd.clo[q];
    H.chi[q] = sd.chi[q];
    H.N[q] = pd.N[q];
    H.k[q] = sd.k[q];
    H.parts[q] = pd.parts[q];
    H.lo[q] = (T)pd.lo[q];
    H.h[q] = (T)pd.h[q];
    H.hd[q] = pd.h[q];
    H.inv2h[q] = (T)(0.5 / pd.h[q]);
    H.invh2[q] = (T)(1.0 / (pd.h[q] * pd.h[q]));
  }
  H.inv4hh[0] = (T)(0.25 / (pd.h[0] * pd.h[1]));  // xy
  H.inv4hh[1] = (T)(0.25 / (pd.h[0] * pd.h[2]));  // xz
  H.inv4hh[2] = (T)(0.25 / (pd.h[1] * pd.h[2]));  // yz
  H.rhs = pd.rhs;
  H.normalize = pd.normalize;
  H.stop_norm = pd.stop_norm;
  H.sub_base = pd.sub_base;
  H.tile_begin = pd.tile_begin;
  H.tile_end = pd.tile_end;
  H.ntiles = pd.tile_end - pd.tile_begin;
  H.dt = (T)pd.dt;
  H.c_lag = (T)ps.c_lag;
  H.corr = (T)ps.corr;
  H.scale_root = (T)(pd.vol / ps.theta_prev);
  H.src = (const T*)sd.v[ps.parity];
  H.dst = (T*)sd.v[ps.parity ^ 1];
  H.psi0 = pd.psi0;
  mon_load<T>(M, pd.mon, pd.dim);
}

// ---------------------------------------------------------------- reductions
template <typename T>
struct Acc {
  T gmax, gmin, dmin;
  int nf;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T big_val();
template <>
__device__ __forceinline__ float big_val<float>() { return FLT_MAX; }
template <>
__device__ __forceinline__ double big_val<double>() { return DBL_MAX; }
__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce the tile's accumulators (in the sweep precision, fixed order) and
// write the tile's partial record.
template <typename T, int NT>
__device__ __forceinline__ void tile_reduce(T th, T l2a, T l2b, T ws, Acc<T> acc, Partial* out,
                                            int sub, T* sh, T* shf, int* shi) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  th = warp_sum(th);
  l2a = warp_sum(l2a);
  l2b = warp_sum(l2b);
  ws = warp_sum(ws);
  T gmax = warp_max(acc.gmax), gmin = warp_min(acc.gmin), dmin = warp_min(acc.dmin);
  int nf = warp_isum(acc.nf);
  if (lane == 0) {
    sh[0 * NW + wid] = th;
    sh[1 * NW + wid] = l2a;
    sh[2 * NW + wid] = l2b;
    sh[3 * NW + wid] = ws;
    shf[0 * NW + wid] = gmax;
    shf[1 * NW + wid] = gmin;
    shf[2 * NW + wid] = dmin;
    shi[wid] = nf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    T m0 = -big_val<T>(), m1 = big_val<T>(), m2 = big_val<T>();
    int c = 0;
    for (int w = 0; w < NW; ++w) {
      s0 += sh[0 * NW + w];
      s1 += sh[1 * NW + w];
      s2 += sh[2 * NW + w];
      s3 += sh[3 * NW + w];
      m0 = fmax(m0, shf[0 * NW + w]);
      m1 = fmin(m1, shf[1 * NW + w]);
      m2 = fmin(m2, shf[2 * NW + w]);
      c += shi[w];
    }
    Partial r;
    r.theta = (double)s0;
    r.l2a = (double)s1;
    r.l2b = (double)s2;
    r.wsum = (double)s3;
    r.gmax = m0;
    r.gmin = m1;
    r.dmin = m2;
    r.nonfinite = c;
    r.sub = sub;
    *out = r;
  }
}

// Fold the partial records of problem p (run by the last block to arrive).
template <int NT>
__device__ void finish_problem(const LaunchArgs& a, int p, int phase) {
  constexpr int NW = NT / 32;
  __shared__ double s_d[NW];
  __shared__ double s_f[NW];
  __shared__ int s_i[NW];
  __shared__ double s_r[NW];
  __shared__ double s_c;
  const ProbDesc& pd = a.probs[p];
  ProbState* ps = a.st + p;
  const int tb = pd.tile_begin, te = pd.tile_end;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  // pass 1: theta (fixed-order sum), non-finite count, min det
  double th = 0.0;
  double dmin = DBL_MAX;
  int nf = 0;
  for (int t = tb + threadIdx.x; t < te; t += NT) {
    const Partial* q = a.part + t;
    th += __ldcg(&q->theta);
    dmin = fmin(dmin, __ldcg(&q->dmin));
    nf += __ldcg(&q->nonfinite);
  }
  th = warp_sum(th);
  dmin = warp_min(dmin);
  nf = warp_isum(nf);
  if (lane == 0) {
    s_d[wid] = th;
    s_f[wid] = dmin;
    s_i[wid] = nf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double T0 = 0.0;
    double dm = DBL_MAX;
    int n = 0;
    for (int w = 0; w < NW; ++w) {
      T0 += s_d[w];
      dm = fmin(dm, s_f[w]);
      n += s_i[w];
    }
    s_d[0] = T0;
    s_f[0] = dm;
    s_i[0] = n;
    double c = 0.0;
    if (pd.rhs == PMA_RHS_LOG && pd.normalize == PMA_NORM_GLOBAL_THETA) c = log(T0 / pd.vol);
    s_c = c;
  }
  __syncthreads();
  const double theta = s_d[0];
  const double dmin_all = s_f[0];
  const int nf_all = s_i[0];
  const double c_n = s_c;

  if (phase == PH_INIT_V) {
    if (threadIdx.x == 0) {
      ps->phase = PH_INIT_THETA;
      ps->tiles_done = 0;
    }
    return;
  }
  const bool tangled = nf_all > 0 || !(dmin_all > 0.0) || !isfinite(theta);
  if (phase == PH_INIT_THETA) {
    if (threadIdx.x == 0) {
      ps->theta = theta;
      ps->theta_prev = theta;
      ps->c_lag = c_n;
      ps->corr = 0.0;
      ps->shift = 0.0;
      ps->min_det = dmin_all;
      if (tangled) {
        ps->status = PMA_ERR_TANGLED;
        ps->phase = PH_DONE;
      } else if (pd.max_steps <= 0) {
        ps->status = PMA_NOT_CONVERGED;
        ps->phase = PH_DONE;
      } else {
        ps->phase = PH_RUN;
      }
      ps->tiles_done = 0;
    }
    return;
  }

  // pass 2: residual per subdomain (one warp per subdomain), then over
  // subdomains by the stop rule (max = ALL, min = ANY)
  const bool any = (pd.stop_rule == PMA_RULE_ANY);
  const double c_lag = ps->c_lag;
  const double delta = c_n - c_lag;
  double r_w = any ? INFINITY : 0.0;
  for (int s = wid; s < pd.nsub; s += NW) {
    const SubDesc& sd = a.subs[pd.sub_base + s];
    double r_s;
    if (pd.stop_norm == PMA_STOP_MAX_UT) {
      double gx = -DBL_MAX, gn = DBL_MAX;
      for (int t = sd.tile_begin + lane; t < sd.tile_end; t += 32) {
        gx = fmax(gx, __ldcg(&a.part[t].gmax));
        gn = fmin(gn, __ldcg(&a.part[t].gmin));
      }
      gx = warp_max(gx);
      gn = warp_min(gn);
      r_s = fmax(gx - c_n, c_n - gn);
    } else {
      double A = 0.0, B = 0.0, W = 0.0;
      for (int t = sd.tile_begin + lane; t < sd.tile_end; t += 32) {
        A += __ldcg(&a.part[t].l2a);
        B += __ldcg(&a.part[t].l2b);
        W += __ldcg(&a.part[t].wsum);
      }
      A = warp_sum(A);
      B = warp_sum(B);
      W = warp_sum(W);
      // sum w (G - c_n)^2 = sum w (G - c_lag - delta)^2
      double q = A - 2.0 * delta * B + delta * delta * W;
      r_s = pd.dt * sqrt(q > 0.0 ? q : 0.0);
    }
    r_w = any ? fmin(r_w, r_s) : fmax(r_w, r_s);
  }
  if (lane == 0) s_r[wid] = r_w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = any ? INFINITY : 0.0;
    for (int w = 0; w < NW; ++w) r = any ? fmin(r, s_r[w]) : fmax(r, s_r[w]);
    ps->theta = theta;
    ps->min_det = dmin_all;
    if (tangled) {
      ps->status = PMA_ERR_TANGLED;
      ps->phase = PH_DONE;
    } else {
      ps->residual = r;
      // transmission nodes written this step carry the old offset
      const double corr = pd.dt * (c_n - c_lag);
      ps->corr = corr;
      ps->shift += corr;
      ps->c_lag = c_n;
      ps->theta_prev = theta;
      ps->parity ^= 1;
      long long step = ps->step + 1;
      ps->step = step;
      if ((step % pd.check_every) == 0 && r <= pd.tol) {
        ps->status = PMA_OK;
        ps->phase = PH_DONE;
      } else if (step >= pd.max_steps) {
        ps->status = PMA_NOT_CONVERGED;
        ps->phase = PH_DONE;
      }
    }
    ps->tiles_done = 0;
  }
}

// Arrival: publish this tile's record, elect the last tile of the problem.
template <int NT>
__device__ __forceinline__ void arrive(const LaunchArgs& a, int prob, int ntiles, int phase,
                                       int* s_last) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(&a.st[prob].tiles_done, 1u);
    *s_last = (prev == (unsigned int)(ntiles - 1));
  }
  __syncthreads();
  if (*s_last) {
    __threadfence();
    finish_problem<NT>(a, prob, phase);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- helpers
// Owner's value at a global node (parallel transmission: previous step).
template <typename T>
__device__ __forceinline__ T gather_owner(const LaunchArgs& a, const TileHdr<T>& H, int gi,
                                          int gj, int gl) {
  const ProbDesc& pd = a.probs[H.prob];
  int kx = owner_k(pd.bcore[0], H.parts[0], gi, H.k[0]);
  int ky = H.dim > 1 ? owner_k(pd.bcore[1], H.parts[1], gj, H.k[1]) : 0;
  int kz = H.dim > 2 ? owner_k(pd.bcore[2], H.parts[2], gl, H.k[2]) : 0;
  const SubDesc& od = a.subs[H.sub_base + (kz * H.parts[1] + ky) * H.parts[0] + kx];
  const T* ov = (const T*)od.v[H.parity];
  long long li = (long long)(gi - od.g0[0]) +
                 (long long)od.n[0] * ((gj - od.g0[1]) + (long long)od.n[1] * (gl - od.g0[2]));
  return ov[li];
}

template <typename T>
__device__ __forceinline__ T init_value(const TileHdr<T>& H, int gi, int gj, int gl) {
  if (!H.psi0) return T(0);
  const long long gflat = (long long)gi + (long long)H.N[0] * (gj + (long long)H.N[1] * gl);
  double q = 0.0;
  const int g[3] = {gi, gj, gl};
  for (int a = 0; a < 3; ++a)
    if (a < H.dim) {
      double xi = (double)H.lo[a] + (double)g[a] * H.hd[a];
      q += 0.5 * xi * xi;
    }
  return (T)(H.psi0[gflat] - q);
}

// Right-hand side at one node from the Hessian entries and mesh point.
// (The theta^0 pass only needs rho det and a finiteness check, so it uses
// the log form whatever the right-hand side.)
template <typename T>
__device__ __forceinline__ T rhs_value(const TileHdr<T>& H, const MonT<T>& M, const T* x, T D,
                                       T& rho) {
  rho = rho_at<T>(M, x);
  if (H.rhs == PMA_RHS_LOG || H.phase != PH_RUN) return Fm<T>::ln(rho * D);
  const T sc = (H.normalize == PMA_NORM_GLOBAL_THETA) ? H.scale_root : T(1);
  const T e = T(1) / (T)H.dim;
  return Fm<T>::pw(sc * rho * D, e) - T(1);
}

template <typename T>
__device__ __forceinline__ void accumulate(const TileHdr<T>& H, T G, T D, T rho, bool owned,
                                           int gi, int gj, int gl, int i, int j, int l, T& th,
                                           T& l2a, T& l2b, T& ws, Acc<T>& acc) {
  if (!(G == G) || !isfinite(G)) acc.nf += 1;
  acc.gmax = fmax(acc.gmax, G);
  acc.gmin = fmin(acc.gmin, G);
  acc.dmin = fmin(acc.dmin, D);
  if (owned) {
    double w = trap_w(gi, H.N[0], H.hd[0]);
    if (H.dim > 1) w *= trap_w(gj, H.N[1], H.hd[1]);
    if (H.dim > 2) w *= trap_w(gl, H.N[2], H.hd[2]);
    th += (T)w * rho * D;
  }
  if (H.stop_norm == PMA_STOP_L2_INCREMENT) {
    double w = trap_w(i, H.n[0], H.hd[0]);
    if (H.dim > 1) w *= trap_w(j, H.n[1], H.hd[1]);
    if (H.dim > 2) w *= trap_w(l, H.n[2], H.hd[2]);
    T d = G - H.c_lag;
    l2a += (T)w * d * d;
    l2b += (T)w * d;
    ws += (T)w;
  }
}

// ---------------------------------------------------------------- 2D sweep
template <typename T, int TX, int TY, int RY>
__global__ void __launch_bounds__(TX * TY / RY) k_sweep2d(LaunchArgs a) {
  constexpr int NT = TX * TY / RY;
  constexpr int SX = TX + 2, SY = TY + 2;
  __shared__ T sv[SY * SX];
  __shared__ TileHdr<T> H;
  __shared__ MonT<T> M;
  __shared__ T red_t[4 * (NT / 32)];
  __shared__ T red_f[3 * (NT / 32)];
  __shared__ int red_i[NT / 32];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const int tx = tid % TX, tyb = tid / TX;

  for (int t = a.t0 + blockIdx.x; t < a.t0 + a.nwork; t += gridDim.x) {
    if (tid == 0) load_header<T>(a, t, H, M);
    __syncthreads();
    const int phase = H.phase;
    if (phase == PH_DONE) {
      __syncthreads();
      continue;
    }
    const int n0 = H.n[0], n1 = H.n[1];
    const bool plx = H.faces & 1, phx = H.faces & 2, ply = H.faces & 4, phy = H.faces & 8;
    T th = 0, l2a = 0, l2b = 0, ws = 0;
    Acc<T> acc{-big_val<T>(), big_val<T>(), big_val<T>(), 0};

    if (phase == PH_INIT_V) {
      // v^0 into both buffers (the next pass reads buffer `parity`)
      for (int r = 0; r < RY; ++r) {
        const int i = H.x0 + tx, j = H.y0 + tyb * RY + r;
        if (i < n0 && j < n1) {
          const T v0 = init_value<T>(H, H.g0[0] + i, H.g0[1] + j, 0);
          H.dst[(long long)j * n0 + i] = v0;
          ((T*)H.src)[(long long)j * n0 + i] = v0;
        }
      }
    } else {
      // stage tile + halo of v^n (mirror on Neumann faces)
      for (int idx = tid; idx < SX * SY; idx += NT) {
        const int ly = idx / SX, lx = idx - ly * SX;
        const int i = reflect_clamp(H.x0 - 1 + lx, n0, plx, phx);
        const int j = reflect_clamp(H.y0 - 1 + ly, n1, ply, phy);
        T val = H.src[(long long)j * n0 + i];
        if (is_dir(H.faces, 2, i, j, 0, n0, n1, 1)) val += H.corr;
        sv[idx] = val;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const int lyy = tyb * RY + r;
        const int i = H.x0 + tx, j = H.y0 + lyy;
        if (i >= n0 || j >= n1) continue;
        const int gi = H.g0[0] + i, gj = H.g0[1] + j;
        if (is_dir(H.faces, 2, i, j, 0, n0, n1, 1)) {
          if (phase == PH_RUN) H.dst[(long long)j * n0 + i] = gather_owner<T>(a, H, gi, gj, 0);
          continue;
        }
        const T* c = sv + (lyy + 1) * SX + (tx + 1);
        const T vc = c[0], ve = c[1], vw = c[-1], vn = c[SX], vs = c[-SX];
        const T vne = c[SX + 1], vnw = c[SX - 1], vse = c[-SX + 1], vsw = c[-SX - 1];
        T x[3];
        x[0] = H.lo[0] + (T)gi * H.h[0] + (ve - vw) * H.inv2h[0];
        x[1] = H.lo[1] + (T)gj * H.h[1] + (vn - vs) * H.inv2h[1];
        x[2] = 0;
        const T hxx = T(1) + (ve - T(2) * vc + vw) * H.invh2[0];
        const T hyy = T(1) + (vn - T(2) * vc + vs) * H.invh2[1];
        const T hxy = ((vne - vse) - (vnw - vsw)) * H.inv4hh[0];
        const T D = hxx * hyy - hxy * hxy;
        T rho;
        const T G = rhs_value<T>(H, M, x, D, rho);
        const bool owned = i >= H.clo[0] && i <= H.chi[0] && j >= H.clo[1] && j <= H.chi[1];
        accumulate<T>(H, G, D, rho, owned, gi, gj, 0, i, j, 0, th, l2a, l2b, ws, acc);
        if (phase == PH_RUN) H.dst[(long long)j * n0 + i] = vc + H.dt * (G - H.c_lag);
      }
    }
    tile_reduce<T, NT>(th, l2a, l2b, ws, acc, a.part + t, H.sub, red_t, red_f, red_i);
    arrive<NT>(a, H.prob, H.ntiles, phase, &s_last);
  }
}

// ---------------------------------------------------------------- 3D sweep
// TX x TY threads, each marching TZ planes of the tile.
template <typename T, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX * TY) k_sweep3d(LaunchArgs a) {
  constexpr int NT = TX * TY;
  constexpr int SX = TX + 2, SY = TY + 2, SZ = TZ + 2;
  __shared__ T sv[SZ * SY * SX];
  __shared__ TileHdr<T> H;
  __shared__ MonT<T> M;
  __shared__ T red_t[4 * (NT / 32)];
  __shared__ T red_f[3 * (NT / 32)];
  __shared__ int red_i[NT / 32];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;

  for (int t = a.t0 + blockIdx.x; t < a.t0 + a.nwork; t += gridDim.x) {
    if (tid == 0) load_header<T>(a, t, H, M);
    __syncthreads();
    const int phase = H.phase;
    if (phase == PH_DONE) {
      __syncthreads();
      continue;
    }
    const int n0 = H.n[0], n1 = H.n[1], n2 = H.n[2];
    const bool plx = H.faces & 1, phx = H.faces & 2, ply = H.faces & 4, phy = H.faces & 8;
    const bool plz = H.faces & 16, phz = H.faces & 32;
    T th = 0, l2a = 0, l2b = 0, ws = 0;
    Acc<T> acc{-big_val<T>(), big_val<T>(), big_val<T>(), 0};
    const long long pitch_z = (long long)n0 * n1;

    if (phase == PH_INIT_V) {
      for (int r = 0; r < TZ; ++r) {
        const int i = H.x0 + tx, j = H.y0 + ty, l = H.z0 + r;
        if (i < n0 && j < n1 && l < n2) {
          const T v0 = init_value<T>(H, H.g0[0] + i, H.g0[1] + j, H.g0[2] + l);
          H.dst[l * pitch_z + (long long)j * n0 + i] = v0;
          ((T*)H.src)[l * pitch_z + (long long)j * n0 + i] = v0;
        }
      }
    } else {
      for (int idx = tid; idx < SX * SY * SZ; idx += NT) {
        const int lz = idx / (SX * SY);
        const int rem = idx - lz * SX * SY;
        const int ly = rem / SX, lx = rem - ly * SX;
        const int i = reflect_clamp(H.x0 - 1 + lx, n0, plx, phx);
        const int j = reflect_clamp(H.y0 - 1 + ly, n1, ply, phy);
        const int l = reflect_clamp(H.z0 - 1 + lz, n2, plz, phz);
        T val = H.src[l * pitch_z + (long long)j * n0 + i];
        if (is_dir(H.faces, 3, i, j, l, n0, n1, n2)) val += H.corr;
        sv[idx] = val;
      }
      __syncthreads();
      const int i = H.x0 + tx, j = H.y0 + ty;
      for (int r = 0; r < TZ; ++r) {
        const int l = H.z0 + r;
        if (i >= n0 || j >= n1 || l >= n2) continue;
        const int gi = H.g0[0] + i, gj = H.g0[1] + j, gl = H.g0[2] + l;
        const long long gidx = l * pitch_z + (long long)j * n0 + i;
        if (is_dir(H.faces, 3, i, j, l, n0, n1, n2)) {
          if (phase == PH_RUN) H.dst[gidx] = gather_owner<T>(a, H, gi, gj, gl);
          continue;
        }
        const T* c = sv + ((r + 1) * SY + (ty + 1)) * SX + (tx + 1);
        constexpr int PY = SX, PZ = SX * SY;
        const T vc = c[0];
        const T vxp = c[1], vxm = c[-1], vyp = c[PY], vym = c[-PY], vzp = c[PZ], vzm = c[-PZ];
        T x[3];
        x[0] = H.lo[0] + (T)gi * H.h[0] + (vxp - vxm) * H.inv2h[0];
        x[1] = H.lo[1] + (T)gj * H.h[1] + (vyp - vym) * H.inv2h[1];
        x[2] = H.lo[2] + (T)gl * H.h[2] + (vzp - vzm) * H.inv2h[2];
        const T hxx = T(1) + (vxp - T(2) * vc + vxm) * H.invh2[0];
        const T hyy = T(1) + (vyp - T(2) * vc + vym) * H.invh2[1];
        const T hzz = T(1) + (vzp - T(2) * vc + vzm) * H.invh2[2];
        const T hxy = ((c[PY + 1] - c[-PY + 1]) - (c[PY - 1] - c[-PY - 1])) * H.inv4hh[0];
        const T hxz = ((c[PZ + 1] - c[-PZ + 1]) - (c[PZ - 1] - c[-PZ - 1])) * H.inv4hh[1];
        const T hyz = ((c[PZ + PY] - c[-PZ + PY]) - (c[PZ - PY] - c[-PZ - PY])) * H.inv4hh[2];
        const T D = hxx * (hyy * hzz - hyz * hyz) - hxy * (hxy * hzz - hyz * hxz) +
                    hxz * (hxy * hyz - hyy * hxz);
        T rho;
        const T G = rhs_value<T>(H, M, x, D, rho);
        const bool owned = i >= H.clo[0] && i <= H.chi[0] && j >= H.clo[1] && j <= H.chi[1] &&
                           l >= H.clo[2] && l <= H.chi[2];
        accumulate<T>(H, G, D, rho, owned, gi, gj, gl, i, j, l, th, l2a, l2b, ws, acc);
        if (phase == PH_RUN) H.dst[gidx] = vc + H.dt * (G - H.c_lag);
      }
    }
    tile_reduce<T, NT>(th, l2a, l2b, ws, acc, a.part + t, H.sub, red_t, red_f, red_i);
    arrive<NT>(a, H.prob, H.ntiles, phase, &s_last);
  }
}

// ---------------------------------------------------------------- dispatch
// Compiled tile shapes.  2D: (TX, TY, RY); 3D: (TX, TY, TZ).
#define PMA_T2D(X) X(32, 16, 2) X(32, 8, 1) X(64, 8, 2) X(16, 16, 2)
#define PMA_T3D(X) X(32, 8, 4) X(32, 4, 8) X(16, 8, 8)

static const Tile2D k_t2d[] = {
#define E(a, b, c) {a, b},
    PMA_T2D(E)
#undef E
};
static const Tile3D k_t3d[] = {
#define E(a, b, c) {a, b, c},
    PMA_T3D(E)
#undef E
};

int tile2d_count() { return (int)(sizeof(k_t2d) / sizeof(k_t2d[0])); }
int tile3d_count() { return (int)(sizeof(k_t3d) / sizeof(k_t3d[0])); }
Tile2D tile2d_shape(int id) { return k_t2d[id]; }
Tile3D tile3d_shape(int id) { return k_t3d[id]; }

template <typename T>
static const void* sweep_fn(int dim, int id, int* nthreads) {
  int k = 0;
  if (dim == 2) {
#define E(a, b, c)                                   \
  if (k++ == id) {                                   \
    *nthreads = (a) * (b) / (c);                     \
    return (const void*)k_sweep2d<T, a, b, c>;       \
  }
    PMA_T2D(E)
#undef E
  } else {
#define E(a, b, c)                                   \
  if (k++ == id) {                                   \
    *nthreads = (a) * (b);                           \
    return (const void*)k_sweep3d<T, a, b, c>;       \
  }
    PMA_T3D(E)
#undef E
  }
  return nullptr;
}

static const void* cls_fn(int cls, int tile_id, int* nthreads) {
  switch (cls) {
    case CLS_2D_F32: return sweep_fn<float>(2, tile_id, nthreads);
    case CLS_2D_F64: return sweep_fn<double>(2, tile_id, nthreads);
    case CLS_3D_F32: return sweep_fn<float>(3, tile_id, nthreads);
    case CLS_3D_F64: return sweep_fn<double>(3, tile_id, nthreads);
  }
  return nullptr;
}

cudaError_t launch_sweep(int cls, int tile_id, const LaunchArgs& a, cudaStream_t s) {
  int nt = 0;
  const void* fn = cls_fn(cls, tile_id, &nt);
  if (!fn) return cudaErrorInvalidValue;
  if (a.nwork <= 0 || a.grid <= 0) return cudaSuccess;
  void* args[] = {(void*)&a};
  return cudaLaunchKernel(fn, dim3(a.grid), dim3(nt), args, 0, s);
}

int sweep_max_blocks_per_sm(int cls, int tile_id) {
  int nt = 0;
  const void* fn = cls_fn(cls, tile_id, &nt);
  if (!fn) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, nt, 0) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

// ---------------------------------------------------------------- combine
// Owner-takes combination: global node g takes x = xi + grad_h v of the
// subdomain whose core holds it (mirror ghost on faces of Omega_c, i.e.
// x_a = xi_a on faces normal to a), and Psi = v - S + |xi|^2/2.
template <typename T>
__device__ __forceinline__ T fetch_v(const SubDesc& sd, const T* v, int dim, int i, int j, int l,
                                     double corr) {
  const int n0 = sd.n[0], n1 = sd.n[1], n2 = sd.n[2];
  i = reflect_clamp(i, n0, sd.faces & 1, sd.faces & 2);
  j = dim > 1 ? reflect_clamp(j, n1, sd.faces & 4, sd.faces & 8) : 0;
  l = dim > 2 ? reflect_clamp(l, n2, sd.faces & 16, sd.faces & 32) : 0;
  T val = v[(long long)i + (long long)n0 * (j + (long long)n1 * l)];
  if (is_dir(sd.faces, dim, i, j, l, n0, n1, n2)) val += (T)corr;
  return val;
}

template <typename T>
__device__ void combine_node(const CombineJob& J, long long g, const SubDesc* subs,
                             const ProbDesc& pd, const ProbState& ps) {
  const int dim = pd.dim;
  const long long N = (long long)pd.N[0] * pd.N[1] * pd.N[2];
  int gi = (int)(g % pd.N[0]);
  long long rest = g / pd.N[0];
  int gj = (int)(rest % pd.N[1]);
  int gl = (int)(rest / pd.N[1]);
  int kx = owner_k(pd.bcore[0], pd.parts[0], gi, 0);
  int ky = owner_k(pd.bcore[1], pd.parts[1], gj, 0);
  int kz = owner_k(pd.bcore[2], pd.parts[2], gl, 0);
  const SubDesc& sd = subs[pd.sub_base + (kz * pd.parts[1] + ky) * pd.parts[0] + kx];
  const T* v = (const T*)sd.v[ps.parity];
  const int i = gi - sd.g0[0], j = gj - sd.g0[1], l = gl - sd.g0[2];
  const int gg[3] = {gi, gj, gl};
  const int li[3] = {i, j, l};
  double q = 0.0;
  for (int a = 0; a < dim; ++a) {
    const double xi = pd.lo[a] + (double)gg[a] * pd.h[a];
    q += 0.5 * xi * xi;
    double xa = xi;
    if (gg[a] > 0 && gg[a] < pd.N[a] - 1) {
      int p[3] = {li[0], li[1], li[2]}, m[3] = {li[0], li[1], li[2]};
      p[a] += 1;
      m[a] -= 1;
      const T vp = fetch_v<T>(sd, v, dim, p[0], p[1], p[2], ps.corr);
      const T vm = fetch_v<T>(sd, v, dim, m[0], m[1], m[2], ps.corr);
      xa = xi + (double)(vp - vm) * (0.5 / pd.h[a]);
    }
    if (J.out_fp64)
      ((double*)J.x)[a * N + g] = xa;
    else
      ((float*)J.x)[a * N + g] = (float)xa;
  }
  if (J.psi) {
    const double vv = (double)v[(long long)i + (long long)sd.n[0] * (j + (long long)sd.n[1] * l)];
    const double psi = vv - ps.shift + q;
    if (J.out_fp64)
      ((double*)J.psi)[g] = psi;
    else
      ((float*)J.psi)[g] = (float)psi;
  }
}

__global__ void k_combine(const CombineJob* jobs, int njobs, const SubDesc* subs,
                          const ProbDesc* probs, const ProbState* st) {
  const CombineJob J = jobs[blockIdx.y];
  const ProbDesc& pd = probs[J.prob];
  const ProbState& ps = st[J.prob];
  const long long N = (long long)pd.N[0] * pd.N[1] * pd.N[2];
  const bool f64 = (pd.cls == CLS_2D_F64 || pd.cls == CLS_3D_F64);
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x) {
    if (f64)
      combine_node<double>(J, g, subs, pd, ps);
    else
      combine_node<float>(J, g, subs, pd, ps);
  }
}

cudaError_t launch_combine(const CombineJob* jobs_dev, int njobs, long long max_nodes,
                           const SubDesc* subs, const ProbDesc* probs, const ProbState* st,
                           cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  long long bx = (max_nodes + 255) / 256;
  if (bx > 4096) bx = 4096;
  if (bx < 1) bx = 1;
  k_combine<<<dim3((unsigned)bx, (unsigned)njobs), 256, 0, s>>>(jobs_dev, njobs, subs, probs, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 check
// det D_h^2 Psi in FP64 at every global node (owner's stencil) and the
// signed measure of every cell of the combined mesh.
__device__ __forceinline__ void atomic_min_double(double* addr, double val) {
  unsigned long long* a = (unsigned long long*)addr;
  unsigned long long old = *a, assumed;
  while (val < __longlong_as_double(old)) {
    assumed = old;
    old = atomicCAS(a, assumed, __double_as_longlong(val));
    if (old == assumed) break;
  }
}

template <typename T>
__device__ void node_x_and_hessian(const SubDesc* subs, const ProbDesc& pd, const ProbState& ps,
                                   const int* gg, double* x, double H[3][3]) {
  const int dim = pd.dim;
  int kk[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) kk[a] = owner_k(pd.bcore[a], pd.parts[a], gg[a], 0);
  const SubDesc& sd = subs[pd.sub_base + (kk[2] * pd.parts[1] + kk[1]) * pd.parts[0] + kk[0]];
  const T* v = (const T*)sd.v[ps.parity];
  const int li[3] = {gg[0] - sd.g0[0], gg[1] - sd.g0[1], gg[2] - sd.g0[2]};
  auto f = [&](int di, int dj, int dl) -> double {
    return (double)fetch_v<T>(sd, v, dim, li[0] + di, li[1] + dj, li[2] + dl, ps.corr);
  };
  const double vc = f(0, 0, 0);
  int e[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) H[a][b] = (a == b && a >= dim) ? 1.0 : 0.0;
  for (int a = 0; a < dim; ++a) {
    const double vp = f(e[a][0], e[a][1], e[a][2]), vm = f(-e[a][0], -e[a][1], -e[a][2]);
    x[a] = pd.lo[a] + gg[a] * pd.h[a] + (vp - vm) / (2.0 * pd.h[a]);
    H[a][a] = 1.0 + (vp - 2.0 * vc + vm) / (pd.h[a] * pd.h[a]);
  }
  for (int a = 0; a < dim; ++a)
    for (int b = a + 1; b < dim; ++b) {
      const int* ea = e[a];
      const int* eb = e[b];
      const double hab = (f(ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2]) -
                          f(ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]) -
                          f(-ea[0] + eb[0], -ea[1] + eb[1], -ea[2] + eb[2]) +
                          f(-ea[0] - eb[0], -ea[1] - eb[1], -ea[2] - eb[2])) /
                         (4.0 * pd.h[a] * pd.h[b]);
      H[a][b] = H[b][a] = hab;
    }
}

template <typename T>
__global__ void k_check(int prob, const SubDesc* subs, const ProbDesc* probs, const ProbState* st,
                        double* out, unsigned long long* cnt) {
  const ProbDesc& pd = probs[prob];
  const ProbState& ps = st[prob];
  const int dim = pd.dim;
  const long long N = (long long)pd.N[0] * pd.N[1] * pd.N[2];
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x) {
    int gg[3] = {(int)(g % pd.N[0]), (int)((g / pd.N[0]) % pd.N[1]),
                 (int)(g / ((long long)pd.N[0] * pd.N[1]))};
    double x[3] = {0, 0, 0}, H[3][3];
    node_x_and_hessian<T>(subs, pd, ps, gg, x, H);
    const double m1 = H[0][0];
    const double m2 = H[0][0] * H[1][1] - H[0][1] * H[1][0];
    const double det = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                       H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                       H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
    atomic_min_double(out + 0, det);
    atomic_min_double(out + 1, dim == 3 ? fmin(m1, m2) : m1);
    // cell with lower corner g
    bool cell = true;
    for (int a = 0; a < dim; ++a) cell = cell && gg[a] < pd.N[a] - 1;
    if (!cell) continue;
    double P[8][3];
    const int nc = 1 << dim;
    for (int c = 0; c < nc; ++c) {
      int q[3] = {gg[0] + (c & 1), gg[1] + ((c >> 1) & 1), gg[2] + ((c >> 2) & 1)};
      double Hd[3][3];
      P[c][0] = P[c][1] = P[c][2] = 0.0;
      node_x_and_hessian<T>(subs, pd, ps, q, P[c], Hd);
    }
    double mu_min = INFINITY;
    if (dim == 2) {
      // corners 0=00 1=10 2=01 3=11; both diagonal splits
      const int tri[4][3] = {{0, 1, 3}, {0, 3, 2}, {0, 1, 2}, {1, 3, 2}};
      for (int k = 0; k < 4; ++k) {
        const double* A = P[tri[k][0]];
        const double* B = P[tri[k][1]];
        const double* C = P[tri[k][2]];
        const double mu = 0.5 * ((B[0] - A[0]) * (C[1] - A[1]) - (C[0] - A[0]) * (B[1] - A[1]));
        mu_min = fmin(mu_min, mu);
      }
    } else {
      const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {1, 0, 2}, {0, 2, 1}, {2, 1, 0}};
      const double sg[6] = {1, 1, 1, -1, -1, -1};
      for (int k = 0; k < 6; ++k) {
        int off = 0;
        int idx[4];
        idx[0] = 0;
        for (int s = 0; s < 3; ++s) {
          off |= 1 << perm[k][s];
          idx[s + 1] = off;
        }
        double A[3][3];
        for (int r = 0; r < 3; ++r)
          for (int cc = 0; cc < 3; ++cc) A[r][cc] = P[idx[r + 1]][cc] - P[idx[0]][cc];
        const double d = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        mu_min = fmin(mu_min, sg[k] * d / 6.0);
      }
    }
    atomic_min_double(out + 2, mu_min);
    if (!(mu_min > 0.0)) atomicAdd(cnt, 1ull);
  }
}

cudaError_t launch_check(int prob, long long nodes, const SubDesc* subs, const ProbDesc* probs,
                         const ProbState* st, double* out, unsigned long long* cnt,
                         cudaStream_t s) {
  // precision of the problem is read on the host side by the caller: try both
  // by class stored in the descriptor
  long long bx = (nodes + 255) / 256;
  if (bx > 2048) bx = 2048;
  if (bx < 1) bx = 1;
  ProbDesc pd;
  cudaError_t e = cudaMemcpyAsync(&pd, probs + prob, sizeof(ProbDesc), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (pd.cls == CLS_2D_F64 || pd.cls == CLS_3D_F64)
    k_check<double><<<(unsigned)bx, 256, 0, s>>>(prob, subs, probs, st, out, cnt);
  else
    k_check<float><<<(unsigned)bx, 256, 0, s>>>(prob, subs, probs, st, out, cnt);
  return cudaGetLastError();
}

}  // namespace pma
