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
#include <cstring>

#include "pma_device.cuh"
#include "pma_internal.h"

namespace pma {

// ---------------------------------------------------------------- tile header
// Shared-memory copy of everything one work item needs: the item, its
// subdomain, its problem's scalars and hot descriptor (copied with 16-byte
// loads spread over the block, so the whole header costs one round trip
// after the work item itself, which is prefetched one item ahead).
template <typename T>
struct SmemHdr {
  WorkItem w;
  SubDesc sd;
  ProbState ps;
  ProbHot<T> ph;
};

template <typename T>
__device__ __forceinline__ const ProbHot<T>* hot_table(const LaunchArgs& a);
template <>
__device__ __forceinline__ const ProbHot<float>* hot_table<float>(const LaunchArgs& a) {
  return a.hotf;
}
template <>
__device__ __forceinline__ const ProbHot<double>* hot_table<double>(const LaunchArgs& a) {
  return a.hotd;
}

// q = e / d for 0 <= e < 2^24, 1 <= d < 2^16, via an FP32 reciprocal; the
// estimate is within one of the quotient and the fix-up makes it exact.
__device__ __forceinline__ int qdiv(int e, int d, float inv_d) {
  int q = __float2int_rz(((float)e + 0.5f) * inv_d);
  const int r = e - q * d;
  if (r < 0) --q;
  else if (r >= d) ++q;
  return q;
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
// FP32 extrema of a warp in one instruction (redux.sync, sm_100 family);
// NaN lanes are ignored, as by fmaxf / fminf.
template <>
__device__ __forceinline__ float warp_max<float>(float v) {
  float r;
  asm("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
template <>
__device__ __forceinline__ float warp_min<float>(float v) {
  float r;
  asm("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
template <typename T>
__device__ __forceinline__ T big_val();
template <>
__device__ __forceinline__ float big_val<float>() { return FLT_MAX; }
template <>
__device__ __forceinline__ double big_val<double>() { return DBL_MAX; }
__device__ __forceinline__ int warp_isum(int v) { return __reduce_add_sync(0xffffffffu, v); }

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

// ---------------------------------------------------------------- finish
// After each sweep launch: one warp per problem folds the problem's tile
// records in a fixed order (lane l takes records l, l+32, ...; xor-tree
// reductions), so the result is bitwise independent of how the sweep was
// scheduled.  It derives theta^n and c^n = log(theta^n/|Omega_c|) (the
// normalised density of Eq. edp), the residual of the stop rule
// (Eq. dd_stop_criterion; Algorithm 1 steps 5-6), checks for tangling, and
// advances the problem's scalars.
__device__ __forceinline__ double warp_dsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// State advance after the theta^0 pass (Sect. 4.4: c^0 from theta^0; the
// lagged constant starts equal to it, so the first step carries no offset).
__device__ __forceinline__ void advance_init(ProbState* ps, double theta, double c_n, double dm,
                                             bool tangled, long long max_steps) {
  ps->theta = theta;
  ps->theta_prev = theta;
  ps->c_lag = c_n;
  ps->corr = 0.0;
  ps->shift = 0.0;
  ps->min_det = dm;
  if (tangled) {
    ps->status = PMA_ERR_TANGLED;
    ps->phase = PH_DONE;
  } else if (max_steps <= 0) {
    ps->status = PMA_NOT_CONVERGED;
    ps->phase = PH_DONE;
  } else {
    ps->phase = PH_RUN;
  }
}

// State advance after a forward-Euler step: the stop test of Eq.
// (dd_stop_criterion) every check_every steps, the step cap, and tangling
// (the state read by the step is kept).  Transmission nodes written by the
// step carry the old normalisation offset: corr = dt (c^n - c^{n-1}).
__device__ __forceinline__ void advance_run(ProbState* ps, double theta, double c_n, double dm,
                                            bool tangled, double r, double dt, int check_every,
                                            double tol, long long max_steps) {
  ps->theta = theta;
  ps->min_det = dm;
  if (tangled) {
    ps->status = PMA_ERR_TANGLED;
    ps->phase = PH_DONE;
    return;
  }
  ps->residual = r;
  const double corr = dt * (c_n - ps->c_lag);
  ps->corr = corr;
  ps->shift += corr;
  ps->c_lag = c_n;
  ps->theta_prev = theta;
  ps->parity ^= 1;
  const long long step = ps->step + 1;
  ps->step = step;
  if ((step % check_every) == 0 && r <= tol) {
    ps->status = PMA_OK;
    ps->phase = PH_DONE;
  } else if (step >= max_steps) {
    ps->status = PMA_NOT_CONVERGED;
    ps->phase = PH_DONE;
  }
}

__global__ void k_finish(const int* __restrict__ list, int n, const SubDesc* __restrict__ subs,
                         const ProbDesc* __restrict__ probs, ProbState* st,
                         const Partial* __restrict__ part, const unsigned int* err) {
  // the next sweep may be launched at once (its CTAs wait for this grid);
  // this grid waits for the sweep before it reads the records
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  const unsigned int e0 = *(const volatile unsigned int*)err;
  const int p = list[w];
  ProbState* ps = st + p;
  const int phase = ps->phase;
  if (phase == PH_DONE) return;
  if (e0 != 0) {
    // a sweep gave up a bounded wait: the step's records are incomplete, so
    // the problem retires with a timeout (later sweeps skip its work)
    if (lane == 0) {
      ps->status = PMA_ERR_TIMEOUT;
      ps->phase = PH_DONE;
    }
    return;
  }
  const ProbDesc& pd = probs[p];
  const int tb = pd.tile_begin, te = pd.tile_end;
  if (phase == PH_INIT_V) {
    if (lane == 0) ps->phase = PH_INIT_THETA;
    return;
  }
  const double c_lag = ps->c_lag;
  // pass 1: theta, extrema of G, min det, non-finite count
  double th = 0.0, gx = -DBL_MAX, gn = DBL_MAX, dm = DBL_MAX;
  int nf = 0;
  for (int t = tb + lane; t < te; t += 32) {
    const Partial& q = part[t];
    th += q.theta;
    gx = fmax(gx, q.gmax);
    gn = fmin(gn, q.gmin);
    dm = fmin(dm, q.dmin);
    nf += q.nonfinite;
  }
  th = warp_dsum(th);
  gx = warp_max(gx);
  gn = warp_min(gn);
  dm = warp_min(dm);
  nf = warp_isum(nf);
  // the rest is scalar (one lane) unless the residual needs per-subdomain
  // folds by the whole warp
  const bool per_sub = pd.stop_norm != PMA_STOP_MAX_UT || pd.stop_rule == PMA_RULE_ANY;
  if (lane != 0 && (phase == PH_INIT_THETA || !per_sub)) return;
  const double theta = th;
  double c_n = 0.0;
  if (pd.rhs == PMA_RHS_LOG && pd.normalize == PMA_NORM_GLOBAL_THETA) c_n = log(theta / pd.vol);
  const bool tangled = nf > 0 || !(dm > 0.0) || !isfinite(theta);
  if (phase == PH_INIT_THETA) {
    if (lane == 0) advance_init(ps, theta, c_n, dm, tangled, pd.max_steps);
    return;
  }
  // residual: per subdomain, combined by the stop rule (max = ALL, min = ANY)
  const bool any = (pd.stop_rule == PMA_RULE_ANY);
  double r;
  if (!per_sub) {
    r = fmax(gx - c_n, c_n - gn);
  } else {
    const double delta = c_n - c_lag;
    r = any ? INFINITY : 0.0;
    for (int s = 0; s < pd.nsub; ++s) {
      const SubDesc& sd = subs[pd.sub_base + s];
      double r_s;
      if (pd.stop_norm == PMA_STOP_MAX_UT) {
        double a1 = -DBL_MAX, a2 = DBL_MAX;
        for (int t = sd.tile_begin + lane; t < sd.tile_end; t += 32) {
          a1 = fmax(a1, part[t].gmax);
          a2 = fmin(a2, part[t].gmin);
        }
        a1 = warp_max(a1);
        a2 = warp_min(a2);
        r_s = fmax(a1 - c_n, c_n - a2);
      } else {
        double A = 0.0, B = 0.0, W = 0.0;
        for (int t = sd.tile_begin + lane; t < sd.tile_end; t += 32) {
          A += part[t].l2a;
          B += part[t].l2b;
          W += part[t].wsum;
        }
        A = warp_dsum(A);
        B = warp_dsum(B);
        W = warp_dsum(W);
        // sum w (G - c_n)^2 = sum w (G - c_lag - delta)^2
        const double q = A - 2.0 * delta * B + delta * delta * W;
        r_s = pd.dt * sqrt(q > 0.0 ? q : 0.0);
      }
      r = any ? fmin(r, r_s) : fmax(r, r_s);
    }
  }
  if (lane == 0)
    advance_run(ps, theta, c_n, dm, tangled, r, pd.dt, pd.check_every, pd.tol, pd.max_steps);
}

cudaError_t launch_finish(const int* list, int n, const SubDesc* subs, const ProbDesc* probs,
                          ProbState* st, const Partial* part, const unsigned int* err,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = (n * 32 + threads - 1) / threads;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_finish, list, n, subs, probs, st, part, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- helpers
// Owner's value at local node (i, j, l) of the item's subdomain (parallel
// transmission: previous step), through the subdomain's neighbour table.  A
// node outside this subdomain's core along an axis belongs to the
// neighbouring block on that side (cores hold >= ceil(o/2)+1 nodes).
// The item's first neighbour entry (3^D per subdomain).
template <typename T, int D>
__device__ __forceinline__ const NbEnt* item_nb(const LaunchArgs& a, const SmemHdr<T>& S) {
  return a.nb + S.ph.nb_base + (S.w.sub - S.ph.sub_base) * (D == 3 ? 27 : 9);
}
template <typename T, int D>
__device__ __forceinline__ T gather_owner(const NbEnt* nbi, const SmemHdr<T>& S, int i, int j,
                                          int l) {
  const int qx = i < S.sd.clo[0] ? 0 : (i > S.sd.chi[0] ? 2 : 1);
  const int qy = j < S.sd.clo[1] ? 0 : (j > S.sd.chi[1] ? 2 : 1);
  const int qz = D == 3 ? (l < S.sd.clo[2] ? 0 : (l > S.sd.chi[2] ? 2 : 1)) : 0;
  const NbEnt* e = nbi + qx + 3 * qy + 9 * qz;
  const T* ov = (const T*)__ldg((const unsigned long long*)&e->v[S.ps.parity]);
  if (ov == nullptr) return T(0);  // no such block: never a transmission node's owner
  const int2 pp = __ldg((const int2*)&e->pitch);
  return __ldcg(ov + i + (long long)pp.x * j + (long long)pp.y * l);
}

// Alternating transmission (Algorithm 1): a transmission node whose owner
// precedes its subdomain in raster order takes the owner's value of the
// current state (already updated this step), read lazily when the box is
// staged.  Overwrites every such position of a staged box (rows of SWp
// elements, SHY rows per plane, SHZ planes; column c holds local i0 + c - 4;
// halo columns 3 / cols + 4 on physical faces are mirror images) with the
// owner's value of buffer `parity` (no offset correction: the owner's
// updated nodes carry the same offset as this subdomain's).
template <typename T, int NT>
__device__ void stage_alternating(const LaunchArgs& a, const SmemHdr<T>& S, T* sv, int SWp,
                                  int SHY, int SHZ, int i0, int j0, int k0, int cols) {
  const SubDesc& sd = S.sd;
  const int n0 = sd.n[0], n1 = sd.n[1], n2 = sd.n[2], faces = sd.faces, dim = S.ph.dim;
  const bool plx = faces & 1, phx = faces & 2, ply = faces & 4, phy = faces & 8;
  const bool plz = faces & 16, phz = faces & 32;
  const int dlx = plx ? -1 : 0, dhx = phx ? -1 : n0 - 1;
  const int dly = ply ? -1 : 0, dhy = phy ? -1 : n1 - 1;
  const int dlz = (dim > 2 && !plz) ? 0 : -1, dhz = (dim > 2 && !phz) ? n2 - 1 : -1;
  const bool left = (i0 == 0), right = (i0 + cols == n0);
  const int PS = SHY * SWp;
  for (int rr = threadIdx.x; rr < SHY * SHZ; rr += NT) {
    const int lz = rr / SHY, ly = rr - lz * SHY;
    const int jj = reflect_clamp(j0 - 1 + ly, n1, ply, phy);
    const int kk = dim > 2 ? reflect_clamp(k0 - 1 + lz, n2, plz, phz) : 0;
    const bool drow = (jj == dly || jj == dhy || kk == dlz || kk == dhz);
    for (int c = 3; c <= cols + 4; ++c) {
      if (left && c == 3 && !plx) continue;          // halo beyond a transmission face
      if (right && c == cols + 4 && !phx) continue;  // (never read by an updated node)
      const int ii = reflect_clamp(i0 + c - 4, n0, plx, phx);
      if (!(drow || ii == dlx || ii == dhx)) continue;
      const int kx = sd.k[0] + (ii < sd.clo[0] ? -1 : (ii > sd.chi[0] ? 1 : 0));
      const int ky = sd.k[1] + (jj < sd.clo[1] ? -1 : (jj > sd.chi[1] ? 1 : 0));
      const int kz = sd.k[2] + (kk < sd.clo[2] ? -1 : (kk > sd.chi[2] ? 1 : 0));
      const int oidx = (kz * S.ph.parts[1] + ky) * S.ph.parts[0] + kx;
      if (oidx >= sd.idx) continue;
      const SubDesc* od = a.subs + S.ph.sub_base + oidx;
      const int ox = sd.g0[0] + ii - __ldg(&od->g0[0]);
      const int oy = sd.g0[1] + jj - __ldg(&od->g0[1]);
      const int oz = sd.g0[2] + kk - __ldg(&od->g0[2]);
      const long long opitch = __ldg(&od->pitch), on1 = __ldg(&od->n[1]);
      const T* ov = (const T*)od->v[S.ps.parity];
      sv[lz * PS + ly * SWp + c] = __ldcg(ov + ox + opitch * (oy + on1 * oz));
    }
  }
}

// Transmission nodes of a 3D box [i0, i0+cols) x [j0, j0+rows) x [k0,
// k0+depth) in a fixed enumeration: whole transmission planes, then in the
// other planes the transmission rows and the transmission columns of the
// remaining rows (each node once).
struct TrBox3 {
  int kp0, kp1, jr0, jr1, ic0, ic1;
  int npl, plane_e, nrow_e, per_plane, total;
  // node e (0 <= e < total); false for an entry already counted elsewhere
  __device__ __forceinline__ bool node(int e, int i0, int j0, int k0, int cols, int rows,
                                       int& i, int& j, int& kk) const {
    if (e < npl * plane_e) {
      const int q = e >= plane_e ? 1 : 0, rem = e - q * plane_e;
      kk = (q == 0 && kp0 >= 0) ? kp0 : kp1;
      const int rr = rem / cols;
      j = j0 + rr;
      i = i0 + rem - rr * cols;
      return true;
    }
    const int e2 = e - npl * plane_e, l = e2 / per_plane;
    kk = k0 + l;
    if (kk == kp0 || kk == kp1) return false;  // done with its plane
    const int e3 = e2 - l * per_plane;
    if (e3 < nrow_e) {
      const int q = e3 >= cols ? 1 : 0;
      j = (q == 0 && jr0 >= 0) ? jr0 : jr1;
      i = i0 + e3 - q * cols;
      return true;
    }
    const int e4 = e3 - nrow_e, q = e4 >= rows ? 1 : 0;
    i = (q == 0 && ic0 >= 0) ? ic0 : ic1;
    j = j0 + e4 - q * rows;
    return !(j == jr0 || j == jr1);  // corner: done with its row
  }
};
__device__ __forceinline__ TrBox3 tr_box3(int dlx, int dhx, int dly, int dhy, int dlz, int dhz,
                                          int i0, int j0, int k0, int cols, int rows,
                                          int depth) {
  TrBox3 t;
  t.kp0 = (dlz >= k0 && dlz < k0 + depth) ? dlz : -1;
  t.kp1 = (dhz >= k0 && dhz < k0 + depth) ? dhz : -1;
  t.jr0 = (dly >= j0 && dly < j0 + rows) ? dly : -1;
  t.jr1 = (dhy >= j0 && dhy < j0 + rows) ? dhy : -1;
  t.ic0 = (dlx >= i0 && dlx < i0 + cols) ? dlx : -1;
  t.ic1 = (dhx >= i0 && dhx < i0 + cols) ? dhx : -1;
  t.npl = (t.kp0 >= 0 ? 1 : 0) + (t.kp1 >= 0 ? 1 : 0);
  const int nrw = (t.jr0 >= 0 ? 1 : 0) + (t.jr1 >= 0 ? 1 : 0);
  const int ncl = (t.ic0 >= 0 ? 1 : 0) + (t.ic1 >= 0 ? 1 : 0);
  t.plane_e = rows * cols;
  t.nrow_e = nrw * cols;
  t.per_plane = t.nrow_e + ncl * rows;
  t.total = t.npl * t.plane_e + depth * t.per_plane;
  return t;
}

// ---------------------------------------------------------------- work queue
// Persistent CTAs pull work items from a per-launch counter (through the
// launch's order table when it has one); the last CTA to run out resets the
// counters for the next launch.  The partial record
// of an item is indexed by the item, so results do not depend on which CTA
// took it.
// The first grid positions of the order go to the CTAs statically (CTA b
// starts with position b, without the queue, so that it can fetch that item
// before the preceding launch has finished); the counter hands out the
// positions after them.
__device__ __forceinline__ int item_of_pos(const LaunchArgs& a, int q) {
  if (a.order == nullptr || q >= a.nwork) return a.t0 + q;
  return a.t0 + __ldg(a.order + q);
}
__device__ __forceinline__ int queue_ticket(const LaunchArgs& a) {
  return (int)atomicAdd(a.queue, 1u) + (int)gridDim.x;
}
__device__ __forceinline__ int pull_item(const LaunchArgs& a) {
  return item_of_pos(a, queue_ticket(a));
}
__device__ __forceinline__ void queue_exit(const LaunchArgs& a) {
  __threadfence();
  const unsigned int done = atomicAdd(a.queue + 1, 1u);
  if (done == gridDim.x - 1) {
    a.queue[0] = 0u;
    a.queue[1] = 0u;
    __threadfence();
  }
}

// ---------------------------------------------------------------- vector I/O
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  float v[4];
  __device__ __forceinline__ void lds(const float* p) {
    const float4 q = *(const float4*)p;
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  __device__ __forceinline__ void stg(float* p) const {
    asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3]));
  }
  __device__ __forceinline__ void sts(float* p) const {
    *(float4*)p = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec4<double> {
  double v[4];
  __device__ __forceinline__ void lds(const double* p) {
    const double2 q0 = *(const double2*)p, q1 = *(const double2*)(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
  }
  __device__ __forceinline__ void stg(double* p) const {
    asm volatile("st.global.v2.f64 [%0], {%1, %2};" ::"l"(p), "d"(v[0]), "d"(v[1]));
    asm volatile("st.global.v2.f64 [%0], {%1, %2};" ::"l"(p + 2), "d"(v[2]), "d"(v[3]));
  }
  __device__ __forceinline__ void sts(double* p) const {
    *(double2*)p = make_double2(v[0], v[1]);
    *(double2*)(p + 2) = make_double2(v[2], v[3]);
  }
};

// Pairs of values of the sweep precision.  FP32 pairs map to the packed
// FFMA2 / FADD2 / FMUL2 instructions of sm_100-family GPUs (two nodes per
// instruction); FP64 pairs are two scalar operations.
template <typename T>
struct P2;
template <>
struct P2<float> {
  float2 v;
  __device__ __forceinline__ float x() const { return v.x; }
  __device__ __forceinline__ float y() const { return v.y; }
  __device__ __forceinline__ static P2 mk(float a, float b) { return P2{make_float2(a, b)}; }
  __device__ __forceinline__ static P2 s(float a) { return P2{make_float2(a, a)}; }
};
template <>
struct P2<double> {
  double a, b;
  __device__ __forceinline__ double x() const { return a; }
  __device__ __forceinline__ double y() const { return b; }
  __device__ __forceinline__ static P2 mk(double p, double q) { return P2{p, q}; }
  __device__ __forceinline__ static P2 s(double p) { return P2{p, p}; }
};
__device__ __forceinline__ P2<float> padd(P2<float> a, P2<float> b) { return P2<float>{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2<float> pmul(P2<float> a, P2<float> b) { return P2<float>{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2<float> pfma(P2<float> a, P2<float> b, P2<float> c) {
  return P2<float>{__ffma2_rn(a.v, b.v, c.v)};
}
// a - b with one rounding, as a scalar subtraction
__device__ __forceinline__ P2<float> psub(P2<float> a, P2<float> b) {
  return P2<float>{__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)};
}
__device__ __forceinline__ P2<double> padd(P2<double> a, P2<double> b) { return {a.a + b.a, a.b + b.b}; }
__device__ __forceinline__ P2<double> pmul(P2<double> a, P2<double> b) { return {a.a * b.a, a.b * b.b}; }
__device__ __forceinline__ P2<double> pfma(P2<double> a, P2<double> b, P2<double> c) {
  return {fma(a.a, b.a, c.a), fma(a.b, b.b, c.b)};
}
__device__ __forceinline__ P2<double> psub(P2<double> a, P2<double> b) { return {a.a - b.a, a.b - b.b}; }
template <typename T>
__device__ __forceinline__ P2<T> pexw(P2<T> a) {
  return P2<T>::mk(Fm<T>::exw(a.x()), Fm<T>::exw(a.y()));
}

// ---------------------------------------------------------------- 2D stencil
// Three-input minimum / maximum (one instruction on sm_100-family GPUs for
// FP32; NaN operands are ignored as by fmin / fmax).
__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ double max3(double a, double b, double c) { return fmax(fmax(a, b), c); }
__device__ __forceinline__ double min3(double a, double b, double c) { return fmin(fmin(a, b), c); }

// Loop invariants of one 2D subdomain (or band) for one step, in registers.
template <typename T>
struct RunK {
  P2<T> NCL, DT2, M2, ONE, I2H0, I2H1, IH20, IH21, INV4, NINV4, BIG, NBIG;
  T c_lag, scale_root, inv_dim, lo0, h0, lo1, h1;
  int nterms;
  bool fast, logrhs, want_l2;
};

template <typename T>
__device__ __forceinline__ RunK<T> make_runk(const ProbHot<T>& ph, const ProbState& ps, int phase) {
  RunK<T> K;
  K.c_lag = (T)ps.c_lag;
  K.logrhs = ph.rhs == PMA_RHS_LOG || phase != PH_RUN;
  K.scale_root = K.inv_dim = T(0);
  if (!K.logrhs) {
    // (|Omega_c| rho det / theta)^(1/d) - 1 with the global normalisation,
    // (rho det)^(1/d) - 1 without it
    K.scale_root = ph.normalize == PMA_NORM_GLOBAL_THETA ? (T)(ph.vol / (T)ps.theta_prev) : T(1);
    K.inv_dim = T(1) / (T)ph.dim;
  }
  K.lo0 = ph.lo[0];
  K.lo1 = ph.lo[1];
  K.h0 = ph.h[0];
  K.h1 = ph.h[1];
  K.NCL = P2<T>::s(-K.c_lag);
  K.DT2 = P2<T>::s(ph.dt);
  K.M2 = P2<T>::s(T(-2));
  K.ONE = P2<T>::s(T(1));
  K.I2H0 = P2<T>::s(ph.inv2h[0]);
  K.I2H1 = P2<T>::s(ph.inv2h[1]);
  K.IH20 = P2<T>::s(ph.invh2[0]);
  K.IH21 = P2<T>::s(ph.invh2[1]);
  K.INV4 = P2<T>::s(ph.inv4hh[0]);
  K.NINV4 = P2<T>::s(-ph.inv4hh[0]);
  K.BIG = P2<T>::s(big_val<T>());
  K.NBIG = P2<T>::s(-big_val<T>());
  K.want_l2 = ph.stop_norm == PMA_STOP_L2_INCREMENT;
  K.nterms = ph.mon.nterms;
  K.fast = ph.mon_fast != 0;
  return K;
}

// G - c_lag of one node from rho det (the update's right-hand side: Eq.
// pmae in log form, or the d-th root form), the same arithmetic per lane as
// the packed evaluation in the stencil.
template <typename T>
__device__ __forceinline__ P2<T> rhs_pair(const RunK<T>& K, P2<T> rD);
template <>
__device__ __forceinline__ P2<float> rhs_pair<float>(const RunK<float>& K, P2<float> rD) {
  if (K.logrhs)
    return pfma(P2<float>::mk(lg2_approx(rD.x()), lg2_approx(rD.y())), P2<float>::s(Fm<float>::kLn2),
                K.NCL);
  return P2<float>::mk(Fm<float>::pw(K.scale_root * rD.x(), K.inv_dim) - 1.0f - K.c_lag,
                       Fm<float>::pw(K.scale_root * rD.y(), K.inv_dim) - 1.0f - K.c_lag);
}
template <>
__device__ __forceinline__ P2<double> rhs_pair<double>(const RunK<double>& K, P2<double> rD) {
  if (K.logrhs) return padd(P2<double>::mk(log(rD.x()), log(rD.y())), K.NCL);
  return P2<double>::mk(pow(K.scale_root * rD.x(), K.inv_dim) - 1.0 - K.c_lag,
                        pow(K.scale_root * rD.y(), K.inv_dim) - 1.0 - K.c_lag);
}

// Partial sums of one thread: theta (owned nodes), sum of G - c over updated
// nodes (a non-finite value anywhere makes it non-finite), extrema of
// rho det over updated nodes (G - c is monotone in it, so the extrema of
// G - c follow from two evaluations per thread), min det, and the
// L2-increment pieces.
template <typename T>
struct RunAcc {
  P2<T> th2, gs2;
  T rmax, rmin, dmin, l2a, l2b, ws;
  __device__ __forceinline__ static RunAcc zero() {
    RunAcc a;
    a.th2 = P2<T>::s(T(0));
    a.gs2 = P2<T>::s(T(0));
    a.rmax = T(0);
    a.rmin = big_val<T>();
    a.dmin = big_val<T>();
    a.l2a = a.l2b = a.ws = T(0);
    return a;
  }
  // extrema of G (= G - c_lag + c_lag), min det and the non-finite flag of
  // the thread's nodes; a thread without updated nodes (or whose largest
  // rho det is not positive: tangled) keeps the neutral extrema
  __device__ __forceinline__ void fold(const RunK<T>& K, Acc<T>& acc) const {
    const P2<T> g = rhs_pair<T>(K, P2<T>::mk(rmax > T(0) ? rmax : T(1), rmin));
    if (rmax > T(0)) acc.gmax = g.x() + K.c_lag;
    if (rmin < big_val<T>()) acc.gmin = g.y() + K.c_lag;
    acc.dmin = dmin;
    if (!isfinite(gs2.x() + gs2.y())) acc.nf += 1;
  }
};

// One run of 4 consecutive x-nodes of a row (Eqs. pmae2d, pmae): reads the
// 3 x 6 window around p (the first node of the run in a shared array of row
// stride SWp, with valid halo columns and rows), forms x = grad_h Psi,
// det D_h^2 Psi, rho(x) and G - c_lag, and returns v + dt (G - c_lag) in o
// (0 at nodes that are not updated: wc/uc/lc are the run's entries of the
// column tables, rowdir marks a transmission row).
// Columns c0-1 .. c0+4 of one staged row (p: column c0 of the row).
template <typename T>
__device__ __forceinline__ void load_row6(const T* p, T* w) {
  Vec4<T> m;
  w[0] = p[-1];
  m.lds(p);
  w[1] = m.v[0]; w[2] = m.v[1]; w[3] = m.v[2]; w[4] = m.v[3];
  w[5] = p[4];
}

// One Gaussian ring (RING) or bump term of the monitor sum at two pairs of
// nodes: amp exp(-width u) with u = ((x - c)^2 - r^2)^2 or (x - c)^2.
template <typename T, bool RING>
__device__ __forceinline__ void sum_terms2(const typename MonT<T>::Term& tm, const P2<T>* X0,
                                           const P2<T>* X1, P2<T>* R) {
  const P2<T> CX = P2<T>::s(tm.c[0]), CY = P2<T>::s(tm.c[1]);
  const P2<T> NWd = P2<T>::s(-tm.width), AMP = P2<T>::s(tm.amp);
#pragma unroll
  for (int pp = 0; pp < 2; ++pp) {
    const P2<T> d0 = psub(X0[pp], CX), d1 = psub(X1[pp], CY);
    P2<T> uu = pfma(d0, d0, pmul(d1, d1));
    if (RING) {
      const P2<T> s2 = psub(uu, P2<T>::s(tm.r2));
      uu = pmul(s2, s2);
    }
    R[pp] = pfma(AMP, pexw<T>(pmul(uu, NWd)), R[pp]);
  }
}
template <typename T, bool RING>
__device__ __forceinline__ void sum_terms3(const typename MonT<T>::Term& tm, const P2<T>* X0,
                                           const P2<T>* X1, const P2<T>* X2, P2<T>* R) {
  const P2<T> CX = P2<T>::s(tm.c[0]), CY = P2<T>::s(tm.c[1]), CZ = P2<T>::s(tm.c[2]);
  const P2<T> NWd = P2<T>::s(-tm.width), AMP = P2<T>::s(tm.amp);
#pragma unroll
  for (int pp = 0; pp < 2; ++pp) {
    const P2<T> d0 = psub(X0[pp], CX), d1 = psub(X1[pp], CY), d2 = psub(X2[pp], CZ);
    P2<T> uu = pfma(d0, d0, pfma(d1, d1, pmul(d2, d2)));
    if (RING) {
      const P2<T> s2 = psub(uu, P2<T>::s(tm.r2));
      uu = pmul(s2, s2);
    }
    R[pp] = pfma(AMP, pexw<T>(pmul(uu, NWd)), R[pp]);
  }
}

// Column tables of a staged band or subdomain, at the run's first column:
// theta weight (owned columns, else 0), 1 at updated columns (else 0), the
// local trapezoid weight, and with TAB the node's xi_x and +big at columns
// that are not updated (else 0); without TAB those two are formed from the
// global column index gi0.
template <typename T>
struct ColTab {
  const T *w, *u, *l, *x, *k;
  int gi0;
};

template <typename T, bool TAB>
__device__ __forceinline__ void stencil_core4(const RunK<T>& K, const MonT<T>& mon, const T* wS,
                                              const T* wC, const T* wN, const ColTab<T>& ct,
                                              bool rowdir, T wyo, T wly, T xi1, Vec4<T>& o,
                                              RunAcc<T>& A);

template <typename T, bool TAB>
__device__ __forceinline__ void stencil_run4(const RunK<T>& K, const MonT<T>& mon, const T* p,
                                             int SWp, const ColTab<T>& ct, bool rowdir, T wyo,
                                             T wly, T xi1, Vec4<T>& o, RunAcc<T>& A) {
  // 3 x 6 window: columns c0-1 .. c0+4 of rows j-1, j, j+1
  T wS[6], wC[6], wN[6];
  load_row6<T>(p - SWp, wS);
  load_row6<T>(p, wC);
  load_row6<T>(p + SWp, wN);
  stencil_core4<T, TAB>(K, mon, wS, wC, wN, ct, rowdir, wyo, wly, xi1, o, A);
}

// The stencil, monitor, update and reductions of one run from its 3 x 6
// window (rows j-1, j, j+1).
template <typename T, bool TAB>
__device__ __forceinline__ void stencil_core4(const RunK<T>& K, const MonT<T>& mon, const T* wS,
                                              const T* wC, const T* wN, const ColTab<T>& ct,
                                              bool rowdir, T wyo, T wly, T xi1, Vec4<T>& o,
                                              RunAcc<T>& A) {
  Vec4<T> wc, uc, xc;
  wc.lds(ct.w);
  uc.lds(ct.u);
  if (TAB) xc.lds(ct.x);
  const P2<T> dA = psub(P2<T>::mk(wN[0], wN[1]), P2<T>::mk(wS[0], wS[1]));
  const P2<T> dB = psub(P2<T>::mk(wN[2], wN[3]), P2<T>::mk(wS[2], wS[3]));
  const P2<T> dC = psub(P2<T>::mk(wN[4], wN[5]), P2<T>::mk(wS[4], wS[5]));
  P2<T> X0[2], X1[2], DD[2], R[2];
#pragma unroll
  for (int pp = 0; pp < 2; ++pp) {
    const P2<T> C = P2<T>::mk(wC[2 * pp + 1], wC[2 * pp + 2]);
    const P2<T> E = P2<T>::mk(wC[2 * pp + 2], wC[2 * pp + 3]);
    const P2<T> Wv = P2<T>::mk(wC[2 * pp], wC[2 * pp + 1]);
    const P2<T> Nn = P2<T>::mk(wN[2 * pp + 1], wN[2 * pp + 2]);
    const P2<T> Ss = P2<T>::mk(wS[2 * pp + 1], wS[2 * pp + 2]);
    const P2<T> XI0 = TAB ? P2<T>::mk(xc.v[2 * pp], xc.v[2 * pp + 1])
                          : P2<T>::mk(fma((T)(ct.gi0 + 2 * pp), K.h0, K.lo0),
                                      fma((T)(ct.gi0 + 2 * pp + 1), K.h0, K.lo0));
    X0[pp] = pfma(psub(E, Wv), K.I2H0, XI0);
    X1[pp] = pfma(psub(Nn, Ss), K.I2H1, P2<T>::s(xi1));
    const P2<T> hxx = pfma(pfma(C, K.M2, padd(E, Wv)), K.IH20, K.ONE);
    const P2<T> hyy = pfma(pfma(C, K.M2, padd(Nn, Ss)), K.IH21, K.ONE);
    const P2<T> df = pp == 0 ? psub(dB, dA) : psub(dC, dB);
    DD[pp] = pfma(pmul(df, K.INV4), pmul(df, K.NINV4), pmul(hxx, hyy));
  }
  if (K.fast) {
    // sum of Gaussian rings, then bumps, two nodes per operation
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) R[pp] = P2<T>::s(mon.base);
    for (int k = 0; k < mon.nring; ++k) sum_terms2<T, true>(mon.t[k], X0, X1, R);
    for (int k = mon.nring; k < K.nterms; ++k) sum_terms2<T, false>(mon.t[k], X0, X1, R);
  } else {
#pragma unroll
    for (int pp = 0; pp < 2; ++pp)
      R[pp] = P2<T>::mk(rho_at<T>(mon, X0[pp].x(), X1[pp].x(), T(0)),
                        rho_at<T>(mon, X0[pp].y(), X1[pp].y(), T(0)));
  }
  // Masks: 1 at updated nodes, 0 at the others (a transmission row or
  // column, or beyond the subdomain, where the window may hold stale
  // values).  The others get rho det := 1 (the one select per node), so
  // every value below stays finite there, their G - c enters the finiteness
  // sum as -c_lag, their theta weight is 0 (they are never owned), and
  // +-big offsets keep them out of the extrema.
  const P2<T> WYO = P2<T>::s(wyo);
  Vec4<T> kc;
  if (TAB) kc.lds(ct.k);
  P2<T> GMX[2], GMN[2], DMN[2], GCs[2], Ms[2];
#pragma unroll
  for (int pp = 0; pp < 2; ++pp) {
    const P2<T> uc2 = P2<T>::mk(uc.v[2 * pp], uc.v[2 * pp + 1]);
    const P2<T> m = rowdir ? P2<T>::s(T(0)) : uc2;
    const P2<T> rd = pmul(R[pp], DD[pp]);
    const P2<T> rD = P2<T>::mk(m.x() != T(0) ? rd.x() : T(1), m.y() != T(0) ? rd.y() : T(1));
    const P2<T> GC = rhs_pair<T>(K, rD);
    const P2<T> vn = pfma(GC, K.DT2, P2<T>::mk(wC[2 * pp + 1], wC[2 * pp + 2]));
    o.v[2 * pp] = vn.x();
    o.v[2 * pp + 1] = vn.y();
    A.gs2 = padd(A.gs2, GC);
    A.th2 = pfma(pmul(P2<T>::mk(wc.v[2 * pp], wc.v[2 * pp + 1]), WYO), rD, A.th2);
    const P2<T> kmn = TAB ? P2<T>::mk(kc.v[2 * pp], kc.v[2 * pp + 1])
                          : pfma(m, K.NBIG, K.BIG);  // 0 or +big
    GMX[pp] = pmul(rD, m);                     // rho det or 0
    GMN[pp] = pfma(rD, m, kmn);                // rho det or +big
    DMN[pp] = pfma(DD[pp], m, kmn);
    GCs[pp] = GC;
    Ms[pp] = m;
  }
  A.rmax = max3(max3(A.rmax, GMX[0].x(), GMX[0].y()), GMX[1].x(), GMX[1].y());
  A.rmin = min3(min3(A.rmin, GMN[0].x(), GMN[0].y()), GMN[1].x(), GMN[1].y());
  A.dmin = min3(min3(A.dmin, DMN[0].x(), DMN[0].y()), DMN[1].x(), DMN[1].y());
  if (K.want_l2) {
    Vec4<T> lc;
    lc.lds(ct.l);
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) {
      const P2<T> w = pmul(pmul(P2<T>::mk(lc.v[2 * pp], lc.v[2 * pp + 1]), P2<T>::s(wly)), Ms[pp]);
      const P2<T> d = pmul(GCs[pp], Ms[pp]);
      A.l2a = fma(w.x() * d.x(), d.x(), A.l2a);
      A.l2b = fma(w.x(), d.x(), A.l2b);
      A.ws += w.x();
      A.l2a = fma(w.y() * d.y(), d.y(), A.l2a);
      A.l2b = fma(w.y(), d.y(), A.l2b);
      A.ws += w.y();
    }
  }
}

// ---------------------------------------------------------------- 2D sweep
// Shared state of the band kernel: the current and the next work item's
// descriptors (the next one is fetched with cp.async while the current band
// is computed), the staged band and the reduction scratch.
template <typename T>
using BandHdr = SmemHdr<T>;

// The first item's descriptors in two parts: the work item, subdomain and
// problem descriptors (unchanged within a window) before the wait for the
// preceding launch, the problem state (which the finish pass writes) after
// it.
template <typename T>
__device__ __forceinline__ void issue_hdr_static(const LaunchArgs& a, BandHdr<T>& H,
                                                 const WorkItem& w) {
  H.w = w;
  const char* s0 = (const char*)(a.subs + w.sub);
  const char* s2 = (const char*)(hot_table<T>(a) + w.prob);
  for (int i = 0; i < (int)(sizeof(SubDesc) / 16); ++i) cp_async16((char*)&H.sd + 16 * i, s0 + 16 * i);
  for (int i = 0; i < (int)(sizeof(ProbHot<T>) / 16); ++i) cp_async16((char*)&H.ph + 16 * i, s2 + 16 * i);
}
template <typename T>
__device__ __forceinline__ void issue_hdr_state(const LaunchArgs& a, BandHdr<T>& H, int prob) {
  const char* s1 = (const char*)(a.st + prob);
  for (int i = 0; i < (int)(sizeof(ProbState) / 16); ++i) cp_async16((char*)&H.ps + 16 * i, s1 + 16 * i);
  cp_async_commit();
}

template <typename T>
__device__ __forceinline__ void issue_hdr(const LaunchArgs& a, BandHdr<T>& H, const WorkItem& w) {
  H.w = w;
  const char* s0 = (const char*)(a.subs + w.sub);
  const char* s1 = (const char*)(a.st + w.prob);
  const char* s2 = (const char*)(hot_table<T>(a) + w.prob);
  for (int i = 0; i < (int)(sizeof(SubDesc) / 16); ++i) cp_async16((char*)&H.sd + 16 * i, s0 + 16 * i);
  for (int i = 0; i < (int)(sizeof(ProbState) / 16); ++i) cp_async16((char*)&H.ps + 16 * i, s1 + 16 * i);
  for (int i = 0; i < (int)(sizeof(ProbHot<T>) / 16); ++i) cp_async16((char*)&H.ph + 16 * i, s2 + 16 * i);
  cp_async_commit();
}

// Thread 0: the pending queue ticket (if any) becomes the following item
// and its work item is loaded (used at the next item's top).
__device__ __forceinline__ void resolve_pull(const LaunchArgs& a, int& t_next, WorkItem& w_next,
                                             int& q_pend, int tend) {
  if (q_pend < 0) return;
  t_next = item_of_pos(a, q_pend);
  if (t_next < tend) w_next = a.work[t_next];
  q_pend = -1;
}

// Warp 0 after the per-warp partials are in shared memory: lane q < 7 folds
// field q of the item's record (theta, the three L2 sums, the extrema of
// G and min det) over the warps in warp order, lane 7 the non-finite count;
// each lane stores its field of the 64-byte record.
template <typename T, int NW>
__device__ __forceinline__ void write_record(const LaunchArgs& a, int t, int sub, const T* red_t,
                                             const T* red_f, const int* red_i, int lane) {
  double* const rec = (double*)(a.part + t);
  if (lane < 4) {
    T s = 0;
    for (int w = 0; w < NW; ++w) s += red_t[lane * NW + w];
    rec[lane] = (double)s;
  } else if (lane == 4) {
    T m = -big_val<T>();
    for (int w = 0; w < NW; ++w) m = fmax(m, red_f[w]);
    rec[4] = (double)m;
  } else if (lane < 7) {
    T m = big_val<T>();
    for (int w = 0; w < NW; ++w) m = fmin(m, red_f[(lane - 4) * NW + w]);
    rec[lane] = (double)m;
  } else if (lane == 7) {
    int cnt = 0;
    for (int w = 0; w < NW; ++w) cnt += red_i[w];
    *(int2*)(rec + 7) = make_int2(cnt, sub);
  }
}

// One work item is a band of `rows` x `cols` nodes of one subdomain (cols a
// multiple of 4 except at the subdomain's right edge; rows padded to a pitch
// of 4 elements in memory).  Staging (one pass): the band plus a one-node
// halo goes to shared memory with 16-byte loads, halo columns on the
// subdomain's x faces take the Neumann mirror, and transmission nodes get
// the offset correction.  Compute: each thread takes runs of 4 consecutive
// nodes of a row, reads the 3 x 6 stencil window with aligned vector loads
// and writes the 4 results with one 16-byte store.  Shared row layout: node
// column c sits at c + 4 (halo columns at 3 and cols + 4), rows are `SWp`
// (a multiple of 4) wide.
// Thread 0: the TMA box of the item whose header is H (its staged rows,
// SWp columns wide) into buffer sv, completing on barrier bar; false when
// the item is staged otherwise (done, first pass, or no tensor map).
template <typename T>
__device__ __forceinline__ bool issue_box2d(const LaunchArgs& a, const SmemHdr<T>& H, T* sv,
                                            unsigned long long* bar) {
  const int pc = H.ps.phase;
  if (pc == PH_DONE || pc == PH_INIT_V || a.tmap == nullptr || H.w.tma_rows <= 0) return false;
  const int swp = (((H.w.ext & 0xffff) + 3) & ~3) + 8;
  fence_proxy_async();
  mbar_expect_tx(bar, (unsigned int)(swp * H.w.tma_rows * (int)sizeof(T) + a.stall_bytes));
  tma_load_2d(sv, (const char*)a.tmap + 128 * ((size_t)H.w.tma_map + H.ps.parity),
              (H.w.ij & 0xffff) - 4, (H.w.ij >> 16) - 1, bar);
  return true;
}

template <typename T, int NT, int SMAX, int MB, bool PF>
__global__ void __launch_bounds__(NT, MB) k_band2d(LaunchArgs a) {
  constexpr int VW = 16 / (int)sizeof(T);
  constexpr int NW = NT / 32;
  // PF: two band buffers; the following item's box is loaded into the
  // other one while this item is computed.  A TMA destination in shared
  // memory must be 128-byte aligned, so the buffer stride SB is SMAX
  // rounded up to 128 bytes.
  constexpr int SB = (SMAX + 128 / (int)sizeof(T) - 1) / (128 / (int)sizeof(T)) * (128 / (int)sizeof(T));
  static_assert((SB * sizeof(T)) % 128 == 0, "band buffers start on 128-byte boundaries");
  __shared__ __align__(128) T sv_all[PF ? 2 * SB : SMAX];
  __shared__ __align__(16) BandHdr<T> HB[2];
  __shared__ __align__(8) unsigned long long tbar_all[2];  // TMA staging barriers
  __shared__ int s_t[2];
  __shared__ T red_t[4 * NW];
  __shared__ T red_f[3 * NW];
  __shared__ int red_i[NW];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tend = a.t0 + a.nwork;
  int t_next = 0;
  WorkItem w_next;
  unsigned int tphs = 0;  // bit k: parity of barrier k's next phase
  int q_pend = -1;        // thread 0: queue ticket not yet resolved
  bool ahead = false;     // thread 0: the current item's box was issued ahead
  if (tid == 0) {
    mbar_init(&tbar_all[0], 1);
    mbar_init(&tbar_all[1], 1);
  }
  // Before the wait for the preceding kernel of the stream (programmatic
  // dependent launch): this CTA's first item (its static position in the
  // order) and the descriptors that no launch of a window writes.
  int t0 = tend;
  if (tid == 0) {
    t0 = item_of_pos(a, (int)blockIdx.x);
    s_t[0] = t0;
    if (t0 < tend) issue_hdr_static<T>(a, HB[0], a.work[t0]);
  }
  // wait until the preceding kernel has completed and its writes are
  // visible; then the first item's state and the following item
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    if (t0 < tend) issue_hdr_state<T>(a, HB[0], HB[0].w.prob);
    t_next = pull_item(a);
    if (t_next < tend) w_next = a.work[t_next];
  }

  for (int it = 0;; ++it) {
    const int b = it & 1;
    if (tid == 0) cp_async_wait_all();
    __syncthreads();  // S1: header `b` complete and visible
    const int t = s_t[b];
    if (t >= tend) break;
    const int bb = PF ? b : 0;  // band buffer and barrier of this item
    T* const sv = sv_all + bb * SB;
    unsigned long long* const tbar = &tbar_all[bb];
    if (tid == 0) {
      // the band's TMA box first (unless it was issued ahead), so that its
      // copy overlaps the prefetch of the following item
      if (!ahead) issue_box2d<T>(a, HB[b], sv, tbar);
      ahead = false;
      // publish the following item, copy its descriptors into the other
      // header buffer and take the queue ticket of the item after it
      // (resolved once this item has been computed, so that the queue
      // atomic and the loads that depend on it do not hold up the staging)
      s_t[b ^ 1] = t_next;
      if (t_next < tend) {
        issue_hdr<T>(a, HB[b ^ 1], w_next);
        q_pend = queue_ticket(a);
      }
    }
    BandHdr<T>& H = HB[b];
    const int phase = H.ps.phase;
    if (phase == PH_DONE) {
      if (tid == 0) resolve_pull(a, t_next, w_next, q_pend, tend);
      continue;
    }
    const int n0 = H.sd.n[0], n1 = H.sd.n[1];
    const long long pitch = H.sd.pitch;
    const int i0 = H.w.ij & 0xffff, j0 = H.w.ij >> 16;
    const int cols = H.w.ext & 0xffff, rows = H.w.ext >> 16;
    const int faces = H.sd.faces;
    const int g00 = H.sd.g0[0], g01 = H.sd.g0[1];
    const T* src = (const T*)H.sd.v[H.ps.parity];
    T* dst = (T*)H.sd.v[H.ps.parity ^ 1];
    const int rpr = (cols + 3) >> 2;  // runs per row
    const int nruns = rows * rpr;
    const float inv_rpr = __fdividef(1.0f, (float)rpr);
    // transmission nodes: local index equal to one of these (-1 = none)
    const int dlx = (faces & 1) ? -1 : 0, dhx = (faces & 2) ? -1 : n0 - 1;
    const int dly = (faces & 4) ? -1 : 0, dhy = (faces & 8) ? -1 : n1 - 1;
    T th = 0, l2a = 0, l2b = 0, ws = 0;
    Acc<T> acc{-big_val<T>(), big_val<T>(), big_val<T>(), 0};

    if (phase == PH_INIT_V) {
      // v^0 into both buffers (the next pass reads buffer `parity`)
      const double* psi0 = a.probs[H.w.prob].psi0;
      const int Nx = H.ph.N[0];
      for (int q = tid; q < nruns; q += NT) {
        const int r = qdiv(q, rpr, inv_rpr), c0 = (q - r * rpr) * 4;
        const int j = j0 + r;
        Vec4<T> o;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + c0 + u;
          T v0 = T(0);
          if (psi0 && i < n0) {
            const int gi = g00 + i, gj = g01 + j;
            const double xi = (double)H.ph.lo[0] + (double)gi * H.ph.hd[0];
            const double et = (double)H.ph.lo[1] + (double)gj * H.ph.hd[1];
            v0 = (T)(psi0[(long long)gj * Nx + gi] - 0.5 * (xi * xi + et * et));
          }
          o.v[u] = v0;
        }
        o.stg(dst + j * pitch + i0 + c0);
        o.stg((T*)src + j * pitch + i0 + c0);
      }
    } else {
      const int SWp = ((cols + 3) & ~3) + 8;
      const int SH = rows + 2;
      const int tr = a.tmap != nullptr ? H.w.tma_rows : 0;
      const int cpr = SWp / VW;  // 16-byte chunks per shared row
      const float inv_cpr = __fdividef(1.0f, (float)cpr);
      const bool plx = faces & 1, phx = faces & 2, ply = faces & 4, phy = faces & 8;
      // (a) the band rows (global columns i0-4 .. i0+SWp-5, rows j0-1 ..
      //     j0+rows): one TMA box where the subdomain has tensor maps (the
      //     box holds SHT >= SH rows; zeros outside the buffer, mirror rows
      //     fixed below), else 16-byte asynchronous copies (chunks outside
      //     the pitched row skipped, rows mirrored / clamped).
      const int SHT = tr > 0 ? tr : SH;
      if (tr > 0) {
        // the box was issued right after S1
      } else {
        for (int e = tid; e < SH * cpr; e += NT) {
          const int r = qdiv(e, cpr, inv_cpr), k = e - r * cpr;
          const int gs = i0 - 4 + k * VW;
          if (gs >= 0 && gs + VW <= pitch) {
            const int jj = reflect_clamp(j0 - 1 + r, n1, ply, phy);
            cp_async16(sv + r * SWp + k * VW, src + jj * pitch + gs);
          }
        }
      }
      cp_async_commit();
      // (b) halo columns on the subdomain's x faces (Neumann mirror; clamp on
      //     transmission faces, where the value is never used): loads issued
      //     now (their latency overlaps the tables and the transmission
      //     pass), written after the copies land.  At most 2 rows per thread.
      const bool left = (i0 == 0), right = (i0 + cols == n0);
      const T corr = (T)H.ps.corr;
      T hl[2], hr[2], hc[2];  // raw halo values and their offset (added at (c))
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int r = tid + q * NT;
        hl[q] = hr[q] = hc[q] = T(0);
        if (r < SH && (left || right)) {
          const int jj = reflect_clamp(j0 - 1 + r, n1, ply, phy);
          hc[q] = (jj == dly || jj == dhy) ? corr : T(0);
          if (left && plx) hl[q] = __ldcg(src + jj * pitch + 1);
          if (right && phx) hr[q] = __ldcg(src + jj * pitch + n0 - 2);
        }
      }
      // Per-column tables of the band (after the staged rows in shared
      // memory): theta weight of owned columns (0 elsewhere), 1 for updated
      // columns (inside the band, not a transmission column), the local
      // trapezoid weight for the L2 increment, xi_x, and +big at columns
      // that are not updated (0 elsewhere).
      const int cr = (cols + 3) & ~3;
      {
      const T h0 = H.ph.h[0], hw0 = H.ph.hw[0], lo0 = H.ph.lo[0];
      const int N0 = H.ph.N[0], clo0 = H.sd.clo[0], chi0 = H.sd.chi[0];
      T* const wcol = sv + SHT * SWp;
      T* const ucol = wcol + cr;
      T* const lcol = ucol + cr;
      T* const xcol = lcol + cr;
      T* const kcol = xcol + cr;
      for (int c = tid; c < cr; c += NT) {
        const int i = i0 + c, gi = g00 + i;
        const bool valid = c < cols;
        const bool upd = valid && i != dlx && i != dhx;
        wcol[c] = (valid && i >= clo0 && i <= chi0) ? ((gi == 0 || gi == N0 - 1) ? hw0 : h0) : T(0);
        ucol[c] = upd ? T(1) : T(0);
        lcol[c] = (i == 0 || i == n0 - 1) ? hw0 : h0;
        xcol[c] = fma((T)gi, h0, lo0);
        kcol[c] = upd ? T(0) : big_val<T>();
      }
      }
      // Transmission nodes of the band (Eq. transmission_condition3): whole
      // transmission rows, then the transmission columns of the other rows,
      // one node per thread, while the staging copies are in flight (the
      // main loop does not store these nodes).  At a step without exchange
      // (exchange_every > 1) the nodes keep their staged values instead,
      // copied once the band has landed (after S2).
      const int jr0 = (dly >= j0 && dly < j0 + rows) ? dly : -1;
      const int jr1 = (dhy >= j0 && dhy < j0 + rows) ? dhy : -1;
      const int ic0 = (dlx >= i0 && dlx < i0 + cols) ? dlx : -1;
      const int ic1 = (dhx >= i0 && dhx < i0 + cols) ? dhx : -1;
      const int nrow_e = ((jr0 >= 0 ? 1 : 0) + (jr1 >= 0 ? 1 : 0)) * cols;
      const int tr_total = nrow_e + ((ic0 >= 0 ? 1 : 0) + (ic1 >= 0 ? 1 : 0)) * rows;
      const int kex = H.ph.exchange_every;
      const bool exch = exchange_step(H.ps.step, kex);
      if (phase == PH_RUN && exch) {
        const int total = tr_total;
        const NbEnt* const nbi = item_nb<T, 2>(a, H);
        for (int e0 = tid; e0 < total; e0 += 2 * NT) {
          // two nodes per thread and pass: both owner loads before the stores
          T val[2];
          T* dp[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int e = e0 + u * NT;
            dp[u] = nullptr;
            val[u] = T(0);
            if (e >= total) continue;
            int i, j;
            if (e < nrow_e) {
              const int q = e >= cols ? 1 : 0;
              j = (q == 0 && jr0 >= 0) ? jr0 : jr1;
              i = i0 + e - q * cols;
            } else {
              const int e2 = e - nrow_e;
              const int q = e2 >= rows ? 1 : 0;
              i = (q == 0 && ic0 >= 0) ? ic0 : ic1;
              j = j0 + e2 - q * rows;
              if (j == jr0 || j == jr1) continue;  // corner: done with its row
            }
            dp[u] = dst + j * pitch + i;
            val[u] = gather_owner<T, 2>(nbi, H, i, j, 0);
          }
#pragma unroll
          for (int u = 0; u < 2; ++u)
            if (dp[u]) st_global(dp[u], val[u]);
        }
      }
      cp_async_wait_all();
      bool gave_up = false;
      if (tr > 0) {
        gave_up = !mbar_wait(tbar, (tphs >> bb) & 1u);
        tphs ^= 1u << bb;
      }
      if (__syncthreads_or(gave_up)) {
        // the box never arrived: report, give the copy one more bounded
        // wait, and leave (the host turns the error word into a status)
        if (tid == 0) {
          atomicOr(a.err, 1u);
          mbar_wait(tbar, ((tphs >> bb) & 1u) ^ 1u);
        }
        break;
      }
      if (tr > 0 && ((ply && j0 == 0) || (phy && j0 + rows == n1))) {
        // Neumann mirror rows of a TMA box (zeros outside the buffer):
        // staged row 0 <- row 2, row rows+1 <- row rows-1 (halo columns
        // are written by (c))
        for (int c = tid; c < SWp; c += NT) {
          if ((left && c == 3) || (right && c == cols + 4)) continue;
          if (ply && j0 == 0) sv[c] = sv[2 * SWp + c];
          if (phy && j0 + rows == n1) sv[(rows + 1) * SWp + c] = sv[(rows - 1) * SWp + c];
        }
        __syncthreads();
      }
      // (c) halo values, and the offset of transmission nodes (only the band's
      //     perimeter can hold them): whole rows whose global row is a
      //     transmission row (halo columns excluded: written by (b)), and the
      //     columns of global column 0 / n0-1 when those are transmission
      //     columns, in the other rows.
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int r = tid + q * NT;
        if (r < SH) {
          if (left) sv[r * SWp + 3] = hl[q] + hc[q];
          if (right) sv[r * SWp + cols + 4] = hr[q] + hc[q];
        }
      }
      const int fl = H.w.flags;
      if (corr != T(0) && fl != 0) {
        const int r0 = (fl & 1) ? 0 : -1, r1 = (fl & 2) ? 1 : -1;
        const int r2 = (fl & 4) ? SH - 2 : -1, r3 = (fl & 8) ? SH - 1 : -1;
        if (fl & 48) {
          const int cl = (fl & 16) ? 4 : -1, ch = (fl & 32) ? cols + 3 : -1;
          for (int r = tid; r < SH; r += NT) {
            if (r != r0 && r != r1 && r != r2 && r != r3) {
              if (cl >= 0) sv[r * SWp + cl] += corr;
              if (ch >= 0) sv[r * SWp + ch] += corr;
            }
          }
        }
        if (fl & 15) {
          const int rr[4] = {r0, r1, r2, r3};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (rr[q] < 0) continue;
            for (int c = tid; c < SWp; c += NT)
              if (!(left && c == 3) && !(right && c == cols + 4)) sv[rr[q] * SWp + c] += corr;
          }
        }
      }
      if (H.ph.alternating && exchange_step(H.ps.step - 1, kex)) {
        __syncthreads();
        stage_alternating<T, NT>(a, H, sv, SWp, SH, 1, i0, j0, 0, cols);
      }
      __syncthreads();  // S2: band staged
      if constexpr (PF) {
        if (tid == 0 && t_next < tend) {
          // the following item's box into the other buffer (its header was
          // requested at this item's top; the buffer's last item is done)
          cp_async_wait_all();
          ahead = issue_box2d<T>(a, HB[b ^ 1], sv_all + (bb ^ 1) * SB, &tbar_all[bb ^ 1]);
        }
      }
      if (phase == PH_RUN && !exch) {
        // interface data frozen between exchanges: every transmission node
        // of the band keeps the value it was staged with (offset included)
        for (int e = tid; e < tr_total; e += NT) {
          int i, j;
          if (e < nrow_e) {
            const int q = e >= cols ? 1 : 0;
            j = (q == 0 && jr0 >= 0) ? jr0 : jr1;
            i = i0 + e - q * cols;
          } else {
            const int e2 = e - nrow_e;
            const int q = e2 >= rows ? 1 : 0;
            i = (q == 0 && ic0 >= 0) ? ic0 : ic1;
            j = j0 + e2 - q * rows;
            if (j == jr0 || j == jr1) continue;  // corner: done with its row
          }
          st_global(dst + j * pitch + i, sv[(j - j0 + 1) * SWp + (i - i0 + 4)]);
        }
      }
      const T h0 = H.ph.h[0], h1 = H.ph.h[1];
      const T hw0 = H.ph.hw[0], hw1 = H.ph.hw[1];
      const int N0 = H.ph.N[0], N1 = H.ph.N[1];
      const int clo0 = H.sd.clo[0], chi0 = H.sd.chi[0], clo1 = H.sd.clo[1], chi1 = H.sd.chi[1];
      const bool run = phase == PH_RUN;
      const T* const wcol = sv + SHT * SWp;
      const T* const ucol = wcol + cr;
      const T* const lcol = ucol + cr;
      const T* const xcol = lcol + cr;
      const T* const kcol = xcol + cr;

      // partial sums: theta, sum of (G - c) over updated nodes (a non-finite
      // value anywhere makes it non-finite), extrema of G - c, min det
      const RunK<T> K = make_runk<T>(H.ph, H.ps, phase);
      RunAcc<T> A = RunAcc<T>::zero();
      // transmission rows (only a band's first or last row can be one) are
      // written by the transmission pass and skipped here
      const int rlo = (j0 == dly) ? 1 : 0;
      const int rhi = (j0 + rows - 1 == dhy) ? rows - 1 : rows;
      const int nrun_u = rhi > rlo ? (rhi - rlo) * rpr : 0;
      for (int q = tid; q < nrun_u; q += NT) {
        const int rq = qdiv(q, rpr, inv_rpr), r = rlo + rq, c0 = (q - rq * rpr) * 4;
        const int j = j0 + r, gj = g01 + j;
        const T wyo = (j >= clo1 && j <= chi1) ? ((gj == 0 || gj == N1 - 1) ? hw1 : h1) : T(0);
        const T wly = (j == 0 || j == n1 - 1) ? hw1 : h1;
        Vec4<T> o;
        const ColTab<T> ct{wcol + c0, ucol + c0, lcol + c0, xcol + c0, kcol + c0, 0};
        stencil_run4<T, true>(K, H.ph.mon, sv + (r + 1) * SWp + c0 + 4, SWp, ct, false, wyo,
                              wly, fma((T)gj, K.h1, K.lo1), o, A);
        if (run) {
          T* const q = dst + j * pitch + i0 + c0;
          if ((i0 + c0 <= dlx) || (i0 + c0 + 3 >= dhx && dhx >= 0)) {
            // a run holding a transmission column: updated nodes only
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int i = i0 + c0 + u;
              if (i != dlx && i != dhx) st_global(q + u, o.v[u]);
            }
          } else {
            o.stg(q);
          }
        }
      }
      A.fold(K, acc);
      l2a = A.l2a;
      l2b = A.l2b;
      ws = A.ws;
      th = A.th2.x() + A.th2.y();
    }
    if (tid == 0) resolve_pull(a, t_next, w_next, q_pend, tend);
    // tile record
    th = warp_sum(th);
    if (H.ph.stop_norm == PMA_STOP_L2_INCREMENT) {
      l2a = warp_sum(l2a);
      l2b = warp_sum(l2b);
      ws = warp_sum(ws);
    }
    const T gmax = warp_max(acc.gmax), gmin = warp_min(acc.gmin), dmin = warp_min(acc.dmin);
    const int nf = warp_isum(acc.nf);
    if (lane == 0) {
      red_t[0 * NW + wid] = th;
      red_t[1 * NW + wid] = l2a;
      red_t[2 * NW + wid] = l2b;
      red_t[3 * NW + wid] = ws;
      red_f[0 * NW + wid] = gmax;
      red_f[1 * NW + wid] = gmin;
      red_f[2 * NW + wid] = dmin;
      red_i[wid] = nf;
    }
    __syncthreads();  // S3
    if (wid == 0) write_record<T, NW>(a, t, H.w.sub, red_t, red_f, red_i, lane);
  }
  if (tid == 0) queue_exit(a);
  // this CTA has run out of work: the next kernel of the stream (launched
  // as a programmatic dependent) may be scheduled while the last CTAs finish
  asm volatile("griddepcontrol.launch_dependents;");
}

// ---------------------------------------------------------------- resident 2D
// k_res2d: one CTA per subdomain, the whole subdomain in shared memory for
// up to `iters` steps of the parallel DD method (Sect. 3), thread-block
// clusters holding all subdomains of a problem.  Per step:
//   1. after the cluster barrier, warp 0 folds the problem's per-subdomain
//      records of the previous step (read from the other CTAs' shared
//      memory, fixed order) into theta, c^n, the residual and the stop test,
//      exactly as the batched finish does;
//   2. transmission nodes (Eq. transmission_condition3): the value copied one
//      step earlier gets the offset correction, and the owner's current value
//      is copied (distributed shared memory) into the next buffer;
//   3. every run of 4 nodes is updated from the current buffer into the next
//      one (same arithmetic as the band kernel), mirror ghosts of physical
//      faces (Eq. nbd) are written alongside;
//   4. the CTA's record goes to its shared memory; cluster barrier.
// Dynamic shared memory: buffer 0 and 1 (`cap` elements each; buffer b holds
// v[b], subdomain row j at (j+1)*SWp, node column i at i+4, one halo row and
// column on every side), then the column tables and the transmission list
// (int2: local position, owner rank << 20 | position in the owner's buffer).
struct ResDecide {
  double vol, dt, tol;
  long long max_steps;
  int nsub, stop_norm, stop_rule, check_every, rhs, normalize;
};

// Step 1 for one problem (warp 0 of each of its CTAs; identical inputs and
// order in every CTA, so all of them take the same decision).
__device__ __forceinline__ void res_decide(ProbState& ps, const ResDecide& dk, const Partial* recs,
                                           int rank0, int lane) {
  const int ph0 = ps.phase;
  const double c_lag = ps.c_lag;
  __syncwarp();
  const bool mine = lane < dk.nsub;
  double th = 0.0, gx = -DBL_MAX, gn = DBL_MAX, dm = DBL_MAX, A = 0.0, B = 0.0, Wt = 0.0;
  int nf = 0;
  if (mine) {
    const unsigned int ra = dsmem_map(recs, (unsigned int)(rank0 + lane));
    th = dsmem_ld(ra + (unsigned int)offsetof(Partial, theta), 0.0);
    A = dsmem_ld(ra + (unsigned int)offsetof(Partial, l2a), 0.0);
    B = dsmem_ld(ra + (unsigned int)offsetof(Partial, l2b), 0.0);
    Wt = dsmem_ld(ra + (unsigned int)offsetof(Partial, wsum), 0.0);
    gx = dsmem_ld(ra + (unsigned int)offsetof(Partial, gmax), 0.0);
    gn = dsmem_ld(ra + (unsigned int)offsetof(Partial, gmin), 0.0);
    dm = dsmem_ld(ra + (unsigned int)offsetof(Partial, dmin), 0.0);
    nf = dsmem_ld(ra + (unsigned int)offsetof(Partial, nonfinite), 0);
  }
  const double gxs = gx, gns = gn;
  th = warp_dsum(th);
  gx = warp_max(gx);
  gn = warp_min(gn);
  dm = warp_min(dm);
  nf = warp_isum(nf);
  const double theta = th;
  double c_n = 0.0;
  if (dk.rhs == PMA_RHS_LOG && dk.normalize == PMA_NORM_GLOBAL_THETA) c_n = log(theta / dk.vol);
  const bool tangled = nf > 0 || !(dm > 0.0) || !isfinite(theta);
  if (ph0 == PH_INIT_THETA) {
    if (lane == 0) advance_init(&ps, theta, c_n, dm, tangled, dk.max_steps);
    __syncwarp();
    return;
  }
  const bool any = (dk.stop_rule == PMA_RULE_ANY);
  double r;
  if (dk.stop_norm == PMA_STOP_MAX_UT && !any) {
    r = fmax(gx - c_n, c_n - gn);
  } else {
    double r_s;
    if (dk.stop_norm == PMA_STOP_MAX_UT) {
      r_s = fmax(gxs - c_n, c_n - gns);
    } else {
      const double delta = c_n - c_lag;
      const double q = A - 2.0 * delta * B + delta * delta * Wt;
      r_s = dk.dt * sqrt(q > 0.0 ? q : 0.0);
    }
    if (!mine) r_s = any ? INFINITY : 0.0;
    r = any ? warp_min(r_s) : warp_max(r_s);
  }
  if (lane == 0)
    advance_run(&ps, theta, c_n, dm, tangled, r, dk.dt, dk.check_every, dk.tol, dk.max_steps);
  __syncwarp();
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? 1024 : 512) / NT) k_res2d(ResArgs a) {
  constexpr int NW = NT / 32;
  constexpr int VW = 16 / (int)sizeof(T);
  extern __shared__ __align__(16) unsigned char res_smem[];
  T* const buf = (T*)res_smem;
  __shared__ __align__(16) SubDesc sd;
  __shared__ __align__(16) ProbHot<T> ph;
  __shared__ __align__(16) ProbState ps;
  __shared__ ResDecide dk;
  __shared__ __align__(16) Partial rec[2];
  __shared__ int act[2];
  __shared__ int rank_cap[kResClusterMax];
  __shared__ int s_ndir, s_exit;
  __shared__ T red_t[4 * NW];
  __shared__ T red_f[3 * NW];
  __shared__ int red_i[NW];

  const int tid = threadIdx.x, lane = tid & 31;
  const ResCta me = a.ctas[blockIdx.x];
  const bool has = me.sub >= 0;
  const int csize = (int)cluster_size();
  const ProbHot<T>* hot = (const ProbHot<T>*)(sizeof(T) == 4 ? (const void*)a.hotf
                                                               : (const void*)a.hotd);
  const int prob = has ? __ldg(&a.subs[me.sub].prob) : 0;
  if (has) {
    coop_copy<NT>(&sd, a.subs + me.sub, (int)sizeof(SubDesc), 0);
    coop_copy<NT>(&ph, hot + prob, (int)sizeof(ProbHot<T>), 0);
    coop_copy<NT>(&ps, a.st + prob, (int)sizeof(ProbState), 0);
    if (tid == 0) {
      const ProbDesc& pd = a.probs[prob];
      dk.vol = pd.vol;
      dk.dt = pd.dt;
      dk.tol = pd.tol;
      dk.max_steps = pd.max_steps;
      dk.nsub = pd.nsub;
      dk.stop_norm = pd.stop_norm;
      dk.stop_rule = pd.stop_rule;
      dk.check_every = pd.check_every;
      dk.rhs = pd.rhs;
      dk.normalize = pd.normalize;
    }
    // buffer capacity of every CTA of the problem (owners of transmission
    // values are read at buffer parity * capacity + position)
    const int nsub = __ldg(&a.probs[prob].nsub), base = __ldg(&a.probs[prob].sub_base);
    if (tid < nsub)
      rank_cap[me.rank0 + tid] =
          res_cap_elems(__ldg(&a.subs[base + tid].n[0]), __ldg(&a.subs[base + tid].n[1]));
  }
  if (tid == 0) {
    act[0] = act[1] = 0;
    s_ndir = 0;
    s_exit = 0;
  }
  __syncthreads();

  int n0 = 4, n1 = 4, cr = 4, SWp = 12, g00 = 0, g01 = 0, cap = 0;
  int clo1 = 0, chi1 = 0, N1 = 1, dlx = -1, dhx = -1, dly = -1, dhy = -1;
  bool plx = true, phx = true, ply = true, phy = true, loaded = false;
  T h1 = 0, hw1 = 0;
  T *wcol = buf, *ucol = buf, *lcol = buf, *dorig = buf;
  int2* dlist = (int2*)buf;
  if (has) {
    n0 = sd.n[0];
    n1 = sd.n[1];
    cr = (n0 + 3) & ~3;
    SWp = cr + 8;
    cap = res_cap_elems(n0, n1);
    g00 = sd.g0[0];
    g01 = sd.g0[1];
    const int faces = sd.faces;
    plx = faces & 1;
    phx = faces & 2;
    ply = faces & 4;
    phy = faces & 8;
    dlx = plx ? -1 : 0;
    dhx = phx ? -1 : n0 - 1;
    dly = ply ? -1 : 0;
    dhy = phy ? -1 : n1 - 1;
    clo1 = sd.clo[1];
    chi1 = sd.chi[1];
    N1 = ph.N[1];
    h1 = ph.h[1];
    hw1 = ph.hw[1];
    wcol = buf + 2 * cap;
    ucol = wcol + cr;
    lcol = ucol + cr;
    dlist = (int2*)(lcol + cr);
    dorig = (T*)(dlist + 2 * (n0 + n1) + 8);
    // column tables: theta weight of owned columns, 1 for updated columns,
    // local trapezoid weight
    {
      const int clo0 = sd.clo[0], chi0 = sd.chi[0], N0 = ph.N[0];
      const T h0 = ph.h[0], hw0 = ph.hw[0];
      for (int c = tid; c < cr; c += NT) {
        const int gi = g00 + c;
        const bool valid = c < n0;
        wcol[c] = (valid && c >= clo0 && c <= chi0) ? ((gi == 0 || gi == N0 - 1) ? hw0 : h0) : T(0);
        ucol[c] = (valid && c != dlx && c != dhx) ? T(1) : T(0);
        lcol[c] = (c == 0 || c == n0 - 1) ? hw0 : h0;
      }
    }
    // transmission nodes on the subdomain's ring, with their owners (the
    // neighbouring block whose core holds the node) and the mirror images
    // that the Neumann faces give them
    const int ring = 2 * n0 + 2 * (n1 - 2);
    for (int e = tid; e < ring; e += NT) {
      int i, j;
      if (e < n0) {
        i = e;
        j = 0;
      } else if (e < 2 * n0) {
        i = e - n0;
        j = n1 - 1;
      } else {
        const int k = e - 2 * n0;
        i = (k & 1) ? n0 - 1 : 0;
        j = 1 + (k >> 1);
      }
      if (!(i == dlx || i == dhx || j == dly || j == dhy)) continue;
      const int kx = sd.k[0] + (i < sd.clo[0] ? -1 : (i > sd.chi[0] ? 1 : 0));
      const int ky = sd.k[1] + (j < sd.clo[1] ? -1 : (j > sd.chi[1] ? 1 : 0));
      const int oidx = ky * ph.parts[0] + kx;
      const SubDesc* od = a.subs + ph.sub_base + oidx;
      const int ox = g00 + i - __ldg(&od->g0[0]);
      const int oy = g01 + j - __ldg(&od->g0[1]);
      const int oswp = ((__ldg(&od->n[0]) + 3) & ~3) + 8;
      const int src = ((me.rank0 + oidx) << 20) | ((oy + 1) * oswp + ox + 4);
      const int xm = (plx && i == 1) ? -1 : ((phx && i == n0 - 2) ? n0 : -2);
      const int ym = (ply && j == 1) ? -1 : ((phy && j == n1 - 2) ? n1 : -2);
      const int nx = xm != -2 ? 2 : 1, ny = ym != -2 ? 2 : 1;
      const int slot = atomicAdd(&s_ndir, nx * ny);
      int q = 0;
      for (int b = 0; b < ny; ++b)
        for (int c = 0; c < nx; ++c) {
          const int jj = b ? ym : j, ii = c ? xm : i;
          dlist[slot + q++] = make_int2((jj + 1) * SWp + ii + 4, src);
        }
    }
    // state v[parity] (or v^0) with mirror / clamp halos into both buffers
    const int phase0 = ps.phase;
    loaded = phase0 != PH_DONE;
    if (loaded) {
      const int par = ps.parity;
      const T* g = (const T*)sd.v[par];
      const long long pitch = sd.pitch;
      const double* psi0 = a.probs[prob].psi0;
      const int Nx = ph.N[0];
      for (int e = tid; e < (n1 + 2) * SWp; e += NT) {
        const int r = e / SWp, c = e - r * SWp;
        const int i = c - 4, j = r - 1;
        T val = T(0);
        if (i >= -1 && i <= n0) {
          const int ii = reflect_clamp(i, n0, plx, phx), jj = reflect_clamp(j, n1, ply, phy);
          if (phase0 == PH_INIT_V) {
            if (psi0) {
              const int gi = g00 + ii, gj = g01 + jj;
              const double xi = (double)ph.lo[0] + (double)gi * ph.hd[0];
              const double et = (double)ph.lo[1] + (double)gj * ph.hd[1];
              val = (T)(psi0[(long long)gj * Nx + gi] - 0.5 * (xi * xi + et * et));
            }
          } else {
            val = __ldcg(g + jj * pitch + ii);
          }
        }
        buf[par * cap + e] = val;
        buf[(par ^ 1) * cap + e] = val;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && has && ps.phase == PH_INIT_V) ps.phase = PH_INIT_THETA;
  // every CTA of the cluster has loaded its state before any other CTA reads
  // it through shared::cluster (the first step's transmission values)
  cluster_arrive();
  cluster_wait();

  const int rpr = cr >> 2;
  const int nruns = n1 * rpr;
  const float inv_rpr = __fdividef(1.0f, (float)rpr);
  bool computed = false;
  int dpar = -1;  // buffer whose transmission values carry the last correction
  for (int it = 0;; ++it) {
    if (it > 0) {
      cluster_wait();
      if (tid < 32) {
        const int slot = (it - 1) & 1;
        int f = 0;
        if (lane < csize) f = dsmem_ld(dsmem_map(&act[slot], (unsigned int)lane), 0);
        const bool any = __any_sync(0xffffffffu, f != 0);
        if (computed) res_decide(ps, dk, &rec[slot], me.rank0, lane);
        if (lane == 0) s_exit = (!any || it >= a.iters) ? 1 : 0;
      }
      __syncthreads();
      if (s_exit) break;
    } else if (a.iters <= 0) {
      break;
    }
    const int phase = has ? ps.phase : PH_DONE;
    computed = (phase == PH_INIT_THETA || phase == PH_RUN);
    if (computed) {
      const int par = ps.parity;
      T* const cur = buf + par * cap;
      T* const nxt = buf + (par ^ 1) * cap;
      const bool run = phase == PH_RUN;
      if (run) {
        const T corr = (T)ps.corr;
        const int nd = s_ndir;
        for (int e = tid; e < nd; e += NT) {
          const int2 d = dlist[e];
          const unsigned int rank = (unsigned int)d.y >> 20;
          const int off = par * rank_cap[rank] + (d.y & 0xfffff);
          const T v0 = cur[d.x];
          dorig[e] = v0;
          cur[d.x] = v0 + corr;
          nxt[d.x] = dsmem_ld(dsmem_map(buf + off, rank), T(0));
        }
        dpar = par;
        __syncthreads();
      }
      const RunK<T> K = make_runk<T>(ph, ps, phase);
      RunAcc<T> A = RunAcc<T>::zero();
      for (int q = tid; q < nruns; q += NT) {
        const int r = qdiv(q, rpr, inv_rpr), c0 = (q - r * rpr) * 4;
        const int j = r, gj = g01 + j;
        const bool rowdir = (j == dly || j == dhy);
        const T wyo = (j >= clo1 && j <= chi1) ? ((gj == 0 || gj == N1 - 1) ? hw1 : h1) : T(0);
        const T wly = (j == 0 || j == n1 - 1) ? hw1 : h1;
        Vec4<T> o;
        const ColTab<T> ct{wcol + c0, ucol + c0, lcol + c0, nullptr, nullptr, g00 + c0};
        stencil_run4<T, false>(K, ph.mon, cur + (r + 1) * SWp + c0 + 4, SWp, ct, rowdir, wyo,
                               wly, fma((T)gj, K.h1, K.lo1), o, A);
        if (run && !rowdir) {
          T* const d = nxt + (r + 1) * SWp + c0 + 4;
          const int jm = (ply && j == 1) ? -1 : ((phy && j == n1 - 2) ? n1 : -2);
          T* const dmr = nxt + (jm + 1) * SWp + c0 + 4;
          if (c0 != 0 && c0 + 3 < n0 - 2) {
            o.sts(d);
            if (jm != -2) o.sts(dmr);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int c = c0 + u;
              if (c < n0 && c != dlx && c != dhx) {
                d[u] = o.v[u];
                if (jm != -2) dmr[u] = o.v[u];
                const int cm = (plx && c == 1) ? -1 : ((phx && c == n0 - 2) ? n0 : -2);
                if (cm != -2) {
                  d[cm - c0] = o.v[u];
                  if (jm != -2) dmr[cm - c0] = o.v[u];
                }
              }
            }
          }
        }
      }
      T th = A.th2.x() + A.th2.y();
      Acc<T> acc{-big_val<T>(), big_val<T>(), big_val<T>(), 0};
      A.fold(K, acc);
      tile_reduce<T, NT>(th, A.l2a, A.l2b, A.ws, acc, &rec[it & 1], me.sub, red_t, red_f, red_i);
      if (tid == 0) act[it & 1] = 1;
    } else {
      if (tid == 0) act[it & 1] = 0;
    }
    cluster_arrive();
  }
  // no CTA leaves while another may still read its shared memory
  cluster_arrive();
  cluster_wait();
  if (has && loaded) {
    const int par = ps.parity;
    T* const cur = buf + par * cap;
    if (dpar == par) {
      // a step that tangled keeps the state it read: its transmission values
      // go back without the correction (still pending in the state)
      const int nd = s_ndir;
      for (int e = tid; e < nd; e += NT) cur[dlist[e].x] = dorig[e];
      __syncthreads();
    }
    T* g = (T*)sd.v[par];
    const int pitch = sd.pitch;
    const int cpr = pitch / VW;
    for (int e = tid; e < n1 * cpr; e += NT) {
      const int r = e / cpr, k = e - r * cpr;
      Vec4<T> o;
      o.lds(cur + (r + 1) * SWp + 4 + k * VW);
      if (VW == 4) {
        o.stg(g + (long long)r * pitch + k * VW);
      } else {
        st_global(g + (long long)r * pitch + k * VW, o.v[0]);
        st_global(g + (long long)r * pitch + k * VW + 1, o.v[1]);
      }
    }
    if ((int)cluster_rank() == me.rank0)
      for (int i = tid; i < (int)(sizeof(ProbState) / 16); i += NT)
        ((int4*)(a.st + prob))[i] = ((const int4*)&ps)[i];
  }
}

// ---------------------------------------------------------------- 3D sweep
// One work item is a box of cols x rows nodes per plane over `depth` planes
// of one subdomain.  Staging mirrors the 2D band kernel (16-byte cp.async
// copies of every staged row, mirror / clamp halos, the transmission offset
// on the box perimeter).  Each thread takes runs of 4 consecutive x-nodes of
// one row and marches them through the planes; per plane it reads the 46
// values of the 19-point stencils of its 4 nodes with aligned vector loads.
template <typename T, int NT, int TZ, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_band3d(LaunchArgs a) {
  constexpr int VW = 16 / (int)sizeof(T);
  constexpr int NW = NT / 32;
  constexpr int HMAX = 8;  // halo rows per thread (host: (rows+2)(TZ+2) <= 8 NT)
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  T* sv = (T*)dyn_smem;     // staged box + column tables (dynamic size)
  __shared__ __align__(16) SmemHdr<T> HB[2];
  __shared__ __align__(8) unsigned long long tbar;  // TMA staging barrier
  __shared__ int s_t[2];
  __shared__ T red_t[4 * NW];
  __shared__ T red_f[3 * NW];
  __shared__ int red_i[NW];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tend = a.t0 + a.nwork;
  int t_next = 0;
  WorkItem w_next;
  unsigned int tph = 0;  // parity of the TMA barrier's next phase
  int q_pend = -1;       // thread 0: queue ticket not yet resolved
  if (tid == 0) mbar_init(&tbar, 1);
  // Before the wait for the preceding kernel of the stream (programmatic
  // dependent launch): this CTA's first item (its static position in the
  // order) and the descriptors that no launch of a window writes.
  int t0 = tend;
  if (tid == 0) {
    t0 = item_of_pos(a, (int)blockIdx.x);
    s_t[0] = t0;
    if (t0 < tend) issue_hdr_static<T>(a, HB[0], a.work[t0]);
  }
  // wait until the preceding kernel has completed and its writes are
  // visible; then the first item's state and the following item
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    if (t0 < tend) issue_hdr_state<T>(a, HB[0], HB[0].w.prob);
    t_next = pull_item(a);
    if (t_next < tend) w_next = a.work[t_next];
  }

  for (int it = 0;; ++it) {
    const int b = it & 1;
    if (tid == 0) cp_async_wait_all();
    __syncthreads();  // header `b` complete and visible
    const int t = s_t[b];
    if (t >= tend) break;
    if (tid == 0) {
      // the box's TMA copy first, so that it overlaps the prefetch of the
      // following item
      const SmemHdr<T>& Hc = HB[b];
      const int pc = Hc.ps.phase;
      if (pc != PH_DONE && pc != PH_INIT_V && a.tmap != nullptr && Hc.w.tma_rows > 0) {
        const int swp = (((Hc.w.ext & 0xffff) + 3) & ~3) + 8;
        const int shy = (Hc.w.ext >> 16) + 2, shz = (Hc.w.kz >> 16) + 2;
        fence_proxy_async();
        mbar_expect_tx(&tbar, (unsigned int)(swp * shy * shz * (int)sizeof(T) + a.stall_bytes));
        tma_load_3d(sv, (const char*)a.tmap + 128 * ((size_t)Hc.w.tma_map + Hc.ps.parity),
                    (Hc.w.ij & 0xffff) - 4, (Hc.w.ij >> 16) - 1, (Hc.w.kz & 0xffff) - 1, &tbar);
      }
      s_t[b ^ 1] = t_next;
      if (t_next < tend) {
        issue_hdr<T>(a, HB[b ^ 1], w_next);
        q_pend = queue_ticket(a);
      }
    }
    SmemHdr<T>& H = HB[b];
    const int phase = H.ps.phase;
    if (phase == PH_DONE) {
      if (tid == 0) resolve_pull(a, t_next, w_next, q_pend, tend);
      continue;
    }
    const int n0 = H.sd.n[0], n1 = H.sd.n[1], n2 = H.sd.n[2];
    const long long pitch = H.sd.pitch, ppitch = pitch * n1;
    const int i0 = H.w.ij & 0xffff, j0 = H.w.ij >> 16;
    const int cols = H.w.ext & 0xffff, rows = H.w.ext >> 16;
    const int k0 = H.w.kz & 0xffff, depth = H.w.kz >> 16;
    const int faces = H.sd.faces;
    const int g00 = H.sd.g0[0], g01 = H.sd.g0[1], g02 = H.sd.g0[2];
    const T* src = (const T*)H.sd.v[H.ps.parity];
    T* dst = (T*)H.sd.v[H.ps.parity ^ 1];
    const int cr = (cols + 3) & ~3;
    const int rpr = cr >> 2;
    const int nruns = rows * rpr;
    const float inv_rpr = __fdividef(1.0f, (float)rpr);
    const int dlx = (faces & 1) ? -1 : 0, dhx = (faces & 2) ? -1 : n0 - 1;
    const int dly = (faces & 4) ? -1 : 0, dhy = (faces & 8) ? -1 : n1 - 1;
    const int dlz = (faces & 16) ? -1 : 0, dhz = (faces & 32) ? -1 : n2 - 1;
    T th = 0, l2a = 0, l2b = 0, ws = 0;
    Acc<T> acc{-big_val<T>(), big_val<T>(), big_val<T>(), 0};

    if (phase == PH_INIT_V) {
      const double* psi0 = a.probs[H.w.prob].psi0;
      const int Nx = H.ph.N[0], Ny = H.ph.N[1];
      for (int q = tid; q < nruns * depth; q += NT) {
        const int l = q / nruns, q2 = q - l * nruns;
        const int r = qdiv(q2, rpr, inv_rpr), c0 = (q2 - r * rpr) * 4;
        const int j = j0 + r, kk = k0 + l;
        Vec4<T> o;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + c0 + u;
          T v0 = T(0);
          if (psi0 && i < n0) {
            const int gi = g00 + i, gj = g01 + j, gk = g02 + kk;
            const double xi = (double)H.ph.lo[0] + (double)gi * H.ph.hd[0];
            const double et = (double)H.ph.lo[1] + (double)gj * H.ph.hd[1];
            const double ze = (double)H.ph.lo[2] + (double)gk * H.ph.hd[2];
            v0 = (T)(psi0[((long long)gk * Ny + gj) * Nx + gi] - 0.5 * (xi * xi + et * et + ze * ze));
          }
          o.v[u] = v0;
        }
        o.stg(dst + kk * ppitch + j * pitch + i0 + c0);
        o.stg((T*)src + kk * ppitch + j * pitch + i0 + c0);
      }
    } else {
      const int SWp = cr + 8, SHY = rows + 2, SHZ = depth + 2;
      const int PS = SHY * SWp;
      const int cpr = SWp / VW;
      const float inv_cpr = __fdividef(1.0f, (float)cpr);
      const int nrow = SHZ * SHY;
      const float inv_shy = 1.0f / (float)SHY;
      const bool plx = faces & 1, phx = faces & 2, ply = faces & 4, phy = faces & 8;
      const bool plz = faces & 16, phz = faces & 32;
      const T corr = (T)H.ps.corr;
      // (a) the staged box: one TMA copy where the subdomain has tensor maps
      //     (zeros outside the buffer, mirror rows and planes fixed below),
      //     else 16-byte asynchronous copies of every staged row
      const bool tma = a.tmap != nullptr && H.w.tma_rows > 0;
      if (tma) {
        // the box was issued right after the header barrier
      } else {
        for (int e = tid; e < nrow * cpr; e += NT) {
          const int rr = qdiv(e, cpr, inv_cpr), k = e - rr * cpr;
          const int gs = i0 - 4 + k * VW;
          if (gs >= 0 && gs + VW <= pitch) {
            const int lz = qdiv(rr, SHY, inv_shy), ly = rr - lz * SHY;
            const int jj = reflect_clamp(j0 - 1 + ly, n1, ply, phy);
            const int kk = reflect_clamp(k0 - 1 + lz, n2, plz, phz);
            cp_async16(sv + lz * PS + ly * SWp + k * VW, src + kk * ppitch + jj * pitch + gs);
          }
        }
      }
      cp_async_commit();
      // Transmission nodes of the box (Eq. transmission_condition3), one
      // per thread while the staging copies are in flight: whole
      // transmission planes, then in the other planes the transmission rows
      // and the transmission columns of the remaining rows.  At a step
      // without exchange (exchange_every > 1) they keep their staged values
      // instead, copied once the box has landed.
      const int kex = H.ph.exchange_every;
      const bool exch = exchange_step(H.ps.step, kex);
      const TrBox3 tb = tr_box3(dlx, dhx, dly, dhy, dlz, dhz, i0, j0, k0, cols, rows, depth);
      if (phase == PH_RUN && exch) {
        const NbEnt* const nbi = item_nb<T, 3>(a, H);
        for (int e = tid; e < tb.total; e += NT) {
          int i, j, kk;
          if (!tb.node(e, i0, j0, k0, cols, rows, i, j, kk)) continue;
          st_global(dst + kk * ppitch + j * pitch + i, gather_owner<T, 3>(nbi, H, i, j, kk));
        }
      }
      // (b) x-halo columns (Neumann mirror; clamp on transmission faces)
      const bool left = (i0 == 0), right = (i0 + cols == n0);
      T hl[HMAX], hr[HMAX];
#pragma unroll
      for (int q = 0; q < HMAX; ++q) {
        const int rr = tid + q * NT;
        hl[q] = hr[q] = T(0);
        if (rr < nrow && (left || right)) {
          const int lz = qdiv(rr, SHY, inv_shy), ly = rr - lz * SHY;
          const int jj = reflect_clamp(j0 - 1 + ly, n1, ply, phy);
          const int kk = reflect_clamp(k0 - 1 + lz, n2, plz, phz);
          const bool dr = (jj == dly || jj == dhy || kk == dlz || kk == dhz);
          const T cc = dr ? corr : T(0);
          const T* row = src + kk * ppitch + jj * pitch;
          if (left && plx) hl[q] = __ldcg(row + 1) + cc;
          if (right && phx) hr[q] = __ldcg(row + n0 - 2) + cc;
        }
      }
      cp_async_wait_all();
      bool gave_up = false;
      if (tma) {
        gave_up = !mbar_wait(&tbar, tph);
        tph ^= 1;
      }
      if (__syncthreads_or(gave_up)) {
        // the box never arrived: report, give the copy one more bounded
        // wait, and leave (the host turns the error word into a status)
        if (tid == 0) {
          atomicOr(a.err, 1u);
          mbar_wait(&tbar, tph ^ 1);
        }
        break;
      }
      if (tma && ((ply && j0 == 0) || (phy && j0 + rows == n1))) {
        // Neumann mirror rows of a TMA box in every staged plane: row 0 <-
        // row 2, row rows+1 <- row rows-1 (x-halo columns: written by (c))
        for (int e = tid; e < SHZ * SWp; e += NT) {
          const int lz = e / SWp, c = e - lz * SWp;
          if ((left && c == 3) || (right && c == cols + 4)) continue;
          T* const pl = sv + lz * PS;
          if (ply && j0 == 0) pl[c] = pl[2 * SWp + c];
          if (phy && j0 + rows == n1) pl[(rows + 1) * SWp + c] = pl[(rows - 1) * SWp + c];
        }
        __syncthreads();
      }
      if (tma && ((plz && k0 == 0) || (phz && k0 + depth == n2))) {
        // then the mirror planes: plane 0 <- plane 2, plane depth+1 <-
        // plane depth-1 (so that edges and corners mirror in both axes)
        for (int e = tid; e < PS; e += NT) {
          const int c = e % SWp;
          if ((left && c == 3) || (right && c == cols + 4)) continue;
          if (plz && k0 == 0) sv[e] = sv[2 * PS + e];
          if (phz && k0 + depth == n2) sv[(depth + 1) * PS + e] = sv[(depth - 1) * PS + e];
        }
        __syncthreads();
      }
      // (c) halos, then the transmission offset on the box perimeter:
      //     transmission planes (whole), rows in other planes (whole),
      //     columns 0 / n0-1 elsewhere; halo columns were written by (b)
#pragma unroll
      for (int q = 0; q < HMAX; ++q) {
        const int rr = tid + q * NT;
        if (rr < nrow) {
          if (left) sv[rr * SWp + 3] = hl[q];
          if (right) sv[rr * SWp + cols + 4] = hr[q];
        }
      }
      if (corr != T(0)) {
        const int cl = (dlx == 0 && i0 == 0) ? 4 : -1;
        const int ch = (dhx >= 0 && right) ? cols + 3 : -1;
        for (int rr = tid; rr < nrow; rr += NT) {
          const int lz = qdiv(rr, SHY, inv_shy), ly = rr - lz * SHY;
          const int jj = reflect_clamp(j0 - 1 + ly, n1, ply, phy);
          const int kk = reflect_clamp(k0 - 1 + lz, n2, plz, phz);
          T* row = sv + rr * SWp;
          if (jj == dly || jj == dhy || kk == dlz || kk == dhz) {
            for (int c = 0; c < SWp; ++c)
              if (!(left && c == 3) && !(right && c == cols + 4)) row[c] += corr;
          } else {
            if (cl >= 0) row[cl] += corr;
            if (ch >= 0) row[ch] += corr;
          }
        }
      }
      if (H.ph.alternating && exchange_step(H.ps.step - 1, kex)) {
        __syncthreads();
        stage_alternating<T, NT>(a, H, sv, SWp, SHY, SHZ, i0, j0, k0, cols);
      }
      const T lo0 = H.ph.lo[0], lo1 = H.ph.lo[1], lo2 = H.ph.lo[2];
      const T h0 = H.ph.h[0], h1 = H.ph.h[1], h2 = H.ph.h[2];
      const T hw0 = H.ph.hw[0], hw1 = H.ph.hw[1], hw2 = H.ph.hw[2];
      const int N0 = H.ph.N[0], N1 = H.ph.N[1], N2 = H.ph.N[2];
      const int clo0 = H.sd.clo[0], chi0 = H.sd.chi[0], clo1 = H.sd.clo[1], chi1 = H.sd.chi[1];
      const int clo2 = H.sd.clo[2], chi2 = H.sd.chi[2];
      const bool want_l2 = H.ph.stop_norm == PMA_STOP_L2_INCREMENT;
      const bool run = phase == PH_RUN;
      const RunK<T> K = make_runk<T>(H.ph, H.ps, phase);
      const int nterms = K.nterms;
      const bool fast = K.fast;
      // column tables after the staged planes: theta weight of owned
      // columns (0 elsewhere), 1 at updated columns (else 0), the local
      // trapezoid weight, xi_x, and +big at columns that are not updated
      T* wcol = sv + SHZ * PS;
      T* ucol = wcol + cr;
      T* lcol = ucol + cr;
      T* xcol = lcol + cr;
      T* kcol = xcol + cr;
      for (int c = tid; c < cr; c += NT) {
        const int i = i0 + c, gi = g00 + i;
        const bool valid = c < cols;
        const bool upd = valid && i != dlx && i != dhx;
        wcol[c] = (valid && i >= clo0 && i <= chi0) ? ((gi == 0 || gi == N0 - 1) ? hw0 : h0) : T(0);
        ucol[c] = upd ? T(1) : T(0);
        lcol[c] = (i == 0 || i == n0 - 1) ? hw0 : h0;
        xcol[c] = fma((T)gi, h0, lo0);
        kcol[c] = upd ? T(0) : big_val<T>();
      }
      __syncthreads();  // box staged
      if (phase == PH_RUN && !exch) {
        // interface data frozen between exchanges: every transmission node
        // of the box keeps the value it was staged with (offset included)
        for (int e = tid; e < tb.total; e += NT) {
          int i, j, kk;
          if (!tb.node(e, i0, j0, k0, cols, rows, i, j, kk)) continue;
          st_global(dst + kk * ppitch + j * pitch + i,
                    sv[(kk - k0 + 1) * PS + (j - j0 + 1) * SWp + (i - i0 + 4)]);
        }
      }
      RunAcc<T> A = RunAcc<T>::zero();
      const P2<T> DT2 = K.DT2;
      const P2<T> M2 = P2<T>::s(T(-2)), ONE = P2<T>::s(T(1));
      const P2<T> I2H0 = P2<T>::s(H.ph.inv2h[0]), I2H1 = P2<T>::s(H.ph.inv2h[1]);
      const P2<T> I2H2 = P2<T>::s(H.ph.inv2h[2]);
      const P2<T> IH20 = P2<T>::s(H.ph.invh2[0]), IH21 = P2<T>::s(H.ph.invh2[1]);
      const P2<T> IH22 = P2<T>::s(H.ph.invh2[2]);
      const P2<T> I4XY = P2<T>::s(H.ph.inv4hh[0]), I4XZ = P2<T>::s(H.ph.inv4hh[1]);
      const P2<T> I4YZ = P2<T>::s(H.ph.inv4hh[2]);
      // transmission rows and planes (only a box's first or last row or
      // plane can be one) are written by the transmission pass, not here
      const int rlo = (j0 == dly) ? 1 : 0, rhi = (j0 + rows - 1 == dhy) ? rows - 1 : rows;
      const int llo = (k0 == dlz) ? 1 : 0, lhi = (k0 + depth - 1 == dhz) ? depth - 1 : depth;
      const int nrun_u = rhi > rlo ? (rhi - rlo) * rpr : 0;
      for (int q = tid; q < nrun_u; q += NT) {
        const int rq = qdiv(q, rpr, inv_rpr), r = rlo + rq, c0 = (q - rq * rpr) * 4;
        const int j = j0 + r, gj = g01 + j;
        Vec4<T> wc, uc, xc;
        wc.lds(wcol + c0);
        uc.lds(ucol + c0);
        xc.lds(xcol + c0);
        const T wyo = (j >= clo1 && j <= chi1) ? ((gj == 0 || gj == N1 - 1) ? hw1 : h1) : T(0);
        const T xi1 = fma((T)gj, h1, lo1);
        P2<T> XI0[2];
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) XI0[pp] = P2<T>::mk(xc.v[2 * pp], xc.v[2 * pp + 1]);
        for (int l = llo; l < lhi; ++l) {
          const int kk = k0 + l, gk = g02 + kk;
          const T* p = sv + (l + 1) * PS + (r + 1) * SWp + c0 + 4;
          // plane z: rows j-1, j, j+1, columns c0-1 .. c0+4
          T cS[6], cC[6], cN[6];
          // planes z-1 / z+1: row j (6 columns) and rows j-1, j+1 (4 columns)
          T dC[6], uC[6];
          Vec4<T> dS, dN, uS, uN;
          {
            Vec4<T> m;
            cS[0] = p[-SWp - 1]; m.lds(p - SWp); cS[5] = p[-SWp + 4];
            cS[1] = m.v[0]; cS[2] = m.v[1]; cS[3] = m.v[2]; cS[4] = m.v[3];
            cC[0] = p[-1]; m.lds(p); cC[5] = p[4];
            cC[1] = m.v[0]; cC[2] = m.v[1]; cC[3] = m.v[2]; cC[4] = m.v[3];
            cN[0] = p[SWp - 1]; m.lds(p + SWp); cN[5] = p[SWp + 4];
            cN[1] = m.v[0]; cN[2] = m.v[1]; cN[3] = m.v[2]; cN[4] = m.v[3];
            const T* pd = p - PS;
            dC[0] = pd[-1]; m.lds(pd); dC[5] = pd[4];
            dC[1] = m.v[0]; dC[2] = m.v[1]; dC[3] = m.v[2]; dC[4] = m.v[3];
            dS.lds(pd - SWp);
            dN.lds(pd + SWp);
            const T* pu = p + PS;
            uC[0] = pu[-1]; m.lds(pu); uC[5] = pu[4];
            uC[1] = m.v[0]; uC[2] = m.v[1]; uC[3] = m.v[2]; uC[4] = m.v[3];
            uS.lds(pu - SWp);
            uN.lds(pu + SWp);
          }
          const T wzo = (kk >= clo2 && kk <= chi2) ? ((gk == 0 || gk == N2 - 1) ? hw2 : h2) : T(0);
          const T xi2 = fma((T)gk, h2, lo2);
          P2<T> X0[2], X1[2], X2[2], DD[2], R[2];
#pragma unroll
          for (int pp = 0; pp < 2; ++pp) {
            const int u0 = 2 * pp;
            const P2<T> C = P2<T>::mk(cC[u0 + 1], cC[u0 + 2]);
            const P2<T> E = P2<T>::mk(cC[u0 + 2], cC[u0 + 3]);
            const P2<T> Wv = P2<T>::mk(cC[u0], cC[u0 + 1]);
            const P2<T> Nn = P2<T>::mk(cN[u0 + 1], cN[u0 + 2]);
            const P2<T> Ss = P2<T>::mk(cS[u0 + 1], cS[u0 + 2]);
            const P2<T> Up = P2<T>::mk(uC[u0 + 1], uC[u0 + 2]);
            const P2<T> Dn = P2<T>::mk(dC[u0 + 1], dC[u0 + 2]);
            X0[pp] = pfma(psub(E, Wv), I2H0, XI0[pp]);
            X1[pp] = pfma(psub(Nn, Ss), I2H1, P2<T>::s(xi1));
            X2[pp] = pfma(psub(Up, Dn), I2H2, P2<T>::s(xi2));
            const P2<T> hxx = pfma(pfma(C, M2, padd(E, Wv)), IH20, ONE);
            const P2<T> hyy = pfma(pfma(C, M2, padd(Nn, Ss)), IH21, ONE);
            const P2<T> hzz = pfma(pfma(C, M2, padd(Up, Dn)), IH22, ONE);
            // cross differences (v_{++} - v_{+-}) - (v_{-+} - v_{--})
            const P2<T> hxy = pmul(psub(psub(P2<T>::mk(cN[u0 + 2], cN[u0 + 3]), P2<T>::mk(cS[u0 + 2], cS[u0 + 3])),
                                        psub(P2<T>::mk(cN[u0], cN[u0 + 1]), P2<T>::mk(cS[u0], cS[u0 + 1]))),
                                   I4XY);
            const P2<T> hxz = pmul(psub(psub(P2<T>::mk(uC[u0 + 2], uC[u0 + 3]), P2<T>::mk(dC[u0 + 2], dC[u0 + 3])),
                                        psub(P2<T>::mk(uC[u0], uC[u0 + 1]), P2<T>::mk(dC[u0], dC[u0 + 1]))),
                                   I4XZ);
            const P2<T> hyz = pmul(psub(psub(P2<T>::mk(uN.v[u0], uN.v[u0 + 1]), P2<T>::mk(uS.v[u0], uS.v[u0 + 1])),
                                        psub(P2<T>::mk(dN.v[u0], dN.v[u0 + 1]), P2<T>::mk(dS.v[u0], dS.v[u0 + 1]))),
                                   I4YZ);
            // det of the symmetric 3x3 matrix by cofactors of the first row
            const P2<T> m1 = psub(pmul(hyy, hzz), pmul(hyz, hyz));
            const P2<T> m2 = psub(pmul(hxy, hzz), pmul(hyz, hxz));
            const P2<T> m3 = psub(pmul(hxy, hyz), pmul(hyy, hxz));
            DD[pp] = pfma(hxz, m3, psub(pmul(hxx, m1), pmul(hxy, m2)));
          }
          if (fast) {
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) R[pp] = P2<T>::s(H.ph.mon.base);
            const int nring = H.ph.mon.nring;
            for (int k = 0; k < nring; ++k) sum_terms3<T, true>(H.ph.mon.t[k], X0, X1, X2, R);
            for (int k = nring; k < nterms; ++k)
              sum_terms3<T, false>(H.ph.mon.t[k], X0, X1, X2, R);
          } else {
#pragma unroll
            for (int pp = 0; pp < 2; ++pp)
              R[pp] = P2<T>::mk(rho_at<T>(H.ph.mon, X0[pp].x(), X1[pp].x(), X2[pp].x()),
                                rho_at<T>(H.ph.mon, X0[pp].y(), X1[pp].y(), X2[pp].y()));
          }
          // masks: 1 at updated nodes, 0 elsewhere (columns only: the
          // transmission rows and planes are skipped); rho det := 1 at the
          // others (see stencil_core4)
          Vec4<T> o, kc;
          kc.lds(kcol + c0);
          const P2<T> WYZ = P2<T>::s(wyo * wzo);
          P2<T> GMX[2], GMN[2], DMN[2], GCs[2], Ms[2];
#pragma unroll
          for (int pp = 0; pp < 2; ++pp) {
            const P2<T> m = P2<T>::mk(uc.v[2 * pp], uc.v[2 * pp + 1]);
            const P2<T> rd = pmul(R[pp], DD[pp]);
            const P2<T> rD = P2<T>::mk(m.x() != T(0) ? rd.x() : T(1), m.y() != T(0) ? rd.y() : T(1));
            const P2<T> GC = rhs_pair<T>(K, rD);
            const P2<T> vn = pfma(GC, DT2, P2<T>::mk(cC[2 * pp + 1], cC[2 * pp + 2]));
            o.v[2 * pp] = vn.x();
            o.v[2 * pp + 1] = vn.y();
            A.gs2 = padd(A.gs2, GC);
            A.th2 = pfma(pmul(P2<T>::mk(wc.v[2 * pp], wc.v[2 * pp + 1]), WYZ), rD, A.th2);
            const P2<T> kmn = P2<T>::mk(kc.v[2 * pp], kc.v[2 * pp + 1]);  // 0 or +big
            GMX[pp] = pmul(rD, m);
            GMN[pp] = pfma(rD, m, kmn);
            DMN[pp] = pfma(DD[pp], m, kmn);
            GCs[pp] = GC;
            Ms[pp] = m;
          }
          A.rmax = max3(max3(A.rmax, GMX[0].x(), GMX[0].y()), GMX[1].x(), GMX[1].y());
          A.rmin = min3(min3(A.rmin, GMN[0].x(), GMN[0].y()), GMN[1].x(), GMN[1].y());
          A.dmin = min3(min3(A.dmin, DMN[0].x(), DMN[0].y()), DMN[1].x(), DMN[1].y());
          if (want_l2) {
            Vec4<T> lc;
            lc.lds(lcol + c0);
            const T wl = ((j == 0 || j == n1 - 1) ? hw1 : h1) * ((kk == 0 || kk == n2 - 1) ? hw2 : h2);
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
              const P2<T> w = pmul(pmul(P2<T>::mk(lc.v[2 * pp], lc.v[2 * pp + 1]), P2<T>::s(wl)), Ms[pp]);
              const P2<T> d = pmul(GCs[pp], Ms[pp]);
              A.l2a = fma(w.x() * d.x(), d.x(), A.l2a);
              A.l2b = fma(w.x(), d.x(), A.l2b);
              A.ws += w.x();
              A.l2a = fma(w.y() * d.y(), d.y(), A.l2a);
              A.l2b = fma(w.y(), d.y(), A.l2b);
              A.ws += w.y();
            }
          }
          if (run) {
            T* const q = dst + kk * ppitch + j * pitch + i0 + c0;
            if ((i0 + c0 <= dlx) || (i0 + c0 + 3 >= dhx && dhx >= 0)) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int i = i0 + c0 + u;
                if (i != dlx && i != dhx) st_global(q + u, o.v[u]);
              }
            } else {
              o.stg(q);
            }
          }
        }
      }
      A.fold(K, acc);
      l2a = A.l2a;
      l2b = A.l2b;
      ws = A.ws;
      th = A.th2.x() + A.th2.y();
    }
    if (tid == 0) resolve_pull(a, t_next, w_next, q_pend, tend);
    // tile record
    th = warp_sum(th);
    if (H.ph.stop_norm == PMA_STOP_L2_INCREMENT) {
      l2a = warp_sum(l2a);
      l2b = warp_sum(l2b);
      ws = warp_sum(ws);
    }
    const T gmax = warp_max(acc.gmax), gmin = warp_min(acc.gmin), dmin = warp_min(acc.dmin);
    const int nf = warp_isum(acc.nf);
    if (lane == 0) {
      red_t[0 * NW + wid] = th;
      red_t[1 * NW + wid] = l2a;
      red_t[2 * NW + wid] = l2b;
      red_t[3 * NW + wid] = ws;
      red_f[0 * NW + wid] = gmax;
      red_f[1 * NW + wid] = gmin;
      red_f[2 * NW + wid] = dmin;
      red_i[wid] = nf;
    }
    __syncthreads();
    if (wid == 0) write_record<T, NW>(a, t, H.w.sub, red_t, red_f, red_i, lane);
  }
  if (tid == 0) queue_exit(a);
  // this CTA has run out of work: the next kernel of the stream (launched
  // as a programmatic dependent) may be scheduled while the last CTAs finish
  asm volatile("griddepcontrol.launch_dependents;");
}

// ---------------------------------------------------------------- dispatch
// Compiled shapes.  2D: (threads, band nodes FP32, band nodes FP64, shared
// elements per band node x 10, FP32 CTAs per SM the registers are budgeted
// for; FP64 budgets for 4): the staged band plus halo and the column
// tables fit in nodes x factor / 10 elements (bands get fewer rows, or
// narrower strips, where the halo would not fit).
#define PMA_T2D(X) X(128, 3072, 1536, 16, 7, 0) X(128, 2048, 1024, 30, 7, 0) \
                   X(128, 4096, 2048, 14, 7, 0) X(128, 5120, 2560, 14, 7, 0) \
                   X(128, 768, 384, 30, 7, 0) X(128, 6144, 3072, 14, 6, 0) \
                   X(128, 4096, 2048, 14, 6, 0) X(128, 4096, 2048, 14, 4, 1) \
                   X(128, 3072, 1536, 16, 5, 1) X(128, 2048, 1024, 16, 8, 1)
#define PMA_SMAX(n, f) (((n) * (f) / 10) & ~3)
// 3D: (threads, nodes per plane box, planes FP32, planes FP64, dynamic
// shared memory in KiB for the staged box and the column tables, FP32 CTAs
// per SM the registers are budgeted for; FP64 budgets for 2).
#define PMA_T3D(X) X(128, 512, 8, 4, 32, 3) X(128, 512, 8, 4, 32, 4) X(128, 512, 8, 4, 64, 3) \
                   X(128, 512, 8, 4, 32, 5) X(128, 512, 8, 4, 32, 6)

static const int k_t2d[][4] = {
#define E(a, b, c, f, m, pf) {a, b, c, f},
    PMA_T2D(E)
#undef E
};
static const int k_t3d[][6] = {
#define E(a, b, c, d, e, m) {a, b, c, d, e, m},
    PMA_T3D(E)
#undef E
};

int tile2d_count() { return (int)(sizeof(k_t2d) / sizeof(k_t2d[0])); }
int tile3d_count() { return (int)(sizeof(k_t3d) / sizeof(k_t3d[0])); }
Tile2D tile2d_shape(int id, bool fp64) {
  Tile2D t;
  t.threads = k_t2d[id][0];
  t.nodes = fp64 ? k_t2d[id][2] : k_t2d[id][1];
  t.smax = PMA_SMAX(t.nodes, k_t2d[id][3]);
  // a one-row band plus halo and the five column tables must fit:
  // 3 * (cols + 8) + 5 * cols <= smax, cols % 4 == 0
  const int cmax = ((t.smax - 24) / 8) & ~3;
  t.cols = cmax < 1024 ? cmax : 1024;
  return t;
}
Tile3D tile3d_shape(int id, bool fp64) {
  Tile3D t;
  t.threads = k_t3d[id][0];
  t.xy = k_t3d[id][1];
  t.tz = fp64 ? k_t3d[id][3] : k_t3d[id][2];
  t.smax = k_t3d[id][4] * 1024 / (fp64 ? 8 : 4);
  // a one-row box: 3 rows x (cols + 8) x (tz + 2) planes + 5 column tables
  const int cmax = ((t.smax / (3 * (t.tz + 2) + 5)) - 8) & ~3;
  t.cols = cmax < 1024 ? cmax : 1024;
  return t;
}

template <typename T>
static const void* sweep_fn(int dim, int id, int* nthreads, int* dyn) {
  int k = 0;
  *dyn = 0;
  if (dim == 2) {
#define E(a, b, c, f, m, pf)                                               \
  if (k++ == id) {                                                         \
    *nthreads = (a);                                                       \
    if constexpr (sizeof(T) == 8)                                          \
      return (const void*)k_band2d<T, a, PMA_SMAX(c, f), 512 / (a), pf>;   \
    else                                                                   \
      return (const void*)k_band2d<T, a, PMA_SMAX(b, f), m, pf>;           \
  }
    PMA_T2D(E)
#undef E
  } else {
#define E(a, b, c, d, e, m)                                                \
  if (k++ == id) {                                                         \
    *nthreads = (a);                                                       \
    *dyn = (e) * 1024;                                                     \
    if constexpr (sizeof(T) == 8)                                          \
      return (const void*)k_band3d<T, a, d, 2>;                            \
    else                                                                   \
      return (const void*)k_band3d<T, a, c, m>;                            \
  }
    PMA_T3D(E)
#undef E
  }
  return nullptr;
}

static const void* cls_fn(int cls, int tile_id, int* nthreads, int* dyn) {
  switch (cls) {
    case CLS_2D_F32: return sweep_fn<float>(2, tile_id, nthreads, dyn);
    case CLS_2D_F64: return sweep_fn<double>(2, tile_id, nthreads, dyn);
    case CLS_3D_F32: return sweep_fn<float>(3, tile_id, nthreads, dyn);
    case CLS_3D_F64: return sweep_fn<double>(3, tile_id, nthreads, dyn);
  }
  return nullptr;
}

// Kernels with dynamic shared memory above 48 KiB must opt in once per
// function (and device); cheap and idempotent.
static cudaError_t opt_in(const void* fn, int dyn) {
  if (dyn <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
}

cudaError_t launch_sweep(int cls, int tile_id, const LaunchArgs& a, cudaStream_t s) {
  int nt = 0, dyn = 0;
  const void* fn = cls_fn(cls, tile_id, &nt, &dyn);
  if (!fn) return cudaErrorInvalidValue;
  if (a.nwork <= 0 || a.grid <= 0) return cudaSuccess;
  void* args[] = {(void*)&a};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.grid);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = (size_t)dyn;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t prepare_sweep_kernels() {
  for (int cls = 0; cls < NUM_CLS; ++cls) {
    const int n = (cls == CLS_2D_F32 || cls == CLS_2D_F64) ? tile2d_count() : tile3d_count();
    for (int id = 0; id < n; ++id) {
      int nt = 0, dyn = 0;
      const void* fn = cls_fn(cls, id, &nt, &dyn);
      const cudaError_t e = opt_in(fn, dyn);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

int sweep_max_blocks_per_sm(int cls, int tile_id) {
  int nt = 0, dyn = 0;
  const void* fn = cls_fn(cls, tile_id, &nt, &dyn);
  if (!fn) return 0;
  if (opt_in(fn, dyn) != cudaSuccess) return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, nt, (size_t)dyn) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

// ---------------------------------------------------------------- resident dispatch
// Classes of the resident path: dynamic shared memory per CTA and threads.
// FP64 uses at most 512 threads (register budget of the FP64 stencil).
static const int k_res[kResClasses][2] = {
    {24 * 1024, 128}, {56 * 1024, 256}, {112 * 1024, 512}, {220 * 1024, 1024}};

static int res_threads(bool fp64, int id) {
  const int nt = k_res[id][1];
  return (fp64 && nt > 512) ? 512 : nt;
}

ResClass res_class(int id, bool fp64) { return ResClass{k_res[id][0], res_threads(fp64, id)}; }

static const void* res_fn(bool fp64, int id) {
  const int nt = k_res[id][1];
  if (fp64) {
    switch (nt) {
      case 128: return (const void*)k_res2d<double, 128>;
      case 256: return (const void*)k_res2d<double, 256>;
      default: return (const void*)k_res2d<double, 512>;
    }
  }
  switch (nt) {
    case 128: return (const void*)k_res2d<float, 128>;
    case 256: return (const void*)k_res2d<float, 256>;
    case 512: return (const void*)k_res2d<float, 512>;
    default: return (const void*)k_res2d<float, 1024>;
  }
}

// Every resident kernel may take the largest class budget (a launch uses
// the largest need among its CTAs).
cudaError_t prepare_res_kernels() {
  for (int f = 0; f < 2; ++f)
    for (int id = 0; id < kResClasses; ++id) {
      const void* fn = res_fn(f == 1, id);
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           k_res[kResClasses - 1][0]);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

static void res_config(bool fp64, int id, int nclusters, int csize, int smem_bytes,
                       cudaStream_t s, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at) {
  *cfg = cudaLaunchConfig_t{};
  cfg->gridDim = dim3((unsigned int)(nclusters * csize), 1, 1);
  cfg->blockDim = dim3((unsigned int)res_threads(fp64, id), 1, 1);
  cfg->dynamicSmemBytes = (size_t)smem_bytes;
  cfg->stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned int)csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg->attrs = at;
  cfg->numAttrs = 1;
}

int res_max_clusters(bool fp64, int id, int csize, int smem_bytes) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  res_config(fp64, id, 1, csize, smem_bytes, nullptr, &cfg, at);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, res_fn(fp64, id), &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_res2d(bool fp64, int id, const ResArgs& a, int nclusters, int csize,
                         int smem_bytes, cudaStream_t s) {
  if (nclusters <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  res_config(fp64, id, nclusters, csize, smem_bytes, s, &cfg, at);
  void* args[] = {(void*)&a};
  return cudaLaunchKernelExC(&cfg, res_fn(fp64, id), args);
}

// ---------------------------------------------------------------- combine
// Owner-takes combination: global node g takes x = xi + grad_h v of the
// subdomain whose core holds it (mirror ghost on faces of Omega_c, i.e.
// x_a = xi_a on faces normal to a), and Psi = v - S + |xi|^2/2.
// A transmission node carries the previous step's offset (corr is added),
// except under alternating transmission after an exchange step when its
// owner precedes the subdomain (alt_new): then the owner's current value is
// the node's value.
template <typename T>
__device__ __forceinline__ T fetch_v(const SubDesc& sd, const T* v, int dim, int i, int j, int l,
                                     double corr, const ProbDesc& pd, const SubDesc* subs,
                                     int parity, bool alt_new) {
  const int n0 = sd.n[0], n1 = sd.n[1], n2 = sd.n[2];
  i = reflect_clamp(i, n0, sd.faces & 1, sd.faces & 2);
  j = dim > 1 ? reflect_clamp(j, n1, sd.faces & 4, sd.faces & 8) : 0;
  l = dim > 2 ? reflect_clamp(l, n2, sd.faces & 16, sd.faces & 32) : 0;
  if (is_dir(sd.faces, dim, i, j, l, n0, n1, n2)) {
    if (alt_new) {
      const int kx = sd.k[0] + (i < sd.clo[0] ? -1 : (i > sd.chi[0] ? 1 : 0));
      const int ky = sd.k[1] + (j < sd.clo[1] ? -1 : (j > sd.chi[1] ? 1 : 0));
      const int kz = sd.k[2] + (l < sd.clo[2] ? -1 : (l > sd.chi[2] ? 1 : 0));
      const int oidx = (kz * pd.parts[1] + ky) * pd.parts[0] + kx;
      if (oidx < sd.idx) {
        const SubDesc& od = subs[pd.sub_base + oidx];
        const T* ov = (const T*)od.v[parity];
        return ov[(long long)(sd.g0[0] + i - od.g0[0]) +
                  (long long)od.pitch * ((sd.g0[1] + j - od.g0[1]) +
                                         (long long)od.n[1] * (sd.g0[2] + l - od.g0[2]))];
      }
    }
    return v[(long long)i + (long long)sd.pitch * (j + (long long)n1 * l)] + (T)corr;
  }
  return v[(long long)i + (long long)sd.pitch * (j + (long long)n1 * l)];
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
  const bool alt = pd.transmission == PMA_TRANSMISSION_ALTERNATING &&
                   exchange_step(ps.step - 1, pd.exchange_every);
  double q = 0.0;
  for (int a = 0; a < dim; ++a) {
    const double xi = pd.lo[a] + (double)gg[a] * pd.h[a];
    q += 0.5 * xi * xi;
    double xa = xi;
    if (gg[a] > 0 && gg[a] < pd.N[a] - 1) {
      int p[3] = {li[0], li[1], li[2]}, m[3] = {li[0], li[1], li[2]};
      p[a] += 1;
      m[a] -= 1;
      const T vp = fetch_v<T>(sd, v, dim, p[0], p[1], p[2], ps.corr, pd, subs, ps.parity, alt);
      const T vm = fetch_v<T>(sd, v, dim, m[0], m[1], m[2], ps.corr, pd, subs, ps.parity, alt);
      xa = xi + (double)(vp - vm) * (0.5 / pd.h[a]);
    }
    if (J.out_fp64)
      ((double*)J.x)[a * N + g] = xa;
    else
      ((float*)J.x)[a * N + g] = (float)xa;
  }
  if (J.psi) {
    const double vv = (double)v[(long long)i + (long long)sd.pitch * (j + (long long)sd.n[1] * l)];
    const double psi = vv - ps.shift + q;
    if (J.out_fp64)
      ((double*)J.psi)[g] = psi;
    else
      ((float*)J.psi)[g] = (float)psi;
  }
}

__global__ void __launch_bounds__(256) k_combine(const CombineJob* jobs, int njobs,
                                                 const SubDesc* subs, const ProbDesc* probs,
                                                 const ProbState* st) {
  __shared__ int s_job;
  if (threadIdx.x == 0) {
    // last job whose first block is <= this block
    int lo = 0, hi = njobs - 1;
    const long long b = blockIdx.x;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].block_begin <= b) lo = mid;
      else hi = mid - 1;
    }
    s_job = lo;
  }
  __syncthreads();
  const CombineJob J = jobs[s_job];
  const ProbDesc& pd = probs[J.prob];
  const ProbState& ps = st[J.prob];
  const long long N = (long long)pd.N[0] * pd.N[1] * pd.N[2];
  const bool f64 = (pd.cls == CLS_2D_F64 || pd.cls == CLS_3D_F64);
  const long long g0 = ((long long)blockIdx.x - J.block_begin) * kCombineNodes;
  for (int k = threadIdx.x; k < kCombineNodes; k += blockDim.x) {
    const long long g = g0 + k;
    if (g >= N) break;
    if (f64)
      combine_node<double>(J, g, subs, pd, ps);
    else
      combine_node<float>(J, g, subs, pd, ps);
  }
}

cudaError_t launch_combine(const CombineJob* jobs_dev, int njobs, long long total_blocks,
                           const SubDesc* subs, const ProbDesc* probs, const ProbState* st,
                           cudaStream_t s) {
  if (njobs <= 0 || total_blocks <= 0) return cudaSuccess;
  k_combine<<<(unsigned)total_blocks, 256, 0, s>>>(jobs_dev, njobs, subs, probs, st);
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
  const bool alt = pd.transmission == PMA_TRANSMISSION_ALTERNATING &&
                   exchange_step(ps.step - 1, pd.exchange_every);
  auto f = [&](int di, int dj, int dl) -> double {
    return (double)fetch_v<T>(sd, v, dim, li[0] + di, li[1] + dj, li[2] + dl, ps.corr, pd, subs,
                              ps.parity, alt);
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
