// pma_internal.h -- device-side tables shared by the sm_103a kernels and the
// host runtime of the DDPMA library.  Not part of the public ABI.
//
// Data layout in HBM (one request = one "problem"):
//   * every subdomain owns two contiguous state buffers v[0], v[1] (ping-pong)
//     of n0*n1*n2 values of the deviation potential v = Psi - |xi|^2/2,
//     x fastest; FP32 or FP64 per request;
//   * the per-step sweep reads v[parity] and writes v[parity^1];
//   * per-tile partial reductions (one 64-byte record per tile) are folded
//     into per-problem scalars by the last tile of each problem;
//   * per-problem scalars (step, normalisation, shift, status) live in a
//     device array indexed by a stable slot number.
#pragma once

#include <cstdint>

#include "pma.h"

namespace pma {

constexpr int kMaxParts = PMA_MAX_PARTS;
constexpr int kMaxTerms = PMA_MAX_TERMS;

// Kernel classes: one work list and one launch per class and step.
enum Cls : int { CLS_2D_F32 = 0, CLS_2D_F64 = 1, CLS_3D_F32 = 2, CLS_3D_F64 = 3, NUM_CLS = 4 };

// Phases of a problem on the device.
enum Phase : int {
  PH_INIT_V = 0,      // next launch writes v^0 (Eq. incond or warm start)
  PH_INIT_THETA = 1,  // next launch computes theta^0 only (no update)
  PH_RUN = 2,         // forward-Euler steps
  PH_DONE = 3
};

struct MonDev {
  int kind, nterms;
  double base, p0;
  pma_term t[kMaxTerms];
};

// Monitor parameters in the sweep precision.  `width` is pre-multiplied by
// log2(e) for the FP32 path (exp(-w q) = 2^(-w log2e q)); k2 = 2k so that
// sin(2 pi k s) = sinpi(k2 s).
template <typename T>
struct alignas(16) MonT {
  int kind, nterms, dim;
  int nring;  // sum of bumps / rings: the terms are stored rings first
              // (nring of them), then bumps; 0 for the other kinds
  T base, p0;
  struct Term {
    int type, axis, along, pad;
    T amp, width, r2, a, k2;
    T c[3];
  } t[kMaxTerms];
  // PMA_MON_TABLE: device copy in the sweep precision (null for the other
  // precision), points per axis, box origin and points per unit length
  const T* table;
  int tn[3], pad2;
  T tlo[3], tsc[3];
};

// Everything one sweep tile needs about its problem, in its precision,
// precomputed on the host (no divisions or FP64 work per tile on device).
template <typename T>
struct alignas(16) ProbHot {
  int dim, rhs, normalize, stop_norm;
  int N[3], sub_base;
  int parts[3], ntiles;
  int alternating;  // 1: alternating transmission (Algorithm 1)
  int mon_fast;     // 1: sum of bump / ring terms (the packed monitor path)
  int nb_base;      // first neighbour entry of the problem's subdomains
  int exchange_every;  // K >= 1: interface data exchanged at steps 0, K, 2K, ...
  T lo[3], h[3], inv2h[3], invh2[3], inv4hh[3], hw[3];
  T dt, vol;
  double hd[3];
  MonT<T> mon;
};

struct ProbDesc {
  int dim;
  int N[3];
  double lo[3];
  double h[3];
  double vol;
  int parts[3];
  int bcore[3][kMaxParts + 1];  // core boundaries b_k per axis
  int sub_base;                 // first subdomain in the subdomain table
  int nsub;
  int tile_begin, tile_end;     // range in this problem's class work list
  int cls;
  int stop_norm, stop_rule, check_every, rhs, normalize, transmission;
  int exchange_every;           // K >= 1 (frozen interface data between exchanges)
  double dt, tol;
  long long max_steps;
  const double* psi0;           // optional warm start (global grid), device
  MonDev mon;
};

struct alignas(16) SubDesc {
  int prob;          // problem slot
  int n[3];          // local node counts (1 on unused axes)
  int g0[3];         // global index of local node 0
  int clo[3], chi[3];// owned core, local indices, inclusive
  int k[3];          // block index per axis
  int faces;         // bit 2a: low face of axis a is physical; bit 2a+1: high
  int idx;           // subdomain index within its problem (raster order)
  int tile_begin, tile_end;  // its tiles in the class work list
  int pitch;         // row stride in elements (n[0] rounded up to 4)
  void* v[2];        // ping-pong state buffers, pitch * n[1] * n[2] values
};

// Step n (the step that computes v^{n+1}) exchanges interface data when
// n is a multiple of K; between exchanges a transmission node keeps the value
// it was staged with.
__host__ __device__ inline bool exchange_step(long long n, int K) {
  return K <= 1 || (n >= 0 && n % K == 0);
}

struct alignas(16) ProbState {
  long long step;       // forward-Euler steps taken
  int phase;            // Phase
  int status;           // pma_status once done
  int parity;           // buffer holding v^step
  unsigned int tiles_done;  // arrival counter of the current launch
  double c_lag;         // normalisation constant used by the next update
  double corr;          // shift of transmission nodes relative to the rest
  double shift;         // S: v_device = v_exact + S at updated nodes
  double theta;         // theta of the last evaluated step
  double theta_prev;    // theta used by the root form (previous step)
  double residual;
  double min_det;
  double pad;
};

// One unit of sweep work: a box of nodes of one subdomain.
//   2D: nodes [i0, i0+cols) x [j0, j0+rows), processed with a flattened
//       node index (row bands: no padding waste on ragged subdomains);
//   3D: an xy tile [i0, i0+cols) x [j0, j0+rows) over planes [k0, k0+depth).
struct alignas(16) WorkItem {
  int sub;
  int prob;
  int ij;    // i0 | j0 << 16
  int ext;   // cols | rows << 16
  int kz;    // 3D: k0 | depth << 16 (planes); 2D: 0
  // 2D: transmission rows and columns of the staged band (halo included):
  // bit q (q < 4) = staged row {0, 1, rows, rows + 1}[q] is a transmission
  // row (each row flagged once); bit 4 / 5 = staged column 4 / cols + 3
  // (local column 0 / n0 - 1) is a transmission column.  3D: 0.
  int flags;
  // TMA staging: 2D: rows of the band's box (the subdomain's full bands
  // plus the halo rows; the box is SWp columns wide); 3D: 1 (the box is the
  // item's staged box); 0 = staged by cp.async.  tma_map: index of the
  // item's tensor map for buffer 0 (buffer 1: the next one).
  int tma_rows;
  int tma_map;
};

struct Partial {
  double theta;   // sum of w rho det over owned nodes
  double l2a;     // sum of w (G - c_lag)^2 over updated nodes (local trapezoid)
  double l2b;     // sum of w (G - c_lag)
  double wsum;    // sum of w
  double gmax, gmin, dmin;
  int nonfinite;
  int sub;
};

static_assert(sizeof(Partial) == 64, "partial record is one 64-byte line");
static_assert(sizeof(WorkItem) == 32, "work item is 32 bytes");

// Work shapes.  2D: a band holds at most `nodes` nodes, at most `cols`
// wide, processed by `threads` threads (shared staging of the band plus a
// one-node halo); 3D: TX x TY threads marching TZ planes.
struct Tile2D { int threads, nodes, smax, cols; };
// 3D: a box of at most `xy` nodes per plane (cols x rows) over `tz` planes.
struct Tile3D { int threads, xy, tz, smax, cols; };

// Cluster-resident 2D path.  A thread-block cluster of up to 16 CTAs holds
// the subdomains of one or more problems, one subdomain per CTA, in shared
// memory for a whole window of steps; transmission values are read from the
// owner's shared memory (distributed shared memory) and theta is reduced
// across the problem's CTAs once per step.  Problems are packed into
// clusters on the host; a CTA without a subdomain only takes part in the
// cluster barriers.
struct ResCta {
  int sub;    // subdomain table index, -1: idle CTA
  int rank0;  // cluster rank of the CTA holding subdomain 0 of the problem
  int pad[2];
};

struct ResArgs {
  const ProbHot<float>* hotf;
  const ProbHot<double>* hotd;
  const ResCta* ctas;  // one entry per CTA of the launch
  const SubDesc* subs;
  const ProbDesc* probs;
  ProbState* st;
  int iters;  // steps of this launch
  int pad;
};

// Shared-memory layout of one resident CTA: two state buffers of
// res_cap_elems() elements (rows of n0 rounded up to 4 plus 8 halo/padding
// columns, n1 + 2 rows), the three column tables, the transmission list (at
// most the subdomain's ring plus 8 mirror images, 8 bytes each) and one
// saved value per list entry.
__host__ __device__ inline int res_cap_elems(int n0, int n1) {
  const int swp = ((n0 + 3) & ~3) + 8;
  return ((n1 + 2) * swp + 3) & ~3;
}
__host__ __device__ inline int res_smem_bytes(int n0, int n1, int esize) {
  const int cr = (n0 + 3) & ~3;
  const int ndir = 2 * (n0 + n1) + 8;
  return (2 * res_cap_elems(n0, n1) + 3 * cr) * esize + ndir * (8 + esize);
}

// Resident classes: shared-memory budget and threads per CTA.
struct ResClass { int smem_bytes, threads; };
constexpr int kResClasses = 4;
constexpr int kResClusterMax = 16;
ResClass res_class(int id, bool fp64);
cudaError_t prepare_res_kernels();
// Clusters of `csize` CTAs of class `id` that fit on the device at once (0:
// the shape cannot be launched).
int res_max_clusters(bool fp64, int id, int csize, int smem_bytes);
cudaError_t launch_res2d(bool fp64, int id, const ResArgs& a, int nclusters, int csize,
                         int smem_bytes, cudaStream_t s);

// Kernel launch entry points (pma_kernels.cu).
// Owners of transmission nodes: for every subdomain, 3^dim entries, one per
// block offset (dx, dy[, dz]) in {-1, 0, 1}^dim (entry (dx + 1) + 3 (dy + 1)
// [+ 9 (dz + 1)]): the neighbouring block's two state buffers, shifted so
// that the owner's value at local node (i, j, l) of THIS subdomain is
// element i + pitch j + plane l of v[parity]; null where there is no such
// block.  A problem's entries start at ProbHot::nb_base.
struct alignas(16) NbEnt {
  const void* v[2];
  int pitch, plane;
  long long pad;
};
static_assert(sizeof(NbEnt) == 32, "neighbour entry is 32 bytes");

struct LaunchArgs {
  const ProbHot<float>* hotf;
  const ProbHot<double>* hotd;
  const WorkItem* work;  // class work list (absolute base)
  int t0;                // first work item of this launch
  int nwork;             // work items of this launch
  const SubDesc* subs;
  const NbEnt* nb;       // neighbour entries (3^dim per subdomain)
  const void* tmap;      // tensor maps (128 B each), see WorkItem::tma_map
  unsigned int* err;     // device error word (bit 0: a bounded wait gave up)
  int stall_bytes;       // test hook: extra bytes announced to the TMA barrier
  const ProbDesc* probs;
  ProbState* st;
  Partial* part;
  unsigned int* queue;   // two counters: next work item, CTAs finished
  int grid;              // CTAs (persistent, pulling work items)
  // Order in which the persistent CTAs take the work items (a permutation
  // of [0, nwork): largest items first, so that the launch ends on small
  // ones), or null for list order.  Records stay indexed by the item, so the
  // order changes no result.
  const int* order;
};

int tile2d_count();
int tile3d_count();
Tile2D tile2d_shape(int id, bool fp64);
Tile3D tile3d_shape(int id, bool fp64);

// cls selects dim/precision; tile_id a compiled tile shape.
cudaError_t launch_sweep(int cls, int tile_id, const LaunchArgs& a, cudaStream_t s);
int sweep_max_blocks_per_sm(int cls, int tile_id);
// Opt every sweep kernel into its dynamic shared-memory size (current
// device); called when a context is created.
cudaError_t prepare_sweep_kernels();

// After a sweep launch: fold the tile records of the listed problem slots
// (one warp each) and advance their scalars.
cudaError_t launch_finish(const int* list, int n, const SubDesc* subs, const ProbDesc* probs,
                          ProbState* st, const Partial* part, const unsigned int* err,
                          cudaStream_t s);

// One combination job: a request's global mesh.  Jobs are laid out on a
// flat grid of blocks of kCombineNodes nodes; block_begin is the job's first
// block (prefix sum over the jobs).
constexpr int kCombineNodes = 1024;
struct CombineJob {
  int prob;        // slot
  int out_fp64;
  void* x;         // dim * N values
  void* psi;       // optional N values
  long long block_begin;
};
cudaError_t launch_combine(const CombineJob* jobs_dev, int njobs, long long total_blocks,
                           const SubDesc* subs, const ProbDesc* probs, const ProbState* st,
                           cudaStream_t s);

// FP64 positivity check of one problem; out (device) receives 4 doubles.
cudaError_t launch_check(int prob, long long nodes, const SubDesc* subs, const ProbDesc* probs,
                         const ProbState* st, double* out, unsigned long long* cnt,
                         cudaStream_t s);

}  // namespace pma
