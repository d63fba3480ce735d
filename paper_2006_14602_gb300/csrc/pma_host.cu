// pma_host.cu -- host runtime behind the C ABI of include/pma.h.
//
// A context owns a CUDA stream, the device tables of every admitted request
// (subdomain descriptors, per-class tile work lists, per-tile partial
// records, per-problem descriptors and scalars) and the requests' state
// buffers.  Work advances in windows of `window` forward-Euler steps: one
// launch per kernel class and step, all captured in one CUDA graph, so a
// window is a single graph launch.  Between windows the host reads the
// per-problem scalars, retires finished requests, admits queued ones while
// the memory budget allows (continuous batching), and rebuilds the tables
// when the set of requests changed.
#include <cuda.h>  // CUtensorMap and its encoder's types (called through the runtime's entry point)
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pma.h"
#include "pma_internal.h"

using namespace pma;

namespace {

thread_local std::string g_err = "";

void set_err(const std::string& s) { g_err = s; }

#define PMA_CK(call)                                                       \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      set_err(std::string(#call) + ": " + cudaGetErrorString(e_));         \
      return PMA_ERR_CUDA;                                                 \
    }                                                                      \
  } while (0)

using Clock = std::chrono::steady_clock;

struct HostSub {
  int n[3], g0[3], clo[3], chi[3], k[3];
  int faces, idx, pitch;
  size_t elems;
  size_t off[2];  // byte offsets of the two buffers in the request block
};

enum ReqState { RQ_QUEUED = 0, RQ_ACTIVE = 1, RQ_FINISHED = 2 };

struct Request {
  uint64_t id = 0;
  pma_grid g{};
  pma_monitor m{};
  pma_decomp d{};
  pma_params p{};
  std::vector<double> psi0;
  std::vector<char> tab_dev;  // tabulated density in the request's precision
  size_t tab_off = 0;
  int dim = 2, cls = 0, esize = 4;
  int parts[3] = {1, 1, 1};
  int bcore[3][kMaxParts + 1];
  std::vector<HostSub> subs;
  long long nodes = 0;       // global nodes
  long long sub_nodes = 0;   // subdomain nodes (with overlap duplicates)
  size_t bytes = 0;          // device bytes
  size_t psi_off = 0;
  char* block = nullptr;     // device allocation
  int slot = -1;
  int res_class = -1;        // resident class, -1: band kernel (fixed at admission)
  int res_smem = 0;          // shared memory one resident CTA of it needs (max over subs)
  int group = 0;             // request group of its class (set by each rebuild)
  ReqState state = RQ_QUEUED;
  pma_info info{};
  Clock::time_point t_submit, t_done;
};

// --------------------------------------------------------------- validation
bool monitor_ok(const pma_monitor& m, int dim) {
  if (m.kind < PMA_MON_SUM || m.kind > PMA_MON_TABLE) return false;
  if ((m.kind == PMA_MON_ARCLEN_BURGERS || m.kind == PMA_MON_ARCLEN_SPIRAL) && dim != 2)
    return false;
  if ((m.kind == PMA_MON_ARCLEN_TANH_SPHERE || m.kind == PMA_MON_ARCLEN_NINE_SPHERES) &&
      dim != 3)
    return false;
  if (m.kind == PMA_MON_ARCLEN_BURGERS && !(m.p0 > 0.0)) return false;
  if (m.kind <= PMA_MON_PRODUCT) {
    if (m.nterms < 0 || m.nterms > PMA_MAX_TERMS) return false;
    for (int t = 0; t < m.nterms; ++t) {
      const pma_term& q = m.term[t];
      if (q.type < PMA_TERM_BUMP || q.type > PMA_TERM_BUMP1) return false;
      if (q.axis < 0 || q.axis >= dim || q.along < 0 || q.along >= dim) return false;
    }
  }
  return true;
}

// Copy a tabulated density into the request (validated; the caller's memory
// is not referenced after this) and its device image in the request's
// precision.
pma_status take_table(Request& r) {
  r.tab_dev.clear();
  if (r.m.kind != PMA_MON_TABLE) {
    r.m.table = nullptr;
    return PMA_OK;
  }
  const int dim = r.g.dim;
  long long cnt = 1;
  for (int a = 0; a < 3; ++a) {
    if (a >= dim) {
      r.m.tn[a] = 1;
      continue;
    }
    if (r.m.tn[a] < 2 || r.m.tn[a] > (1 << 16) || !(r.m.thi[a] > r.m.tlo[a])) {
      set_err("monitor.table: 2 <= tn <= 65536 and thi > tlo on every axis");
      return PMA_ERR_INVALID;
    }
    cnt *= r.m.tn[a];
  }
  if (!r.m.table || cnt > (1LL << 28)) {
    set_err("monitor.table: missing or larger than 2^28 values");
    return PMA_ERR_INVALID;
  }
  const int esize = (r.p.precision == PMA_FP64) ? 8 : 4;
  r.tab_dev.resize((size_t)cnt * esize);
  for (long long i = 0; i < cnt; ++i) {
    const double v = r.m.table[i];
    if (!(v > 0.0) || !std::isfinite(v)) {
      r.tab_dev.clear();
      set_err("monitor.table: values must be positive and finite");
      return PMA_ERR_INVALID;
    }
    if (esize == 8) {
      memcpy(r.tab_dev.data() + 8 * i, &v, 8);
    } else {
      const float f = (float)v;
      memcpy(r.tab_dev.data() + 4 * i, &f, 4);
    }
  }
  r.m.table = nullptr;
  return PMA_OK;
}

// Core partition b_k = round(k N / p); part k spans
// [b_k - floor(o/2), b_{k+1} - 1 + ceil(o/2)] clipped to [0, N-1].
bool axis_parts(int n, int parts, int overlap, int* b, int* lo, int* hi) {
  if (parts < 1 || parts > kMaxParts) return false;
  if (parts > 1 && overlap < 2) return false;
  const int ol = overlap / 2, oh = overlap - overlap / 2;
  for (int k = 0; k <= parts; ++k) b[k] = (int)((2LL * k * n + parts) / (2LL * parts));
  for (int k = 0; k < parts; ++k) {
    lo[k] = (k == 0) ? 0 : b[k] - ol;
    hi[k] = (k == parts - 1) ? n - 1 : b[k + 1] - 1 + oh;
    if (parts > 1 && b[k + 1] - b[k] < oh + 1) return false;
    if (hi[k] - lo[k] + 1 < 3) return false;
  }
  return true;
}

pma_status build_request(Request& r) {
  const pma_grid& g = r.g;
  if (g.dim < 2 || g.dim > 3) {
    set_err("grid.dim must be 2 or 3");
    return PMA_ERR_INVALID;
  }
  r.dim = g.dim;
  const pma_params& p = r.p;
  if (!(p.dt > 0.0) || !std::isfinite(p.dt) || p.max_steps < 0 || !(p.tol >= 0.0)) {
    set_err("params: dt > 0, tol >= 0, max_steps >= 0 required");
    return PMA_ERR_INVALID;
  }
  if (p.stop_norm < 0 || p.stop_norm > 1 || p.stop_rule < 0 || p.stop_rule > 1 || p.rhs < 0 ||
      p.rhs > 1 || p.normalize < 0 || p.normalize > 1 || p.precision < 0 || p.precision > 1) {
    set_err("params: option out of range");
    return PMA_ERR_INVALID;
  }
  if (r.d.transmission != PMA_TRANSMISSION_PARALLEL &&
      r.d.transmission != PMA_TRANSMISSION_ALTERNATING) {
    set_err("decomp.transmission: unknown form");
    return PMA_ERR_INVALID;
  }
  if (r.d.exchange_every < 0) {
    set_err("decomp.exchange_every must be >= 0 (0 and 1: every step)");
    return PMA_ERR_INVALID;
  }
  if (!monitor_ok(r.m, r.dim)) {
    set_err("monitor: bad kind, term or axis");
    return PMA_ERR_INVALID;
  }
  int lo[3][kMaxParts], hi[3][kMaxParts];
  r.nodes = 1;
  for (int a = 0; a < 3; ++a) {
    if (a >= r.dim) {
      r.parts[a] = 1;
      r.bcore[a][0] = 0;
      r.bcore[a][1] = 1;
      lo[a][0] = hi[a][0] = 0;
      continue;
    }
    if (g.n[a] < 3 || g.n[a] > 65535 || !(g.hi[a] > g.lo[a])) {
      set_err("grid: 3 <= n <= 65535 and hi > lo on every axis");
      return PMA_ERR_INVALID;
    }
    r.parts[a] = r.d.parts[a] < 1 ? 1 : r.d.parts[a];
    if (!axis_parts(g.n[a], r.parts[a], r.d.overlap, r.bcore[a], lo[a], hi[a])) {
      set_err("decomp: parts/overlap incompatible with the grid (core >= ceil(o/2)+1)");
      return PMA_ERR_INVALID;
    }
    r.nodes *= g.n[a];
  }
  for (int a = r.dim; a < 3; ++a)
    for (int k = 2; k <= kMaxParts; ++k) r.bcore[a][k] = 1;
  for (int a = 0; a < r.dim; ++a)
    for (int k = r.parts[a] + 1; k <= kMaxParts; ++k) r.bcore[a][k] = g.n[a];
  r.cls = (r.dim == 2) ? (p.precision == PMA_FP64 ? CLS_2D_F64 : CLS_2D_F32)
                       : (p.precision == PMA_FP64 ? CLS_3D_F64 : CLS_3D_F32);
  r.esize = (p.precision == PMA_FP64) ? 8 : 4;
  r.subs.clear();
  size_t off = 0;
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  int idx = 0;
  for (int kz = 0; kz < r.parts[2]; ++kz)
    for (int ky = 0; ky < r.parts[1]; ++ky)
      for (int kx = 0; kx < r.parts[0]; ++kx, ++idx) {
        HostSub s{};
        const int kk[3] = {kx, ky, kz};
        s.faces = 0;
        for (int a = 0; a < 3; ++a) {
          s.k[a] = kk[a];
          s.g0[a] = lo[a][kk[a]];
          s.n[a] = hi[a][kk[a]] - lo[a][kk[a]] + 1;
          s.clo[a] = r.bcore[a][kk[a]] - s.g0[a];
          s.chi[a] = r.bcore[a][kk[a] + 1] - 1 - s.g0[a];
          if (a >= r.dim) {
            s.clo[a] = s.chi[a] = 0;
            s.n[a] = 1;
          }
          if (kk[a] == 0) s.faces |= 1 << (2 * a);
          if (kk[a] == r.parts[a] - 1) s.faces |= 1 << (2 * a + 1);
        }
        s.idx = idx;
        s.pitch = (s.n[0] + 3) & ~3;
        s.elems = (size_t)s.pitch * s.n[1] * s.n[2];
        r.sub_nodes += (long long)s.n[0] * s.n[1] * s.n[2];
        for (int b = 0; b < 2; ++b) {
          s.off[b] = off;
          off = align(off + s.elems * r.esize);
        }
        r.subs.push_back(s);
      }
  r.psi_off = off;
  if (!r.psi0.empty()) off = align(off + (size_t)r.nodes * sizeof(double));
  r.tab_off = off;
  if (!r.tab_dev.empty()) off = align(off + r.tab_dev.size());
  r.bytes = off;
  return PMA_OK;
}

}  // namespace

// ============================================================== context
// Request groups per class (see pma_ctx::ngroups) and the position of the
// device error word after the groups' queue counters.
constexpr int kGroups = 2;
constexpr int kErrWord = 2 * NUM_CLS * kGroups;

struct pma_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0, used = 0;
  int num_sms = 1;

  std::mutex mu;
  std::condition_variable cv;
  uint64_t next_id = 1;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::deque<uint64_t> queue;
  std::vector<uint64_t> active;

  // slots
  int slot_cap = 0;
  std::vector<int> free_slots;
  ProbDesc* d_probs = nullptr;
  ProbState* d_state = nullptr;
  ProbHot<float>* d_hotf = nullptr;
  ProbHot<double>* d_hotd = nullptr;
  std::vector<ProbDesc> h_probs;
  std::vector<ProbHot<float>> h_hotf;
  std::vector<ProbHot<double>> h_hotd;
  ProbState* h_state = nullptr;  // pinned mirror

  // tables
  SubDesc* d_subs = nullptr;
  NbEnt* d_nb = nullptr;
  size_t nb_cap = 0;
  CUtensorMap* d_tmap = nullptr;  // two per subdomain (2D bands staged by TMA)
  size_t tmap_cap = 0;
  size_t subs_cap = 0;
  WorkItem* d_work[NUM_CLS] = {};
  Partial* d_part[NUM_CLS] = {};
  size_t work_cap[NUM_CLS] = {};
  int nwork[NUM_CLS] = {};
  // Request groups: the live requests of a class are split into kGroups
  // groups of about equal node count; each group's items are a contiguous
  // range of the class work list and run as their own sweep + finish chain
  // on their own stream, so that one group's finish pass and launch tail
  // overlap the other group's sweep.  Index kg = k * kGroups + g.
  int ngroups = 1;                        // PMA_OPT_GROUPS (1 or kGroups)
  int gbeg[NUM_CLS * kGroups] = {};       // first item of the group
  int gcnt[NUM_CLS * kGroups] = {};       // items of the group
  int* d_fin[NUM_CLS * kGroups] = {};     // live problem slots per group
  size_t fin_cap[NUM_CLS * kGroups] = {};
  int nfin[NUM_CLS * kGroups] = {};
  std::vector<int> h_fin[NUM_CLS * kGroups];
  // 2 counters per class and group, then the error word (kErrWord)
  unsigned int* d_queue = nullptr;
  int grid[NUM_CLS * kGroups] = {};
  cudaStream_t gstream[kGroups] = {};     // [0] = the context's stream
  cudaEvent_t ev_gfork = nullptr, ev_gjoin[kGroups] = {};
  int tile_id[NUM_CLS] = {};
  std::vector<SubDesc> h_subs;
  std::vector<NbEnt> h_nb;
  std::vector<CUtensorMap> h_tmap;
  unsigned int h_err = 0;
  std::vector<WorkItem> h_work[NUM_CLS];
  // largest-first order of each group's items (relative to the group start)
  std::vector<int> h_order[NUM_CLS * kGroups];
  int* d_order[NUM_CLS * kGroups] = {};
  size_t order_cap[NUM_CLS * kGroups] = {};
  bool dirty = true;
  long long dead_tiles = 0, live_tiles = 0;

  // resident path: per precision and class, the CTA table of the packed
  // clusters; a side stream runs it beside the band kernels
  struct ResGroup {
    std::vector<ResCta> h;
    ResCta* d = nullptr;
    size_t cap = 0;
    int nclusters = 0;
    int smem = 0;
  };
  ResGroup rg[2][kResClasses];
  int res_csize[2][kResClasses] = {};  // cluster size per class (0: unusable)
  bool res_dirty = true;
  long long res_packed = 0, res_live = 0;  // subdomain CTAs packed / still running
  cudaStream_t side[2 * kResClasses] = {};  // one per precision and class
  cudaEvent_t ev_fork = nullptr, ev_join[2 * kResClasses] = {};

  // graphs
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = 0;
  bool graph_valid = false;

  // combine scratch
  CombineJob* d_jobs = nullptr;
  int jobs_cap = 0;
  double* d_stage = nullptr;  // device staging of pma_get_mesh_batch
  size_t stage_cap = 0;       // in doubles
  double* d_check = nullptr;

  // options
  int window = 32;
  int use_graphs = 1;
  int launch_mode = PMA_LAUNCH_BATCHED;
  int opt_tile2d = 0, opt_tile3d = 0;
  int max_active = 0;
  int opt_resident = 0;
  int opt_res_steps = 0;  // steps of a resident launch per window (0: the window's)

  // counters (pma_get_stats)
  pma_stats stats{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // PMA_OPT_TIME_SWEEPS = k: a pair of timing events around the sweep
  // launches of every k-th step of a window (external event records inside
  // the window's graph)
  int opt_time_sweeps = 0;
  int opt_test_stall = 0;  // test hook of the bounded TMA wait
  bool time_this_step = false;
  std::vector<cudaEvent_t> tev;
  std::vector<int> tev_groups;  // per timed (step, class): groups, 2 events each
  int tev_used = 0;
  bool capturing = false;
  int graph_steps_timed = 0;

  // server
  std::thread server;
  std::atomic<bool> stop{false};
  bool serving = false;
  pma_status server_err = PMA_OK;
};

namespace {

pma_status ensure_slots(pma_ctx* c, int need) {
  if (need <= c->slot_cap) return PMA_OK;
  int cap = std::max(need, std::max(64, c->slot_cap * 2));
  ProbDesc* np = nullptr;
  ProbState* ns = nullptr;
  ProbState* hs = nullptr;
  if (c->d_hotf) cudaFree(c->d_hotf);
  if (c->d_hotd) cudaFree(c->d_hotd);
  c->d_hotf = nullptr;
  c->d_hotd = nullptr;
  PMA_CK(cudaMalloc(&c->d_hotf, sizeof(ProbHot<float>) * cap));
  PMA_CK(cudaMalloc(&c->d_hotd, sizeof(ProbHot<double>) * cap));
  PMA_CK(cudaMalloc(&np, sizeof(ProbDesc) * cap));
  PMA_CK(cudaMalloc(&ns, sizeof(ProbState) * cap));
  PMA_CK(cudaMallocHost(&hs, sizeof(ProbState) * cap));
  PMA_CK(cudaMemsetAsync(ns, 0, sizeof(ProbState) * cap, c->stream));
  if (c->slot_cap) {
    PMA_CK(cudaMemcpyAsync(ns, c->d_state, sizeof(ProbState) * c->slot_cap,
                           cudaMemcpyDeviceToDevice, c->stream));
    PMA_CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->d_probs);
    cudaFree(c->d_state);
    memcpy(hs, c->h_state, sizeof(ProbState) * c->slot_cap);
    cudaFreeHost(c->h_state);
  }
  for (int s = cap - 1; s >= c->slot_cap; --s) c->free_slots.push_back(s);
  c->h_probs.resize(cap);
  c->h_hotf.resize(cap);
  c->h_hotd.resize(cap);
  c->d_probs = np;
  c->d_state = ns;
  c->h_state = hs;
  c->slot_cap = cap;
  c->dirty = true;
  c->graph_valid = false;
  return PMA_OK;
}

template <typename X>
pma_status ensure_buf(X** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return PMA_OK;
  size_t nc = std::max<size_t>(need, std::max<size_t>(256, *cap * 2));
  if (*p) cudaFree(*p);
  *p = nullptr;
  PMA_CK(cudaMalloc(p, sizeof(X) * nc));
  *cap = nc;
  return PMA_OK;
}

void fill_probdesc(const Request& r, ProbDesc& pd) {
  memset(&pd, 0, sizeof(pd));
  pd.dim = r.dim;
  pd.vol = 1.0;
  for (int a = 0; a < 3; ++a) {
    if (a < r.dim) {
      pd.N[a] = r.g.n[a];
      pd.lo[a] = r.g.lo[a];
      pd.h[a] = (r.g.hi[a] - r.g.lo[a]) / (double)(r.g.n[a] - 1);
      pd.vol *= r.g.hi[a] - r.g.lo[a];
    } else {
      pd.N[a] = 1;
      pd.lo[a] = 0.0;
      pd.h[a] = 1.0;
    }
    pd.parts[a] = r.parts[a];
    for (int k = 0; k <= kMaxParts; ++k) pd.bcore[a][k] = r.bcore[a][k];
  }
  pd.nsub = (int)r.subs.size();
  pd.cls = r.cls;
  pd.stop_norm = r.p.stop_norm;
  pd.stop_rule = r.p.stop_rule;
  pd.check_every = r.p.check_every > 0 ? r.p.check_every : 1;
  pd.rhs = r.p.rhs;
  pd.normalize = r.p.normalize;
  pd.transmission = r.d.transmission;
  pd.exchange_every = r.d.exchange_every > 1 ? r.d.exchange_every : 1;
  pd.dt = r.p.dt;
  pd.tol = r.p.tol;
  pd.max_steps = r.p.max_steps;
  pd.psi0 = r.psi0.empty() ? nullptr : (const double*)(r.block + r.psi_off);
  pd.mon.kind = r.m.kind;
  pd.mon.nterms = r.m.nterms;
  pd.mon.base = r.m.base;
  pd.mon.p0 = r.m.p0;
  for (int t = 0; t < kMaxTerms; ++t) pd.mon.t[t] = r.m.term[t];
}

template <typename T>
void fill_hot(const Request& r, const ProbDesc& pd, ProbHot<T>& h) {
  memset(&h, 0, sizeof(h));
  h.dim = pd.dim;
  h.rhs = pd.rhs;
  h.normalize = pd.normalize;
  h.stop_norm = pd.stop_norm;
  h.sub_base = pd.sub_base;
  h.ntiles = pd.tile_end - pd.tile_begin;
  h.alternating = pd.transmission == PMA_TRANSMISSION_ALTERNATING ? 1 : 0;
  h.exchange_every = pd.exchange_every;
  for (int a = 0; a < 3; ++a) {
    h.N[a] = pd.N[a];
    h.parts[a] = pd.parts[a];
    h.lo[a] = (T)pd.lo[a];
    h.h[a] = (T)pd.h[a];
    h.hd[a] = pd.h[a];
    h.hw[a] = (T)(0.5 * pd.h[a]);
    h.inv2h[a] = (T)(0.5 / pd.h[a]);
    h.invh2[a] = (T)(1.0 / (pd.h[a] * pd.h[a]));
  }
  h.inv4hh[0] = (T)(0.25 / (pd.h[0] * pd.h[1]));
  h.inv4hh[1] = (T)(0.25 / (pd.h[0] * pd.h[2]));
  h.inv4hh[2] = (T)(0.25 / (pd.h[1] * pd.h[2]));
  h.dt = (T)pd.dt;
  h.vol = (T)pd.vol;
  // exp(-w q) is evaluated as 2^(-w log2(e) q) by the FP32 path
  const double wscale = (sizeof(T) == 4) ? 1.4426950408889634 : 1.0;
  h.mon.kind = r.m.kind;
  h.mon.nterms = r.m.nterms;
  h.mon.dim = pd.dim;
  h.mon.table = (r.m.kind == PMA_MON_TABLE && (int)sizeof(T) == r.esize && r.block)
                    ? (const T*)(r.block + r.tab_off)
                    : nullptr;
  for (int a = 0; a < 3; ++a) {
    h.mon.tn[a] = (a < pd.dim && r.m.kind == PMA_MON_TABLE) ? r.m.tn[a] : 1;
    h.mon.tlo[a] = (T)r.m.tlo[a];
    h.mon.tsc[a] = (a < pd.dim && r.m.kind == PMA_MON_TABLE)
                       ? (T)((double)(r.m.tn[a] - 1) / (r.m.thi[a] - r.m.tlo[a]))
                       : T(0);
  }
  h.mon.base = (T)r.m.base;
  h.mon.p0 = (T)r.m.p0;
  h.mon_fast = r.m.kind == PMA_MON_SUM ? 1 : 0;
  for (int t = 0; t < r.m.nterms && t < kMaxTerms; ++t)
    if (r.m.term[t].type != PMA_TERM_BUMP && r.m.term[t].type != PMA_TERM_RING) h.mon_fast = 0;
  for (int t = 0; t < kMaxTerms; ++t) {
    const pma_term& q = r.m.term[t];
    auto& o = h.mon.t[t];
    o.type = q.type;
    o.axis = q.axis;
    o.along = q.along;
    o.amp = (T)q.amp;
    o.width = (T)(q.width * wscale);
    o.r2 = (T)q.r2;
    o.a = (T)q.a;
    o.k2 = (T)(2.0 * q.k);
    for (int a = 0; a < 3; ++a) o.c[a] = (T)q.c[a];
  }
  h.mon.nring = 0;
  if (h.mon_fast) {
    // rings first, then bumps (the sweep evaluates the two kinds in two
    // branch-free loops); the sum is the same up to rounding order
    typename MonT<T>::Term sorted[kMaxTerms];
    int n = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int t = 0; t < r.m.nterms && t < kMaxTerms; ++t)
        if ((h.mon.t[t].type == PMA_TERM_RING) == (pass == 0)) sorted[n++] = h.mon.t[t];
    for (int t = 0; t < n; ++t) {
      h.mon.t[t] = sorted[t];
      if (sorted[t].type == PMA_TERM_RING) h.mon.nring = t + 1;
    }
  }
}

int pick_tile(pma_ctx* c, int cls) {
  if (cls == CLS_2D_F32 || cls == CLS_2D_F64) {
    int id = c->opt_tile2d;
    return (id >= 0 && id < tile2d_count()) ? id : 0;
  }
  int id = c->opt_tile3d;
  return (id >= 0 && id < tile3d_count()) ? id : 0;
}

// Work items of one subdomain (entry sidx of the subdomain table).
//   2D: bands of full-width rows (strips of at most t2.cols columns), sized
//       so that the staged band, its halo and the column tables fit;
//   3D: boxes of cols x rows nodes per plane over tz planes.
// Mirror of a node index across a physical face, clamp across a
// transmission face (the staged halo of a band).
static int reflect_host(int i, int n, bool phys_lo, bool phys_hi) {
  if (i < 0) i = phys_lo ? -i : 0;
  if (i >= n) i = phys_hi ? 2 * (n - 1) - i : n - 1;
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Transmission rows / columns of a staged 2D band (WorkItem::flags).
static int band_flags(const HostSub& hs, int i0, int j0, int cols, int rows) {
  const int n0 = hs.n[0], n1 = hs.n[1], f = hs.faces;
  const bool plx = f & 1, phx = f & 2, ply = f & 4, phy = f & 8;
  const int dly = ply ? -1 : 0, dhy = phy ? -1 : n1 - 1;
  const int sh = rows + 2;
  const int cand[4] = {0, 1, sh - 2, sh - 1};
  int fl = 0;
  for (int q = 0; q < 4; ++q) {
    bool dup = false;
    for (int p = 0; p < q; ++p) dup = dup || cand[p] == cand[q];
    if (dup) continue;
    const int jj = reflect_host(j0 - 1 + cand[q], n1, ply, phy);
    if (jj == dly || jj == dhy) fl |= 1 << q;
  }
  if (!plx && i0 == 0) fl |= 16;
  if (!phx && i0 + cols == n0) fl |= 32;
  return fl;
}

void push_items(const HostSub& hs, int dim, bool fp64, int tile_id, int sidx, int slot,
                std::vector<WorkItem>& wl) {
  if (dim == 2) {
    const Tile2D t2 = tile2d_shape(tile_id, fp64);
    for (int x = 0; x < hs.n[0]; x += t2.cols) {
      const int cols = std::min(t2.cols, hs.n[0] - x);
      const int cr = (cols + 3) & ~3;
      const int swp = cr + 8;
      int rows = std::max(1, std::min(hs.n[1], t2.nodes / cr));
      while (rows > 1 && ((rows + 2) * swp + 5 * cr > t2.smax || rows + 2 > 2 * t2.threads))
        --rows;
      // one TMA box per band where the subdomain is one strip and the box
      // fits the copy engine's 256 x 256 limit
      const int tr = (cols == hs.n[0] && swp <= 256 && rows + 2 <= 256) ? rows + 2 : 0;
      for (int y = 0; y < hs.n[1]; y += rows) {
        const int rr = std::min(rows, hs.n[1] - y);
        wl.push_back(WorkItem{sidx, slot, x | (y << 16), cols | (rr << 16), 0,
                              band_flags(hs, x, y, cols, rr), tr, -1});
      }
    }
  } else {
    const Tile3D t3 = tile3d_shape(tile_id, fp64);
    for (int x = 0; x < hs.n[0]; x += t3.cols) {
      const int cols = std::min(t3.cols, hs.n[0] - x);
      const int cr = (cols + 3) & ~3;
      const int swp = cr + 8;
      int rows = std::max(1, std::min(hs.n[1], t3.xy / cr));
      while (rows > 1 && ((rows + 2) * swp * (t3.tz + 2) + 5 * cr > t3.smax ||
                          (rows + 2) * (t3.tz + 2) > 8 * t3.threads))
        --rows;
      // one TMA box per item where the subdomain is one strip and the box
      // fits the copy engine's 256 x 256 x 256 limit
      const int t3ok = (cols == hs.n[0] && swp <= 256 && rows + 2 <= 256 && t3.tz + 2 <= 256);
      for (int y = 0; y < hs.n[1]; y += rows) {
        const int rr = std::min(rows, hs.n[1] - y);
        for (int z = 0; z < hs.n[2]; z += t3.tz) {
          const int d = std::min(t3.tz, hs.n[2] - z);
          wl.push_back(WorkItem{sidx, slot, x | (y << 16), cols | (rr << 16), z | (d << 16), 0,
                                t3ok, -1});
        }
      }
    }
  }
}

// The driver's tiled tensor-map encoder, found once through the runtime
// (no link-time dependency on the driver library); null if unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// Tensor maps of a subdomain's two state buffers for the TMA staging of its
// work items: the buffer as a (pitch x n1 [x n2]) array, boxes of
// (SWp x box_rows [x box_planes]) elements, zero fill outside.  Returns
// false (the items then stage with cp.async) if the encoder is missing or
// refuses.
bool encode_box_maps(const SubDesc& sd, int dim, int esize, int cols, int box_rows,
                     int box_planes, CUtensorMap out[2]) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)sd.pitch, (cuuint64_t)sd.n[1], (cuuint64_t)sd.n[2]};
  const cuuint64_t strides[2] = {(cuuint64_t)sd.pitch * (cuuint64_t)esize,
                                 (cuuint64_t)sd.pitch * (cuuint64_t)sd.n[1] * (cuuint64_t)esize};
  const cuuint32_t box[3] = {(cuuint32_t)(((cols + 3) & ~3) + 8), (cuuint32_t)box_rows,
                             (cuuint32_t)box_planes};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int p = 0; p < 2; ++p) {
    if (fn(&out[p], esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
           (cuuint32_t)dim, sd.v[p], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// Tensor maps for the TMA items of one subdomain (items wl[b, e)): 2D, one
// pair for the subdomain's band box; 3D, one pair per distinct box extent
// (full / last rows x full / last planes).  Items whose maps cannot be
// encoded fall back to cp.async.
void assign_maps(const SubDesc& sd, int dim, int esize, int n0, WorkItem* w, int n,
                 std::vector<CUtensorMap>& maps) {
  if (n <= 0 || w[0].tma_rows <= 0) return;
  if (dim == 2) {
    const size_t base = maps.size();
    maps.resize(base + 2);
    if (encode_box_maps(sd, 2, esize, n0, w[0].tma_rows, 1, &maps[base])) {
      for (int t = 0; t < n; ++t) w[t].tma_map = (int)base;
    } else {
      maps.resize(base);
      for (int t = 0; t < n; ++t) w[t].tma_rows = 0;
    }
    return;
  }
  int ext[4][3], nm = 0;  // (rows, planes, map index)
  for (int t = 0; t < n; ++t) {
    const int rr = w[t].ext >> 16, d = w[t].kz >> 16;
    int m = -1;
    bool seen = false;
    for (int q = 0; q < nm; ++q)
      if (ext[q][0] == rr && ext[q][1] == d) {
        m = ext[q][2];
        seen = true;
      }
    if (!seen && nm < 4) {
      const size_t base = maps.size();
      maps.resize(base + 2);
      if (encode_box_maps(sd, 3, esize, n0, rr + 2, d + 2, &maps[base])) {
        m = (int)base;
      } else {
        maps.resize(base);
      }
      ext[nm][0] = rr;
      ext[nm][1] = d;
      ext[nm][2] = m;
      ++nm;
    }
    if (m < 0) {
      w[t].tma_rows = 0;
    } else {
      w[t].tma_map = m;
    }
  }
}

// Neighbour entries of the subdomains subs[0..n) of one problem (blocks in
// raster order over parts), appended to `out` (see NbEnt).
void fill_nb(const SubDesc* subs, int n, int dim, const int parts[3], int esize,
             std::vector<NbEnt>& out) {
  const int per = dim == 3 ? 27 : 9;
  for (int s = 0; s < n; ++s) {
    const SubDesc& me = subs[s];
    for (int q = 0; q < per; ++q) {
      const int d[3] = {q % 3 - 1, (q / 3) % 3 - 1, per == 27 ? q / 9 - 1 : 0};
      int k[3];
      bool ok = true;
      for (int a = 0; a < 3; ++a) {
        k[a] = me.k[a] + d[a];
        ok = ok && k[a] >= 0 && k[a] < parts[a];
      }
      NbEnt e{};
      if (ok) {
        const SubDesc& o = subs[(k[2] * parts[1] + k[1]) * parts[0] + k[0]];
        const long long pitch = o.pitch, plane = (long long)o.pitch * o.n[1];
        const long long c0 = (me.g0[0] - o.g0[0]) + pitch * (me.g0[1] - o.g0[1]) +
                             plane * (me.g0[2] - o.g0[2]);
        for (int p = 0; p < 2; ++p) e.v[p] = (const char*)o.v[p] + c0 * esize;
        e.pitch = (int)pitch;
        e.plane = (int)plane;
      }
      out.push_back(e);
    }
  }
}

// Rebuild subdomain table, work lists and problem descriptors for the
// current active + finished requests.  Only active requests get tiles.
pma_status rebuild(pma_ctx* c) {
  const auto t_rb = Clock::now();
  c->h_subs.clear();
  c->h_nb.clear();
  c->h_tmap.clear();
  const int G = (c->launch_mode == PMA_LAUNCH_BATCHED) ? std::max(1, std::min(c->ngroups, kGroups)) : 1;
  for (int k = 0; k < NUM_CLS; ++k) {
    c->h_work[k].clear();
    for (int g = 0; g < kGroups; ++g) c->h_fin[k * kGroups + g].clear();
    c->tile_id[k] = pick_tile(c, k);
  }
  c->live_tiles = 0;
  c->dead_tiles = 0;
  // groups: per class, the live band requests in decreasing subdomain-node
  // count, each to the group with the fewest nodes so far (ties: lower group)
  auto is_live = [](const Request& r) {
    return r.state == RQ_ACTIVE && r.slot >= 0 && r.res_class < 0;
  };
  {
    std::vector<Request*> byc[NUM_CLS];
    for (auto& kv : c->reqs)
      if (is_live(*kv.second)) byc[kv.second->cls].push_back(kv.second.get());
    for (int k = 0; k < NUM_CLS; ++k) {
      std::stable_sort(byc[k].begin(), byc[k].end(), [](const Request* a, const Request* b) {
        return a->sub_nodes > b->sub_nodes;
      });
      long long load[kGroups] = {};
      for (Request* r : byc[k]) {
        int g = 0;
        for (int q = 1; q < G; ++q)
          if (load[q] < load[g]) g = q;
        r->group = g;
        load[g] += r->sub_nodes;
      }
    }
  }
  // pass g emits the requests of group g (pass 0 also those without band
  // items: finished, or on the resident path), so every group's items are
  // one contiguous range of its class list
  for (int g = 0; g < G; ++g) {
    for (int k = 0; k < NUM_CLS; ++k) c->gbeg[k * kGroups + g] = (int)c->h_work[k].size();
    for (auto& kv : c->reqs) {
      Request& r = *kv.second;
      if (r.state == RQ_QUEUED || r.slot < 0) continue;
      const bool live = is_live(r);
      if (live ? r.group != g : g != 0) continue;
      ProbDesc& pd = c->h_probs[r.slot];
      fill_probdesc(r, pd);
      pd.sub_base = (int)c->h_subs.size();
      std::vector<WorkItem>& wl = c->h_work[r.cls];
      pd.tile_begin = (int)wl.size();
      for (size_t si = 0; si < r.subs.size(); ++si) {
        const HostSub& hs = r.subs[si];
        SubDesc sd{};
        sd.prob = r.slot;
        for (int a = 0; a < 3; ++a) {
          sd.n[a] = hs.n[a];
          sd.g0[a] = hs.g0[a];
          sd.clo[a] = hs.clo[a];
          sd.chi[a] = hs.chi[a];
          sd.k[a] = hs.k[a];
        }
        sd.faces = hs.faces;
        sd.idx = hs.idx;
        sd.pitch = hs.pitch;
        sd.v[0] = r.block + hs.off[0];
        sd.v[1] = r.block + hs.off[1];
        sd.tile_begin = (int)wl.size();
        if (live)
          push_items(hs, r.dim, r.esize == 8, c->tile_id[r.cls], (int)c->h_subs.size(), r.slot,
                     wl);
        sd.tile_end = (int)wl.size();
        assign_maps(sd, r.dim, r.esize, hs.n[0], wl.data() + sd.tile_begin,
                    sd.tile_end - sd.tile_begin, c->h_tmap);
        c->h_subs.push_back(sd);
      }
      pd.tile_end = (int)wl.size();
      const int nb_base = (int)c->h_nb.size();
      fill_nb(c->h_subs.data() + pd.sub_base, (int)r.subs.size(), r.dim, pd.parts, r.esize,
              c->h_nb);
      if (live) {
        c->live_tiles += pd.tile_end - pd.tile_begin;
        c->h_fin[r.cls * kGroups + g].push_back(r.slot);
      }
      fill_hot<float>(r, pd, c->h_hotf[r.slot]);
      fill_hot<double>(r, pd, c->h_hotd[r.slot]);
      c->h_hotf[r.slot].nb_base = nb_base;
      c->h_hotd[r.slot].nb_base = nb_base;
    }
    for (int k = 0; k < NUM_CLS; ++k)
      c->gcnt[k * kGroups + g] = (int)c->h_work[k].size() - c->gbeg[k * kGroups + g];
  }
  for (int k = 0; k < NUM_CLS; ++k)
    for (int g = G; g < kGroups; ++g) {
      c->gbeg[k * kGroups + g] = (int)c->h_work[k].size();
      c->gcnt[k * kGroups + g] = 0;
    }
  pma_status st;
  if ((st = ensure_buf(&c->d_subs, &c->subs_cap, c->h_subs.size() + 1)) != PMA_OK) return st;
  if ((st = ensure_buf(&c->d_nb, &c->nb_cap, c->h_nb.size() + 1)) != PMA_OK) return st;
  if ((st = ensure_buf(&c->d_tmap, &c->tmap_cap, c->h_tmap.size() + 2)) != PMA_OK) return st;
  if (!c->h_subs.empty()) {
    PMA_CK(cudaMemcpyAsync(c->d_subs, c->h_subs.data(), sizeof(SubDesc) * c->h_subs.size(),
                           cudaMemcpyHostToDevice, c->stream));
    PMA_CK(cudaMemcpyAsync(c->d_nb, c->h_nb.data(), sizeof(NbEnt) * c->h_nb.size(),
                           cudaMemcpyHostToDevice, c->stream));
    PMA_CK(cudaMemcpyAsync(c->d_tmap, c->h_tmap.data(), sizeof(CUtensorMap) * c->h_tmap.size(),
                           cudaMemcpyHostToDevice, c->stream));
  }
  for (int k = 0; k < NUM_CLS; ++k) {
    const size_t cap = c->work_cap[k];
    if ((st = ensure_buf(&c->d_work[k], &c->work_cap[k], c->h_work[k].size() + 1)) != PMA_OK)
      return st;
    if (c->work_cap[k] != cap || !c->d_part[k]) {
      if (c->d_part[k]) cudaFree(c->d_part[k]);
      c->d_part[k] = nullptr;
      PMA_CK(cudaMalloc(&c->d_part[k], sizeof(Partial) * c->work_cap[k]));
    }
    c->nwork[k] = (int)c->h_work[k].size();
    if (c->nwork[k])
      PMA_CK(cudaMemcpyAsync(c->d_work[k], c->h_work[k].data(),
                             sizeof(WorkItem) * c->nwork[k], cudaMemcpyHostToDevice,
                             c->stream));
    const std::vector<WorkItem>& wl = c->h_work[k];
    auto size_of = [&](int t) {
      const WorkItem& w = wl[t];
      const long long d = (k == CLS_3D_F32 || k == CLS_3D_F64) ? (w.kz >> 16) : 1;
      return (long long)(w.ext & 0xffff) * (long long)(w.ext >> 16) * d;
    };
    const int per_sm = sweep_max_blocks_per_sm(k, c->tile_id[k]);
    for (int g = 0; g < kGroups; ++g) {
      const int kg = k * kGroups + g;
      c->nfin[kg] = (int)c->h_fin[kg].size();
      if ((st = ensure_buf(&c->d_fin[kg], &c->fin_cap[kg], c->h_fin[kg].size() + 1)) != PMA_OK)
        return st;
      if (c->nfin[kg])
        PMA_CK(cudaMemcpyAsync(c->d_fin[kg], c->h_fin[kg].data(), sizeof(int) * c->nfin[kg],
                               cudaMemcpyHostToDevice, c->stream));
      // largest items first (ties in list order), relative to the group's
      // first item: the persistent CTAs then end the launch on the smallest
      // items instead of a few large ones
      std::vector<int>& ord = c->h_order[kg];
      const int b = c->gbeg[kg], n = c->gcnt[kg];
      ord.resize(n);
      for (int t = 0; t < n; ++t) ord[t] = t;
      std::stable_sort(ord.begin(), ord.end(),
                       [&](int x, int y) { return size_of(b + x) > size_of(b + y); });
      if ((st = ensure_buf(&c->d_order[kg], &c->order_cap[kg], ord.size() + 1)) != PMA_OK)
        return st;
      if (n)
        PMA_CK(cudaMemcpyAsync(c->d_order[kg], ord.data(), sizeof(int) * ord.size(),
                               cudaMemcpyHostToDevice, c->stream));
      c->grid[kg] = std::min(n, per_sm * c->num_sms);
    }
  }
  PMA_CK(cudaMemcpyAsync(c->d_probs, c->h_probs.data(), sizeof(ProbDesc) * c->slot_cap,
                         cudaMemcpyHostToDevice, c->stream));
  PMA_CK(cudaMemcpyAsync(c->d_hotf, c->h_hotf.data(), sizeof(ProbHot<float>) * c->slot_cap,
                         cudaMemcpyHostToDevice, c->stream));
  PMA_CK(cudaMemcpyAsync(c->d_hotd, c->h_hotd.data(), sizeof(ProbHot<double>) * c->slot_cap,
                         cudaMemcpyHostToDevice, c->stream));
  c->stats.h2d_bytes += (double)(sizeof(SubDesc) * c->h_subs.size() + sizeof(NbEnt) * c->h_nb.size() +
                                 sizeof(CUtensorMap) * c->h_tmap.size() +
                                 (sizeof(ProbDesc) + sizeof(ProbHot<float>) +
                                  sizeof(ProbHot<double>)) * c->slot_cap);
  for (int k = 0; k < NUM_CLS; ++k) c->stats.h2d_bytes += (double)sizeof(WorkItem) * c->nwork[k];
  // The host-side vectors must stay alive until the copies complete.
  PMA_CK(cudaStreamSynchronize(c->stream));
  c->stats.rebuild_ms += std::chrono::duration<double, std::milli>(Clock::now() - t_rb).count();
  c->dirty = false;
  c->graph_valid = false;
  c->res_dirty = true;
  return PMA_OK;
}

// Resident class of a request (at admission; never changes afterwards, so a
// request's arithmetic does not depend on what else is admitted): the first
// class whose shared-memory budget holds every subdomain and whose cluster
// holds all of them.  -1: the band kernels.
int pick_res_class(const pma_ctx* c, const Request& r, int* smem) {
  *smem = 0;
  if (!c->opt_resident || c->launch_mode != PMA_LAUNCH_BATCHED || r.dim != 2) return -1;
  if (r.d.transmission != PMA_TRANSMISSION_PARALLEL) return -1;
  if (r.d.exchange_every > 1) return -1;
  const int nsub = (int)r.subs.size();
  if (nsub > kResClusterMax) return -1;
  int need = 0;
  for (const HostSub& hs : r.subs) {
    if (hs.n[0] < 4 || hs.n[1] < 4) return -1;
    need = std::max(need, res_smem_bytes(hs.n[0], hs.n[1], r.esize));
  }
  const int f = r.esize == 8 ? 1 : 0;
  const int nclass = std::min(c->opt_resident, kResClasses);
  for (int id = 0; id < nclass; ++id)
    if (need <= res_class(id, f == 1).smem_bytes && nsub <= c->res_csize[f][id]) {
      *smem = need;
      return id;
    }
  return -1;
}

// Pack the active resident requests of every class into clusters (first fit
// over requests by decreasing subdomain count; the CTAs of one request are
// consecutive ranks of one cluster, in subdomain order).
pma_status rebuild_res(pma_ctx* c) {
  for (int f = 0; f < 2; ++f)
    for (int id = 0; id < kResClasses; ++id) {
      pma_ctx::ResGroup& g = c->rg[f][id];
      g.h.clear();
      g.nclusters = 0;
      g.smem = 0;
    }
  c->res_packed = c->res_live = 0;
  std::vector<const Request*> rs;
  for (uint64_t id : c->active) {
    const Request& r = *c->reqs[id];
    if (r.res_class >= 0 && c->h_state[r.slot].phase != PH_DONE) rs.push_back(&r);
  }
  std::stable_sort(rs.begin(), rs.end(), [](const Request* a, const Request* b) {
    return a->subs.size() > b->subs.size();
  });
  std::vector<int> fill[2][kResClasses];
  for (const Request* rp : rs) {
    const Request& r = *rp;
    const int f = r.esize == 8 ? 1 : 0, id = r.res_class;
    const int cs = c->res_csize[f][id], nsub = (int)r.subs.size();
    pma_ctx::ResGroup& g = c->rg[f][id];
    std::vector<int>& fl = fill[f][id];
    int bin = -1;
    for (size_t b = 0; b < fl.size(); ++b)
      if (fl[b] + nsub <= cs) {
        bin = (int)b;
        break;
      }
    if (bin < 0) {
      bin = (int)fl.size();
      fl.push_back(0);
      g.h.resize((size_t)cs * fl.size(), ResCta{-1, 0, {0, 0}});
    }
    const int rank0 = fl[bin];
    const int base = c->h_probs[r.slot].sub_base;
    for (int s2 = 0; s2 < nsub; ++s2) g.h[(size_t)bin * cs + rank0 + s2] = ResCta{base + s2, rank0, {0, 0}};
    fl[bin] += nsub;
    g.smem = std::max(g.smem, r.res_smem);
    c->res_packed += nsub;
  }
  c->res_live = c->res_packed;
  for (int f = 0; f < 2; ++f)
    for (int id = 0; id < kResClasses; ++id) {
      pma_ctx::ResGroup& g = c->rg[f][id];
      const int cs = c->res_csize[f][id];
      g.nclusters = cs > 0 ? (int)(g.h.size() / cs) : 0;
      if (g.h.empty()) continue;
      pma_status st = ensure_buf(&g.d, &g.cap, g.h.size());
      if (st != PMA_OK) return st;
      PMA_CK(cudaMemcpyAsync(g.d, g.h.data(), sizeof(ResCta) * g.h.size(),
                             cudaMemcpyHostToDevice, c->stream));
      c->stats.h2d_bytes += (double)sizeof(ResCta) * g.h.size();
    }
  PMA_CK(cudaStreamSynchronize(c->stream));
  c->res_dirty = false;
  return PMA_OK;
}

int res_launches(const pma_ctx* c) {
  int n = 0;
  for (int f = 0; f < 2; ++f)
    for (int id = 0; id < kResClasses; ++id) n += c->rg[f][id].nclusters > 0 ? 1 : 0;
  return n;
}

// One window of the resident path: one launch per precision and class, each
// on its own stream so that they run side by side (ordered after everything
// already on the context's stream, which waits for all of them).
pma_status launch_res_window(pma_ctx* c, int steps) {
  PMA_CK(cudaEventRecord(c->ev_fork, c->stream));
  for (int f = 0; f < 2; ++f)
    for (int id = 0; id < kResClasses; ++id) {
      const pma_ctx::ResGroup& g = c->rg[f][id];
      if (g.nclusters == 0) continue;
      cudaStream_t ss = c->side[f * kResClasses + id];
      PMA_CK(cudaStreamWaitEvent(ss, c->ev_fork, 0));
      ResArgs a;
      a.hotf = c->d_hotf;
      a.hotd = c->d_hotd;
      a.ctas = g.d;
      a.subs = c->d_subs;
      a.probs = c->d_probs;
      a.st = c->d_state;
      a.iters = c->opt_res_steps > 0 ? c->opt_res_steps : steps;
      a.pad = 0;
      PMA_CK(launch_res2d(f == 1, id, a, g.nclusters, c->res_csize[f][id], g.smem, ss));
      PMA_CK(cudaEventRecord(c->ev_join[f * kResClasses + id], ss));
    }
  return PMA_OK;
}

pma_status join_res_window(pma_ctx* c) {
  for (int f = 0; f < 2; ++f)
    for (int id = 0; id < kResClasses; ++id)
      if (c->rg[f][id].nclusters > 0)
        PMA_CK(cudaStreamWaitEvent(c->stream, c->ev_join[f * kResClasses + id], 0));
  return PMA_OK;
}

LaunchArgs args_for(pma_ctx* c, int k, int t0, int n) {
  LaunchArgs a;
  a.hotf = c->d_hotf;
  a.hotd = c->d_hotd;
  a.work = c->d_work[k];
  a.t0 = t0;
  a.nwork = n;
  a.subs = c->d_subs;
  a.nb = c->d_nb;
  a.tmap = c->d_tmap;
  a.err = c->d_queue + kErrWord;
  a.stall_bytes = c->opt_test_stall ? 16 : 0;
  a.probs = c->d_probs;
  a.st = c->d_state;
  a.part = c->d_part[k];
  a.queue = c->d_queue + 2 * (k * kGroups);
  a.grid = std::min(n, c->grid[k * kGroups] > 0 ? c->grid[k * kGroups] : n);
  a.order = nullptr;  // the per-subdomain launches take their items in list order
  return a;
}

// The launch of group g of class k: its contiguous item range, its queue
// counters, largest items first.
LaunchArgs args_for_group(pma_ctx* c, int k, int g) {
  const int kg = k * kGroups + g;
  LaunchArgs a = args_for(c, k, c->gbeg[kg], c->gcnt[kg]);
  a.queue = c->d_queue + 2 * kg;
  a.grid = std::min(c->gcnt[kg], c->grid[kg] > 0 ? c->grid[kg] : c->gcnt[kg]);
  a.order = c->d_order[kg];
  return a;
}

// Timing events of the timed steps (PMA_OPT_TIME_SWEEPS): one pair per
// group launch, on the group's stream.
pma_status time_mark(pma_ctx* c, cudaStream_t s) {
  if (!c->time_this_step || c->tev_used >= (int)c->tev.size()) return PMA_OK;
  PMA_CK(cudaEventRecordWithFlags(c->tev[c->tev_used++], s,
                                  c->capturing ? cudaEventRecordExternal
                                               : cudaEventRecordDefault));
  return PMA_OK;
}

int groups_with_work(const pma_ctx* c, int k) {
  int n = 0;
  for (int g = 0; g < kGroups; ++g) n += c->gcnt[k * kGroups + g] > 0 ? 1 : 0;
  return n;
}

pma_status launch_step(pma_ctx* c) {
  for (int k = 0; k < NUM_CLS; ++k) {
    if (c->nwork[k] == 0) continue;
    pma_status st;
    if (c->launch_mode == PMA_LAUNCH_PER_SUBDOMAIN) {
      if (c->time_this_step) c->tev_groups.push_back(1);
      if ((st = time_mark(c, c->stream)) != PMA_OK) return st;
      for (const SubDesc& sd : c->h_subs) {
        const int n = sd.tile_end - sd.tile_begin;
        if (n <= 0 || c->h_probs[sd.prob].cls != k) continue;
        LaunchArgs a = args_for(c, k, sd.tile_begin, n);
        PMA_CK(launch_sweep(k, c->tile_id[k], a, c->stream));
      }
      if ((st = time_mark(c, c->stream)) != PMA_OK) return st;
      PMA_CK(launch_finish(c->d_fin[k * kGroups], c->nfin[k * kGroups], c->d_subs, c->d_probs,
                           c->d_state, c->d_part[k], c->d_queue + kErrWord, c->stream));
      continue;
    }
    // one sweep + finish chain per group, each on its own stream
    if (c->time_this_step) c->tev_groups.push_back(groups_with_work(c, k));
    for (int g = 0; g < kGroups; ++g) {
      const int kg = k * kGroups + g;
      if (c->gcnt[kg] == 0) continue;
      cudaStream_t s = c->gstream[g];
      if ((st = time_mark(c, s)) != PMA_OK) return st;
      PMA_CK(launch_sweep(k, c->tile_id[k], args_for_group(c, k, g), s));
      if ((st = time_mark(c, s)) != PMA_OK) return st;
      PMA_CK(launch_finish(c->d_fin[kg], c->nfin[kg], c->d_subs, c->d_probs, c->d_state,
                           c->d_part[k], c->d_queue + kErrWord, s));
    }
  }
  return PMA_OK;
}

// The band steps of a window: the other groups' streams fork from the
// context's stream before the first step and join it after the last.
bool uses_group_streams(const pma_ctx* c) {
  if (c->launch_mode != PMA_LAUNCH_BATCHED) return false;
  for (int k = 0; k < NUM_CLS; ++k)
    for (int g = 1; g < kGroups; ++g)
      if (c->gcnt[k * kGroups + g] > 0) return true;
  return false;
}

pma_status launch_steps(pma_ctx* c, int steps) {
  const bool fork = uses_group_streams(c);
  if (fork) {
    PMA_CK(cudaEventRecord(c->ev_gfork, c->stream));
    for (int g = 1; g < kGroups; ++g) PMA_CK(cudaStreamWaitEvent(c->gstream[g], c->ev_gfork, 0));
  }
  pma_status st = PMA_OK;
  for (int s = 0; s < steps && st == PMA_OK; ++s) {
    c->time_this_step = c->opt_time_sweeps > 0 && (s % c->opt_time_sweeps) == 0;
    st = launch_step(c);
  }
  c->time_this_step = false;
  if (fork) {
    // joined even after a failed launch, so that a capture can end
    for (int g = 1; g < kGroups; ++g) {
      PMA_CK(cudaEventRecord(c->ev_gjoin[g], c->gstream[g]));
      PMA_CK(cudaStreamWaitEvent(c->stream, c->ev_gjoin[g], 0));
    }
  }
  return st;
}

// Sweep launches per step (one per class and request group, or one per
// subdomain in the per-subdomain mode) and finish launches per step (one per
// class and group).
int sweeps_per_step(pma_ctx* c) {
  int n = 0;
  for (int k = 0; k < NUM_CLS; ++k) {
    if (c->nwork[k] == 0) continue;
    if (c->launch_mode == PMA_LAUNCH_PER_SUBDOMAIN) {
      for (const SubDesc& sd : c->h_subs)
        if (sd.tile_end > sd.tile_begin && c->h_probs[sd.prob].cls == k) ++n;
    } else {
      n += groups_with_work(c, k);
    }
  }
  return n;
}
int finishes_per_step(pma_ctx* c) {
  int n = 0;
  for (int k = 0; k < NUM_CLS; ++k) {
    if (c->nwork[k] == 0) continue;
    n += c->launch_mode == PMA_LAUNCH_PER_SUBDOMAIN ? 1 : groups_with_work(c, k);
  }
  return n;
}
int launches_per_step(pma_ctx* c) { return sweeps_per_step(c) + finishes_per_step(c); }

pma_status run_window(pma_ctx* c, int steps) {
  if (c->dirty) {
    pma_status st = rebuild(c);
    if (st != PMA_OK) return st;
  }
  if (c->res_dirty) {
    pma_status st = rebuild_res(c);
    if (st != PMA_OK) return st;
  }
  const bool graphs = c->use_graphs && c->launch_mode == PMA_LAUNCH_BATCHED;
  const int nres = res_launches(c);
  const int nband = launches_per_step(c);
  if (c->opt_time_sweeps) {
    const size_t need = (size_t)2 * kGroups * NUM_CLS * steps;
    if (c->tev.size() < need) {
      while (c->tev.size() < need) {
        cudaEvent_t e = nullptr;
        PMA_CK(cudaEventCreate(&e));
        c->tev.push_back(e);
      }
      c->graph_valid = false;
    }
  }
  c->tev_used = 0;
  if (!graphs) c->tev_groups.clear();
  PMA_CK(cudaEventRecord(c->ev0, c->stream));
  if (nres > 0) {
    pma_status st = launch_res_window(c, steps);
    if (st != PMA_OK) return st;
  }
  if (nband == 0) {
    // resident work only
  } else if (graphs) {
    if (!c->graph_valid || c->graph_steps != steps) {
      if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
      }
      cudaGraph_t g = nullptr;
      c->tev_groups.clear();
      PMA_CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      c->capturing = true;
      pma_status st = launch_steps(c, steps);
      c->capturing = false;
      c->graph_steps_timed = c->tev_used;
      cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
      if (st != PMA_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      PMA_CK(ce);
      cudaError_t ie = cudaGraphInstantiate(&c->gexec, g, 0);
      cudaGraphDestroy(g);
      PMA_CK(ie);
      c->graph_steps = steps;
      c->graph_valid = true;
    }
    c->tev_used = c->graph_steps_timed;
    PMA_CK(cudaGraphLaunch(c->gexec, c->stream));
  } else {
    pma_status st = launch_steps(c, steps);
    if (st != PMA_OK) return st;
  }
  if (nres > 0) {
    pma_status st = join_res_window(c);
    if (st != PMA_OK) return st;
  }
  PMA_CK(cudaEventRecord(c->ev1, c->stream));
  PMA_CK(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(ProbState) * c->slot_cap,
                         cudaMemcpyDeviceToHost, c->stream));
  PMA_CK(cudaMemcpyAsync(&c->h_err, c->d_queue + kErrWord, sizeof(unsigned int),
                         cudaMemcpyDeviceToHost, c->stream));
  PMA_CK(cudaStreamSynchronize(c->stream));
  if (c->h_err != 0) {
    // clear the word so that the context can run again
    c->h_err = 0;
    PMA_CK(cudaMemsetAsync(c->d_queue + kErrWord, 0, sizeof(unsigned int), c->stream));
    PMA_CK(cudaStreamSynchronize(c->stream));
    set_err("a sweep kernel gave up waiting for its staging copies (bounded wait)");
    return PMA_ERR_TIMEOUT;
  }
  float ms = 0.f;
  PMA_CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->stats.windows += 1;
  c->stats.window_ms += ms;
  // timed (step, class) pairs: from the first group's sweep start to the
  // latest sweep end (the groups' sweeps run at the same time)
  for (size_t q = 0, i = 0; q < c->tev_groups.size(); ++q) {
    const int ng = c->tev_groups[q];
    if ((int)i + 2 * ng > c->tev_used) break;
    float lo = 0.f, hi = 0.f;
    for (int g = 0; g < ng; ++g) {
      float t0 = 0.f, t1 = 0.f;
      if (g > 0) PMA_CK(cudaEventElapsedTime(&t0, c->tev[i], c->tev[i + 2 * g]));
      PMA_CK(cudaEventElapsedTime(&t1, c->tev[i], c->tev[i + 2 * g + 1]));
      lo = std::min(lo, t0);
      hi = std::max(hi, t1);
    }
    i += 2 * ng;
    c->stats.sweep_kernel_ms += hi - lo;
    c->stats.sweep_kernel_launches += 1;
  }
  for (int k = 0; k < NUM_CLS; ++k) c->stats.sweep_steps += c->nwork[k] > 0 ? steps : 0;
  c->stats.sweep_launches += (int64_t)steps * sweeps_per_step(c) + nres;
  c->stats.other_launches += (int64_t)steps * finishes_per_step(c);
  c->stats.res_launches += nres;
  c->stats.d2h_bytes += (double)sizeof(ProbState) * c->slot_cap;
  return PMA_OK;
}

// Retire finished requests (lock held).
void collect(pma_ctx* c) {
  std::vector<uint64_t> still;
  const auto now = Clock::now();
  for (uint64_t id : c->active) {
    Request& r = *c->reqs[id];
    const ProbState& ps = c->h_state[r.slot];
    if (ps.phase == PH_DONE) {
      if (r.res_class >= 0) c->res_live -= (long long)r.subs.size();
      r.state = RQ_FINISHED;
      r.t_done = now;
      r.info.steps = ps.step;
      r.info.residual = ps.residual;
      r.info.theta = ps.theta;
      r.info.min_det = ps.min_det;
      r.info.shift = ps.shift;
      r.info.status = ps.status;
      r.info.latency_us =
          std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
    } else {
      still.push_back(id);
    }
  }
  if (still.size() != c->active.size()) {
    // compact the work lists when most tiles belong to finished requests
    long long live = 0;
    for (uint64_t id : still) {
      const Request& r = *c->reqs[id];
      const ProbDesc& pd = c->h_probs[r.slot];
      live += pd.tile_end - pd.tile_begin;
    }
    if (live * 2 < c->live_tiles) c->dirty = true;
    // repack the clusters when most resident CTAs idle
    if (c->res_live * 2 < c->res_packed) c->res_dirty = true;
    c->active.swap(still);
    c->cv.notify_all();
  }
}

// Admit queued requests while memory and slots allow (lock held).
pma_status admit(pma_ctx* c) {
  const auto t0 = Clock::now();
  bool admitted = false;
  while (!c->queue.empty()) {
    if (c->max_active > 0 && (int)c->active.size() >= c->max_active) break;
    Request& r = *c->reqs[c->queue.front()];
    if (c->budget && c->used + r.bytes > c->budget) break;
    pma_status st = ensure_slots(c, (int)(c->slot_cap - c->free_slots.size()) + 1);
    if (st != PMA_OK) return st;
    void* blk = nullptr;
    cudaError_t e = cudaMallocAsync(&blk, r.bytes, c->stream);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      if (c->active.empty()) {
        set_err(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        return PMA_ERR_NOMEM;
      }
      break;  // wait for memory to free up
    }
    r.block = (char*)blk;
    c->used += r.bytes;
    if (!r.tab_dev.empty()) {
      PMA_CK(cudaMemcpyAsync(r.block + r.tab_off, r.tab_dev.data(), r.tab_dev.size(),
                             cudaMemcpyHostToDevice, c->stream));
      c->stats.h2d_bytes += (double)r.tab_dev.size();
    }
    if (!r.psi0.empty()) {
      PMA_CK(cudaMemcpyAsync(r.block + r.psi_off, r.psi0.data(), sizeof(double) * r.nodes,
                             cudaMemcpyHostToDevice, c->stream));
      c->stats.h2d_bytes += (double)sizeof(double) * r.nodes;
    }
    r.slot = c->free_slots.back();
    c->free_slots.pop_back();
    r.res_class = pick_res_class(c, r, &r.res_smem);
    // the pinned mirror entry is the copy's source: it is not touched again
    // before the synchronisation at the end of this admission pass
    ProbState& ps = c->h_state[r.slot];
    ps = ProbState{};
    ps.phase = PH_INIT_V;
    ps.status = PMA_PENDING;
    PMA_CK(cudaMemcpyAsync(c->d_state + r.slot, &ps, sizeof(ps), cudaMemcpyHostToDevice,
                           c->stream));
    c->stats.h2d_bytes += (double)sizeof(ps);
    admitted = true;
    r.state = RQ_ACTIVE;
    c->active.push_back(r.id);
    c->queue.pop_front();
    c->dirty = true;
  }
  // tables, warm starts and initial states of every admitted request are in
  // flight on the stream; their host sources must outlive the copies
  if (admitted) PMA_CK(cudaStreamSynchronize(c->stream));
  c->stats.admit_ms += std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  return PMA_OK;
}

void free_request(pma_ctx* c, Request& r) {
  if (r.block) {
    cudaFreeAsync(r.block, c->stream);
    r.block = nullptr;
    c->used -= r.bytes;
  }
  if (r.slot >= 0) {
    c->free_slots.push_back(r.slot);
    r.slot = -1;
  }
  // A freed slot is only reused through admit(), which rebuilds the tables
  // before the next window, so finished requests need no rebuild here.
}

pma_status ensure_jobs(pma_ctx* c, int n) {
  if (n <= c->jobs_cap) return PMA_OK;
  if (c->d_jobs) cudaFree(c->d_jobs);
  c->d_jobs = nullptr;
  PMA_CK(cudaMalloc(&c->d_jobs, sizeof(CombineJob) * n));
  c->jobs_cap = n;
  return PMA_OK;
}

// Combine one finished request into device buffers (lock held).
pma_status combine_into(pma_ctx* c, Request& r, void* x, int out_fp64, void* psi) {
  if (c->dirty) {
    pma_status st = rebuild(c);
    if (st != PMA_OK) return st;
  }
  pma_status st = ensure_jobs(c, 1);
  if (st != PMA_OK) return st;
  CombineJob j{r.slot, out_fp64, x, psi, 0};
  const long long nb = (r.nodes + kCombineNodes - 1) / kCombineNodes;
  PMA_CK(cudaMemcpyAsync(c->d_jobs, &j, sizeof(j), cudaMemcpyHostToDevice, c->stream));
  PMA_CK(launch_combine(c->d_jobs, 1, nb, c->d_subs, c->d_probs, c->d_state, c->stream));
  // the job record lives on this stack frame: wait for the copy
  PMA_CK(cudaStreamSynchronize(c->stream));
  c->stats.h2d_bytes += sizeof(j);
  c->stats.other_launches += 1;
  return PMA_OK;
}

pma_status loop_once(pma_ctx* c, std::unique_lock<std::mutex>& lk, bool* idle) {
  pma_status st = admit(c);
  if (st != PMA_OK) return st;
  *idle = c->active.empty();
  if (*idle) return PMA_OK;
  std::vector<long long> before(c->active.size());
  for (size_t i = 0; i < c->active.size(); ++i)
    before[i] = c->h_state[c->reqs[c->active[i]]->slot].step;
  const std::vector<uint64_t> ids = c->active;
  st = run_window(c, c->window);
  if (st != PMA_OK) return st;
  for (size_t i = 0; i < ids.size(); ++i) {
    const Request& r = *c->reqs[ids[i]];
    const long long d = c->h_state[r.slot].step - before[i];
    c->stats.node_updates += d * r.sub_nodes;
    if (r.res_class >= 0) {
      c->stats.res_node_updates += d * r.sub_nodes;
      c->stats.sweep_bytes += 2.0 * r.esize * (double)r.sub_nodes;
    } else {
      c->stats.sweep_bytes += 2.0 * r.esize * (double)(d * r.sub_nodes);
    }
  }
  collect(c);
  (void)lk;
  return PMA_OK;
}

}  // namespace

// ============================================================== C ABI
extern "C" {

const char* pma_status_str(int32_t s) {
  switch (s) {
    case PMA_OK: return "ok";
    case PMA_NOT_CONVERGED: return "not converged";
    case PMA_PENDING: return "pending";
    case PMA_ERR_INVALID: return "invalid argument";
    case PMA_ERR_NOMEM: return "out of device memory";
    case PMA_ERR_TANGLED: return "mesh tangled";
    case PMA_ERR_TIMEOUT: return "timeout";
    case PMA_ERR_CUDA: return "CUDA error";
    case PMA_ERR_BUSY: return "busy";
    case PMA_ERR_NOT_FOUND: return "unknown request";
  }
  return "unknown status";
}

const char* pma_last_error(void) { return g_err.c_str(); }

int32_t pma_abi_version(void) { return PMA_ABI_VERSION; }

pma_status pma_create(pma_ctx** out, int device, size_t mem_budget_bytes, void* stream) {
  if (!out) return PMA_ERR_INVALID;
  *out = nullptr;
  std::unique_ptr<pma_ctx> c(new pma_ctx());
  c->device = device;
  PMA_CK(cudaSetDevice(device));
  PMA_CK(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    PMA_CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  c->budget = mem_budget_bytes;
  PMA_CK(prepare_sweep_kernels());
  PMA_CK(prepare_res_kernels());
  // largest cluster (16, else 8, 4) each resident class can launch at its
  // full budget on this device
  for (int f = 0; f < 2; ++f)
    for (int id = 0; id < kResClasses; ++id) {
      c->res_csize[f][id] = 0;
      for (int cs = kResClusterMax; cs >= 4; cs /= 2)
        if (res_max_clusters(f == 1, id, cs, res_class(id, f == 1).smem_bytes) > 0) {
          c->res_csize[f][id] = cs;
          break;
        }
    }
  for (int k = 0; k < 2 * kResClasses; ++k) {
    PMA_CK(cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking));
    PMA_CK(cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming));
  }
  PMA_CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  pma_status st = ensure_slots(c.get(), 64);
  if (st != PMA_OK) return st;
  PMA_CK(cudaMalloc(&c->d_check, sizeof(double) * 4 + sizeof(unsigned long long)));
  PMA_CK(cudaMalloc(&c->d_queue, sizeof(unsigned int) * (kErrWord + 1)));
  PMA_CK(cudaMemset(c->d_queue, 0, sizeof(unsigned int) * (kErrWord + 1)));
  c->gstream[0] = c->stream;
  for (int g = 1; g < kGroups; ++g) {
    PMA_CK(cudaStreamCreateWithFlags(&c->gstream[g], cudaStreamNonBlocking));
    PMA_CK(cudaEventCreateWithFlags(&c->ev_gjoin[g], cudaEventDisableTiming));
  }
  PMA_CK(cudaEventCreateWithFlags(&c->ev_gfork, cudaEventDisableTiming));
  PMA_CK(cudaEventCreate(&c->ev0));
  PMA_CK(cudaEventCreate(&c->ev1));
  *out = c.release();
  return PMA_OK;
}

pma_status pma_destroy(pma_ctx* c) {
  if (!c) return PMA_ERR_INVALID;
  pma_serve_stop(c);
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto& kv : c->reqs)
    if (kv.second->block) cudaFreeAsync(kv.second->block, c->stream);
  cudaStreamSynchronize(c->stream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  cudaFree(c->d_probs);
  cudaFree(c->d_state);
  cudaFree(c->d_hotf);
  cudaFree(c->d_hotd);
  cudaFreeHost(c->h_state);
  cudaFree(c->d_subs);
  cudaFree(c->d_nb);
  cudaFree(c->d_tmap);
  for (int k = 0; k < NUM_CLS; ++k) {
    cudaFree(c->d_work[k]);
    cudaFree(c->d_part[k]);
  }
  for (int kg = 0; kg < NUM_CLS * kGroups; ++kg) {
    cudaFree(c->d_order[kg]);
    cudaFree(c->d_fin[kg]);
  }
  cudaFree(c->d_jobs);
  cudaFree(c->d_stage);
  cudaFree(c->d_check);
  cudaFree(c->d_queue);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
  for (int f = 0; f < 2; ++f)
    for (int id = 0; id < kResClasses; ++id) cudaFree(c->rg[f][id].d);
  for (int k = 0; k < 2 * kResClasses; ++k) {
    if (c->side[k]) {
      cudaStreamSynchronize(c->side[k]);
      cudaStreamDestroy(c->side[k]);
    }
    if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  for (int g = 1; g < kGroups; ++g) {
    if (c->gstream[g]) {
      cudaStreamSynchronize(c->gstream[g]);
      cudaStreamDestroy(c->gstream[g]);
    }
    if (c->ev_gjoin[g]) cudaEventDestroy(c->ev_gjoin[g]);
  }
  if (c->ev_gfork) cudaEventDestroy(c->ev_gfork);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return PMA_OK;
}

pma_status pma_set_option(pma_ctx* c, int32_t opt, int64_t v) {
  if (!c) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  switch (opt) {
    case PMA_OPT_WINDOW_STEPS:
      if (v < 1 || v > 100000) return PMA_ERR_INVALID;
      c->window = (int)v;
      break;
    case PMA_OPT_USE_GRAPHS: c->use_graphs = v ? 1 : 0; break;
    case PMA_OPT_LAUNCH_MODE:
      if (v != PMA_LAUNCH_BATCHED && v != PMA_LAUNCH_PER_SUBDOMAIN) return PMA_ERR_INVALID;
      c->launch_mode = (int)v;
      c->dirty = true;  // the request groups depend on the launch mode
      break;
    case PMA_OPT_GROUPS:
      if (v < 1 || v > kGroups) return PMA_ERR_INVALID;
      c->ngroups = (int)v;
      c->dirty = true;
      break;
    case PMA_OPT_TILE_2D:
      if (v < 0 || v >= tile2d_count()) return PMA_ERR_INVALID;
      c->opt_tile2d = (int)v;
      c->dirty = true;
      break;
    case PMA_OPT_TILE_3D:
      if (v < 0 || v >= tile3d_count()) return PMA_ERR_INVALID;
      c->opt_tile3d = (int)v;
      c->dirty = true;
      break;
    case PMA_OPT_MAX_ACTIVE:
      if (v < 0) return PMA_ERR_INVALID;
      c->max_active = (int)v;
      break;
    case PMA_OPT_RESIDENT_STEPS:
      if (v < 0 || v > (1 << 20)) return PMA_ERR_INVALID;
      c->opt_res_steps = (int)v;
      break;
    case PMA_OPT_TIME_SWEEPS:
      if (v < 0) return PMA_ERR_INVALID;
      c->opt_time_sweeps = (int)std::min<int64_t>(v, 1 << 20);
      break;
    case PMA_OPT_RESIDENT:
      if (v < 0) return PMA_ERR_INVALID;
      c->opt_resident = (int)std::min<int64_t>(v, kResClasses);
      break;
    case PMA_OPT_TEST_STALL:
      if (v < 0 || v > 1) return PMA_ERR_INVALID;
      c->opt_test_stall = (int)v;
      break;
    default: return PMA_ERR_INVALID;
  }
  c->graph_valid = false;
  return PMA_OK;
}

pma_status pma_get_option(pma_ctx* c, int32_t opt, int64_t* v) {
  if (!c || !v) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  switch (opt) {
    case PMA_OPT_WINDOW_STEPS: *v = c->window; break;
    case PMA_OPT_USE_GRAPHS: *v = c->use_graphs; break;
    case PMA_OPT_LAUNCH_MODE: *v = c->launch_mode; break;
    case PMA_OPT_TILE_2D: *v = c->opt_tile2d; break;
    case PMA_OPT_TILE_3D: *v = c->opt_tile3d; break;
    case PMA_OPT_MAX_ACTIVE: *v = c->max_active; break;
    case PMA_OPT_RESIDENT: *v = c->opt_resident; break;
    case PMA_OPT_TIME_SWEEPS: *v = c->opt_time_sweeps; break;
    case PMA_OPT_RESIDENT_STEPS: *v = c->opt_res_steps; break;
    case PMA_OPT_TEST_STALL: *v = c->opt_test_stall; break;
    case PMA_OPT_GROUPS: *v = c->ngroups; break;
    default: return PMA_ERR_INVALID;
  }
  return PMA_OK;
}

pma_status pma_submit(pma_ctx* c, const pma_grid* grid, const pma_monitor* mon,
                      const pma_decomp* dec, const pma_params* par, const double* psi0,
                      uint64_t* req_id) {
  if (!c || !grid || !mon || !par || !req_id) return PMA_ERR_INVALID;
  std::unique_ptr<Request> r(new Request());
  r->g = *grid;
  r->m = *mon;
  if (dec) {
    r->d = *dec;
  } else {
    r->d.parts[0] = r->d.parts[1] = r->d.parts[2] = 1;
    r->d.overlap = 0;
    r->d.transmission = PMA_TRANSMISSION_PARALLEL;
  }
  r->p = *par;
  if (psi0) {
    long long n = 1;
    for (int a = 0; a < grid->dim && a < 3; ++a) n *= grid->n[a] > 0 ? grid->n[a] : 0;
    if (n <= 0) return PMA_ERR_INVALID;
    r->psi0.assign(psi0, psi0 + n);
  }
  pma_status st = take_table(*r);
  if (st != PMA_OK) return st;
  st = build_request(*r);
  if (st != PMA_OK) return st;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->budget && r->bytes > c->budget) {
    set_err("request larger than the memory budget");
    return PMA_ERR_NOMEM;
  }
  r->id = c->next_id++;
  r->t_submit = Clock::now();
  r->info.status = PMA_PENDING;
  *req_id = r->id;
  c->queue.push_back(r->id);
  c->reqs[r->id] = std::move(r);
  c->cv.notify_all();
  return PMA_OK;
}

pma_status pma_run(pma_ctx* c, int64_t max_windows, int32_t* n_active) {
  if (!c) return PMA_ERR_INVALID;
  std::unique_lock<std::mutex> lk(c->mu);
  if (c->serving) return PMA_ERR_BUSY;
  PMA_CK(cudaSetDevice(c->device));
  int64_t w = 0;
  pma_status st = PMA_OK;
  while (max_windows <= 0 || w < max_windows) {
    bool idle = false;
    st = loop_once(c, lk, &idle);
    if (st != PMA_OK) break;
    if (idle) {
      if (c->queue.empty()) break;
      // a queued request that cannot be admitted with nothing active
      set_err("queued request cannot be admitted");
      st = PMA_ERR_NOMEM;
      break;
    }
    ++w;
  }
  if (n_active) *n_active = (int32_t)(c->active.size() + c->queue.size());
  return st;
}

static void server_main(pma_ctx* c) {
  cudaSetDevice(c->device);
  std::unique_lock<std::mutex> lk(c->mu);
  while (!c->stop.load()) {
    bool idle = false;
    pma_status st = loop_once(c, lk, &idle);
    if (st != PMA_OK) {
      c->server_err = st;
      // fail every pending request so that waiters return
      for (auto& kv : c->reqs)
        if (kv.second->state != RQ_FINISHED) {
          kv.second->state = RQ_FINISHED;
          kv.second->info.status = st;
        }
      c->active.clear();
      c->queue.clear();
      c->cv.notify_all();
      break;
    }
    if (idle) c->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

pma_status pma_serve_start(pma_ctx* c) {
  if (!c) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->serving) return PMA_ERR_BUSY;
  c->stop = false;
  c->serving = true;
  c->server = std::thread(server_main, c);
  return PMA_OK;
}

pma_status pma_serve_stop(pma_ctx* c) {
  if (!c) return PMA_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->serving) return PMA_OK;
    c->stop = true;
    c->cv.notify_all();
  }
  if (c->server.joinable()) c->server.join();
  std::lock_guard<std::mutex> lk(c->mu);
  c->serving = false;
  return c->server_err;
}

pma_status pma_poll(pma_ctx* c, uint64_t id, int32_t* done) {
  if (!c || !done) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->reqs.find(id);
  if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
  *done = it->second->state == RQ_FINISHED ? 1 : 0;
  return PMA_OK;
}

pma_status pma_wait(pma_ctx* c, uint64_t id, int64_t timeout_us) {
  if (!c) return PMA_ERR_INVALID;
  std::unique_lock<std::mutex> lk(c->mu);
  auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  for (;;) {
    auto it = c->reqs.find(id);
    if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
    if (it->second->state == RQ_FINISHED) return (pma_status)it->second->info.status;
    if (!c->serving) {
      // drive the work on this thread
      lk.unlock();
      int32_t n = 0;
      pma_status st = pma_run(c, 1, &n);
      lk.lock();
      if (st != PMA_OK) return st;
      continue;
    }
    if (timeout_us < 0) {
      c->cv.wait(lk);
    } else if (c->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto it2 = c->reqs.find(id);
      if (it2 != c->reqs.end() && it2->second->state == RQ_FINISHED)
        return (pma_status)it2->second->info.status;
      return PMA_ERR_TIMEOUT;
    }
  }
}

pma_status pma_get_mesh_device(pma_ctx* c, uint64_t id, void* x_dev, int32_t out_fp64,
                               void* psi_dev, pma_info* info) {
  if (!c || !x_dev) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->reqs.find(id);
  if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
  Request& r = *it->second;
  if (r.state != RQ_FINISHED) return PMA_ERR_BUSY;
  if (!r.block) return (pma_status)r.info.status;
  PMA_CK(cudaSetDevice(c->device));
  pma_status st = combine_into(c, r, x_dev, out_fp64 ? 1 : 0, psi_dev);
  if (st != PMA_OK) return st;
  if (info) *info = r.info;
  return (pma_status)r.info.status;
}

pma_status pma_get_mesh(pma_ctx* c, uint64_t id, double* x_out, double* psi_out,
                        pma_info* info) {
  if (!c || !x_out) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->reqs.find(id);
  if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
  Request& r = *it->second;
  if (r.state != RQ_FINISHED) return PMA_ERR_BUSY;
  if (!r.block) return (pma_status)r.info.status;
  PMA_CK(cudaSetDevice(c->device));
  const size_t nx = (size_t)r.dim * r.nodes, np = psi_out ? (size_t)r.nodes : 0;
  double* tmp = nullptr;
  PMA_CK(cudaMallocAsync(&tmp, sizeof(double) * (nx + np), c->stream));
  pma_status st = combine_into(c, r, tmp, 1, psi_out ? tmp + nx : nullptr);
  if (st == PMA_OK) {
    cudaError_t e = cudaMemcpyAsync(x_out, tmp, sizeof(double) * nx, cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess && psi_out)
      e = cudaMemcpyAsync(psi_out, tmp + nx, sizeof(double) * np, cudaMemcpyDeviceToHost,
                          c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      set_err(std::string("mesh copy: ") + cudaGetErrorString(e));
      st = PMA_ERR_CUDA;
    }
    c->stats.d2h_bytes += (double)sizeof(double) * (nx + np);
  }
  cudaFreeAsync(tmp, c->stream);
  if (st != PMA_OK) return st;
  if (info) *info = r.info;
  pma_status fin = (pma_status)r.info.status;
  free_request(c, r);
  c->reqs.erase(it);
  return fin;
}

pma_status pma_check_mesh(pma_ctx* c, uint64_t id, double* out4) {
  if (!c || !out4) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->reqs.find(id);
  if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
  Request& r = *it->second;
  if (r.state != RQ_FINISHED || !r.block) return PMA_ERR_BUSY;
  PMA_CK(cudaSetDevice(c->device));
  if (c->dirty) {
    pma_status st = rebuild(c);
    if (st != PMA_OK) return st;
  }
  double init[4] = {INFINITY, INFINITY, INFINITY, 0.0};
  PMA_CK(cudaMemcpyAsync(c->d_check, init, sizeof(double) * 3, cudaMemcpyHostToDevice,
                         c->stream));
  unsigned long long* cnt = (unsigned long long*)(c->d_check + 3);
  PMA_CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), c->stream));
  PMA_CK(launch_check(r.slot, r.nodes, c->d_subs, c->d_probs, c->d_state, c->d_check, cnt,
                      c->stream));
  double res[3];
  unsigned long long n = 0;
  PMA_CK(cudaMemcpyAsync(res, c->d_check, sizeof(double) * 3, cudaMemcpyDeviceToHost,
                         c->stream));
  PMA_CK(cudaMemcpyAsync(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
  PMA_CK(cudaStreamSynchronize(c->stream));
  out4[0] = res[0];
  out4[1] = res[1];
  out4[2] = res[2];
  out4[3] = (double)n;
  return PMA_OK;
}

pma_status pma_get_info(pma_ctx* c, uint64_t id, pma_info* info) {
  if (!c || !info) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->reqs.find(id);
  if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
  *info = it->second->info;
  if (it->second->state != RQ_FINISHED) info->status = PMA_PENDING;
  return PMA_OK;
}

pma_status pma_release(pma_ctx* c, uint64_t id) {
  if (!c) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  auto it = c->reqs.find(id);
  if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
  Request& r = *it->second;
  if (r.state == RQ_ACTIVE) {
    // its tiles are in the work lists: drop them before the next window
    cudaStreamSynchronize(c->stream);
    c->active.erase(std::remove(c->active.begin(), c->active.end(), id), c->active.end());
    c->dirty = true;
  } else if (r.state == RQ_QUEUED) {
    c->queue.erase(std::remove(c->queue.begin(), c->queue.end(), id), c->queue.end());
  }
  free_request(c, r);
  c->reqs.erase(it);
  return PMA_OK;
}

pma_status pma_counts(pma_ctx* c, int32_t* queued, int32_t* active, int32_t* finished) {
  if (!c) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  int f = 0;
  for (auto& kv : c->reqs)
    if (kv.second->state == RQ_FINISHED) ++f;
  if (queued) *queued = (int32_t)c->queue.size();
  if (active) *active = (int32_t)c->active.size();
  if (finished) *finished = f;
  return PMA_OK;
}

pma_status pma_admit(pma_ctx* c) {
  if (!c) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if (c->serving) return PMA_ERR_BUSY;
  PMA_CK(cudaSetDevice(c->device));
  pma_status st = admit(c);
  if (st != PMA_OK) return st;
  if (c->dirty) st = rebuild(c);
  return st;
}

pma_status pma_get_mesh_device_batch(pma_ctx* c, int32_t n, const uint64_t* ids,
                                     void* const* x_dev, int32_t out_fp64) {
  if (!c || n < 0 || (n > 0 && (!ids || !x_dev))) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  PMA_CK(cudaSetDevice(c->device));
  std::vector<CombineJob> jobs;
  long long blocks = 0;
  for (int i = 0; i < n; ++i) {
    auto it = c->reqs.find(ids[i]);
    if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
    Request& r = *it->second;
    if (r.state != RQ_FINISHED || !r.block) return PMA_ERR_BUSY;
    if (!x_dev[i]) return PMA_ERR_INVALID;
    jobs.push_back(CombineJob{r.slot, out_fp64 ? 1 : 0, x_dev[i], nullptr, blocks});
    blocks += (r.nodes + kCombineNodes - 1) / kCombineNodes;
  }
  if (jobs.empty()) return PMA_OK;
  if (c->dirty) {
    pma_status st = rebuild(c);
    if (st != PMA_OK) return st;
  }
  pma_status st = ensure_jobs(c, (int)jobs.size());
  if (st != PMA_OK) return st;
  PMA_CK(cudaMemcpyAsync(c->d_jobs, jobs.data(), sizeof(CombineJob) * jobs.size(),
                         cudaMemcpyHostToDevice, c->stream));
  PMA_CK(launch_combine(c->d_jobs, (int)jobs.size(), blocks, c->d_subs, c->d_probs, c->d_state,
                        c->stream));
  PMA_CK(cudaStreamSynchronize(c->stream));
  c->stats.h2d_bytes += (double)sizeof(CombineJob) * jobs.size();
  c->stats.other_launches += 1;
  return PMA_OK;
}

pma_status pma_get_mesh_batch(pma_ctx* c, int32_t n, const uint64_t* ids, double* x_out,
                              pma_info* infos) {
  if (!c || n < 0 || (n > 0 && (!ids || !x_out))) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  if (n == 0) return PMA_OK;
  PMA_CK(cudaSetDevice(c->device));
  const auto t0 = Clock::now();
  std::vector<Request*> rs;
  std::vector<size_t> off;
  size_t total = 0;
  long long blocks = 0;
  for (int i = 0; i < n; ++i) {
    auto it = c->reqs.find(ids[i]);
    if (it == c->reqs.end()) return PMA_ERR_NOT_FOUND;
    Request& r = *it->second;
    if (r.state != RQ_FINISHED || !r.block) return PMA_ERR_BUSY;
    for (Request* q : rs)
      if (q == &r) {
        set_err("pma_get_mesh_batch: request id listed twice");
        return PMA_ERR_INVALID;
      }
    rs.push_back(&r);
    off.push_back(total);
    total += (size_t)r.dim * (size_t)r.nodes;
  }
  // Page-locked host memory is mapped into the device's address space: the
  // combination kernel then writes the meshes straight into it (all SMs
  // writing over the host link, no staging buffer and no separate copy).
  // Pageable memory goes through a device staging buffer and one copy.
  double* direct = nullptr;
  {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, x_out) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer != nullptr)
      direct = (double*)pa.devicePointer;
    else
      cudaGetLastError();  // an unregistered pointer is not an error here
  }
  if (!direct && total > c->stage_cap) {
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_cap = 0;
    PMA_CK(cudaMalloc(&c->d_stage, sizeof(double) * total));
    c->stage_cap = total;
  }
  double* const dst = direct ? direct : c->d_stage;
  std::vector<CombineJob> jobs;
  for (int i = 0; i < n; ++i) {
    jobs.push_back(CombineJob{rs[i]->slot, 1, dst + off[i], nullptr, blocks});
    blocks += (rs[i]->nodes + kCombineNodes - 1) / kCombineNodes;
  }
  if (c->dirty) {
    pma_status st = rebuild(c);
    if (st != PMA_OK) return st;
  }
  pma_status st = ensure_jobs(c, n);
  if (st != PMA_OK) return st;
  PMA_CK(cudaMemcpyAsync(c->d_jobs, jobs.data(), sizeof(CombineJob) * jobs.size(),
                         cudaMemcpyHostToDevice, c->stream));
  PMA_CK(launch_combine(c->d_jobs, n, blocks, c->d_subs, c->d_probs, c->d_state, c->stream));
  if (!direct)
    PMA_CK(cudaMemcpyAsync(x_out, c->d_stage, sizeof(double) * total, cudaMemcpyDeviceToHost,
                           c->stream));
  PMA_CK(cudaStreamSynchronize(c->stream));
  c->stats.h2d_bytes += (double)sizeof(CombineJob) * jobs.size();
  c->stats.d2h_bytes += (double)sizeof(double) * total;
  c->stats.other_launches += 1;
  for (int i = 0; i < n; ++i) {
    if (infos) infos[i] = rs[i]->info;
    const uint64_t id = rs[i]->id;
    free_request(c, *rs[i]);
    c->reqs.erase(id);
  }
  c->stats.combine_ms += std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  return PMA_OK;
}

pma_status pma_get_stats(pma_ctx* c, pma_stats* out, int32_t reset) {
  if (!c || !out) return PMA_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->stats;
  if (reset) c->stats = pma_stats{};
  return PMA_OK;
}

pma_status pma_solve(int device, const pma_grid* grid, const pma_monitor* mon,
                     const pma_decomp* dec, const pma_params* par, const double* psi0,
                     double* x_out, double* psi_out, pma_info* info) {
  pma_ctx* c = nullptr;
  pma_status st = pma_create(&c, device, 0, nullptr);
  if (st != PMA_OK) return st;
  uint64_t id = 0;
  st = pma_submit(c, grid, mon, dec, par, psi0, &id);
  if (st == PMA_OK) {
    int32_t n = 0;
    st = pma_run(c, 0, &n);
    if (st == PMA_OK) st = pma_get_mesh(c, id, x_out, psi_out, info);
  }
  pma_destroy(c);
  return st;
}

}  // extern "C"

// ============================================================== no-allocation solve
// pma_solve_static runs one request with every intermediate buffer (state,
// tables, tile records, counters) carved out of one fixed scratch array
// that belongs to this library's device code, for callers that must not
// allocate device memory.  The array is reserved on each GPU the library is
// loaded on and held until the process exits.
namespace {

static __device__ __align__(256) unsigned char g_static_scratch[PMA_STATIC_SCRATCH_BYTES];

// Device address of the scratch array on device `dev` (current).  In host
// code the array's name is only a stand-in, so the address is looked up on
// every call: after a device reset, or when the primary context is released
// and created again, the module is loaded anew and the array may sit at a
// new address, so a cached pointer could go stale.
pma_status static_scratch(int dev, void** out) {
  if (dev < 0) {
    set_err("pma_solve_static: no current device");
    return PMA_ERR_INVALID;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    set_err(std::string("pma_solve_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return PMA_ERR_CUDA;
  }
  *out = p;
  return PMA_OK;
}

struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 255) & ~(size_t)255;
    return o;
  }
};

}  // namespace

extern "C" pma_status pma_solve_static(const pma_grid* grid, const pma_monitor* mon,
                                       const pma_decomp* dec, const pma_params* par,
                                       const double* psi0_dev, double* x_dev, pma_info* info,
                                       void* cuda_stream) {
  if (!grid || !mon || !par || !x_dev) return PMA_ERR_INVALID;
  Request r;
  r.g = *grid;
  r.m = *mon;
  if (dec) {
    r.d = *dec;
  } else {
    r.d.parts[0] = r.d.parts[1] = r.d.parts[2] = 1;
    r.d.overlap = 0;
    r.d.transmission = PMA_TRANSMISSION_PARALLEL;
  }
  r.p = *par;
  pma_status st = take_table(r);
  if (st != PMA_OK) return st;
  st = build_request(r);  // state layout (no warm start block)
  if (st != PMA_OK) return st;
  int dev = 0;
  PMA_CK(cudaGetDevice(&dev));
  void* base = nullptr;
  if ((st = static_scratch(dev, &base)) != PMA_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const auto t_start = Clock::now();

  // work items of the request (default work shapes), slot 0
  const int cls = r.cls;
  r.slot = 0;
  std::vector<SubDesc> subs;
  std::vector<WorkItem> work;
  for (size_t si = 0; si < r.subs.size(); ++si) {
    const HostSub& hs = r.subs[si];
    SubDesc sd{};
    sd.prob = 0;
    for (int a = 0; a < 3; ++a) {
      sd.n[a] = hs.n[a];
      sd.g0[a] = hs.g0[a];
      sd.clo[a] = hs.clo[a];
      sd.chi[a] = hs.chi[a];
      sd.k[a] = hs.k[a];
    }
    sd.faces = hs.faces;
    sd.idx = hs.idx;
    sd.pitch = hs.pitch;
    sd.tile_begin = (int)work.size();
    push_items(hs, r.dim, r.esize == 8, 0, (int)si, 0, work);
    sd.tile_end = (int)work.size();
    subs.push_back(sd);
  }
  for (WorkItem& w : work) w.tma_rows = 0;  // the static path stages with cp.async

  // scratch layout; everything must fit the fixed array
  Carve cv;
  const size_t o_subs = cv.take(sizeof(SubDesc) * subs.size());
  const size_t o_nb = cv.take(sizeof(NbEnt) * 27 * subs.size());
  const size_t o_work = cv.take(sizeof(WorkItem) * work.size());
  const size_t o_part = cv.take(sizeof(Partial) * work.size());
  const size_t o_prob = cv.take(sizeof(ProbDesc));
  const size_t o_hotf = cv.take(sizeof(ProbHot<float>));
  const size_t o_hotd = cv.take(sizeof(ProbHot<double>));
  const size_t o_st = cv.take(sizeof(ProbState));
  const size_t o_q = cv.take(sizeof(unsigned int) * (2 * NUM_CLS + 1));
  const size_t o_fin = cv.take(sizeof(int));
  const size_t o_job = cv.take(sizeof(CombineJob));
  const size_t o_v = cv.take(r.bytes);
  if (cv.off > (size_t)PMA_STATIC_SCRATCH_BYTES) {
    set_err("pma_solve_static: request needs " + std::to_string(cv.off) +
            " bytes of scratch, the fixed area holds " +
            std::to_string((size_t)PMA_STATIC_SCRATCH_BYTES));
    return PMA_ERR_NOMEM;
  }
  char* B = (char*)base;
  r.block = B + o_v;
  for (SubDesc& sd : subs) {
    const HostSub& hs = r.subs[sd.idx];
    sd.v[0] = r.block + hs.off[0];
    sd.v[1] = r.block + hs.off[1];
  }
  ProbDesc pd;
  fill_probdesc(r, pd);
  std::vector<NbEnt> nb;
  fill_nb(subs.data(), (int)subs.size(), r.dim, pd.parts, r.esize, nb);
  pd.sub_base = 0;
  pd.tile_begin = 0;
  pd.tile_end = (int)work.size();
  pd.psi0 = psi0_dev;
  ProbHot<float> hf;
  ProbHot<double> hd;
  fill_hot<float>(r, pd, hf);
  fill_hot<double>(r, pd, hd);
  ProbState ps{};
  ps.phase = PH_INIT_V;
  ps.status = PMA_PENDING;
  const int fin = 0;

  // upload (clears the counters and the problem scalars of any earlier call)
  PMA_CK(cudaMemcpyAsync(B + o_subs, subs.data(), sizeof(SubDesc) * subs.size(),
                         cudaMemcpyHostToDevice, s));
  PMA_CK(cudaMemcpyAsync(B + o_nb, nb.data(), sizeof(NbEnt) * nb.size(), cudaMemcpyHostToDevice,
                         s));
  PMA_CK(cudaMemcpyAsync(B + o_work, work.data(), sizeof(WorkItem) * work.size(),
                         cudaMemcpyHostToDevice, s));
  PMA_CK(cudaMemcpyAsync(B + o_prob, &pd, sizeof(pd), cudaMemcpyHostToDevice, s));
  PMA_CK(cudaMemcpyAsync(B + o_hotf, &hf, sizeof(hf), cudaMemcpyHostToDevice, s));
  PMA_CK(cudaMemcpyAsync(B + o_hotd, &hd, sizeof(hd), cudaMemcpyHostToDevice, s));
  PMA_CK(cudaMemcpyAsync(B + o_st, &ps, sizeof(ps), cudaMemcpyHostToDevice, s));
  if (!r.tab_dev.empty())
    PMA_CK(cudaMemcpyAsync(r.block + r.tab_off, r.tab_dev.data(), r.tab_dev.size(),
                           cudaMemcpyHostToDevice, s));
  PMA_CK(cudaMemcpyAsync(B + o_fin, &fin, sizeof(fin), cudaMemcpyHostToDevice, s));
  PMA_CK(cudaMemsetAsync(B + o_q, 0, sizeof(unsigned int) * (2 * NUM_CLS + 1), s));
  PMA_CK(cudaStreamSynchronize(s));

  int num_sms = 1;
  PMA_CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  PMA_CK(prepare_sweep_kernels());
  LaunchArgs la;
  la.hotf = (const ProbHot<float>*)(B + o_hotf);
  la.hotd = (const ProbHot<double>*)(B + o_hotd);
  la.work = (const WorkItem*)(B + o_work);
  la.t0 = 0;
  la.nwork = (int)work.size();
  la.subs = (const SubDesc*)(B + o_subs);
  la.nb = (const NbEnt*)(B + o_nb);
  la.tmap = nullptr;
  la.err = (unsigned int*)(B + o_q) + 2 * NUM_CLS;
  la.stall_bytes = 0;
  la.probs = (const ProbDesc*)(B + o_prob);
  la.st = (ProbState*)(B + o_st);
  la.part = (Partial*)(B + o_part);
  la.queue = (unsigned int*)(B + o_q) + 2 * cls;
  la.order = nullptr;
  la.grid = std::min(la.nwork, sweep_max_blocks_per_sm(cls, 0) * num_sms);

  // step in windows until the request is done: the first window also
  // covers the initial-state and theta^0 passes; windows then double (16 up
  // to 256 steps) and never run past the step cap, so a request that stops
  // early is followed by at most one window of launches that skip it
  const long long cap = r.p.max_steps;
  long long taken = 0;  // steps taken at the last read-back
  long long w = 16;
  for (bool first = true;; first = false) {
    const long long n = std::min(w, std::max(1LL, cap - taken)) + (first ? 2 : 0);
    for (long long k = 0; k < n; ++k) {
      PMA_CK(launch_sweep(cls, 0, la, s));
      PMA_CK(launch_finish((const int*)(B + o_fin), 1, la.subs, la.probs, la.st, la.part, la.err,
                           s));
    }
    PMA_CK(cudaMemcpyAsync(&ps, B + o_st, sizeof(ps), cudaMemcpyDeviceToHost, s));
    PMA_CK(cudaStreamSynchronize(s));
    if (ps.phase == PH_DONE) break;
    taken = ps.step;
    w = std::min(2 * w, 256LL);
  }

  // owner-takes combination into the caller's buffer
  const CombineJob job{0, 1, x_dev, nullptr, 0};
  PMA_CK(cudaMemcpyAsync(B + o_job, &job, sizeof(job), cudaMemcpyHostToDevice, s));
  PMA_CK(launch_combine((const CombineJob*)(B + o_job), 1,
                        (r.nodes + kCombineNodes - 1) / kCombineNodes, la.subs, la.probs, la.st,
                        s));
  PMA_CK(cudaStreamSynchronize(s));
  if (info) {
    info->steps = ps.step;
    info->residual = ps.residual;
    info->theta = ps.theta;
    info->min_det = ps.min_det;
    info->shift = ps.shift;
    info->status = ps.status;
    info->reserved = 0;
    info->latency_us = std::chrono::duration<double, std::micro>(Clock::now() - t_start).count();
  }
  return (pma_status)ps.status;
}

// ============================================================== self-test
// Host-only consistency checks of the tables the sweep kernels index (no
// device is touched; buffer addresses are offsets into a dummy block):
//   * the neighbour table: for sampled local nodes of every subdomain, the
//     entry the kernels select (block offset by core ranges, 3^dim entries
//     per subdomain) addresses the same element as the owner found directly
//     from the core boundaries of the decomposition (Eq.
//     transmission_condition3 with the owner-takes reading of the overlap);
//   * the transmission-row and -column flags of every staged 2D band
//     against a direct classification of its staged rows and columns;
//   * the work items of every compiled shape: an exact tiling of each
//     subdomain, the shared-memory budget, and the TMA box limits.
// Returns the number of failed checks; the first failure is described by
// pma_last_error.
extern "C" int32_t pma_selftest_tables(void) {
  struct Case {
    int dim, n[3], parts[3], o;
  };
  const Case cases[] = {{2, {45, 37, 1}, {3, 2, 1}, 5},    {2, {97, 65, 1}, {4, 3, 1}, 8},
                        {2, {150, 400, 1}, {2, 2, 1}, 6},  {2, {513, 17, 1}, {16, 1, 1}, 4},
                        {2, {2300, 40, 1}, {2, 1, 1}, 6},  {3, {19, 17, 15}, {2, 2, 2}, 4},
                        {3, {30, 44, 27}, {1, 2, 2}, 4},   {3, {40, 9, 11}, {3, 1, 1}, 3}};
  int bad = 0;
  std::string first;
  auto fail = [&](const std::string& what) {
    if (bad++ == 0) first = what;
  };
  for (const Case& cs : cases) {
    for (int esize : {4, 8}) {
      Request r;
      r.g.dim = cs.dim;
      for (int a = 0; a < 3; ++a) {
        r.g.n[a] = cs.n[a];
        r.g.lo[a] = 0.0;
        r.g.hi[a] = 1.0;
        r.d.parts[a] = cs.parts[a];
      }
      r.d.overlap = cs.o;
      r.d.transmission = PMA_TRANSMISSION_PARALLEL;
      r.m.kind = PMA_MON_SUM;
      r.m.nterms = 0;
      r.m.base = 1.0;
      r.p.dt = 1e-4;
      r.p.tol = 0.0;
      r.p.max_steps = 1;
      r.p.check_every = 1;
      r.p.precision = esize == 8 ? PMA_FP64 : PMA_FP32;
      if (build_request(r) != PMA_OK) {
        fail("build_request refused a self-test case");
        continue;
      }
      // buffer addresses inside a host block: compared, never dereferenced
      std::vector<char> host_block(r.bytes + 64);
      char* const block = host_block.data();
      std::vector<SubDesc> subs;
      for (const HostSub& hs : r.subs) {
        SubDesc sd{};
        for (int a = 0; a < 3; ++a) {
          sd.n[a] = hs.n[a];
          sd.g0[a] = hs.g0[a];
          sd.clo[a] = hs.clo[a];
          sd.chi[a] = hs.chi[a];
          sd.k[a] = hs.k[a];
        }
        sd.faces = hs.faces;
        sd.idx = hs.idx;
        sd.pitch = hs.pitch;
        sd.v[0] = block + hs.off[0];
        sd.v[1] = block + hs.off[1];
        subs.push_back(sd);
      }
      // neighbour table against the owner from the core boundaries
      std::vector<NbEnt> nb;
      fill_nb(subs.data(), (int)subs.size(), r.dim, r.parts, esize, nb);
      const int per = r.dim == 3 ? 27 : 9;
      if ((int)nb.size() != per * (int)subs.size()) fail("neighbour table size");
      for (size_t s = 0; s < subs.size() && nb.size() == per * subs.size(); ++s) {
        const SubDesc& me = subs[s];
        int samp[3][4], ns[3];
        for (int a = 0; a < 3; ++a) {
          const int n = me.n[a];
          ns[a] = 0;
          for (int v : {0, 1, n / 2, n - 1})
            if (v >= 0 && v < n) samp[a][ns[a]++] = v;
        }
        for (int ia = 0; ia < ns[0]; ++ia)
          for (int ja = 0; ja < ns[1]; ++ja)
            for (int la = 0; la < ns[2]; ++la) {
              const int loc[3] = {samp[0][ia], samp[1][ja], samp[2][la]};
              int kk[3], q[3];
              for (int a = 0; a < 3; ++a) {
                const int g = me.g0[a] + loc[a];
                kk[a] = 0;
                while (kk[a] + 1 < r.parts[a] && g >= r.bcore[a][kk[a] + 1]) ++kk[a];
                q[a] = loc[a] < me.clo[a] ? 0 : (loc[a] > me.chi[a] ? 2 : 1);
              }
              const SubDesc& o = subs[(kk[2] * r.parts[1] + kk[1]) * r.parts[0] + kk[0]];
              const NbEnt& e = nb[s * per + q[0] + 3 * q[1] + (per == 27 ? 9 * q[2] : 0)];
              for (int p = 0; p < 2; ++p) {
                const long long want =
                    (long long)((const char*)o.v[p] - block) / esize + (me.g0[0] + loc[0] - o.g0[0]) +
                    (long long)o.pitch * ((me.g0[1] + loc[1] - o.g0[1]) +
                                          (long long)o.n[1] * (me.g0[2] + loc[2] - o.g0[2]));
                const long long got = e.v[p] == nullptr
                                          ? -1
                                          : (long long)((const char*)e.v[p] - block) / esize +
                                                loc[0] + (long long)e.pitch * loc[1] +
                                                (long long)e.plane * loc[2];
                if (want != got) fail("neighbour entry addresses the wrong owner element");
              }
            }
      }
      // work items of every compiled shape
      const int nshape = r.dim == 2 ? tile2d_count() : tile3d_count();
      for (int id = 0; id < nshape; ++id) {
        for (size_t si = 0; si < r.subs.size(); ++si) {
          const HostSub& hs = r.subs[si];
          std::vector<WorkItem> wl;
          push_items(hs, r.dim, esize == 8, id, (int)si, 0, wl);
          std::vector<unsigned char> cover((size_t)hs.n[0] * hs.n[1] * hs.n[2], 0);
          for (const WorkItem& w : wl) {
            const int i0 = w.ij & 0xffff, j0 = w.ij >> 16;
            const int cols = w.ext & 0xffff, rows = w.ext >> 16;
            const int k0 = r.dim == 3 ? (w.kz & 0xffff) : 0, dep = r.dim == 3 ? (w.kz >> 16) : 1;
            const int cr = (cols + 3) & ~3, swp = cr + 8;
            for (int l = k0; l < k0 + dep; ++l)
              for (int j = j0; j < j0 + rows; ++j)
                for (int i = i0; i < i0 + cols; ++i) {
                  if (i >= hs.n[0] || j >= hs.n[1] || l >= hs.n[2]) {
                    fail("work item beyond its subdomain");
                    continue;
                  }
                  cover[((size_t)l * hs.n[1] + j) * hs.n[0] + i] += 1;
                }
            if (r.dim == 2) {
              const Tile2D t2 = tile2d_shape(id, esize == 8);
              const int box = w.tma_rows > 0 ? w.tma_rows : rows + 2;
              if (box * swp + 5 * cr > t2.smax) fail("2D band exceeds its shared memory");
              if (w.tma_rows > 0 && (cols != hs.n[0] || swp > 256 || w.tma_rows > 256 ||
                                     w.tma_rows < rows + 2))
                fail("2D TMA box outside the copy engine's limits");
              // transmission flags against the staged rows and columns
              const int n1 = hs.n[1], f = hs.faces;
              const int dly = (f & 4) ? -1 : 0, dhy = (f & 8) ? -1 : n1 - 1;
              const int sh = rows + 2;
              const int cand[4] = {0, 1, sh - 2, sh - 1};
              for (int rr = 0; rr < sh; ++rr) {
                const int jj = reflect_host(j0 - 1 + rr, n1, f & 4, f & 8);
                const bool trans = jj == dly || jj == dhy;
                bool flagged = false;
                for (int qq = 0; qq < 4; ++qq)
                  if ((w.flags >> qq) & 1) flagged = flagged || cand[qq] == rr;
                if (trans != flagged) fail("2D band transmission-row flags");
              }
              const bool cl = !(f & 1) && i0 == 0, ch = !(f & 2) && i0 + cols == hs.n[0];
              if (((w.flags >> 4) & 1) != (cl ? 1 : 0) || ((w.flags >> 5) & 1) != (ch ? 1 : 0))
                fail("2D band transmission-column flags");
            } else {
              const Tile3D t3 = tile3d_shape(id, esize == 8);
              if ((rows + 2) * swp * (dep + 2) + 5 * cr > t3.smax)
                fail("3D box exceeds its shared memory");
              if (w.tma_rows > 0 && (cols != hs.n[0] || swp > 256 || rows + 2 > 256))
                fail("3D TMA box outside the copy engine's limits");
            }
          }
          for (unsigned char c : cover)
            if (c != 1) {
              fail("work items do not tile the subdomain exactly once");
              break;
            }
        }
      }
    }
  }
  if (bad) set_err("pma_selftest_tables: " + std::to_string(bad) + " failed checks; first: " + first);
  return bad;
}
