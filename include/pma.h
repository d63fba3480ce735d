/*
 * pma.h -- C ABI of the GB300 (sm_103a) domain-decomposition parabolic
 * Monge-Ampere (DDPMA) adaptive mesh generator.
 *
 * Method: Sulman, Nguyen, Haynes & Huang, "Domain Decomposition Parabolic
 * Monge-Ampere Approach for Fast Generation of Adaptive Moving Meshes".
 * A mesh x(xi) = grad Psi(xi) on a box Omega_c (Sect. 2, Eq. AdpMesh) is the
 * steady state of the parabolic Monge-Ampere flow
 *     Psi_tau = log(|Omega_c| rho(grad Psi) det D^2 Psi)          (Eq. pmae)
 * from Psi^0 = |xi|^2/2 (Eq. incond) with grad Psi . n = xi . n on the
 * boundary (Eq. nbd).  Omega_c is split into overlapping subdomains that are
 * advanced independently and exchange one layer of Dirichlet data per step
 * (Sect. 3, Eq. transmission_condition3); the subdomain meshes are combined
 * into one global mesh (Sects. 4.4-4.5).
 *
 * Everything here is plain C: host pointers, device pointers passed as
 * void*, sizes and plain structs.  No exception or process exit crosses the
 * boundary: every call returns a pma_status.
 *
 * Threading: one pma_ctx may be driven by one thread at a time, except that
 * pma_submit, pma_poll and pma_wait may be called from any thread while a
 * pma_serve_start() server thread runs.
 *
 * Layouts: global arrays are x-fastest, row-major over (z, y, x); a mesh is
 * component-major: x_out[a * N + node] for a = 0..dim-1, N = prod(n[0..dim-1]).
 */
#ifndef PMA_H
#define PMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMA_ABI_VERSION 2
#define PMA_MAX_TERMS 4
#define PMA_MAX_PARTS 32 /* subdomains per axis */

/* ---------------------------------------------------------------- status */
typedef enum {
  PMA_OK = 0,             /* converged: residual <= tol                     */
  PMA_NOT_CONVERGED = 1,  /* stopped at max_steps; the mesh is still valid  */
  PMA_PENDING = 2,        /* request still running                          */
  PMA_ERR_INVALID = -1,   /* bad argument or unsupported option             */
  PMA_ERR_NOMEM = -2,     /* device memory budget or allocation exhausted   */
  PMA_ERR_TANGLED = -3,   /* det D_h^2 Psi <= 0 or a non-finite value: the
                             mesh of the last valid step is returned        */
  PMA_ERR_TIMEOUT = -4,   /* pma_wait ran out of time                       */
  PMA_ERR_CUDA = -5,      /* a CUDA call failed (see pma_last_error)        */
  PMA_ERR_BUSY = -6,      /* operation not allowed in the current state     */
  PMA_ERR_NOT_FOUND = -7  /* unknown or already released request id         */
} pma_status;

/* ------------------------------------------------------------ problem */

/* Computational box Omega_c = prod_a [lo[a], hi[a]] with n[a] >= 3 nodes on
 * axis a (Sect. 4: uniform grids such as 65x65 or 81x81x81).  Axes >= dim
 * are ignored.                                                             */
typedef struct {
  int32_t dim;      /* 2 or 3 */
  int32_t n[3];
  double lo[3];
  double hi[3];
} pma_grid;

/* Monitor density rho(x) (Sect. 2, Eq. edp1; Sect. 4, Eq. monitfn).
 * Term shapes, x the physical mesh point:
 *   PMA_TERM_BUMP : amp * exp(-width * |x - c|^2)
 *   PMA_TERM_RING : amp * exp(-width * (|x - c|^2 - r2)^2)
 *   PMA_TERM_SINE : amp * exp(-width * (x[axis] - c[axis]
 *                                       - a * sin(2 pi k x[along]))^2)
 *   PMA_TERM_BUMP1: amp * exp(-width * (x[axis] - c[axis])^2)
 * Kinds:
 *   PMA_MON_SUM     rho = base + sum of nterms terms
 *   PMA_MON_PRODUCT rho = prod over terms of (base + term), separable
 *   PMA_MON_ARCLEN_* rho = sqrt(1 + |grad u|^2) of the paper's test
 *                    functions: BURGERS Eq. test_fn1 (eps = p0), SPIRAL
 *                    Eq. test_fn2, TANH_SPHERE Eq. test_fn3d1, NINE_SPHERES
 *                    Eq. test_fn3d2.  nterms is ignored.
 *   PMA_MON_TABLE   rho sampled on a uniform grid of tn[a] >= 2 points over
 *                    [tlo[a], thi[a]] per axis a < dim (values x fastest,
 *                    all > 0 and finite), as a physical solution is sampled
 *                    in the moving-mesh loop of Sect. 2; evaluated by
 *                    multilinear interpolation with the point clamped to the
 *                    table's box.  `table` is host memory, copied at submit;
 *                    it is stored on the device in the request's precision.
 * The density need not be normalised: the normalisation of Eq. (edp) is
 * applied by the solver (see pma_params.normalize).                        */
enum { PMA_TERM_BUMP = 0, PMA_TERM_RING = 1, PMA_TERM_SINE = 2, PMA_TERM_BUMP1 = 3 };
enum { PMA_MON_SUM = 0, PMA_MON_PRODUCT = 1, PMA_MON_ARCLEN_BURGERS = 2,
       PMA_MON_ARCLEN_SPIRAL = 3, PMA_MON_ARCLEN_TANH_SPHERE = 4,
       PMA_MON_ARCLEN_NINE_SPHERES = 5, PMA_MON_TABLE = 6 };

typedef struct {
  int32_t type;
  int32_t axis;
  int32_t along;
  int32_t reserved;
  double amp, width, r2, a, k;
  double c[3];
} pma_term;

typedef struct {
  int32_t kind;
  int32_t nterms;   /* 0..PMA_MAX_TERMS */
  double base;
  double p0;
  pma_term term[PMA_MAX_TERMS];
  const double *table;  /* PMA_MON_TABLE only (else ignored)         */
  int32_t tn[3];        /* table points per axis (1 on axes >= dim)  */
  int32_t reserved;
  double tlo[3], thi[3];
} pma_monitor;

/* Overlapping decomposition (Sect. 3).  parts[a] subdomains along axis a
 * (slabs when one axis is split, blocks otherwise); neighbours share
 * `overlap` node indices (>= 2 when any axis is split; Sect. 4.1 uses 3,
 * Sect. 4.4 studies 5..15).  Core partition b_k = round(k N / p); part k
 * spans [b_k - floor(o/2), b_{k+1} - 1 + ceil(o/2)] clipped to the grid; the
 * owned core is [b_k, b_{k+1} - 1] and must hold >= ceil(o/2) + 1 nodes.
 * transmission: PMA_TRANSMISSION_PARALLEL (Eq. transmission_condition3,
 * every subdomain takes its neighbours' previous-step values) or
 * PMA_TRANSMISSION_ALTERNATING (Algorithm 1: a subdomain takes the new value
 * of an owner that precedes it in raster order).
 * exchange_every: K >= 1 (0 reads as 1).  The subdomains exchange interface
 * data at steps 0, K, 2K, ... only; in between, every transmission node keeps
 * the value of the last exchange, as when each subdomain is integrated over
 * a pseudo-time interval with its neighbours' data frozen at the interval's
 * start (Sect. 3, the paragraph after Algorithm 1).  K = 1 is one exchange
 * per step (bitwise the K = 1 behaviour of either transmission form).
 * Negative values are rejected with PMA_ERR_INVALID.                       */
enum { PMA_TRANSMISSION_PARALLEL = 0, PMA_TRANSMISSION_ALTERNATING = 1 };

typedef struct {
  int32_t parts[3];
  int32_t overlap;
  int32_t transmission;
  int32_t exchange_every;
} pma_decomp;

/* Pseudo-time integration and stopping (Sects. 2, 4.4).
 *   dt          forward-Euler step (Sect. 4.4 uses 0.015..0.12 * h^2)
 *   tol         stop when residual <= tol at a checked step
 *   max_steps   hard cap (PMA_NOT_CONVERGED when reached)
 *   stop_norm   PMA_STOP_MAX_UT: residual = max |Psi_tau| over updated nodes;
 *               PMA_STOP_L2_INCREMENT: ||Psi^{n+1} - Psi^n||_2 of
 *               Eq. (dd_stop_criterion), trapezoid rule per subdomain
 *   stop_rule   PMA_RULE_ALL: every subdomain below tol (max);
 *               PMA_RULE_ANY: min over subdomains (Algorithm 1, step 6)
 *   check_every test the stop rule after every check_every steps (>= 1)
 *   rhs         PMA_RHS_LOG (Eq. pmae) or PMA_RHS_ROOT:
 *               (|Omega_c| rho det / theta)^(1/dim) - 1, with theta of the
 *               previous step (same steady state)
 *   normalize   PMA_NORM_GLOBAL_THETA: rho is normalised by
 *               theta = sum_nodes w rho det D_h^2 Psi over the combined mesh
 *               (the discrete int_Omega rho of Eq. edp) every step;
 *               PMA_NORM_NONE: the subdomain equations of Eq. (pmae1a) as
 *               printed, log(rho det D^2 Psi)
 *   precision   PMA_FP32 (sweep in FP32, reductions and stop test in FP64)
 *               or PMA_FP64                                                */
enum { PMA_STOP_MAX_UT = 0, PMA_STOP_L2_INCREMENT = 1 };
enum { PMA_RULE_ALL = 0, PMA_RULE_ANY = 1 };
enum { PMA_RHS_LOG = 0, PMA_RHS_ROOT = 1 };
enum { PMA_NORM_GLOBAL_THETA = 0, PMA_NORM_NONE = 1 };
enum { PMA_FP32 = 0, PMA_FP64 = 1 };

typedef struct {
  double dt;
  double tol;
  int64_t max_steps;
  int32_t stop_norm;
  int32_t stop_rule;
  int32_t check_every;
  int32_t rhs;
  int32_t normalize;
  int32_t precision;
} pma_params;

/* Outcome of one request. */
typedef struct {
  int64_t steps;       /* pseudo-time steps taken                          */
  double residual;     /* residual of the last step (stop_norm)            */
  double theta;        /* normalisation sum of the last step               */
  double min_det;      /* min det D_h^2 Psi over updated nodes, last step  */
  double shift;        /* internal uniform offset already removed from Psi */
  int32_t status;      /* pma_status of the request                        */
  int32_t reserved;
  double latency_us;   /* admission to completion, host clock              */
} pma_info;

typedef struct pma_ctx pma_ctx;

/* ------------------------------------------------------------ context */

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t, NULL = a new non-blocking stream owned by the context).
 * mem_budget_bytes caps the device memory held by admitted requests (0 = no
 * cap); requests beyond it wait for admission.  The context owns all device
 * memory it allocates and frees it in pma_destroy.
 * Errors: PMA_ERR_INVALID (NULL ctx), PMA_ERR_CUDA.                         */
pma_status pma_create(pma_ctx **ctx, int device, size_t mem_budget_bytes, void *cuda_stream);

/* Stop a running server, wait for the device and free everything. */
pma_status pma_destroy(pma_ctx *ctx);

/* Tuning knobs.  Window, graphs and admission cap leave results bitwise
 * unchanged; tile shapes and the resident path change the order in which
 * theta is summed, so results agree to rounding only.
 *   PMA_OPT_WINDOW_STEPS   steps per CUDA-graph window (default 32)
 *   PMA_OPT_USE_GRAPHS     1 = capture windows in CUDA graphs (default)
 *   PMA_OPT_LAUNCH_MODE    PMA_LAUNCH_BATCHED: all subdomains of all admitted
 *                          requests in one launch per step (default);
 *                          PMA_LAUNCH_PER_SUBDOMAIN: the plain reference path,
 *                          one launch per subdomain per step, no graphs
 *   PMA_OPT_TILE_2D        2D tile shape id (0 = auto)
 *   PMA_OPT_TILE_3D        3D tile shape id (0 = auto)
 *   PMA_OPT_MAX_ACTIVE     cap on concurrently admitted requests (0 = none)
 *   PMA_OPT_RESIDENT       k > 0: 2D requests of at most 16 subdomains (parallel
 *                          transmission, one exchange per step) whose
 *                          subdomains fit the first k shared-memory classes
 *                          (24, 56, 112, 220 KiB per subdomain) run
 *                          cluster-resident: one CTA per subdomain for a whole
 *                          window, transmission values and theta exchanged
 *                          through distributed shared memory; 0 = band
 *                          kernels only (default).  Batched launch mode only;
 *                          decided per request when it is admitted.
 *   PMA_OPT_TIME_SWEEPS    k > 0: time the sweep launches of every k-th step
 *                          of a window with CUDA events, a pair around each
 *                          group's sweep on the group's stream (recorded
 *                          inside the windows' graphs; each pair costs about a
 *                          microsecond, so k = 1 slows a step by several per
 *                          cent); a timed (step, class) counts from its first
 *                          sweep's start to its last sweep's end (the groups'
 *                          sweeps overlap); sums in pma_stats
 *                          (sweep_kernel_ms, sweep_kernel_launches).
 *                          0 = off (default).
 *   PMA_OPT_RESIDENT_STEPS steps a resident launch takes per window (0 = the
 *                          window's steps, default).  A resident step costs
 *                          a few microseconds against tens for a band step,
 *                          so resident requests can run several band windows'
 *                          worth of steps while the band work of a window
 *                          runs beside them (results do not depend on it).
 *   PMA_OPT_TEST_STALL     test hook of the bounded waits: 1 = the 2D and 3D
 *                          sweep kernels announce 16 more bytes to their TMA
 *                          staging barrier than the copy delivers, so the wait
 *                          gives up after about a second; the kernel records
 *                          the failure in the device error word and leaves,
 *                          the step's finish pass retires every active request
 *                          with PMA_ERR_TIMEOUT (later sweeps skip their work)
 *                          and pma_run returns PMA_ERR_TIMEOUT; the context
 *                          stays usable.  0 = off (default).
 *   PMA_OPT_GROUPS         request groups per kernel class in the batched
 *                          mode, 1 (default) or 2: the admitted requests of
 *                          a class are split into groups of about equal node
 *                          count, and each group's sweep and finish launches
 *                          run on their own stream (captured in the same
 *                          graph), so that one group's finish pass and launch
 *                          tail overlap the other's sweep.  Requests are
 *                          independent, so results do not depend on it
 *                          (bitwise). */
enum { PMA_OPT_WINDOW_STEPS = 1, PMA_OPT_USE_GRAPHS = 2, PMA_OPT_LAUNCH_MODE = 3,
       PMA_OPT_TILE_2D = 4, PMA_OPT_TILE_3D = 5, PMA_OPT_MAX_ACTIVE = 6,
       PMA_OPT_RESIDENT = 7, PMA_OPT_TIME_SWEEPS = 8, PMA_OPT_RESIDENT_STEPS = 9,
       PMA_OPT_TEST_STALL = 10, PMA_OPT_GROUPS = 11 };
enum { PMA_LAUNCH_BATCHED = 0, PMA_LAUNCH_PER_SUBDOMAIN = 1 };
pma_status pma_set_option(pma_ctx *ctx, int32_t option, int64_t value);
pma_status pma_get_option(pma_ctx *ctx, int32_t option, int64_t *value);

/* ------------------------------------------------------------ requests */

/* Queue one mesh-generation request.  All inputs are copied; psi0 (optional,
 * host, N doubles, NULL = Eq. incond) is a warm start such as the previous
 * steady state (Sect. 2).  The request is admitted to the device at the next
 * window boundary when its memory fits the budget.
 * Errors: PMA_ERR_INVALID (bad grid/decomposition/params), PMA_ERR_NOMEM
 * (larger than the whole budget).                                          */
pma_status pma_submit(pma_ctx *ctx, const pma_grid *grid, const pma_monitor *monitor,
                      const pma_decomp *decomp, const pma_params *params,
                      const double *psi0, uint64_t *req_id);

/* Advance every admitted request on the calling thread until all queued and
 * admitted requests are finished or max_windows windows have run (<= 0: no
 * limit).  *n_active (optional) receives the number still unfinished.     */
pma_status pma_run(pma_ctx *ctx, int64_t max_windows, int32_t *n_active);

/* Continuous batching on a context-owned host thread: requests submitted
 * at any time are admitted at window boundaries as memory frees up, and
 * retire when they finish.  pma_serve_stop waits for the thread.           */
pma_status pma_serve_start(pma_ctx *ctx);
pma_status pma_serve_stop(pma_ctx *ctx);

/* Admit queued requests now (allocate their device memory, upload their
 * tables and warm starts) without advancing them, so that a later pma_run
 * starts with every input resident in device memory.                     */
pma_status pma_admit(pma_ctx *ctx);

/* Non-blocking completion test (*done = 1 when finished). */
pma_status pma_poll(pma_ctx *ctx, uint64_t req_id, int32_t *done);

/* Block until the request finishes or timeout_us elapses (< 0: forever);
 * PMA_ERR_TIMEOUT on expiry, otherwise the request's final status.        */
pma_status pma_wait(pma_ctx *ctx, uint64_t req_id, int64_t timeout_us);

/* Combined mesh of a finished request into caller-owned HOST memory:
 * x_out dim*N doubles (component-major), psi_out optional N doubles
 * (combined Psi), info optional.  Combination is owner-takes: each global
 * node takes grad_h Psi from the subdomain whose core holds it.  Releases
 * the request.  Returns the request's final status (PMA_OK,
 * PMA_NOT_CONVERGED or PMA_ERR_TANGLED) or an error.                        */
pma_status pma_get_mesh(pma_ctx *ctx, uint64_t req_id, double *x_out, double *psi_out,
                        pma_info *info);

/* Same into caller-owned DEVICE memory on the context's stream, without a
 * host copy and without releasing: x_dev holds dim*N values of type double
 * (out_fp64 = 1) or float (0); psi_dev optional N values of the same type.
 * The copy is complete when the context's stream reaches it.              */
pma_status pma_get_mesh_device(pma_ctx *ctx, uint64_t req_id, void *x_dev, int32_t out_fp64,
                               void *psi_dev, pma_info *info);

/* Batched form of pma_get_mesh_device: one combine launch for n finished
 * requests; x_dev[i] receives request ids[i]'s mesh (dim_i * N_i values).  */
pma_status pma_get_mesh_device_batch(pma_ctx *ctx, int32_t n, const uint64_t *ids,
                                     void *const *x_dev, int32_t out_fp64);

/* Batched pma_get_mesh into ONE caller-owned HOST buffer: the meshes of the
 * n finished requests ids[0..n-1] are packed back to back in that order,
 * request i's dim_i * N_i doubles (component-major) starting right after
 * request i-1's.  Into page-locked memory (cudaHostAlloc, cudaHostRegister)
 * one combination launch writes the meshes directly through the buffer's
 * device mapping; into pageable memory one combination launch into a
 * device staging buffer and one device-to-host copy.  infos (optional) receives n
 * records.  Releases the requests.  Errors (nothing is released):
 * PMA_ERR_NOT_FOUND (unknown id), PMA_ERR_BUSY (a request not finished or
 * without a mesh), PMA_ERR_INVALID (NULL buffers, an id listed twice),
 * PMA_ERR_CUDA.  Per-request outcomes are in infos[i].status.              */
pma_status pma_get_mesh_batch(pma_ctx *ctx, int32_t n, const uint64_t *ids, double *x_out,
                              pma_info *infos);

/* FP64 positivity check of a finished request: recomputes det D_h^2 Psi in
 * FP64 at every global node (Sylvester minors of the symmetric FD Hessian)
 * and the signed measure of every mesh cell (2 triangles per quad in both
 * diagonal splits; 6 tetrahedra per hexahedron).  out[0] = min det,
 * out[1] = min leading minor, out[2] = min cell measure, out[3] = number of
 * non-positive cells.                                                     */
pma_status pma_check_mesh(pma_ctx *ctx, uint64_t req_id, double *out4);

/* Outcome so far of a request without releasing it (status PMA_PENDING
 * while it runs). */
pma_status pma_get_info(pma_ctx *ctx, uint64_t req_id, pma_info *info);

/* Drop a request (finished or not) and free its device memory. */
pma_status pma_release(pma_ctx *ctx, uint64_t req_id);

/* Number of requests queued, admitted and finished-but-unreleased. */
pma_status pma_counts(pma_ctx *ctx, int32_t *queued, int32_t *active, int32_t *finished);

/* Counters of the context since creation or the last reset.
 * sweep_launches counts the sweep kernels (band or resident), other_launches
 * the per-problem finish and the combination kernels.  window_ms is
 * the device time of the stepping windows, measured with CUDA events on
 * the context's stream around the sweep launches only; node_updates counts
 * subdomain nodes advanced by one step; sweep_bytes is the algorithmic HBM
 * traffic of those updates (band kernels: one read and one write of v per
 * node and step; resident path: one read and one write of v per node and
 * window); h2d/d2h_bytes are the host<->device copies the context issued;
 * res_launches and res_node_updates are the resident path's share of
 * sweep_launches and node_updates.                                        */
typedef struct {
  int64_t windows;
  int64_t sweep_launches;
  int64_t other_launches;
  int64_t node_updates;
  double sweep_bytes;
  double window_ms;
  double h2d_bytes;
  double d2h_bytes;
  int64_t res_launches;
  int64_t res_node_updates;
  double sweep_kernel_ms;         /* PMA_OPT_TIME_SWEEPS: device time of the sweeps
                                     of the timed (step, class) pairs            */
  int64_t sweep_kernel_launches;  /* and the number of timed (step, class) pairs   */
  double admit_ms;                /* host wall time of admission passes            */
  double rebuild_ms;              /* host wall time of table rebuilds              */
  double combine_ms;              /* host wall time of pma_get_mesh_batch calls    */
  int64_t sweep_steps;            /* (step, kernel class) pairs the band sweeps ran;
                                     sweep_bytes / sweep_steps = bytes per step   */
} pma_stats;
pma_status pma_get_stats(pma_ctx *ctx, pma_stats *out, int32_t reset);

/* ------------------------------------------------------------ one shot */

/* Synchronous convenience on device `device` (its own context and stream):
 * submit, run to completion and copy the mesh to host x_out (dim*N doubles).
 * Returns the request's final status.                                     */
pma_status pma_solve(int device, const pma_grid *grid, const pma_monitor *monitor,
                     const pma_decomp *decomp, const pma_params *params, const double *psi0,
                     double *x_out, double *psi_out, pma_info *info);

/* Allocation-free solve (the paper has no counterpart: this is a service
 * for callers that must not allocate device memory).  Some programs cannot
 * call cudaMalloc at this point: a host application that reserved the whole
 * device for its own memory pool up front, a framework whose caching
 * allocator owns every byte it hands out, or latency-critical code that may
 * not risk the device-wide synchronisation an allocation or a free can
 * cause.  This call runs one request to completion on the current device
 * using only a fixed scratch area that lives inside this library
 * (PMA_STATIC_SCRATCH_BYTES per GPU, reserved when the library is loaded on
 * a device and held until the process exits); it calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   grid, monitor, decomp, params  the request (host structs, as pma_submit)
 *   psi0_dev   optional warm start, DEVICE memory, N doubles (NULL: Psi^0 =
 *              |xi|^2/2)
 *   x_dev      output, DEVICE memory, dim*N doubles, component-major
 *   info       optional, host
 *   cuda_stream  stream to run on (NULL: the legacy default stream); the
 *              call returns after the stream has finished its work.
 * Requests whose state, tables and records do not fit the scratch area are
 * rejected with PMA_ERR_NOMEM (pma_last_error gives the bytes needed).  Both
 * transmission forms and every exchange_every are accepted.  Every call
 * shares the same scratch area: calls that overlap on the GPU (two streams,
 * two host threads, or a call racing a previous call still in flight on
 * another stream) corrupt each other.  Each call looks up the scratch area's
 * device address on the current device (so a device reset between calls
 * is harmless); the first call on a device also loads the library's device
 * code there, so make the first call on each device before any stream
 * capture begins.
 * Returns the request's final status (PMA_OK, PMA_NOT_CONVERGED,
 * PMA_ERR_TANGLED) or an error.                                             */
#define PMA_STATIC_SCRATCH_BYTES (32u << 20)
pma_status pma_solve_static(const pma_grid *grid, const pma_monitor *monitor,
                            const pma_decomp *decomp, const pma_params *params,
                            const double *psi0_dev, double *x_dev, pma_info *info,
                            void *cuda_stream);

/* ------------------------------------------------------------ misc */
const char *pma_status_str(int32_t status);
/* Last CUDA / validation error text of this thread (never NULL). */
const char *pma_last_error(void);
int32_t pma_abi_version(void);
/* Host-only consistency checks of the library's device tables (neighbour
 * entries of the transmission gathers against the owner of each node by
 * the decomposition's core boundaries, transmission-row/column flags of the
 * staged 2D bands, exact tiling and shared-memory / TMA limits of the work
 * items of every compiled shape) on built-in decompositions.  Touches no
 * device.  Returns the number of failed checks (0 = pass); the first
 * failure is described by pma_last_error.                                */
int32_t pma_selftest_tables(void);

#ifdef __cplusplus
}
#endif
#endif /* PMA_H */
