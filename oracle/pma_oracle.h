/*
 * pma_oracle.h -- FP64 CPU oracle of the (domain-decomposition) parabolic
 * Monge-Ampere mesh generator of Sulman, Nguyen, Haynes & Huang
 * ("Domain Decomposition Parabolic Monge-Ampere Approach for Fast Generation
 * of Adaptive Moving Meshes").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path.  Only
 * the test suite, the package smoke test and the CPU-baseline leg of the
 * benchmark may load it; the product path never does.  It shares no code,
 * header, table or constant with the CUDA library: every definition below is
 * restated here from the paper on its own.
 *
 * Everything is plain double precision, single threaded, straightforward
 * loops in the order the paper states the method:
 *   Sect. 2, Eq. (pmae)/(incond)/(nbd)       the PMA flow, its initial and
 *                                             Neumann boundary conditions
 *   Sect. 3, Eqs. (pmae1d)/(pmae2d)           centred finite differences
 *   Sect. 3, Algorithm 1 and Eq.
 *            (transmission_condition3)       alternating / parallel DD
 *   Sect. 2, Eq. (dd_stop_criterion)          stopping rule
 *   Sect. 4.4, forward Euler in pseudo time  the time integrator
 *   Sect. 4.5, Eq. (quality_measure)          mesh quality E_adp
 */
#ifndef PMA_ORACLE_H
#define PMA_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_TERMS 4
#define OR_MAX_PARTS 32

/* Status codes (same meaning as the library's, defined independently). */
enum { OR_OK = 0, OR_NOT_CONVERGED = 1, OR_ERR_INVALID = -1, OR_ERR_NOMEM = -2,
       OR_ERR_TANGLED = -3 };

/* Box Omega_c = prod [lo_a, hi_a] with n_a nodes per axis (n_a >= 3). */
typedef struct {
  int dim;
  long n[3];
  double lo[3], hi[3];
} or_grid;

/* Monitor density rho(x).  Term shapes (x in physical coordinates):
 *   BUMP : amp * exp(-width * |x - c|^2)
 *   RING : amp * exp(-width * (|x - c|^2 - r2)^2)
 *   SINE : amp * exp(-width * (x[axis] - c[axis] - a*sin(2*pi*k*x[along]))^2)
 *   BUMP1: amp * exp(-width * (x[axis] - c[axis])^2)      (one axis only)
 * Monitor kinds:
 *   SUM     : rho = base + sum_t term_t(x)
 *   PRODUCT : rho = prod_t (base + term_t(x)), each term a BUMP1
 *   ARCLEN_*: rho = sqrt(1 + |grad u(x)|^2), Eq. (monitfn), with u the test
 *             functions of Sect. 4: BURGERS Eq. (test_fn1) (eps = p0),
 *             SPIRAL Eq. (test_fn2), TANH_SPHERE Eq. (test_fn3d1),
 *             NINE_SPHERES Eq. (test_fn3d2).
 *   TABLE   : rho given at the nodes of a uniform grid of tn[a] >= 2 points
 *             on [tlo[a], thi[a]] per axis (x fastest), as a solution
 *             computed on a physical mesh would be sampled (Sect. 2, the
 *             moving-mesh loop); evaluated by multilinear interpolation,
 *             the point first clamped to the table's box.                  */
enum { OR_TERM_BUMP = 0, OR_TERM_RING = 1, OR_TERM_SINE = 2, OR_TERM_BUMP1 = 3 };
enum { OR_MON_SUM = 0, OR_MON_PRODUCT = 1, OR_MON_ARCLEN_BURGERS = 2,
       OR_MON_ARCLEN_SPIRAL = 3, OR_MON_ARCLEN_TANH_SPHERE = 4,
       OR_MON_ARCLEN_NINE_SPHERES = 5, OR_MON_TABLE = 6 };

typedef struct {
  int type;
  int axis, along;
  double amp, width, r2, a, k;
  double c[3];
} or_term;

typedef struct {
  int kind;
  int nterms;
  double base;
  double p0;
  or_term term[OR_MAX_TERMS];
  const double *table; /* TABLE: tn[0] * tn[1] * tn[2] values, x fastest  */
  int tn[3];           /* TABLE: points per axis (1 on axes >= dim)      */
  double tlo[3], thi[3];
} or_monitor;

/* Overlapping decomposition (Sect. 3): parts[a] subdomains along axis a,
 * neighbours share `overlap` node indices.  alternating = 0 is the parallel
 * (Jacobi) transmission of Eq. (transmission_condition3); 1 is Algorithm 1,
 * where a subdomain takes the new value of an owner that precedes it.
 * exchange_every = K >= 1 (0 reads as 1): the interface data are exchanged
 * at steps n = 0, K, 2K, ... only and stay frozen in between, the way the
 * paper integrates each subdomain over an interval Delta tau with the
 * neighbours' data of the interval's start (Sect. 3, the ode113 paragraph
 * after Algorithm 1).  K = 1 is one exchange per step.                     */
typedef struct {
  int parts[3];
  int overlap;
  int alternating;
  int exchange_every;
} or_decomp;

enum { OR_STOP_MAX_UT = 0, OR_STOP_L2_INCREMENT = 1 };
enum { OR_RULE_ALL = 0, OR_RULE_ANY = 1 };
enum { OR_RHS_LOG = 0, OR_RHS_ROOT = 1 };
enum { OR_NORM_GLOBAL_THETA = 0, OR_NORM_NONE = 1 };

typedef struct {
  double dt, tol;
  long max_steps;
  int stop_norm;
  int stop_rule;
  int check_every;
  int rhs;
  int normalize;
  int lag_theta;   /* ROOT only: use theta of the previous step (0 = exact) */
} or_params;

typedef struct {
  long steps;
  double residual;
  double theta;
  double min_det;
  int status;
} or_info;

/* Full solve.  psi0: optional warm start on the global grid (Sect. 2, the
 * previous steady state), NULL for Eq. (incond).  x_out: dim * N values,
 * component-major, x fastest.  psi_out (optional): combined Psi.  res_hist
 * (optional): residual of every step, max_steps entries.                   */
int or_solve(const or_grid *g, const or_monitor *m, const or_decomp *dd,
             const or_params *p, const double *psi0, double *x_out,
             double *psi_out, double *res_hist, or_info *info);

/* or_solve, and det_out (optional, N values): det D_h^2 Psi at every global
 * node from the stencil of the node's owner, the stencil the combined mesh
 * is taken from.                                                          */
int or_solve_det(const or_grid *g, const or_monitor *m, const or_decomp *dd,
                 const or_params *p, const double *psi0, double *x_out,
                 double *psi_out, double *det_out, double *res_hist, or_info *info);

/* rho at npts points x (point-major, dim values each). */
int or_monitor_eval(const or_monitor *m, int dim, const double *x, long npts,
                    double *rho_out);

/* Single-domain operator at every node of the global grid for the
 * deviation potential v = Psi - |xi|^2/2 (Neumann ghost mirror at all faces):
 * mesh point (dim*N, component-major), det of the FD Hessian, rho and
 * G = log(rho * det).                                                        */
int or_operator(const or_grid *g, const or_monitor *m, const double *v,
                double *x_out, double *det_out, double *rho_out, double *G_out);

/* Subdomain extents along one axis: lo/hi (inclusive global indices) and the
 * owned core [clo, chi] of every part.                                       */
int or_extents(long n, int parts, int overlap, long *lo, long *hi, long *clo,
               long *chi);

/* Mesh quality of Eq. (quality_measure) on a combined global Psi:
 * E = |Omega_c| rho(grad_h Psi) det D_h^2 Psi / theta, theta = sum w rho det.
 * out[0] = E_2 = (sum w E^2 / sum w)^(1/2), out[1] = E_max, out[2] = min det,
 * out[3] = min signed cell measure (2D: both triangle splits; 3D: 6 tets),
 * out[4] = theta.                                                           */
int or_quality(const or_grid *g, const or_monitor *m, const double *psi,
               double *out);

#ifdef __cplusplus
}
#endif
#endif
