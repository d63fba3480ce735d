/*
 * pma_oracle.c -- FP64 CPU oracle of the (DD) parabolic Monge-Ampere mesh
 * generator.  TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke test
 * and the CPU-baseline leg of the benchmark, never by the product path.
 *
 * The state is the deviation potential v = Psi - |xi|^2/2 (Psi of Eq. (pmae));
 * the flow and every operator below are written for v, which is the same
 * PDE: grad Psi = xi + grad v and D^2 Psi = I + D^2 v.
 *
 * One forward-Euler step (Sect. 4.4) of the parallel DD method
 * (Eq. (transmission_condition3)), in the order the method states it:
 *   1. on every subdomain, at every node that is not a transmission
 *      (Dirichlet) node, the centred differences of Eqs. (pmae1d)/(pmae2d):
 *      x = grad_h Psi, H = D_h^2 Psi, det H, rho(x), G = log(rho det H);
 *      Neumann faces use the mirror ghost v_{-1} = v_1, the centred form of
 *      Eq. (nbd) (grad Psi . n = xi . n  <=>  dv/dn = 0);
 *   2. normalisation: theta = sum over global nodes of w rho det H taken on
 *      the owning subdomain, c = log(theta/|Omega_c|) -- the discrete form of
 *      the normalised density of Eq. (edp);
 *   3. v^{n+1} = v^n + dt (G - c) at updated nodes;
 *   4. transmission nodes take the owner's v^n (parallel form) or, for an
 *      owner that precedes the subdomain, its v^{n+1} (Algorithm 1), at
 *      every exchange step (every step, or every K-th with the interface
 *      data frozen in between);
 *   5. residual per subdomain and the stop rule (Algorithm 1, steps 5-6;
 *      Eq. (dd_stop_criterion)).
 */
#include "pma_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Monitor functions                                                        */
/* ------------------------------------------------------------------------ */

static double sech2(double z) {
  double c = cosh(z);
  return 1.0 / (c * c);
}

/* One additive term of a SUM monitor, or one factor term of a PRODUCT. */
static double term_value(const or_term *t, int dim, const double *x) {
  double q = 0.0;
  int a;
  switch (t->type) {
    case OR_TERM_BUMP:
      for (a = 0; a < dim; ++a) q += (x[a] - t->c[a]) * (x[a] - t->c[a]);
      return t->amp * exp(-t->width * q);
    case OR_TERM_RING: {
      double s;
      for (a = 0; a < dim; ++a) q += (x[a] - t->c[a]) * (x[a] - t->c[a]);
      s = q - t->r2;
      return t->amp * exp(-t->width * s * s);
    }
    case OR_TERM_SINE: {
      double s = x[t->axis] - t->c[t->axis] - t->a * sin(2.0 * OR_PI * t->k * x[t->along]);
      return t->amp * exp(-t->width * s * s);
    }
    case OR_TERM_BUMP1: {
      double s = x[t->axis] - t->c[t->axis];
      return t->amp * exp(-t->width * s * s);
    }
  }
  return NAN;
}

/* grad u of the test functions of Sect. 4 (Eqs. test_fn1, test_fn2,
 * test_fn3d1, test_fn3d2), differentiated by hand; rho = sqrt(1+|grad u|^2)
 * is Eq. (monitfn).                                                        */
static double arclen_rho(const or_monitor *m, const double *x) {
  double gu[3] = {0.0, 0.0, 0.0};
  switch (m->kind) {
    case OR_MON_ARCLEN_BURGERS: {
      /* u = 1/(1+exp(s)), s = (x+y-1)/(2 eps): du/ds = -sech^2(s/2)/4 */
      double eps = m->p0;
      double s = (x[0] + x[1] - 1.0) / (2.0 * eps);
      double d = -0.25 * sech2(0.5 * s) / (2.0 * eps);
      gu[0] = d;
      gu[1] = d;
      break;
    }
    case OR_MON_ARCLEN_SPIRAL: {
      /* u = 1 + 9/(1+q), q = 100 r^2 cos^2(phi), phi = theta - 20 r^2,
       * d = x - (0.7, 0.5), r^2 = |d|^2, r^2 grad theta = (-d_y, d_x).     */
      double dx = x[0] - 0.7, dy = x[1] - 0.5;
      double r2 = dx * dx + dy * dy;
      double phi = atan2(dy, dx) - 20.0 * r2;
      double cphi = cos(phi), s2phi = sin(2.0 * phi);
      double q = 100.0 * r2 * cphi * cphi;
      /* grad q = 100 [2 cos^2(phi) d - sin(2 phi) (r^2 grad theta - 40 r^2 d)] */
      double gqx = 100.0 * (2.0 * cphi * cphi * dx - s2phi * (-dy - 40.0 * r2 * dx));
      double gqy = 100.0 * (2.0 * cphi * cphi * dy - s2phi * (dx - 40.0 * r2 * dy));
      double f = -9.0 / ((1.0 + q) * (1.0 + q));
      gu[0] = f * gqx;
      gu[1] = f * gqy;
      break;
    }
    case OR_MON_ARCLEN_TANH_SPHERE: {
      /* u = tanh(100 (|x|^2 - 0.125)) */
      double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
      double f = 200.0 * sech2(100.0 * (r2 - 0.125));
      gu[0] = f * x[0];
      gu[1] = f * x[1];
      gu[2] = f * x[2];
      break;
    }
    case OR_MON_ARCLEN_NINE_SPHERES: {
      /* u = sum_k tanh(50 (|x - x_k|^2 - 0.1875)), centres as printed */
      static const double cx[9] = {0, 0.5, 0.5, -0.5, -0.5, 0.5, 0.5, -0.5, -0.5};
      static const double cy[9] = {0, 0.5, -0.5, 0.5, -0.5, 0.5, -0.5, 0.5, -0.5};
      static const double cz[9] = {0, 0.5, 0.5, 0.5, 0.5, -0.5, -0.5, -0.5, -0.5};
      int k;
      for (k = 0; k < 9; ++k) {
        double ex = x[0] - cx[k], ey = x[1] - cy[k], ez = x[2] - cz[k];
        double f = 100.0 * sech2(50.0 * (ex * ex + ey * ey + ez * ez - 0.1875));
        gu[0] += f * ex;
        gu[1] += f * ey;
        gu[2] += f * ez;
      }
      break;
    }
    default:
      return NAN;
  }
  return sqrt(1.0 + gu[0] * gu[0] + gu[1] * gu[1] + gu[2] * gu[2]);
}

/* Multilinear interpolation of a tabulated density: along each axis the
 * point is clamped to [tlo, thi], located in its table cell (the last cell
 * on the upper face) and weighted by its fractional position; the 2^dim
 * corner values are combined with the product weights.                     */
static double table_rho(const or_monitor *m, int dim, const double *x) {
  long base[3] = {0, 0, 0};
  double frac[3] = {0.0, 0.0, 0.0};
  long stride[3];
  double r = 0.0;
  int a, corner;
  stride[0] = 1;
  stride[1] = m->tn[0];
  stride[2] = (long)m->tn[0] * m->tn[1];
  for (a = 0; a < dim; ++a) {
    const double h = (m->thi[a] - m->tlo[a]) / (double)(m->tn[a] - 1);
    double s = (x[a] - m->tlo[a]) / h;
    long k;
    if (s < 0.0) s = 0.0;
    if (s > (double)(m->tn[a] - 1)) s = (double)(m->tn[a] - 1);
    k = (long)floor(s);
    if (k > m->tn[a] - 2) k = m->tn[a] - 2;
    base[a] = k;
    frac[a] = s - (double)k;
  }
  for (corner = 0; corner < (1 << dim); ++corner) {
    double w = 1.0;
    long idx = 0;
    for (a = 0; a < dim; ++a) {
      const int up = (corner >> a) & 1;
      w *= up ? frac[a] : 1.0 - frac[a];
      idx += (base[a] + up) * stride[a];
    }
    r += w * m->table[idx];
  }
  return r;
}

static double rho_at(const or_monitor *m, int dim, const double *x) {
  int t;
  if (m->kind == OR_MON_TABLE) return table_rho(m, dim, x);
  if (m->kind == OR_MON_SUM) {
    double r = m->base;
    for (t = 0; t < m->nterms; ++t) r += term_value(&m->term[t], dim, x);
    return r;
  }
  if (m->kind == OR_MON_PRODUCT) {
    double r = 1.0;
    for (t = 0; t < m->nterms; ++t) r *= m->base + term_value(&m->term[t], dim, x);
    return r;
  }
  return arclen_rho(m, x);
}

int or_monitor_eval(const or_monitor *m, int dim, const double *x, long npts,
                    double *rho_out) {
  long i;
  if (!m || !x || !rho_out || dim < 1 || dim > 3) return OR_ERR_INVALID;
  for (i = 0; i < npts; ++i) rho_out[i] = rho_at(m, dim, x + i * dim);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Decomposition (Sect. 3: overlapping slabs / blocks)                      */
/* ------------------------------------------------------------------------ */

/* Core partition b_k = round(k N / p); part k spans
 * [b_k - floor(o/2), b_{k+1} - 1 + ceil(o/2)] clipped to the grid, so two
 * neighbours share exactly o node indices.  The owned core is
 * [b_k, b_{k+1} - 1].                                                      */
int or_extents(long n, int parts, int overlap, long *lo, long *hi, long *clo,
               long *chi) {
  int k;
  long ol = overlap / 2, oh = overlap - overlap / 2;
  if (n < 3 || parts < 1 || parts > OR_MAX_PARTS) return OR_ERR_INVALID;
  if (parts > 1 && overlap < 2) return OR_ERR_INVALID;
  for (k = 0; k < parts; ++k) {
    long b0 = (2 * (long)k * n + parts) / (2 * parts);
    long b1 = (2 * (long)(k + 1) * n + parts) / (2 * parts);
    clo[k] = b0;
    chi[k] = b1 - 1;
    lo[k] = (k == 0) ? 0 : b0 - ol;
    hi[k] = (k == parts - 1) ? n - 1 : b1 - 1 + oh;
    if (parts > 1 && (b1 - b0) < oh + 1) return OR_ERR_INVALID;
    if (hi[k] - lo[k] + 1 < 3) return OR_ERR_INVALID;
  }
  return OR_OK;
}

typedef struct {
  long lo[3], hi[3], clo[3], chi[3], n[3], size;
  int k[3];
  int phys_lo[3], phys_hi[3];
  double *v, *vn, *G, *D, *R;
  unsigned char *upd;
} sub_t;

typedef struct {
  int dim;
  long N[3];
  double lo[3], h[3];
  double vol;
  int parts[3], nsub;
  long plo[3][OR_MAX_PARTS], phi[3][OR_MAX_PARTS];
  long pclo[3][OR_MAX_PARTS], pchi[3][OR_MAX_PARTS];
  sub_t *sub;
} dd_t;

static long sidx(const sub_t *s, long i, long j, long l) {
  return (l * s->n[1] + j) * s->n[0] + i;
}

/* Mirror ghost across a Neumann face: index -1 -> 1, n -> n - 2. */
static long mirror(long i, long n) {
  if (i < 0) return -i;
  if (i >= n) return 2 * (n - 1) - i;
  return i;
}

static double vget(const sub_t *s, const double *v, long i, long j, long l) {
  return v[sidx(s, mirror(i, s->n[0]), mirror(j, s->n[1]), mirror(l, s->n[2]))];
}

/* Trapezoid weight of global index gi on axis a. */
static double tw(const dd_t *d, int a, long gi) {
  return (gi == 0 || gi == d->N[a] - 1) ? 0.5 * d->h[a] : d->h[a];
}

static double det_sym(int dim, double H[3][3]) {
  if (dim == 1) return H[0][0];
  if (dim == 2) return H[0][0] * H[1][1] - H[0][1] * H[1][0];
  return H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
         H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
         H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
}

/* Centred FD gradient and Hessian of Psi at local node (i,j,l)
 * (Eqs. pmae1d/pmae2d), mesh point x = grad_h Psi (Eq. AdpMesh).          */
static void node_op(const dd_t *d, const sub_t *s, const double *v, long i,
                    long j, long l, double *x, double H[3][3]) {
  long c[3] = {i, j, l};
  int a, b;
  double vc = vget(s, v, i, j, l);
  for (a = 0; a < 3; ++a)
    for (b = 0; b < 3; ++b) H[a][b] = 0.0;
  for (a = 0; a < d->dim; ++a) {
    long p[3] = {i, j, l}, q[3] = {i, j, l};
    double vp, vm, xi;
    p[a] += 1;
    q[a] -= 1;
    vp = vget(s, v, p[0], p[1], p[2]);
    vm = vget(s, v, q[0], q[1], q[2]);
    xi = d->lo[a] + (double)(s->lo[a] + c[a]) * d->h[a];
    x[a] = xi + (vp - vm) / (2.0 * d->h[a]);
    H[a][a] = 1.0 + (vp - 2.0 * vc + vm) / (d->h[a] * d->h[a]);
  }
  for (a = 0; a < d->dim; ++a)
    for (b = a + 1; b < d->dim; ++b) {
      long pp[3] = {i, j, l}, pm[3] = {i, j, l}, mp[3] = {i, j, l}, mm[3] = {i, j, l};
      double hab;
      pp[a] += 1; pp[b] += 1;
      pm[a] += 1; pm[b] -= 1;
      mp[a] -= 1; mp[b] += 1;
      mm[a] -= 1; mm[b] -= 1;
      hab = (vget(s, v, pp[0], pp[1], pp[2]) - vget(s, v, pm[0], pm[1], pm[2]) -
             vget(s, v, mp[0], mp[1], mp[2]) + vget(s, v, mm[0], mm[1], mm[2])) /
            (4.0 * d->h[a] * d->h[b]);
      H[a][b] = hab;
      H[b][a] = hab;
    }
}

static void dd_free(dd_t *d) {
  int s;
  if (!d->sub) return;
  for (s = 0; s < d->nsub; ++s) {
    free(d->sub[s].v);
    free(d->sub[s].vn);
    free(d->sub[s].G);
    free(d->sub[s].D);
    free(d->sub[s].R);
    free(d->sub[s].upd);
  }
  free(d->sub);
  d->sub = NULL;
}

static int dd_build(dd_t *d, const or_grid *g, const or_decomp *dd) {
  int a, s, kx, ky, kz;
  memset(d, 0, sizeof(*d));
  if (!g || g->dim < 1 || g->dim > 3) return OR_ERR_INVALID;
  d->dim = g->dim;
  d->vol = 1.0;
  for (a = 0; a < 3; ++a) {
    int parts = (dd && a < g->dim) ? dd->parts[a] : 1;
    int ov = dd ? dd->overlap : 0;
    if (a >= g->dim) {
      d->N[a] = 1;
      d->lo[a] = 0.0;
      d->h[a] = 1.0;
      d->parts[a] = 1;
      d->plo[a][0] = d->phi[a][0] = d->pclo[a][0] = d->pchi[a][0] = 0;
      continue;
    }
    if (g->n[a] < 3 || !(g->hi[a] > g->lo[a])) return OR_ERR_INVALID;
    if (parts < 1) parts = 1;
    d->N[a] = g->n[a];
    d->lo[a] = g->lo[a];
    d->h[a] = (g->hi[a] - g->lo[a]) / (double)(g->n[a] - 1);
    d->vol *= g->hi[a] - g->lo[a];
    d->parts[a] = parts;
    if (or_extents(g->n[a], parts, ov, d->plo[a], d->phi[a], d->pclo[a], d->pchi[a]) != OR_OK)
      return OR_ERR_INVALID;
  }
  d->nsub = d->parts[0] * d->parts[1] * d->parts[2];
  d->sub = (sub_t *)calloc((size_t)d->nsub, sizeof(sub_t));
  if (!d->sub) return OR_ERR_NOMEM;
  s = 0;
  for (kz = 0; kz < d->parts[2]; ++kz)
    for (ky = 0; ky < d->parts[1]; ++ky)
      for (kx = 0; kx < d->parts[0]; ++kx, ++s) {
        sub_t *u = &d->sub[s];
        int kk[3] = {kx, ky, kz};
        long i, j, l;
        for (a = 0; a < 3; ++a) {
          u->k[a] = kk[a];
          u->lo[a] = d->plo[a][kk[a]];
          u->hi[a] = d->phi[a][kk[a]];
          u->clo[a] = d->pclo[a][kk[a]];
          u->chi[a] = d->pchi[a][kk[a]];
          u->n[a] = u->hi[a] - u->lo[a] + 1;
          u->phys_lo[a] = (kk[a] == 0);
          u->phys_hi[a] = (kk[a] == d->parts[a] - 1);
        }
        u->size = u->n[0] * u->n[1] * u->n[2];
        u->v = (double *)calloc((size_t)u->size, sizeof(double));
        u->vn = (double *)calloc((size_t)u->size, sizeof(double));
        u->G = (double *)calloc((size_t)u->size, sizeof(double));
        u->D = (double *)calloc((size_t)u->size, sizeof(double));
        u->R = (double *)calloc((size_t)u->size, sizeof(double));
        u->upd = (unsigned char *)calloc((size_t)u->size, 1);
        if (!u->v || !u->vn || !u->G || !u->D || !u->R || !u->upd) return OR_ERR_NOMEM;
        for (l = 0; l < u->n[2]; ++l)
          for (j = 0; j < u->n[1]; ++j)
            for (i = 0; i < u->n[0]; ++i) {
              long c[3] = {i, j, l};
              int dir = 0;
              for (a = 0; a < d->dim; ++a) {
                if (c[a] == 0 && !u->phys_lo[a]) dir = 1;
                if (c[a] == u->n[a] - 1 && !u->phys_hi[a]) dir = 1;
              }
              u->upd[sidx(u, i, j, l)] = (unsigned char)(!dir);
            }
      }
  return OR_OK;
}

/* Subdomain that owns global node gidx (the one whose core contains it). */
static int owner_of(const dd_t *d, const long *gidx) {
  int a, kk[3] = {0, 0, 0};
  for (a = 0; a < 3; ++a) {
    int k;
    for (k = 0; k < d->parts[a]; ++k)
      if (gidx[a] >= d->pclo[a][k] && gidx[a] <= d->pchi[a][k]) {
        kk[a] = k;
        break;
      }
  }
  return (kk[2] * d->parts[1] + kk[1]) * d->parts[0] + kk[0];
}

static int is_owned(const sub_t *s, int dim, const long *gidx) {
  int a;
  for (a = 0; a < dim; ++a)
    if (gidx[a] < s->clo[a] || gidx[a] > s->chi[a]) return 0;
  return 1;
}

/* Combined output (owner-takes): x_g = grad_h Psi of the owning subdomain,
 * and optionally det D_h^2 Psi from the same (owner's) stencil.            */
static void dd_output(const dd_t *d, int use_new, double *x_out, double *psi_out,
                      double *det_out) {
  long gi, gj, gl;
  long Ntot = d->N[0] * d->N[1] * d->N[2];
  for (gl = 0; gl < d->N[2]; ++gl)
    for (gj = 0; gj < d->N[1]; ++gj)
      for (gi = 0; gi < d->N[0]; ++gi) {
        long gidx[3] = {gi, gj, gl};
        long gflat = (gl * d->N[1] + gj) * d->N[0] + gi;
        int o = owner_of(d, gidx);
        const sub_t *s = &d->sub[o];
        const double *v = use_new ? s->vn : s->v;
        long i = gi - s->lo[0], j = gj - s->lo[1], l = gl - s->lo[2];
        double x[3], H[3][3];
        int a;
        node_op(d, s, v, i, j, l, x, H);
        if (x_out)
          for (a = 0; a < d->dim; ++a) x_out[a * Ntot + gflat] = x[a];
        if (det_out) det_out[gflat] = det_sym(d->dim, H);
        if (psi_out) {
          double q = 0.0;
          for (a = 0; a < d->dim; ++a) {
            double xi = d->lo[a] + (double)gidx[a] * d->h[a];
            q += 0.5 * xi * xi;
          }
          psi_out[gflat] = v[sidx(s, i, j, l)] + q;
        }
      }
}

int or_solve(const or_grid *g, const or_monitor *m, const or_decomp *ddp,
             const or_params *p, const double *psi0, double *x_out,
             double *psi_out, double *res_hist, or_info *info) {
  return or_solve_det(g, m, ddp, p, psi0, x_out, psi_out, NULL, res_hist, info);
}

int or_solve_det(const or_grid *g, const or_monitor *m, const or_decomp *ddp,
                 const or_params *p, const double *psi0, double *x_out,
                 double *psi_out, double *det_out, double *res_hist, or_info *info) {
  dd_t d;
  or_decomp one = {{1, 1, 1}, 0, 0, 1};
  int rc, s, status = OR_NOT_CONVERGED, a;
  long n, steps = 0;
  double theta = 0.0, theta_prev = 0.0, last_res = INFINITY, min_det_last = INFINITY;
  int check_every, exchange_every, exchange;

  if (!g || !m || !p || !x_out) return OR_ERR_INVALID;
  if (!(p->dt > 0.0) || p->max_steps < 0) return OR_ERR_INVALID;
  if (!ddp) ddp = &one;
  rc = dd_build(&d, g, ddp);
  if (rc != OR_OK) {
    dd_free(&d);
    return rc;
  }
  check_every = p->check_every > 0 ? p->check_every : 1;
  if (ddp->exchange_every < 0) {
    dd_free(&d);
    return OR_ERR_INVALID;
  }
  exchange_every = ddp->exchange_every > 0 ? ddp->exchange_every : 1;

  /* Eq. (incond): Psi^0 = |xi|^2/2, i.e. v^0 = 0; or the warm start of
   * Sect. 2 (previous steady state) restricted to every subdomain.        */
  for (s = 0; s < d.nsub; ++s) {
    sub_t *u = &d.sub[s];
    long i, j, l;
    for (l = 0; l < u->n[2]; ++l)
      for (j = 0; j < u->n[1]; ++j)
        for (i = 0; i < u->n[0]; ++i) {
          double val = 0.0;
          if (psi0) {
            long gidx[3] = {u->lo[0] + i, u->lo[1] + j, u->lo[2] + l};
            long gflat = (gidx[2] * d.N[1] + gidx[1]) * d.N[0] + gidx[0];
            double q = 0.0;
            for (a = 0; a < d.dim; ++a) {
              double xi = d.lo[a] + (double)gidx[a] * d.h[a];
              q += 0.5 * xi * xi;
            }
            val = psi0[gflat] - q;
          }
          u->v[sidx(u, i, j, l)] = val;
        }
  }

  for (n = 0; n < p->max_steps; ++n) {
    int tangled = 0;
    double min_det = INFINITY, c = 0.0, rmax = 0.0, rmin = INFINITY;

    /* 1. operator at every updated node, theta over owned nodes */
    theta = 0.0;
    for (s = 0; s < d.nsub; ++s) {
      sub_t *u = &d.sub[s];
      long i, j, l;
      for (l = 0; l < u->n[2]; ++l)
        for (j = 0; j < u->n[1]; ++j)
          for (i = 0; i < u->n[0]; ++i) {
            long k = sidx(u, i, j, l);
            long gidx[3] = {u->lo[0] + i, u->lo[1] + j, u->lo[2] + l};
            double x[3], H[3][3], D, rho;
            if (!u->upd[k]) continue;
            node_op(&d, u, u->v, i, j, l, x, H);
            D = det_sym(d.dim, H);
            rho = rho_at(m, d.dim, x);
            u->D[k] = D;
            u->R[k] = rho;
            if (D < min_det) min_det = D;
            if (!(D > 0.0) || !isfinite(rho) || !isfinite(D)) tangled = 1;
            if (is_owned(u, d.dim, gidx)) {
              double w = 1.0;
              for (a = 0; a < d.dim; ++a) w *= tw(&d, a, gidx[a]);
              theta += w * rho * D;
            }
          }
    }
    if (tangled || !isfinite(theta)) {
      status = OR_ERR_TANGLED;
      min_det_last = min_det;
      break;
    }

    /* 2. normalisation constant (Eq. edp, normalised density) */
    if (n == 0) theta_prev = theta;
    if (p->normalize == OR_NORM_GLOBAL_THETA) c = log(theta / d.vol);

    /* 3. forward Euler at updated nodes, with the residual pieces */
    for (s = 0; s < d.nsub; ++s) {
      sub_t *u = &d.sub[s];
      long i, j, l;
      double rs = 0.0;
      for (l = 0; l < u->n[2]; ++l)
        for (j = 0; j < u->n[1]; ++j)
          for (i = 0; i < u->n[0]; ++i) {
            long k = sidx(u, i, j, l);
            long c3[3] = {i, j, l};
            double F;
            if (!u->upd[k]) continue;
            if (p->rhs == OR_RHS_LOG) {
              /* Eq. (pmae): log(|Omega_c| rho det D^2 Psi), rho/theta normalised */
              F = log(u->R[k] * u->D[k]) - c;
            } else {
              /* root form: (|Omega_c| rho det / theta)^(1/d) - 1 */
              double th = (p->lag_theta ? theta_prev : theta);
              double sc = (p->normalize == OR_NORM_GLOBAL_THETA) ? d.vol / th : 1.0;
              F = pow(sc * u->R[k] * u->D[k], 1.0 / (double)d.dim) - 1.0;
            }
            u->G[k] = F;
            u->vn[k] = u->v[k] + p->dt * F;
            if (p->stop_norm == OR_STOP_MAX_UT) {
              if (fabs(F) > rs) rs = fabs(F);
            } else {
              double w = 1.0, inc = u->vn[k] - u->v[k];
              for (a = 0; a < d.dim; ++a)
                w *= (c3[a] == 0 || c3[a] == u->n[a] - 1) ? 0.5 * d.h[a] : d.h[a];
              rs += w * inc * inc;
            }
          }
      if (p->stop_norm == OR_STOP_L2_INCREMENT) rs = sqrt(rs);
      if (rs > rmax) rmax = rs;
      if (rs < rmin) rmin = rs;
    }
    theta_prev = theta;

    /* 4. transmission (Dirichlet) nodes from their owner at an exchange
     * step; between exchanges they keep the data of the last exchange    */
    exchange = (n % exchange_every) == 0;
    for (s = 0; s < d.nsub; ++s) {
      sub_t *u = &d.sub[s];
      long i, j, l;
      for (l = 0; l < u->n[2]; ++l)
        for (j = 0; j < u->n[1]; ++j)
          for (i = 0; i < u->n[0]; ++i) {
            long k = sidx(u, i, j, l);
            long gidx[3] = {u->lo[0] + i, u->lo[1] + j, u->lo[2] + l};
            int o;
            const sub_t *w;
            long ko;
            if (u->upd[k]) continue;
            if (!exchange) {
              u->vn[k] = u->v[k];
              continue;
            }
            o = owner_of(&d, gidx);
            w = &d.sub[o];
            ko = sidx(w, gidx[0] - w->lo[0], gidx[1] - w->lo[1], gidx[2] - w->lo[2]);
            u->vn[k] = (ddp->alternating && o < s) ? w->vn[ko] : w->v[ko];
          }
    }

    /* 5. residual and stop rule */
    /* ALL: every subdomain below TOL (max); ANY: Algorithm 1 step 6 (min) */
    last_res = (p->stop_rule == OR_RULE_ANY) ? rmin : rmax;
    if (res_hist) res_hist[n] = last_res;
    min_det_last = min_det;
    for (s = 0; s < d.nsub; ++s) {
      double *t = d.sub[s].v;
      d.sub[s].v = d.sub[s].vn;
      d.sub[s].vn = t;
    }
    steps = n + 1;
    if ((steps % check_every) == 0 && last_res <= p->tol) {
      status = OR_OK;
      break;
    }
  }

  dd_output(&d, 0, x_out, psi_out, det_out);
  if (info) {
    info->steps = steps;
    info->residual = last_res;
    info->theta = theta;
    info->min_det = min_det_last;
    info->status = status;
  }
  dd_free(&d);
  return status;
}

int or_operator(const or_grid *g, const or_monitor *m, const double *v,
                double *x_out, double *det_out, double *rho_out, double *G_out) {
  dd_t d;
  int rc;
  long i, j, l, Ntot;
  sub_t *u;
  if (!g || !m || !v) return OR_ERR_INVALID;
  rc = dd_build(&d, g, NULL);
  if (rc != OR_OK) {
    dd_free(&d);
    return rc;
  }
  u = &d.sub[0];
  memcpy(u->v, v, (size_t)u->size * sizeof(double));
  Ntot = u->size;
  for (l = 0; l < u->n[2]; ++l)
    for (j = 0; j < u->n[1]; ++j)
      for (i = 0; i < u->n[0]; ++i) {
        long k = sidx(u, i, j, l);
        double x[3], H[3][3], D, rho;
        int a;
        node_op(&d, u, u->v, i, j, l, x, H);
        D = det_sym(d.dim, H);
        rho = rho_at(m, d.dim, x);
        if (x_out)
          for (a = 0; a < d.dim; ++a) x_out[a * Ntot + k] = x[a];
        if (det_out) det_out[k] = D;
        if (rho_out) rho_out[k] = rho;
        if (G_out) G_out[k] = log(rho * D);
      }
  dd_free(&d);
  return OR_OK;
}

/* Signed measure of a simplex given by its vertices (dim+1 points). */
static double simplex_measure(int dim, const double P[4][3]) {
  if (dim == 1) return P[1][0] - P[0][0];
  if (dim == 2)
    return 0.5 * ((P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) -
                  (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]));
  {
    double A[3][3];
    int r, c;
    for (r = 0; r < 3; ++r)
      for (c = 0; c < 3; ++c) A[r][c] = P[r + 1][c] - P[0][c];
    return (A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
            A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
            A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0])) / 6.0;
  }
}

int or_quality(const or_grid *g, const or_monitor *m, const double *psi,
               double *out) {
  dd_t d;
  int rc, a;
  long i, j, l, Ntot;
  sub_t *u;
  double theta = 0.0, sw = 0.0, swe2 = 0.0, emax = 0.0, min_det = INFINITY;
  double min_cell = INFINITY;
  double *X;
  if (!g || !m || !psi || !out) return OR_ERR_INVALID;
  rc = dd_build(&d, g, NULL);
  if (rc != OR_OK) {
    dd_free(&d);
    return rc;
  }
  u = &d.sub[0];
  Ntot = u->size;
  X = (double *)malloc((size_t)(3 * Ntot) * sizeof(double));
  if (!X) {
    dd_free(&d);
    return OR_ERR_NOMEM;
  }
  for (l = 0; l < u->n[2]; ++l)
    for (j = 0; j < u->n[1]; ++j)
      for (i = 0; i < u->n[0]; ++i) {
        long c3[3] = {i, j, l};
        double q = 0.0;
        for (a = 0; a < d.dim; ++a) {
          double xi = d.lo[a] + (double)c3[a] * d.h[a];
          q += 0.5 * xi * xi;
        }
        u->v[sidx(u, i, j, l)] = psi[sidx(u, i, j, l)] - q;
      }
  for (l = 0; l < u->n[2]; ++l)
    for (j = 0; j < u->n[1]; ++j)
      for (i = 0; i < u->n[0]; ++i) {
        long k = sidx(u, i, j, l);
        long c3[3] = {i, j, l};
        double x[3] = {0, 0, 0}, H[3][3], D, rho, w = 1.0;
        node_op(&d, u, u->v, i, j, l, x, H);
        D = det_sym(d.dim, H);
        rho = rho_at(m, d.dim, x);
        u->D[k] = D;
        u->R[k] = rho;
        for (a = 0; a < 3; ++a) X[a * Ntot + k] = x[a];
        for (a = 0; a < d.dim; ++a) w *= tw(&d, a, c3[a]);
        theta += w * rho * D;
        if (D < min_det) min_det = D;
      }
  for (l = 0; l < u->n[2]; ++l)
    for (j = 0; j < u->n[1]; ++j)
      for (i = 0; i < u->n[0]; ++i) {
        long k = sidx(u, i, j, l);
        long c3[3] = {i, j, l};
        double w = 1.0, E = d.vol * u->R[k] * u->D[k] / theta;
        for (a = 0; a < d.dim; ++a) w *= tw(&d, a, c3[a]);
        sw += w;
        swe2 += w * E * E;
        if (E > emax) emax = E;
      }
  /* cell measures */
  {
    long ci, cj, cl;
    long nc[3] = {u->n[0] - 1, d.dim > 1 ? u->n[1] - 1 : 1, d.dim > 2 ? u->n[2] - 1 : 1};
    for (cl = 0; cl < nc[2]; ++cl)
      for (cj = 0; cj < nc[1]; ++cj)
        for (ci = 0; ci < nc[0]; ++ci) {
          double P[4][3];
          if (d.dim == 1) {
            P[0][0] = X[sidx(u, ci, 0, 0)];
            P[1][0] = X[sidx(u, ci + 1, 0, 0)];
            double mu = simplex_measure(1, P);
            if (mu < min_cell) min_cell = mu;
          } else if (d.dim == 2) {
            /* quad corners 00,10,11,01 split along both diagonals */
            long k00 = sidx(u, ci, cj, 0), k10 = sidx(u, ci + 1, cj, 0);
            long k11 = sidx(u, ci + 1, cj + 1, 0), k01 = sidx(u, ci, cj + 1, 0);
            long tri[4][3] = {{k00, k10, k11}, {k00, k11, k01}, {k00, k10, k01}, {k10, k11, k01}};
            int t, vtx;
            for (t = 0; t < 4; ++t) {
              double mu;
              for (vtx = 0; vtx < 3; ++vtx) {
                P[vtx][0] = X[0 * Ntot + tri[t][vtx]];
                P[vtx][1] = X[1 * Ntot + tri[t][vtx]];
              }
              mu = simplex_measure(2, P);
              if (mu < min_cell) min_cell = mu;
            }
          } else {
            /* hex split into 6 tets along the 000-111 diagonal, one per
             * axis permutation, sign-corrected by the permutation parity   */
            static const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1},
                                           {1, 0, 2}, {0, 2, 1}, {2, 1, 0}};
            static const double sgn[6] = {1, 1, 1, -1, -1, -1};
            int t, vtx, b;
            for (t = 0; t < 6; ++t) {
              long off[3] = {0, 0, 0};
              double mu;
              for (vtx = 0; vtx < 4; ++vtx) {
                long k;
                if (vtx > 0) off[perm[t][vtx - 1]] = 1;
                k = sidx(u, ci + off[0], cj + off[1], cl + off[2]);
                for (b = 0; b < 3; ++b) P[vtx][b] = X[b * Ntot + k];
              }
              mu = sgn[t] * simplex_measure(3, P);
              if (mu < min_cell) min_cell = mu;
            }
          }
        }
  }
  out[0] = sqrt(swe2 / sw);
  out[1] = emax;
  out[2] = min_det;
  out[3] = min_cell;
  out[4] = theta;
  free(X);
  dd_free(&d);
  return OR_OK;
}
