/*
 * Seeded synthetic geometry for the cut-cell Poisson method: exact-to-rounding
 * integrals over cut cells, grid faces and embedded-boundary (EB) patches.
 *
 * This file is an INPUT GENERATOR shared by the FP64 oracle and the GPU path.
 * It holds none of the discretisation's arithmetic (no stencils, no least
 * squares, no operator): it only integrates given functions over the pieces of
 * a Cartesian grid cut by circles (2D) or spheres (3D).  The paper takes these
 * moments from a separate geometry generator (Sec. 2.1, the volume/face/normal
 * moment definitions; Sec. 3.1 asks for O(h^{6+D}) accurate moments); here they
 * are computed to rounding level by iterated Gauss-Kronrod quadrature.
 *
 * Method (per element, in cell-normalised coordinates xi = (x - centre)/h, the
 * element being [-1/2,1/2]^D):
 *   - 2D cells and 3D faces: a square cut by one circle.  Outer integral in u
 *     by adaptive 15-point Gauss-Kronrod, split at every u where the piece
 *     structure changes (circle tangents and circle/edge crossings), with the
 *     substitution u = a + (b-a) sin^2(pi s / 2) which turns the square-root
 *     behaviour at circle tangents into an analytic integrand.  Inner integral
 *     in v is closed form (antiderivatives of the integrand's v factor).
 *   - 3D cells: a height direction k is chosen (largest |normal component|);
 *     the k-integral of the integrand's k factor over the fluid part of the
 *     vertical line is closed form; the remaining (u,v) integral uses the same
 *     square machinery with adaptive inner quadrature, split at the circles
 *     where the sphere crosses the cell's top and bottom faces.
 *   - 3D EB patches: the sphere as a graph t(u,v) over the same square, area
 *     element R/|t - C_k|, split at the same circles.
 *   - 2D EB arcs: the circle parametrised by angle, split where it crosses
 *     the cell's edges.
 * Integrands are products f(x) = prod_d g_d(x_d) of 1-D functions (powers of
 * (x_d - o_d)/h, or sin(w x_d + th) and its derivative), optionally times a
 * component of the EB normal that points out of the fluid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GEO_OK 0
#define GEO_ERR_MULTIBODY 1
#define GEO_ERR_ARG 2

#define MAXFN 16
#define MAXT 512

typedef struct {
  int dim;
  int n[3];
  double h;
  int inside;          /* 1: fluid inside the single body; 0: fluid outside all bodies */
  int nbody;
  const double* center; /* [nbody][3], physical */
  const double* radius; /* [nbody] */
} geo_t;

/* 1-D function families per dimension. kind 0: ((x - o)/h)^p with o = pow_center
 * (NaN -> element centre); kind 1: amp*sin(w x + th); kind 2: amp*w*cos(w x + th). */
typedef struct {
  int nfn[3];
  int kind[3][MAXFN];
  int pw[3][MAXFN];
  double pow_center[3];
  double w[3], th[3], amp[3];
} basis_t;

/* ---------------------------------------------------------------- 1-D basis */

typedef struct {
  const basis_t* b;
  double ec[3];   /* element centre (physical) */
  double h;
  double o[3];    /* power centre offset, normalised */
} bctx_t;

static void bctx_init(bctx_t* c, const basis_t* b, const double ec[3], double h) {
  c->b = b;
  c->h = h;
  for (int d = 0; d < 3; ++d) {
    c->ec[d] = ec[d];
    c->o[d] = isnan(b->pow_center[d]) ? 0.0 : (b->pow_center[d] - ec[d]) / h;
  }
}

static void fn_eval(const bctx_t* c, int d, double xi, double* v) {
  const basis_t* b = c->b;
  double x = c->ec[d] + c->h * xi;
  double t = xi - c->o[d];
  for (int i = 0; i < b->nfn[d]; ++i) {
    switch (b->kind[d][i]) {
      case 0: {
        double r = 1.0;
        for (int p = 0; p < b->pw[d][i]; ++p) r *= t;
        v[i] = r;
      } break;
      case 1: v[i] = b->amp[d] * sin(b->w[d] * x + b->th[d]); break;
      default: v[i] = b->amp[d] * b->w[d] * cos(b->w[d] * x + b->th[d]); break;
    }
  }
}

/* antiderivative with respect to xi */
static void fn_anti(const bctx_t* c, int d, double xi, double* v) {
  const basis_t* b = c->b;
  double x = c->ec[d] + c->h * xi;
  double t = xi - c->o[d];
  for (int i = 0; i < b->nfn[d]; ++i) {
    double w = b->w[d];
    switch (b->kind[d][i]) {
      case 0: {
        int p = b->pw[d][i];
        double r = t;
        for (int q = 0; q < p; ++q) r *= t;
        v[i] = r / (p + 1);
      } break;
      case 1:
        if (w == 0.0) v[i] = b->amp[d] * sin(b->th[d]) * xi;
        else v[i] = -b->amp[d] * cos(w * x + b->th[d]) / (w * c->h);
        break;
      default:
        if (w == 0.0) v[i] = 0.0;
        else v[i] = b->amp[d] * sin(w * x + b->th[d]) / c->h;
        break;
    }
  }
}

/* ---------------------------------------------------------- Gauss-Kronrod 15 */

static const double XGK[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                              0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                              0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                              0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double WGK[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                              0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                              0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                              0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double WG[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                             0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

typedef void (*vfun_t)(void* ctx, double x, double* out);

#define GEO_RTOL 1e-13
#define GEO_ATOL 2e-16
#define GEO_MAXDEPTH 40

/* Adaptive GK15 of a vector integrand over [a,b] with the sin^2 substitution
 * x = a + (b-a) sin^2(pi s/2), s in [0,1].  res[0..nt) += integral. */
static void adapt_sub(vfun_t f, void* ctx, double a, double b, int nt, double* res) {
  if (!(b > a)) return;
  double stk_s0[2 * GEO_MAXDEPTH + 4], stk_s1[2 * GEO_MAXDEPTH + 4];
  int stk_d[2 * GEO_MAXDEPTH + 4];
  int sp = 0;
  stk_s0[0] = 0.0; stk_s1[0] = 1.0; stk_d[0] = 0; sp = 1;
  double fk[MAXT], gk[MAXT], tmp[MAXT];
  const double HP = 1.5707963267948966192;
  while (sp > 0) {
    --sp;
    double s0 = stk_s0[sp], s1 = stk_s1[sp];
    int dep = stk_d[sp];
    double sc = 0.5 * (s0 + s1), hl = 0.5 * (s1 - s0);
    for (int i = 0; i < nt; ++i) { fk[i] = 0.0; gk[i] = 0.0; }
    for (int j = 0; j < 15; ++j) {
      int idx = j < 8 ? j : 14 - j;
      double xs = j < 8 ? -XGK[idx] : XGK[idx];
      double s = sc + hl * xs;
      double sn = sin(HP * s);
      double x = a + (b - a) * sn * sn;
      double jac = (b - a) * HP * sin(2.0 * HP * s);
      f(ctx, x, tmp);
      double wk = WGK[idx] * jac * hl;
      double wg = (idx & 1) ? WG[idx >> 1] * jac * hl : 0.0;
      for (int i = 0; i < nt; ++i) { fk[i] += wk * tmp[i]; gk[i] += wg * tmp[i]; }
    }
    /* QUADPACK-style acceptance: |K - G| is a pessimistic bound on the K15
     * error (which behaves like (|K-G|)^{3/2}); differences at the rounding
     * level of the panel's absolute sum count as converged. */
    double err = 0.0, mag = 0.0;
    for (int i = 0; i < nt; ++i) {
      double e = fabs(fk[i] - gk[i]);
      if (e > err) err = e;
      if (fabs(fk[i]) > mag) mag = fabs(fk[i]);
    }
    /* QUADPACK's scaling of |K-G| into an estimate of the K15 error */
    if (mag > 0.0) {
      double r = 200.0 * err / mag;
      err = r < 1.0 ? mag * r * sqrt(r) : err;
    }
    double tol = GEO_RTOL * mag + GEO_ATOL * 2.0 * hl;
    if (err <= tol || dep >= GEO_MAXDEPTH || sp + 2 >= 2 * GEO_MAXDEPTH + 4) {
      for (int i = 0; i < nt; ++i) res[i] += fk[i];
    } else {
      stk_s0[sp] = sc; stk_s1[sp] = s1; stk_d[sp] = dep + 1; ++sp;
      stk_s0[sp] = s0; stk_s1[sp] = sc; stk_d[sp] = dep + 1; ++sp;
    }
  }
}

/* test hook: one GK15 panel of x^k on [0,1] (no substitution); kronrod or gauss */
double geo_gk15_panel_pow(int k, int gauss) {
  double s = 0.0;
  for (int j = 0; j < 15; ++j) {
    int idx = j < 8 ? j : 14 - j;
    double xs = j < 8 ? -XGK[idx] : XGK[idx];
    double x = 0.5 + 0.5 * xs;
    double w = gauss ? ((idx & 1) ? WG[idx >> 1] : 0.0) : WGK[idx];
    s += 0.5 * w * pow(x, k);
  }
  return s;
}

/* ------------------------------------------------------------- small sorts */

static int sort_unique(double* p, int n) {
  for (int i = 1; i < n; ++i) {
    double v = p[i];
    int j = i - 1;
    while (j >= 0 && p[j] > v) { p[j + 1] = p[j]; --j; }
    p[j + 1] = v;
  }
  int m = 0;
  for (int i = 0; i < n; ++i) {
    if (m == 0 || p[i] - p[m - 1] > 1e-15) p[m++] = p[i];
  }
  return m;
}

/* critical u for the square [-1/2,1/2]^2 and circles centred (cu,cv) */
static int crit_u(double cu, double cv, const double* R, int nR, double* pts) {
  int m = 0;
  pts[m++] = -0.5;
  pts[m++] = 0.5;
  for (int j = 0; j < nR; ++j) {
    double r = R[j];
    if (!(r > 0)) continue;
    double c[2] = {cu - r, cu + r};
    for (int q = 0; q < 2; ++q)
      if (c[q] > -0.5 && c[q] < 0.5) pts[m++] = c[q];
    for (int e = 0; e < 2; ++e) {
      double dv = (e ? 0.5 : -0.5) - cv;
      if (fabs(dv) < r) {
        double s = sqrt(r * r - dv * dv);
        if (cu - s > -0.5 && cu - s < 0.5) pts[m++] = cu - s;
        if (cu + s > -0.5 && cu + s < 0.5) pts[m++] = cu + s;
      }
    }
  }
  return sort_unique(pts, m);
}

static int crit_v(double u, double cu, double cv, const double* R, int nR, double* pts) {
  int m = 0;
  pts[m++] = -0.5;
  pts[m++] = 0.5;
  for (int j = 0; j < nR; ++j) {
    double r = R[j];
    if (!(r > 0)) continue;
    double du = u - cu;
    if (fabs(du) < r) {
      double s = sqrt(r * r - du * du);
      if (cv - s > -0.5 && cv - s < 0.5) pts[m++] = cv - s;
      if (cv + s > -0.5 && cv + s < 0.5) pts[m++] = cv + s;
    }
  }
  return sort_unique(pts, m);
}

/* --------------------------------------------------------- term bookkeeping */

typedef struct {
  int nt;
  const int* terms; /* [nt][3] function index per physical dim */
} terms_t;

/* ------------------------------------------- square cut by one circle (2D) */
/* Region: [-1/2,1/2]^2 in (u,v) = physical dims (du,dv) intersected with the
 * outside (inside=0) or inside (inside=1) of the circle (cu,cv,R).  Integrand:
 * prod of the u and v factors times `fixed[d]` for the remaining dims (their
 * functions evaluated at a fixed coordinate, e.g. a face's normal coordinate). */
typedef struct {
  const bctx_t* bc;
  const terms_t* T;
  int du, dv, dfix;          /* dfix: fixed dim (3D faces) or -1 */
  double fixval[MAXFN];      /* values of fixed-dim functions */
  double cu, cv, R;
  int inside;
  int has_circle;
} sq_t;

static void sq_outer(void* vctx, double u, double* out) {
  sq_t* q = (sq_t*)vctx;
  const basis_t* b = q->bc->b;
  int nt = q->T->nt;
  double fu[MAXFN], Ga[MAXFN], Gb[MAXFN], acc[MAXFN];
  fn_eval(q->bc, q->du, u, fu);
  int nfv = b->nfn[q->dv];
  for (int i = 0; i < nfv; ++i) acc[i] = 0.0;
  double pts[8];
  int np;
  if (q->has_circle) np = crit_v(u, q->cu, q->cv, &q->R, 1, pts);
  else { pts[0] = -0.5; pts[1] = 0.5; np = 2; }
  for (int k = 0; k + 1 < np; ++k) {
    double va = pts[k], vb = pts[k + 1];
    int fluid = 1;
    if (q->has_circle) {
      double vm = 0.5 * (va + vb), du = u - q->cu, dv = vm - q->cv;
      int in = du * du + dv * dv < q->R * q->R;
      fluid = q->inside ? in : !in;
    }
    if (!fluid) continue;
    fn_anti(q->bc, q->dv, va, Ga);
    fn_anti(q->bc, q->dv, vb, Gb);
    for (int i = 0; i < nfv; ++i) acc[i] += Gb[i] - Ga[i];
  }
  for (int t = 0; t < nt; ++t) {
    const int* tt = q->T->terms + 3 * t;
    double v = fu[tt[q->du]] * acc[tt[q->dv]];
    if (q->dfix >= 0) v *= q->fixval[tt[q->dfix]];
    out[t] = v;
  }
}

static void sq_integrate(sq_t* q, double* res) {
  int nt = q->T->nt;
  for (int t = 0; t < nt; ++t) res[t] = 0.0;
  double pts[16];
  int np;
  if (q->has_circle) np = crit_u(q->cu, q->cv, &q->R, 1, pts);
  else { pts[0] = -0.5; pts[1] = 0.5; np = 2; }
  for (int k = 0; k + 1 < np; ++k) adapt_sub(sq_outer, q, pts[k], pts[k + 1], nt, res);
}

/* ---------------------------------------------------- 3D cell, sphere cut */

typedef struct {
  const bctx_t* bc;
  const terms_t* T;
  int du, dv, dk;
  double C[3];
  double R;
  int inside;
  int eb;        /* 0 volume, 1 EB patch */
  int ncomp;     /* EB: normal component (-1: none) */
  double Rc[3];  /* circle radii in the (u,v) plane */
  int nRc;
  double u;      /* current outer coordinate */
  double fu[MAXFN];
} cell3_t;

/* fluid t-intervals on the vertical line through (u,v) */
static int tset(const cell3_t* q, double u, double v, double* ta, double* tb) {
  double du = u - q->C[q->du], dv = v - q->C[q->dv];
  double rho2 = du * du + dv * dv, R2 = q->R * q->R;
  double ck = q->C[q->dk];
  if (rho2 >= R2) {
    if (q->inside) return 0;
    ta[0] = -0.5; tb[0] = 0.5;
    return 1;
  }
  double s = sqrt(R2 - rho2);
  double lo = ck - s, hi = ck + s;
  if (q->inside) {
    double a = lo > -0.5 ? lo : -0.5, b = hi < 0.5 ? hi : 0.5;
    if (b > a) { ta[0] = a; tb[0] = b; return 1; }
    return 0;
  }
  int m = 0;
  double a0 = -0.5, b0 = lo < 0.5 ? lo : 0.5;
  if (b0 > a0) { ta[m] = a0; tb[m] = b0; ++m; }
  double a1 = hi > -0.5 ? hi : -0.5, b1 = 0.5;
  if (b1 > a1) { ta[m] = a1; tb[m] = b1; ++m; }
  return m;
}

static void cell3_point(void* vctx, double v, double* out) {
  cell3_t* q = (cell3_t*)vctx;
  const basis_t* b = q->bc->b;
  int nt = q->T->nt;
  double u = q->u;
  const double* fu = q->fu;
  double fv[MAXFN];
  fn_eval(q->bc, q->dv, v, fv);
  if (!q->eb) {
    double ta[2], tb[2], Ga[MAXFN], Gb[MAXFN], acc[MAXFN];
    int nk = b->nfn[q->dk];
    for (int i = 0; i < nk; ++i) acc[i] = 0.0;
    int m = tset(q, u, v, ta, tb);
    for (int j = 0; j < m; ++j) {
      fn_anti(q->bc, q->dk, ta[j], Ga);
      fn_anti(q->bc, q->dk, tb[j], Gb);
      for (int i = 0; i < nk; ++i) acc[i] += Gb[i] - Ga[i];
    }
    for (int t = 0; t < nt; ++t) {
      const int* tt = q->T->terms + 3 * t;
      out[t] = fu[tt[q->du]] * fv[tt[q->dv]] * acc[tt[q->dk]];
    }
    return;
  }
  int nout = q->ncomp == -2 ? 4 * nt : nt;
  for (int t = 0; t < nout; ++t) out[t] = 0.0;
  double du = u - q->C[q->du], dv = v - q->C[q->dv];
  double rho2 = du * du + dv * dv, R2 = q->R * q->R;
  if (rho2 >= R2) return;
  double s = sqrt(R2 - rho2);
  for (int sg = -1; sg <= 1; sg += 2) {
    double t = q->C[q->dk] + sg * s;
    if (t < -0.5 || t > 0.5) continue;
    double fk[MAXFN];
    fn_eval(q->bc, q->dk, t, fk);
    double wgt = q->R / s;
    if (q->ncomp >= 0) {
      double xi[3];
      xi[q->du] = u; xi[q->dv] = v; xi[q->dk] = t;
      double nrm = (xi[q->ncomp] - q->C[q->ncomp]) / q->R;
      if (!q->inside) nrm = -nrm; /* outward from the fluid */
      wgt *= nrm;
    }
    if (q->ncomp == -2) {
      double xi[3];
      xi[q->du] = u; xi[q->dv] = v; xi[q->dk] = t;
      double nv[3];
      for (int d = 0; d < 3; ++d) nv[d] = (q->inside ? 1.0 : -1.0) * (xi[d] - q->C[d]) / q->R;
      for (int tt = 0; tt < nt; ++tt) {
        const int* ti = q->T->terms + 3 * tt;
        double f = wgt * fu[ti[q->du]] * fv[ti[q->dv]] * fk[ti[q->dk]];
        out[tt] += f;
        for (int d = 0; d < 3; ++d) out[(d + 1) * nt + tt] += f * nv[d];
      }
      continue;
    }
    for (int tt = 0; tt < nt; ++tt) {
      const int* ti = q->T->terms + 3 * tt;
      out[tt] += wgt * fu[ti[q->du]] * fv[ti[q->dv]] * fk[ti[q->dk]];
    }
  }
}

static void cell3_outer(void* vctx, double u, double* out) {
  cell3_t* q = (cell3_t*)vctx;
  int nt = (q->eb && q->ncomp == -2) ? 4 * q->T->nt : q->T->nt;
  for (int t = 0; t < nt; ++t) out[t] = 0.0;
  q->u = u;
  fn_eval(q->bc, q->du, u, q->fu);
  double pts[16];
  int np = crit_v(u, q->C[q->du], q->C[q->dv], q->Rc, q->nRc, pts);
  for (int k = 0; k + 1 < np; ++k) adapt_sub(cell3_point, q, pts[k], pts[k + 1], nt, out);
}

static int cell3_integrate(cell3_t* q, double* res) {
  int nt = (q->eb && q->ncomp == -2) ? 4 * q->T->nt : q->T->nt;
  for (int t = 0; t < nt; ++t) res[t] = 0.0;
  /* circles: sphere crossing t=-1/2, t=+1/2, and the silhouette */
  double ck = q->C[q->dk], R2 = q->R * q->R;
  q->nRc = 0;
  for (int e = 0; e < 2; ++e) {
    double dt = (e ? 0.5 : -0.5) - ck;
    if (R2 - dt * dt > 0) q->Rc[q->nRc++] = sqrt(R2 - dt * dt);
  }
  q->Rc[q->nRc++] = q->R;
  double pts[32];
  int np = crit_u(q->C[q->du], q->C[q->dv], q->Rc, q->nRc, pts);
  /* cell3_point evaluates at u stored in the context: keep it reentrant per cell */
  for (int k = 0; k + 1 < np; ++k) {
    cell3_t local = *q;
    adapt_sub(cell3_outer, &local, pts[k], pts[k + 1], nt, res);
  }
  return GEO_OK;
}

/* choose the height direction: largest |C_d| such that the silhouette circle
 * misses the (u,v) square */
static int pick_height(const double C[3], double R, int* dk) {
  int order[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (fabs(C[order[j]]) > fabs(C[order[i]])) { int t = order[i]; order[i] = order[j]; order[j] = t; }
  for (int i = 0; i < 3; ++i) {
    int k = order[i];
    int u = (k + 1) % 3, v = (k + 2) % 3;
    double fu = fabs(C[u]) + 0.5, fv = fabs(C[v]) + 0.5;
    if (fu * fu + fv * fv < R * R) { *dk = k; return GEO_OK; }
  }
  /* no direction keeps the silhouette out of the square: the quadrature still
   * splits at the silhouette circle, with the endpoint substitution removing
   * its square-root behaviour */
  *dk = order[0];
  return GEO_OK;
}

/* --------------------------------------------------------- 2D EB arc */

typedef struct {
  const bctx_t* bc;
  const terms_t* T;
  double C[2];
  double R;
  int inside;
  int ncomp;
} arc_t;

static void arc_point(void* vctx, double th, double* out) {
  arc_t* q = (arc_t*)vctx;
  double c = cos(th), s = sin(th);
  double u = q->C[0] + q->R * c, v = q->C[1] + q->R * s;
  double fu[MAXFN], fv[MAXFN];
  fn_eval(q->bc, 0, u, fu);
  fn_eval(q->bc, 1, v, fv);
  double wgt = q->R;
  double sg = q->inside ? 1.0 : -1.0;
  if (q->ncomp == -2) {
    int nt = q->T->nt;
    for (int t = 0; t < nt; ++t) {
      const int* tt = q->T->terms + 3 * t;
      double f = wgt * fu[tt[0]] * fv[tt[1]];
      out[t] = f;
      out[nt + t] = f * sg * c;
      out[2 * nt + t] = f * sg * s;
      out[3 * nt + t] = 0.0;
    }
    return;
  }
  if (q->ncomp >= 0) {
    double nrm = q->ncomp == 0 ? c : s;
    if (!q->inside) nrm = -nrm;
    wgt *= nrm;
  }
  for (int t = 0; t < q->T->nt; ++t) {
    const int* tt = q->T->terms + 3 * t;
    out[t] = wgt * fu[tt[0]] * fv[tt[1]];
  }
}

static void arc_integrate(arc_t* q, double* res) {
  int nt = q->ncomp == -2 ? 4 * q->T->nt : q->T->nt;
  for (int t = 0; t < nt; ++t) res[t] = 0.0;
  const double PI = 3.14159265358979323846;
  double pts[16];
  int m = 0;
  pts[m++] = -PI;
  pts[m++] = PI;
  for (int d = 0; d < 2; ++d)
    for (int e = 0; e < 2; ++e) {
      double w = ((e ? 0.5 : -0.5) - q->C[d]) / q->R;
      if (w > -1.0 && w < 1.0) {
        double a = d == 0 ? acos(w) : asin(w);
        if (d == 0) { pts[m++] = a; pts[m++] = -a; }
        else { pts[m++] = a; pts[m++] = (a >= 0 ? PI - a : -PI - a); }
      }
    }
  m = sort_unique(pts, m);
  for (int k = 0; k + 1 < m; ++k) {
    double tm = 0.5 * (pts[k] + pts[k + 1]);
    double u = q->C[0] + q->R * cos(tm), v = q->C[1] + q->R * sin(tm);
    if (u < -0.5 || u > 0.5 || v < -0.5 || v > 0.5) continue;
    adapt_sub(arc_point, q, pts[k], pts[k + 1], nt, res);
  }
}

/* --------------------------------------------------------- classification */

static void box_dist(const double* c, const double* lo, const double* hi, int dim, double* dmin, double* dmax) {
  double a = 0.0, b = 0.0;
  for (int d = 0; d < dim; ++d) {
    double q = c[d] < lo[d] ? lo[d] - c[d] : (c[d] > hi[d] ? c[d] - hi[d] : 0.0);
    a += q * q;
    double f = fabs(c[d] - lo[d]) > fabs(c[d] - hi[d]) ? fabs(c[d] - lo[d]) : fabs(c[d] - hi[d]);
    b += f * f;
  }
  *dmin = sqrt(a);
  *dmax = sqrt(b);
}

/* flag: 0 covered, 1 full, 2 cut; body index of the cutting body (or -1) */
static int classify_box(const geo_t* g, const double* lo, const double* hi, int8_t* flag, int32_t* body) {
  *body = -1;
  if (g->nbody == 0) { *flag = 1; return GEO_OK; }
  if (g->inside) {
    double dmin, dmax;
    box_dist(g->center, lo, hi, g->dim, &dmin, &dmax);
    double r = g->radius[0];
    if (dmax <= r) *flag = 1;
    else if (dmin >= r) *flag = 0;
    else { *flag = 2; *body = 0; }
    return GEO_OK;
  }
  int ncut = 0;
  *flag = 1;
  for (int b = 0; b < g->nbody; ++b) {
    double dmin, dmax;
    box_dist(g->center + 3 * b, lo, hi, g->dim, &dmin, &dmax);
    double r = g->radius[b];
    if (dmax <= r) { *flag = 0; *body = -1; return GEO_OK; }
    if (dmin < r) { ++ncut; *body = b; }
  }
  if (ncut > 1) return GEO_ERR_MULTIBODY;
  if (ncut == 1) *flag = 2;
  return GEO_OK;
}

static void cell_box(const geo_t* g, int64_t idx, double* lo, double* hi, double* ctr) {
  int64_t i[3] = {0, 0, 0};
  int64_t r = idx;
  for (int d = 0; d < g->dim; ++d) { i[d] = r % g->n[d]; r /= g->n[d]; }
  for (int d = 0; d < 3; ++d) {
    if (d < g->dim) {
      lo[d] = i[d] * g->h; hi[d] = (i[d] + 1) * g->h; ctr[d] = (i[d] + 0.5) * g->h;
    } else { lo[d] = hi[d] = ctr[d] = 0.0; }
  }
}

/* faces normal to d: index over (n_d+1) along d and n along the others */
static void face_box(const geo_t* g, int dir, int64_t idx, double* lo, double* hi, double* ctr) {
  int64_t i[3] = {0, 0, 0};
  int64_t r = idx;
  for (int d = 0; d < g->dim; ++d) {
    int64_t nd = g->n[d] + (d == dir);
    i[d] = r % nd; r /= nd;
  }
  for (int d = 0; d < 3; ++d) {
    if (d >= g->dim) { lo[d] = hi[d] = ctr[d] = 0.0; continue; }
    if (d == dir) { lo[d] = hi[d] = ctr[d] = i[d] * g->h; }
    else { lo[d] = i[d] * g->h; hi[d] = (i[d] + 1) * g->h; ctr[d] = (i[d] + 0.5) * g->h; }
  }
}

int geo_classify_cells(const geo_t* g, int8_t* flag, int32_t* body) {
  int64_t nc = 1;
  for (int d = 0; d < g->dim; ++d) nc *= g->n[d];
  int err = GEO_OK;
#pragma omp parallel for schedule(static) reduction(max : err)
  for (int64_t c = 0; c < nc; ++c) {
    double lo[3], hi[3], ctr[3];
    cell_box(g, c, lo, hi, ctr);
    int e = classify_box(g, lo, hi, flag + c, body + c);
    if (e > err) err = e;
  }
  return err;
}

int geo_classify_faces(const geo_t* g, int dir, int8_t* flag, int32_t* body) {
  int64_t nf = 1;
  for (int d = 0; d < g->dim; ++d) nf *= g->n[d] + (d == dir);
  int err = GEO_OK;
#pragma omp parallel for schedule(static) reduction(max : err)
  for (int64_t f = 0; f < nf; ++f) {
    double lo[3], hi[3], ctr[3];
    face_box(g, dir, f, lo, hi, ctr);
    int e = classify_box(g, lo, hi, flag + f, body + f);
    if (e > err) err = e;
  }
  return err;
}

/* ---------------------------------------------------------- integrations */

static void norm_body(const geo_t* g, int b, const double* ctr, double* C, double* R) {
  for (int d = 0; d < 3; ++d) C[d] = d < g->dim ? (g->center[3 * b + d] - ctr[d]) / g->h : 0.0;
  *R = g->radius[b] / g->h;
}

/* Integrals over the fluid part of cells, normalised by h^D.
 * cells[i]: linear cell index; body[i]: cutting body or -1 (full cell). */
int geo_cell_integrals(const geo_t* g, int64_t ncell, const int64_t* cells, const int32_t* body, const basis_t* b,
                       int nt, const int* terms, double* out) {
  if (nt > MAXT) return GEO_ERR_ARG;
  terms_t T = {nt, terms};
  int err = GEO_OK;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : err)
  for (int64_t i = 0; i < ncell; ++i) {
    double lo[3], hi[3], ctr[3];
    cell_box(g, cells[i], lo, hi, ctr);
    bctx_t bc;
    bctx_init(&bc, b, ctr, g->h);
    double* res = out + i * nt;
    int bd = body[i];
    if (g->dim == 1 || bd < 0) {
      /* full cell: product of 1-D integrals */
      double A[3][MAXFN], Ga[MAXFN], Gb[MAXFN];
      for (int d = 0; d < 3; ++d) {
        if (d >= g->dim) { for (int k = 0; k < MAXFN; ++k) A[d][k] = 1.0; continue; }
        fn_anti(&bc, d, -0.5, Ga);
        fn_anti(&bc, d, 0.5, Gb);
        for (int k = 0; k < b->nfn[d]; ++k) A[d][k] = Gb[k] - Ga[k];
      }
      for (int t = 0; t < nt; ++t) {
        const int* tt = terms + 3 * t;
        res[t] = A[0][tt[0]] * (g->dim > 1 ? A[1][tt[1]] : 1.0) * (g->dim > 2 ? A[2][tt[2]] : 1.0);
      }
      continue;
    }
    double C[3], R;
    norm_body(g, bd, ctr, C, &R);
    if (g->dim == 2) {
      sq_t q;
      q.bc = &bc; q.T = &T; q.du = 0; q.dv = 1; q.dfix = -1;
      q.cu = C[0]; q.cv = C[1]; q.R = R; q.inside = g->inside; q.has_circle = 1;
      sq_integrate(&q, res);
    } else {
      cell3_t q;
      memset(&q, 0, sizeof(q));
      q.bc = &bc; q.T = &T;
      int dk;
      int e = pick_height(C, R, &dk);
      if (e > err) err = e;
      q.dk = dk; q.du = (dk + 1) % 3; q.dv = (dk + 2) % 3;
      for (int d = 0; d < 3; ++d) q.C[d] = C[d];
      q.R = R; q.inside = g->inside; q.eb = 0; q.ncomp = -1;
      cell3_integrate(&q, res);
    }
  }
  return err;
}

/* Integrals over the fluid part of grid faces normal to `dir`, normalised by h^(D-1). */
int geo_face_integrals(const geo_t* g, int dir, int64_t nface, const int64_t* faces, const int32_t* body,
                       const basis_t* b, int nt, const int* terms, double* out) {
  if (nt > MAXT) return GEO_ERR_ARG;
  terms_t T = {nt, terms};
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nface; ++i) {
    double lo[3], hi[3], ctr[3];
    face_box(g, dir, faces[i], lo, hi, ctr);
    bctx_t bc;
    bctx_init(&bc, b, ctr, g->h);
    double* res = out + i * nt;
    double fix[MAXFN];
    fn_eval(&bc, dir, 0.0, fix);
    int bd = body[i];
    int others[2], no = 0;
    for (int d = 0; d < g->dim; ++d)
      if (d != dir) others[no++] = d;
    if (bd < 0 || g->dim == 1) {
      double A[3][MAXFN], Ga[MAXFN], Gb[MAXFN];
      for (int d = 0; d < 3; ++d) {
        if (d >= g->dim) { for (int k = 0; k < MAXFN; ++k) A[d][k] = 1.0; continue; }
        if (d == dir) { for (int k = 0; k < b->nfn[d]; ++k) A[d][k] = fix[k]; continue; }
        fn_anti(&bc, d, -0.5, Ga);
        fn_anti(&bc, d, 0.5, Gb);
        for (int k = 0; k < b->nfn[d]; ++k) A[d][k] = Gb[k] - Ga[k];
      }
      for (int t = 0; t < nt; ++t) {
        const int* tt = terms + 3 * t;
        res[t] = A[0][tt[0]] * (g->dim > 1 ? A[1][tt[1]] : 1.0) * (g->dim > 2 ? A[2][tt[2]] : 1.0);
      }
      continue;
    }
    double C[3], R;
    norm_body(g, bd, ctr, C, &R);
    double R2f = R * R - C[dir] * C[dir];
    if (g->dim == 2) {
      int v = others[0];
      double Ga[MAXFN], Gb[MAXFN], acc[MAXFN];
      for (int k = 0; k < b->nfn[v]; ++k) acc[k] = 0.0;
      double seg[4];
      int ns = 0;
      if (R2f > 0) {
        double rf = sqrt(R2f);
        double a = C[v] - rf, bb = C[v] + rf;
        if (g->inside) {
          double x0 = a > -0.5 ? a : -0.5, x1 = bb < 0.5 ? bb : 0.5;
          if (x1 > x0) { seg[0] = x0; seg[1] = x1; ns = 1; }
        } else {
          double x1 = a < 0.5 ? a : 0.5;
          if (x1 > -0.5) { seg[2 * ns] = -0.5; seg[2 * ns + 1] = x1; ++ns; }
          double x0 = bb > -0.5 ? bb : -0.5;
          if (0.5 > x0) { seg[2 * ns] = x0; seg[2 * ns + 1] = 0.5; ++ns; }
        }
      } else if (!g->inside) { seg[0] = -0.5; seg[1] = 0.5; ns = 1; }
      for (int s = 0; s < ns; ++s) {
        fn_anti(&bc, v, seg[2 * s], Ga);
        fn_anti(&bc, v, seg[2 * s + 1], Gb);
        for (int k = 0; k < b->nfn[v]; ++k) acc[k] += Gb[k] - Ga[k];
      }
      for (int t = 0; t < nt; ++t) {
        const int* tt = terms + 3 * t;
        res[t] = fix[tt[dir]] * acc[tt[v]];
      }
    } else {
      sq_t q;
      q.bc = &bc; q.T = &T; q.du = others[0]; q.dv = others[1]; q.dfix = dir;
      for (int k = 0; k < b->nfn[dir]; ++k) q.fixval[k] = fix[k];
      q.cu = C[others[0]]; q.cv = C[others[1]]; q.inside = g->inside;
      if (R2f > 0) { q.R = sqrt(R2f); q.has_circle = 1; }
      else { q.R = 0; q.has_circle = 0; }
      if (!q.has_circle && g->inside) { for (int t = 0; t < nt; ++t) res[t] = 0.0; continue; }
      sq_integrate(&q, res);
    }
  }
  return GEO_OK;
}

/* Integrals over the EB patch of cut cells, normalised by h^(D-1); ncomp >= 0
 * multiplies by that component of the unit normal pointing out of the fluid. */
int geo_eb_integrals(const geo_t* g, int64_t ncell, const int64_t* cells, const int32_t* body, const basis_t* b,
                     int ncomp, int nt, const int* terms, double* out) {
  if ((ncomp == -2 ? 4 * nt : nt) > MAXT) return GEO_ERR_ARG;
  terms_t T = {nt, terms};
  int err = GEO_OK;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : err)
  for (int64_t i = 0; i < ncell; ++i) {
    double lo[3], hi[3], ctr[3];
    cell_box(g, cells[i], lo, hi, ctr);
    bctx_t bc;
    bctx_init(&bc, b, ctr, g->h);
    int nout = ncomp == -2 ? 4 * nt : nt;
    double* res = out + i * nout;
    int bd = body[i];
    if (bd < 0 || g->dim == 1) { for (int t = 0; t < nout; ++t) res[t] = 0.0; continue; }
    double C[3], R;
    norm_body(g, bd, ctr, C, &R);
    if (g->dim == 2) {
      arc_t q;
      q.bc = &bc; q.T = &T; q.C[0] = C[0]; q.C[1] = C[1]; q.R = R; q.inside = g->inside; q.ncomp = ncomp;
      arc_integrate(&q, res);
    } else {
      cell3_t q;
      memset(&q, 0, sizeof(q));
      q.bc = &bc; q.T = &T;
      int dk;
      int e = pick_height(C, R, &dk);
      if (e > err) err = e;
      q.dk = dk; q.du = (dk + 1) % 3; q.dv = (dk + 2) % 3;
      for (int d = 0; d < 3; ++d) q.C[d] = C[d];
      q.R = R; q.inside = g->inside; q.eb = 1; q.ncomp = ncomp;
      cell3_integrate(&q, res);
    }
  }
  return err;
}

int geo_abi_version(void) { return 1; }
