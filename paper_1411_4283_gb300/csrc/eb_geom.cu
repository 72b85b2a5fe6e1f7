// Moment tables of cut-cell geometries computed on the device (Sec. 2.1): the
// volume moments m^p_v, the face moments m^p_f of the grid faces and the
// moments of the EB patch (plain and weighted by each normal component) that
// the least squares of Sec. 2.2.1 consume.  Sec. 3.1 asks for moments accurate
// to O(h^{6+D}); these are exact to rounding.
//
// Geometry: the unit square minus circles (or the inside of one circle).  A
// cell (or face) box is covered when one disk contains it, full when no circle
// reaches into it, and cut by the one circle that crosses it (two circles in
// one box are refused, EB_ERR_MULTIVALUED).  Moments are in h-scaled
// coordinates about the cell or face centre and divided by h^D (volumes) or
// h^(D-1) (faces, EB patches), graded monomial order (eb.h).
//   face moments    the fluid part of a face is the face segment minus (or, for
//                   the inside of a circle, intersected with) the chord inside
//                   the circle: integrals of t^q in closed form;
//   EB moments      the arcs of the circle inside the cell (angles from the
//                   intersections with the cell edges), Gauss-Legendre in the
//                   angle on pieces of at most pi/4: the integrand is a
//                   trigonometric polynomial of low degree, integrated to
//                   rounding; the normal points out of the fluid;
//   volume moments  the divergence theorem, int_V xi^p = 1/(p_d+1) oint
//                   xi^(p+e_d) n_d, in the direction d most tangent to the
//                   boundary in the cell (so that a thin sliver is not the small
//                   difference of terms of size one): the fluid parts of the two
//                   edges normal to d in closed form and the arcs.
// Cells whose volume fraction is at most 1e-14 count as covered and those at
// least 1 - 1e-14 as full, faces likewise; a face next to a covered cell is
// closed.  The lists of cut cells and cut faces are ascending.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "eb_internal.cuh"
#include "eb_scan.cuh"

struct eb_geometry {
  eb_geom desc;
  std::vector<void*> allocs;  // device arrays the descriptor points into
  // the shape parameters and, per cell and per face, the body whose boundary cuts it (-1: none); the
  // moment tables' shape derivatives are recomputed from these
  int n_body = 0, inside = 0;
  double centers[64][3] = {};
  double radii[64] = {};
  int32_t* cell_body = nullptr;     // [ncell]
  int32_t* face_body[3] = {nullptr, nullptr, nullptr};
};

namespace eb {

constexpr int GEO_MAXB = 64;     // bodies
constexpr int GEO_GL = 20;       // Gauss-Legendre points per arc piece
constexpr int GEO_MAXQ = 6;      // moment degree
constexpr double GEO_EPS = 1e-14;

struct Circles {
  int n, inside;
  double c[GEO_MAXB][2];
  double r[GEO_MAXB];
};

template <int NG>
struct GlRuleN {
  double x[NG], w[NG];  // nodes and weights on [-1, 1]
};
using GlRule = GlRuleN<GEO_GL>;
constexpr int GEO_GLT = 48;  // sin^2-mapped panels in the polar angle and along face chords
using GlRuleT = GlRuleN<GEO_GLT>;

// Gauss-Legendre rule by Newton's method on P_n (three-term recurrence), from the Chebyshev guesses
template <int NG = GEO_GL>
static GlRuleN<NG> gl_rule() {
  GlRuleN<NG> g;
  const int n = NG;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    const double w = 2.0 / ((1.0 - x * x) * dp * dp);
    g.x[i] = -x;
    g.w[i] = w;
    g.x[n - 1 - i] = x;
    g.w[n - 1 - i] = w;
  }
  return g;
}

// distances from a point to the nearest and farthest points of a box (2-D)
__device__ __forceinline__ void box_dist2(const double* c, const double* lo, const double* hi, double* dmin,
                                          double* dmax) {
  double a = 0.0, b = 0.0;
  for (int d = 0; d < 2; ++d) {
    const double n = fmin(fmax(c[d], lo[d]), hi[d]) - c[d];
    const double f = fmax(fabs(c[d] - lo[d]), fabs(c[d] - hi[d]));
    a += n * n;
    b += f * f;
  }
  *dmin = sqrt(a);
  *dmax = sqrt(b);
}

// 0 covered, 1 full, 2 cut (body in *body); 3: two circles reach into the box
__device__ int classify_box2(const Circles& B, const double* lo, const double* hi, int* body) {
  *body = -1;
  if (B.n == 0) return 1;
  double dmin, dmax;
  if (B.inside) {
    box_dist2(B.c[0], lo, hi, &dmin, &dmax);
    if (dmax <= B.r[0]) return 1;
    if (dmin >= B.r[0]) return 0;
    *body = 0;
    return 2;
  }
  int ncut = 0;
  for (int b = 0; b < B.n; ++b) {
    box_dist2(B.c[b], lo, hi, &dmin, &dmax);
    if (dmax <= B.r[b]) {
      *body = -1;
      return 0;
    }
    if (dmin < B.r[b]) {
      ++ncut;
      *body = b;
    }
  }
  if (ncut > 1) return 3;
  return ncut ? 2 : 1;
}

// cells (dir < 0) or faces normal to dir: flag and cutting body; err set for two bodies in one box
__global__ void k_geo_classify2(Circles B, int nx, int ny, double h, int dir, int64_t n, uint8_t* flag,
                                int32_t* body, int32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int mx = nx + (dir == 0), ix = (int)(i % mx), iy = (int)(i / mx);
  double lo[2] = {ix * h, iy * h}, hi[2] = {(ix + 1) * h, (iy + 1) * h};
  if (dir >= 0) hi[dir] = lo[dir];
  int b;
  int f = classify_box2(B, lo, hi, &b);
  if (f == 3) {
    atomicExch(err, 1);
    f = 2;
  }
  flag[i] = (uint8_t)f;
  body[i] = b;
}

__global__ void k_geo_is(const uint8_t* flag, int64_t n, uint8_t v, int32_t* sel) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) sel[i] = flag[i] == v;
}

__global__ void k_geo_compact(const int32_t* sel, const int64_t* pos, int64_t n, int32_t* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && sel[i]) out[pos[i]] = (int32_t)i;
}

// graded monomials of degree <= q in 2-D: (p0, p1), degree by degree, p0 descending
__device__ __forceinline__ void mon2(int i, int* p0, int* p1) {
  int q = 0;
  while (i > q) {
    i -= q + 1;
    ++q;
  }
  *p0 = q - i;
  *p1 = i;
}

// fluid intervals of the segment [-1/2, 1/2] of a line at signed distance dn from the circle centre, with
// the circle's chord at tangential position ct: outside fluid keeps the segment minus the chord,
// inside fluid the segment's part within it.  Returns the count (<= 2).
__device__ int fluid_intervals(double dn, double ct, double R, int inside, double* a, double* b) {
  const double s2 = R * R - dn * dn;
  if (s2 <= 0.0) {
    if (inside) return 0;
    a[0] = -0.5;
    b[0] = 0.5;
    return 1;
  }
  const double s = sqrt(s2), lo = ct - s, hi = ct + s;
  if (inside) {
    const double u = fmax(lo, -0.5), v = fmin(hi, 0.5);
    if (v <= u) return 0;
    a[0] = u;
    b[0] = v;
    return 1;
  }
  int k = 0;
  if (lo > -0.5) {
    a[k] = -0.5;
    b[k] = fmin(lo, 0.5);
    ++k;
  }
  if (hi < 0.5) {
    a[k] = fmax(hi, -0.5);
    b[k] = 0.5;
    ++k;
  }
  return k;
}

// int_a^b t^k dt for k = 0..q
__device__ __forceinline__ void seg_powers(double a, double b, int q, double* out) {
  double pa = a, pb = b;
  for (int k = 0; k <= q; ++k) {
    out[k] = (pb - pa) / (k + 1);
    pa *= a;
    pb *= b;
  }
}

struct GeoOut2 {
  int q, K;          // moment degree and its monomial count
  double* vol;       // [n][K]
  double* eb;        // [n][K]
  double* ebn;       // [n][2][K]
};

// moments of the cut cells (one thread per cell)
__global__ void k_circle_cells(Circles B, GlRule gl, int nx, double h, const int32_t* __restrict__ cells, int64_t n,
                               const int32_t* __restrict__ body, GeoOut2 o) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int c = cells[t];
  const int ix = c % nx, iy = c / nx;
  const int b = body[c];
  const double cx = (B.c[b][0] - (ix + 0.5) * h) / h, cy = (B.c[b][1] - (iy + 0.5) * h) / h, R = B.r[b] / h;
  const int q = o.q, K = o.K, inside = B.inside;
  double vol[28], eb[28], ebn[2][28];
  for (int k = 0; k < K; ++k) vol[k] = eb[k] = ebn[0][k] = ebn[1][k] = 0.0;
  // ---- arcs inside the cell: angles where the circle meets the cell edges
  double ang[8];
  int na = 0;
  for (int s = -1; s <= 1; s += 2) {
    const double e = 0.5 * s;
    double d2 = R * R - (e - cx) * (e - cx);  // edge x = e
    if (d2 >= 0.0) {
      const double w = sqrt(d2);
      for (int u = -1; u <= 1; u += 2) {
        const double yy = cy + u * w;
        if (yy >= -0.5 && yy <= 0.5) ang[na++] = atan2(yy - cy, e - cx);
      }
    }
    d2 = R * R - (e - cy) * (e - cy);  // edge y = e
    if (d2 >= 0.0) {
      const double w = sqrt(d2);
      for (int u = -1; u <= 1; u += 2) {
        const double xx = cx + u * w;
        if (xx >= -0.5 && xx <= 0.5) ang[na++] = atan2(e - cy, xx - cx);
      }
    }
  }
  for (int i = 1; i < na; ++i)  // insertion sort
    for (int j = i; j > 0 && ang[j] < ang[j - 1]; --j) {
      const double tmp = ang[j];
      ang[j] = ang[j - 1];
      ang[j - 1] = tmp;
    }
  int narc = 0;
  double arc0[8], arc1[8];
  if (na == 0) {  // the whole circle lies in the cell
    arc0[0] = -M_PI;
    arc1[0] = M_PI;
    narc = 1;
  } else {
    for (int i = 0; i < na; ++i) {
      const double a = ang[i], e = i + 1 < na ? ang[i + 1] : ang[0] + 2.0 * M_PI;
      if (e - a <= 0.0) continue;
      const double m = 0.5 * (a + e);
      const double px = cx + R * cos(m), py = cy + R * sin(m);
      if (px > -0.5 && px < 0.5 && py > -0.5 && py < 0.5) {
        arc0[narc] = a;
        arc1[narc] = e;
        ++narc;
      }
    }
  }
  const double sgn = inside ? 1.0 : -1.0;  // normal out of the fluid: +radial inside the circle, -radial outside
  // divergence-theorem direction dd: the one most tangent to the boundary in this cell (the smaller
  // component of the centre offset), so that a thin sliver of fluid along an edge is not the small
  // difference of edge and arc terms of size one
  const int dd = fabs(cx) <= fabs(cy) ? 0 : 1;
  double arcx[28];                         // int xi^(p + e_dd) n_dd ds over the arcs
  for (int k = 0; k < K; ++k) arcx[k] = 0.0;
  for (int a = 0; a < narc; ++a) {
    const int npc = (int)ceil((arc1[a] - arc0[a]) / (0.25 * M_PI));
    const double span = (arc1[a] - arc0[a]) / npc;
    for (int pc = 0; pc < npc; ++pc) {
      const double m = arc0[a] + (pc + 0.5) * span, hw = 0.5 * span;
      for (int g = 0; g < GEO_GL; ++g) {
        const double th = m + hw * gl.x[g], wt = gl.w[g] * hw * R;  // ds = R dtheta
        const double ct = cos(th), st = sin(th);
        const double x = cx + R * ct, y = cy + R * st, n0 = sgn * ct, n1 = sgn * st;
        double xp[GEO_MAXQ + 2], yp[GEO_MAXQ + 2];
        xp[0] = yp[0] = 1.0;
        for (int k = 1; k <= q + 1; ++k) {
          xp[k] = xp[k - 1] * x;
          yp[k] = yp[k - 1] * y;
        }
        for (int k = 0; k < K; ++k) {
          int p0, p1;
          mon2(k, &p0, &p1);
          const double v = wt * xp[p0] * yp[p1];
          eb[k] += v;
          ebn[0][k] += v * n0;
          ebn[1][k] += v * n1;
          arcx[k] += dd == 0 ? wt * xp[p0 + 1] * yp[p1] * n0 : wt * xp[p0] * yp[p1 + 1] * n1;
        }
      }
    }
  }
  // ---- volume moments: the two edges normal to dd (fluid intervals, closed form) and the arcs
  for (int s = -1; s <= 1; s += 2) {
    const double e = 0.5 * s;
    double ia[2], ib[2];
    const int ni = dd == 0 ? fluid_intervals(e - cx, cy, R, inside, ia, ib) : fluid_intervals(e - cy, cx, R, inside, ia, ib);
    for (int j = 0; j < ni; ++j) {
      double sp[GEO_MAXQ + 1];
      seg_powers(ia[j], ib[j], q, sp);
      for (int k = 0; k < K; ++k) {
        int p0, p1;
        mon2(k, &p0, &p1);
        // n_dd = s on the edge xi_dd = s/2; the tangential exponent is the other one
        vol[k] += dd == 0 ? s * pow(e, p0 + 1) * sp[p1] : s * pow(e, p1 + 1) * sp[p0];
      }
    }
  }
  for (int k = 0; k < K; ++k) {
    int p0, p1;
    mon2(k, &p0, &p1);
    vol[k] = (vol[k] + arcx[k]) / ((dd == 0 ? p0 : p1) + 1);
  }
  for (int k = 0; k < K; ++k) {
    o.vol[t * K + k] = vol[k];
    o.eb[t * K + k] = eb[k];
    o.ebn[(t * 2 + 0) * K + k] = ebn[0][k];
    o.ebn[(t * 2 + 1) * K + k] = ebn[1][k];
  }
}

// moments of the cut faces normal to dir (one thread per face): int t^q dt over the fluid intervals
__global__ void k_circle_faces(Circles B, int nx, int dir, double h, const int32_t* __restrict__ faces, int64_t n,
                               const int32_t* __restrict__ body, int q, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int f = faces[t];
  const int mx = nx + (dir == 0), ix = f % mx, iy = f / mx;
  const int b = body[f];
  // face centre; normal coordinate dir, tangential coordinate 1 - dir
  const double fc[2] = {dir == 0 ? ix * h : (ix + 0.5) * h, dir == 1 ? iy * h : (iy + 0.5) * h};
  const double dn = (fc[dir] - B.c[b][dir]) / h, ct = (B.c[b][1 - dir] - fc[1 - dir]) / h, R = B.r[b] / h;
  double ia[2], ib[2];
  const int ni = fluid_intervals(dn, ct, R, B.inside, ia, ib);
  double acc[GEO_MAXQ + 1];
  for (int k = 0; k <= q; ++k) acc[k] = 0.0;
  for (int j = 0; j < ni; ++j) {
    double sp[GEO_MAXQ + 1];
    seg_powers(ia[j], ib[j], q, sp);
    for (int k = 0; k <= q; ++k) acc[k] += sp[k];
  }
  for (int k = 0; k <= q; ++k) out[t * (q + 1) + k] = acc[k];
}

// volume fractions at the ends: a cut cell at most GEO_EPS becomes covered, at least 1 - GEO_EPS full
__global__ void k_geo_settle(const int32_t* __restrict__ list, int64_t n, const double* __restrict__ mom, int K,
                             uint8_t* flag, int32_t* keep) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double k0 = mom[t * K];
  uint8_t f = 2;
  if (k0 >= 1.0 - GEO_EPS) f = 1;
  else if (k0 <= GEO_EPS) f = 0;
  flag[list[t]] = f;
  keep[t] = f == 2;
}

// a face next to a covered cell closes (2-D)
__global__ void k_geo_close_faces(const uint8_t* __restrict__ cflag, int nx, int ny, int dir, int64_t n,
                                  uint8_t* fflag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || fflag[i] == 0) return;
  const int mx = nx + (dir == 0), ix = (int)(i % mx), iy = (int)(i / mx);
  int lx = ix, ly = iy;
  if (dir == 0) --lx;
  else --ly;
  const bool lo_cov = lx >= 0 && ly >= 0 && cflag[lx + (int64_t)nx * ly] == 0;
  const bool hi_cov = ix < nx && iy < ny && cflag[ix + (int64_t)nx * iy] == 0;
  if (lo_cov || hi_cov) fflag[i] = 0;
}

__global__ void k_geo_keep_open(const int32_t* __restrict__ list, int64_t n, const uint8_t* __restrict__ fflag,
                                int32_t* keep) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) keep[t] = keep[t] && fflag[list[t]] == 2;
}

// rows of src kept (keep[t]) packed in order: dst[pos[t]] = src[t] (width w doubles)
__global__ void k_geo_pack(const int32_t* keep, const int64_t* pos, int64_t n, int w, const double* src,
                           double* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * w) return;
  const int64_t t = i / w;
  if (keep[t]) dst[pos[t] * w + i % w] = src[i];
}

__global__ void k_geo_pack_idx(const int32_t* keep, const int64_t* pos, int64_t n, const int32_t* src, int32_t* dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && keep[t]) dst[pos[t]] = src[t];
}

// ---------------------------------------------------------------- shape derivatives
//
// Derivatives of the moment tables when the boundary moves with a normal speed V(x) along
// N = (x - c)/r, the direction out of the body (ShapeVel: V = 1 on one body for its radius; V = -/+ f for
// the amplitude of a level-set mode psi + a f with f = sin(2 pi k . x + theta), at a = 0, the sign
// that of -psi's gradient along N: - for the outside of the bodies, + for the inside of one).  The cut
// sets are held fixed.  With n = sgn N the normal out of the fluid (sgn = -1 outside, +1 inside), the
// transport theorem on the patch gives (curvature 1/r in 2-D, mean curvature sum 2/r in 3-D)
//   volume moments  d int_V xi^p = sgn int_patch xi^p V dA;
//   EB moments      d int_patch F dA = int (grad F . N + curv F) V dA + oint_edges F V_e dl;
//   normal moments  d int_patch F n dA = sgn [int (grad F . N + curv F) V N dA - int F grad_G V dA
//                   + oint_edges F V_e N dl]   (d N = -grad_G V, the surface gradient);
//   face moments    the disk (chord) the body cuts from a face plane grows along its rim with speed
//                   V r / rho (rho its radius, its half-length in 2-D), the fluid part by sgn times that.
// The edges of a patch lie on the cell's faces; an edge point moves within its face plane with the
// in-surface speed V_e = -V (N . n_p) / (1 - (N . n_p)^2)^(1/2), n_p the face's normal out of the cell;
// in 2-D the edges are the arc ends, which slide along the cell edges they lie on with the arc-angle
// speed V t' (t' = cos t / (r sin t) on an x edge, -sin t / (r cos t) on a y edge).

// the normal speed of sv at the physical point X of body b's boundary, and its gradient
__device__ __forceinline__ double shape_speed(const ShapeVel& sv, int inside, int b, const double* X, int D,
                                              double* gV) {
  if (sv.kind == 0) {
    for (int d = 0; d < D; ++d) gV[d] = 0.0;
    return b == sv.body ? 1.0 : 0.0;
  }
  double a = sv.theta;
  for (int d = 0; d < D; ++d) a += 2.0 * M_PI * sv.k[d] * X[d];
  const double sg = inside ? 1.0 : -1.0, ca = cos(a);
  for (int d = 0; d < D; ++d) gV[d] = sg * 2.0 * M_PI * sv.k[d] * ca;
  return sg * sin(a);
}

__device__ __forceinline__ bool shape_moves(const ShapeVel& sv, int b) {
  return b >= 0 && (sv.kind != 0 || b == sv.body);
}

__global__ void k_circle_cells_dv(Circles B, GlRule gl, int nx, double h, ShapeVel sv,
                                  const int32_t* __restrict__ cells, int64_t n, const int32_t* __restrict__ cbody,
                                  int q, int K, double* dvol, double* deb, double* debn) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int c = cells[t];
  const int b = cbody[c];
  double dv[28], de[28], dn[2][28];
  for (int k = 0; k < K; ++k) dv[k] = de[k] = dn[0][k] = dn[1][k] = 0.0;
  if (shape_moves(sv, b)) {
    const int ix = c % nx, iy = c / nx;
    const double cx = (B.c[b][0] - (ix + 0.5) * h) / h, cy = (B.c[b][1] - (iy + 0.5) * h) / h;
    const double R = B.r[b] / h;
    // arc ends: angle, d(angle)/dR (R in units of h), sorted by angle
    double ang[8], dang[8];
    int na = 0;
    for (int sd = -1; sd <= 1; sd += 2) {
      const double e = 0.5 * sd;
      double d2 = R * R - (e - cx) * (e - cx);
      if (d2 > 0.0) {
        const double w = sqrt(d2);
        for (int u = -1; u <= 1; u += 2) {
          const double yy = cy + u * w;
          if (yy > -0.5 && yy < 0.5) {
            const double th = atan2(yy - cy, e - cx);
            ang[na] = th;
            dang[na++] = cos(th) / (R * sin(th));
          }
        }
      }
      d2 = R * R - (e - cy) * (e - cy);
      if (d2 > 0.0) {
        const double w = sqrt(d2);
        for (int u = -1; u <= 1; u += 2) {
          const double xx = cx + u * w;
          if (xx > -0.5 && xx < 0.5) {
            const double th = atan2(e - cy, xx - cx);
            ang[na] = th;
            dang[na++] = -sin(th) / (R * cos(th));
          }
        }
      }
    }
    for (int i = 1; i < na; ++i)
      for (int j = i; j > 0 && ang[j] < ang[j - 1]; --j) {
        double tmp = ang[j];
        ang[j] = ang[j - 1];
        ang[j - 1] = tmp;
        tmp = dang[j];
        dang[j] = dang[j - 1];
        dang[j - 1] = tmp;
      }
    const double sgn = B.inside ? 1.0 : -1.0;  // n = sgn N, out of the fluid
    for (int i = 0; i < na; ++i) {
      const double a = ang[i], e = i + 1 < na ? ang[i + 1] : ang[0] + 2.0 * M_PI;
      const double da = dang[i], dE = i + 1 < na ? dang[i + 1] : dang[0];
      if (e - a <= 0.0) continue;
      const double m = 0.5 * (a + e);
      const double px = cx + R * cos(m), py = cy + R * sin(m);
      if (!(px > -0.5 && px < 0.5 && py > -0.5 && py < 0.5)) continue;
      const int npc = (int)ceil((e - a) / (0.25 * M_PI));
      const double span = (e - a) / npc;
      for (int pc = 0; pc < npc; ++pc) {
        const double mm = a + (pc + 0.5) * span, hw = 0.5 * span;
        for (int g = 0; g < GEO_GL; ++g) {
          const double th = mm + hw * gl.x[g], ds = gl.w[g] * hw * R;  // arc length / h
          const double ct = cos(th), st = sin(th);
          const double x = cx + R * ct, y = cy + R * st;
          const double X[2] = {B.c[b][0] + h * R * ct, B.c[b][1] + h * R * st};
          double gv[2];
          const double V = shape_speed(sv, B.inside, b, X, 2, gv);
          const double gn = gv[0] * ct + gv[1] * st;
          const double gG[2] = {h * (gv[0] - gn * ct), h * (gv[1] - gn * st)};
          double xp[GEO_MAXQ + 1], yp[GEO_MAXQ + 1];
          xp[0] = yp[0] = 1.0;
          for (int k = 1; k <= q; ++k) {
            xp[k] = xp[k - 1] * x;
            yp[k] = yp[k - 1] * y;
          }
          for (int k = 0; k < K; ++k) {
            int p0, p1;
            mon2(k, &p0, &p1);
            const double f = xp[p0] * yp[p1];
            double gN = 0.0;  // grad_xi f . N
            if (p0 > 0) gN += p0 * xp[p0 - 1] * yp[p1] * ct;
            if (p1 > 0) gN += p1 * xp[p0] * yp[p1 - 1] * st;
            const double v = ds * V * (gN + f / R);
            dv[k] += sgn * ds * f * V;
            de[k] += v;
            dn[0][k] += sgn * (v * ct - ds * f * gG[0]);
            dn[1][k] += sgn * (v * st - ds * f * gG[1]);
          }
        }
      }
      // ends: + f(t_b) V R t_b' - f(t_a) V R t_a'
      for (int end = 0; end < 2; ++end) {
        const double th = end ? e : a, dth = end ? dE : da, sg = end ? 1.0 : -1.0;
        const double ct = cos(th), st = sin(th);
        const double x = cx + R * ct, y = cy + R * st;
        const double X[2] = {B.c[b][0] + h * R * ct, B.c[b][1] + h * R * st};
        double gv[2];
        const double se = sg * shape_speed(sv, B.inside, b, X, 2, gv) * R * dth;
        for (int k = 0; k < K; ++k) {
          int p0, p1;
          mon2(k, &p0, &p1);
          const double v = pow(x, p0) * pow(y, p1) * se;
          de[k] += v;
          dn[0][k] += v * sgn * ct;
          dn[1][k] += v * sgn * st;
        }
      }
    }
    // the integrals above are per unit h (lengths in units of h): d/dt of the tables is (1/h) times them
    for (int k = 0; k < K; ++k) {
      dv[k] /= h;
      de[k] /= h;
      dn[0][k] /= h;
      dn[1][k] /= h;
    }
  }
  for (int k = 0; k < K; ++k) {
    dvol[t * K + k] = dv[k];
    deb[t * K + k] = de[k];
    debn[(t * 2 + 0) * K + k] = dn[0][k];
    debn[(t * 2 + 1) * K + k] = dn[1][k];
  }
}

__global__ void k_circle_faces_dv(Circles B, int nx, int dir, double h, ShapeVel sv, const int32_t* __restrict__ faces,
                                  int64_t n, const int32_t* __restrict__ fbody, int q, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int f = faces[t];
  const int b = fbody[f];
  double acc[GEO_MAXQ + 1];
  for (int k = 0; k <= q; ++k) acc[k] = 0.0;
  if (shape_moves(sv, b)) {
    const int mx = nx + (dir == 0), ix = f % mx, iy = f / mx;
    const double fc[2] = {dir == 0 ? ix * h : (ix + 0.5) * h, dir == 1 ? iy * h : (iy + 0.5) * h};
    const double dn = (fc[dir] - B.c[b][dir]) / h, ct = (B.c[b][1 - dir] - fc[1 - dir]) / h;
    const double R = B.r[b] / h, s2 = R * R - dn * dn;
    if (s2 > 0.0) {
      const double s = sqrt(s2);
      // outside fluid loses length at both chord ends; inside fluid gains it
      const double sg = B.inside ? 1.0 : -1.0;
      for (int e = -1; e <= 1; e += 2) {
        const double end = ct + e * s;
        if (end > -0.5 && end < 0.5) {
          double X[2], gv[2];
          X[dir] = fc[dir];
          X[1 - dir] = fc[1 - dir] + h * end;
          const double speed = shape_speed(sv, B.inside, b, X, 2, gv) * R / s;  // d(end) per unit parameter / h
          double p = 1.0;
          for (int k = 0; k <= q; ++k) {
            acc[k] += sg * p * speed;
            p *= end;
          }
        }
      }
    }
    for (int k = 0; k <= q; ++k) acc[k] /= h;
  }
  for (int k = 0; k <= q; ++k) out[t * (q + 1) + k] = acc[k];
}

// ---------------------------------------------------------------- 3-D: the cube minus spheres
//
// Face moments: the fluid part of a face square is the square minus (inside fluid: intersected with)
// the disk the sphere cuts from the face plane; in tangential coordinates (u, v) the disk's chord at u
// is |v - c_v| < (rho^2 - (u - c_u)^2)^(1/2): the v-integral in closed form, the u-integral by
// Gauss-Legendre on panels split where the chord ends cross v = +-1/2 and mapped by
// u = a + (b - a) sin^2(pi s / 2), which flattens the square-root behaviour at the disk's edge.
// EB moments: the area element of a sphere in (z, phi) is R dz dphi (Archimedes); at each z the patch
// is the arcs of the circle of radius (R^2 - (z - c_z)^2)^(1/2) inside the cell's x-y square.  The
// outer integral runs over the polar angle th (z = c_z + R cos th, dA = R^2 sin th dth dphi), split
// where the arcs change (tangencies with the square's edge lines and corners) and mapped by the same
// sin^2 substitution with 48 points per panel: in z the circle's radius has a square-root branch at
// the poles, which slows convergence in the cells next to them; in th it is R sin th.  Volume moments: the divergence theorem with the
// x-derivative, int_V xi^p = 1/(p_0+1) oint xi^(p+e_0) n_0 dA, over the two x faces' fluid parts and
// the patch.

struct Spheres {
  int n, inside;
  double c[GEO_MAXB][3];
  double r[GEO_MAXB];
};

__device__ __forceinline__ void box_dist3(const double* c, const double* lo, const double* hi, double* dmin,
                                          double* dmax) {
  double a = 0.0, b = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double n = fmin(fmax(c[d], lo[d]), hi[d]) - c[d];
    const double f = fmax(fabs(c[d] - lo[d]), fabs(c[d] - hi[d]));
    a += n * n;
    b += f * f;
  }
  *dmin = sqrt(a);
  *dmax = sqrt(b);
}

__device__ int classify_box3(const Spheres& B, const double* lo, const double* hi, int* body) {
  *body = -1;
  if (B.n == 0) return 1;
  double dmin, dmax;
  if (B.inside) {
    box_dist3(B.c[0], lo, hi, &dmin, &dmax);
    if (dmax <= B.r[0]) return 1;
    if (dmin >= B.r[0]) return 0;
    *body = 0;
    return 2;
  }
  int ncut = 0;
  for (int b = 0; b < B.n; ++b) {
    box_dist3(B.c[b], lo, hi, &dmin, &dmax);
    if (dmax <= B.r[b]) {
      *body = -1;
      return 0;
    }
    if (dmin < B.r[b]) {
      ++ncut;
      *body = b;
    }
  }
  if (ncut > 1) return 3;
  return ncut ? 2 : 1;
}

__global__ void k_geo_classify3(Spheres B, int N, double h, int dir, int64_t n, uint8_t* flag, int32_t* body,
                                int32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m0 = N + (dir == 0), m1 = N + (dir == 1);
  const int ix = (int)(i % m0), iy = (int)((i / m0) % m1), iz = (int)(i / ((int64_t)m0 * m1));
  double lo[3] = {ix * h, iy * h, iz * h}, hi[3] = {(ix + 1) * h, (iy + 1) * h, (iz + 1) * h};
  if (dir >= 0) hi[dir] = lo[dir];
  int b;
  int f = classify_box3(B, lo, hi, &b);
  if (f == 3) {
    atomicExch(err, 1);
    f = 2;
  }
  flag[i] = (uint8_t)f;
  body[i] = b;
}

// graded monomials of degree <= q in 3-D: degree by degree, p0 descending, then p1 descending
__device__ __forceinline__ void mon3(int i, int* p) {
  int q = 0;
  while (i >= (q + 1) * (q + 2) / 2) {
    i -= (q + 1) * (q + 2) / 2;
    ++q;
  }
  int a = 0;  // within degree q: p0 = q - a, then p1 from a down to 0
  while (i > a) {
    i -= a + 1;
    ++a;
  }
  p[0] = q - a;
  p[1] = a - i;
  p[2] = i;
}

// mon3's exponents packed p0 | p1 << 4 | p2 << 8, for loops unrolled over a compile-time count (the
// accumulators of such loops stay in registers)
__host__ __device__ constexpr int mon3_packed(int i) {
  int q = 0;
  while (i >= (q + 1) * (q + 2) / 2) {
    i -= (q + 1) * (q + 2) / 2;
    ++q;
  }
  int a = 0;
  while (i > a) {
    i -= a + 1;
    ++a;
  }
  return (q - a) | ((a - i) << 4) | (i << 8);
}

__device__ __forceinline__ void sort_small(double* v, int n) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && v[j] < v[j - 1]; --j) {
      const double t = v[j];
      v[j] = v[j - 1];
      v[j - 1] = t;
    }
}

// arcs of the circle (cx, cy, rho) inside the square [-1/2, 1/2]^2: angle intervals; returns the count
__device__ int square_arcs(double cx, double cy, double rho, double* a0, double* a1) {
  double ang[8];
  int na = 0;
  for (int s = -1; s <= 1; s += 2) {
    const double e = 0.5 * s;
    double d2 = rho * rho - (e - cx) * (e - cx);
    if (d2 >= 0.0) {
      const double w = sqrt(d2);
      for (int u = -1; u <= 1; u += 2) {
        const double yy = cy + u * w;
        if (yy >= -0.5 && yy <= 0.5) ang[na++] = atan2(yy - cy, e - cx);
      }
    }
    d2 = rho * rho - (e - cy) * (e - cy);
    if (d2 >= 0.0) {
      const double w = sqrt(d2);
      for (int u = -1; u <= 1; u += 2) {
        const double xx = cx + u * w;
        if (xx >= -0.5 && xx <= 0.5) ang[na++] = atan2(e - cy, xx - cx);
      }
    }
  }
  if (na == 0) {  // the circle lies inside the square, or outside it (or around it)
    if (cx - rho > -0.5 && cx + rho < 0.5 && cy - rho > -0.5 && cy + rho < 0.5) {
      a0[0] = -M_PI;
      a1[0] = M_PI;
      return 1;
    }
    return 0;
  }
  sort_small(ang, na);
  int narc = 0;
  for (int i = 0; i < na; ++i) {
    const double a = ang[i], e = i + 1 < na ? ang[i + 1] : ang[0] + 2.0 * M_PI;
    if (e - a <= 0.0) continue;
    const double m = 0.5 * (a + e);
    const double px = cx + rho * cos(m), py = cy + rho * sin(m);
    if (px > -0.5 && px < 0.5 && py > -0.5 && py < 0.5) {
      a0[narc] = a;
      a1[narc] = e;
      ++narc;
    }
  }
  return narc;
}

// sin^2-mapped Gauss-Legendre node g on the panel [a, b]: position and weight
__device__ __forceinline__ void sin2_node(const GlRuleT& gl, int g, double a, double b, double* t, double* w) {
  const double s = 0.5 * gl.x[g] + 0.5;
  const double sn = sin(0.5 * M_PI * s), cs = cos(0.5 * M_PI * s);
  *t = a + (b - a) * sn * sn;
  *w = 0.5 * gl.w[g] * (b - a) * M_PI * sn * cs;
}

// moments int u^a v^b over the fluid part of the square [-1/2,1/2]^2 of a plane the sphere cuts in the
// disk (cu, cv, rho) (rho <= 0: no disk), for the graded 2-D monomials of degree <= q; disk[] holds the
// quadrature over the disk's u-range of the chord (inside fluid) or of the column minus the chord
__device__ void disk_square(double cu, double cv, double rho, int inside, int q, const GlRuleT& gl, double* out) {
  const int K2 = (q + 1) * (q + 2) / 2;
  double su[GEO_MAXQ + 2], sv[GEO_MAXQ + 2];
  seg_powers(-0.5, 0.5, q, su);
  seg_powers(-0.5, 0.5, q, sv);
  double disk[28];
  int pa[28], pb[28];
  for (int k = 0; k < K2; ++k) {
    disk[k] = 0.0;
    mon2(k, &pa[k], &pb[k]);
  }
  const double lo = fmax(-0.5, cu - rho), hi = fmin(0.5, cu + rho);
  if (rho > 0.0 && hi > lo) {
    double br[6];
    int nb = 0;
    br[nb++] = lo;
    br[nb++] = hi;
    for (int e = -1; e <= 1; e += 2) {
      const double dv = 0.5 * e - cv;
      if (fabs(dv) < rho) {
        const double w = sqrt(rho * rho - dv * dv);
        for (int sg = -1; sg <= 1; sg += 2) {
          const double uu = cu + sg * w;
          if (uu > lo && uu < hi) br[nb++] = uu;
        }
      }
    }
    sort_small(br, nb);
    for (int pnl = 0; pnl + 1 < nb; ++pnl) {
      if (br[pnl + 1] <= br[pnl]) continue;
      for (int g = 0; g < GEO_GLT; ++g) {
        double u, wu;
        sin2_node(gl, g, br[pnl], br[pnl + 1], &u, &wu);
        const double hw = sqrt(fmax(rho * rho - (u - cu) * (u - cu), 0.0));
        const double va = fmin(fmax(cv - hw, -0.5), 0.5), vb = fmin(fmax(cv + hw, -0.5), 0.5);
        double vp[GEO_MAXQ + 2];
        if (inside) {
          seg_powers(va, vb, q, vp);
        } else {  // [-1/2, va] and [vb, 1/2]
          double v1[GEO_MAXQ + 2], v2[GEO_MAXQ + 2];
          seg_powers(-0.5, va, q, v1);
          seg_powers(vb, 0.5, q, v2);
          for (int k = 0; k <= q; ++k) vp[k] = v1[k] + v2[k];
        }
        double up = 1.0, upow[GEO_MAXQ + 1];
        for (int k = 0; k <= q; ++k) {
          upow[k] = up;
          up *= u;
        }
        for (int k = 0; k < K2; ++k) disk[k] += wu * upow[pa[k]] * vp[pb[k]];
      }
    }
  }
  if (inside) {
    for (int k = 0; k < K2; ++k) out[k] = disk[k];
    return;
  }
  // outside fluid, integrated directly (a nearly closed face is not the small difference of the square
  // and the disk): the full columns outside the disk's u-range in closed form, and inside it the parts
  // of the column outside the chord
  double full[28];
  for (int k = 0; k < K2; ++k) full[k] = 0.0;
  {
    double ua[2], ub[2];
    int nu = 0;
    if (!(rho > 0.0) || hi <= lo) {
      ua[0] = -0.5;
      ub[0] = 0.5;
      nu = 1;
    } else {
      if (lo > -0.5) { ua[nu] = -0.5; ub[nu] = lo; ++nu; }
      if (hi < 0.5) { ua[nu] = hi; ub[nu] = 0.5; ++nu; }
    }
    for (int j = 0; j < nu; ++j) {
      double up2[GEO_MAXQ + 2];
      seg_powers(ua[j], ub[j], q, up2);
      for (int k = 0; k < K2; ++k) full[k] += up2[pa[k]] * sv[pb[k]];
    }
  }
  for (int k = 0; k < K2; ++k) out[k] = full[k] + disk[k];
}

// fn(x, y, z, ex, ey, ez, w) at the quadrature nodes of the patch of the sphere (cx, cy, cz, R) inside
// the cell [-1/2, 1/2]^3 (cell-centred coordinates in units of h): (x, y, z) the node, (ex, ey, ez) =
// node - centre = R N, w its area weight in units of h^2 (the rule of k_sphere_patch)
template <class Fn>
__device__ void sphere_patch_quad(double cx, double cy, double cz, double R, const GlRule& gl, const GlRuleT& glt,
                                  Fn&& fn) {
  // z breakpoints: the range ends, tangencies with the edge lines x, y = +-1/2 and passes through the
  // square's corners
  const double zl = fmax(-0.5, cz - R), zh = fmin(0.5, cz + R);
  double br[20];
  int nb = 0;
  br[nb++] = zl;
  br[nb++] = zh;
  for (int e = -1; e <= 1; e += 2) {
    const double dd[2] = {(0.5 * e - cx) * (0.5 * e - cx), (0.5 * e - cy) * (0.5 * e - cy)};
    for (int j = 0; j < 2; ++j) {
      const double qq = R * R - dd[j];
      if (qq > 0.0)
        for (int sg = -1; sg <= 1; sg += 2) {
          const double zz = cz + sg * sqrt(qq);
          if (zz > zl && zz < zh) br[nb++] = zz;
        }
    }
    for (int e2 = -1; e2 <= 1; e2 += 2) {
      const double qq = R * R - (0.5 * e - cx) * (0.5 * e - cx) - (0.5 * e2 - cy) * (0.5 * e2 - cy);
      if (qq > 0.0)
        for (int sg = -1; sg <= 1; sg += 2) {
          const double zz = cz + sg * sqrt(qq);
          if (zz > zl && zz < zh) br[nb++] = zz;
        }
    }
  }
  // the z breakpoints as polar angles from the +z axis: z = cz + R cos(th), rho = R sin(th), and
  // dA = R dz dphi = R^2 sin(th) dth dphi; the angle keeps the integrand analytic up to the poles
  // (rho = (R^2 - (z - cz)^2)^(1/2) is not at z = cz +- R)
  for (int i = 0; i < nb; ++i) br[i] = acos(fmin(1.0, fmax(-1.0, (br[i] - cz) / R)));
  sort_small(br, nb);
  for (int pnl = 0; pnl + 1 < nb; ++pnl) {
    if (br[pnl + 1] <= br[pnl]) continue;
    for (int gz = 0; gz < GEO_GLT; ++gz) {
      double th, wth;
      sin2_node(glt, gz, br[pnl], br[pnl + 1], &th, &wth);
      const double z = cz + R * cos(th), rho = R * sin(th);
      const double wz = wth * rho;  // R dz = R^2 sin(th) dth: the factor R is applied with dphi below
      if (rho <= 0.0) continue;
      double a0[4], a1[4];
      const int narc = square_arcs(cx, cy, rho, a0, a1);
      for (int a = 0; a < narc; ++a) {
        const int npc = (int)ceil((a1[a] - a0[a]) / (0.25 * M_PI));
        const double span = (a1[a] - a0[a]) / npc;
        for (int pc = 0; pc < npc; ++pc) {
          const double mm = a0[a] + (pc + 0.5) * span, hw = 0.5 * span;
          for (int g = 0; g < GEO_GL; ++g) {
            const double ph = mm + hw * gl.x[g];
            const double cp = cos(ph), sp = sin(ph);
            fn(cx + rho * cp, cy + rho * sp, z, rho * cp, rho * sp, z - cz, wz * gl.w[g] * hw * R);  // dA = R dz dphi
          }
        }
      }
    }
  }
}

// one table of a cut cell's EB patch integrals (thread per cell and table): t = 0 int xi^p dA, t = 1..3
// int xi^p n_(t-1) dA, t = 4 int xi^(p+e_d) n_d dA (the patch part of the volume moments, d the cell's
// divergence direction); divided by h^2
template <int Q>
__global__ void k_sphere_patch(Spheres B, GlRule gl, GlRuleT glt, int N, double h, const int32_t* __restrict__ cells,
                               int64_t n, const int32_t* __restrict__ cbody, double* eb, double* ebn, double* volp) {
  constexpr int K = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  const int64_t tt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tt >= 5 * n) return;
  const int64_t t = tt / 5;
  const int table = (int)(tt % 5);
  const int c = cells[t];
  const int ix = c % N, iy = (c / N) % N, iz = c / (N * N);
  const int b = cbody[c];
  const double cx = (B.c[b][0] - (ix + 0.5) * h) / h, cy = (B.c[b][1] - (iy + 0.5) * h) / h;
  const double cz = (B.c[b][2] - (iz + 0.5) * h) / h, R = B.r[b] / h;
  const double sgn = B.inside ? 1.0 : -1.0;  // normal out of the fluid: sgn (x - c) / R
  // divergence-theorem direction (table 4): the smallest component of the centre offset, the direction
  // most tangent to the patch (see k_sphere_vol)
  const int dd = (fabs(cx) <= fabs(cy) && fabs(cx) <= fabs(cz)) ? 0 : (fabs(cy) <= fabs(cz) ? 1 : 2);
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  sphere_patch_quad(cx, cy, cz, R, gl, glt,
                    [&](double x, double y, double z, double ex, double ey, double ez, double w) {
                      double f = w;
                      if (table >= 1 && table <= 3) {
                        const double e = table == 1 ? ex : (table == 2 ? ey : ez);
                        f *= sgn * e / R;
                      } else if (table == 4) {
                        f *= sgn * (dd == 0 ? ex : (dd == 1 ? ey : ez)) / R;
                      }
                      double xp[Q + 2], yp[Q + 2], zp[Q + 2];
                      xp[0] = yp[0] = zp[0] = 1.0;
#pragma unroll
                      for (int k = 1; k <= Q + 1; ++k) {
                        xp[k] = xp[k - 1] * x;
                        yp[k] = yp[k - 1] * y;
                        zp[k] = zp[k - 1] * z;
                      }
                      const int ex4 = table == 4 && dd == 0, ey4 = table == 4 && dd == 1, ez4 = table == 4 && dd == 2;
#pragma unroll
                      for (int k = 0; k < K; ++k) {
                        const int pk = mon3_packed(k);
                        acc[k] += f * xp[(pk & 15) + ex4] * yp[((pk >> 4) & 15) + ey4] * zp[(pk >> 8) + ez4];
                      }
                    });
  double* dst = table == 0 ? eb + t * K : (table == 4 ? volp + t * K : ebn + (t * 3 + table - 1) * K);
#pragma unroll
  for (int k = 0; k < K; ++k) dst[k] = acc[k];
}

// volume moments from the patch part and the two x faces' fluid parts (thread per cell)
__global__ void k_sphere_vol(Spheres B, GlRuleT gl, int N, double h, const int32_t* __restrict__ cells, int64_t n,
                             const int32_t* __restrict__ cbody, int q, int K, const double* __restrict__ volp,
                             double* vol) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int c = cells[t];
  const int ix = c % N, iy = (c / N) % N, iz = c / (N * N);
  const int b = cbody[c];
  const double cx = (B.c[b][0] - (ix + 0.5) * h) / h, cy = (B.c[b][1] - (iy + 0.5) * h) / h;
  const double cz = (B.c[b][2] - (iz + 0.5) * h) / h, R = B.r[b] / h;
  // the direction most tangent to the patch (as in k_sphere_patch) and the two faces normal to it
  const double cc[3] = {cx, cy, cz};
  const int dd = (fabs(cx) <= fabs(cy) && fabs(cx) <= fabs(cz)) ? 0 : (fabs(cy) <= fabs(cz) ? 1 : 2);
  const int u = dd == 0 ? 1 : 0, v = dd == 2 ? 1 : 2;
  double acc[35];
  for (int k = 0; k < K; ++k) acc[k] = volp[t * K + k];
  for (int s = -1; s <= 1; s += 2) {
    const double xe = 0.5 * s, d2 = R * R - (xe - cc[dd]) * (xe - cc[dd]);
    double fm[28];
    disk_square(cc[u], cc[v], d2 > 0.0 ? sqrt(d2) : 0.0, B.inside, q, gl, fm);
    for (int k = 0; k < K; ++k) {
      int p[3];
      mon3(k, p);
      const int dg = p[u] + p[v];
      const int k2 = dg * (dg + 1) / 2 + p[v];  // (p_u, p_v) in the graded 2-D order
      acc[k] += s * pow(xe, p[dd] + 1) * fm[k2];
    }
  }
  for (int k = 0; k < K; ++k) {
    int p[3];
    mon3(k, p);
    vol[t * K + k] = acc[k] / (p[dd] + 1);
  }
}

// tangential moments of the cut faces normal to dir (thread per face)
__global__ void k_sphere_faces(Spheres B, GlRuleT gl, int N, int dir, double h, const int32_t* __restrict__ faces,
                               int64_t n, const int32_t* __restrict__ fbody, int q, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int f = faces[t];
  const int m0 = N + (dir == 0), m1 = N + (dir == 1);
  const int i3[3] = {f % m0, (f / m0) % m1, f / (m0 * m1)};
  const int b = fbody[f];
  const int u = dir == 0 ? 1 : 0, v = dir == 2 ? 1 : 2;  // tangential dims, ascending
  const double dn = (i3[dir] * h - B.c[b][dir]) / h;
  const double cu = (B.c[b][u] - (i3[u] + 0.5) * h) / h, cv = (B.c[b][v] - (i3[v] + 0.5) * h) / h;
  const double R = B.r[b] / h, d2 = R * R - dn * dn;
  const int K2 = (q + 1) * (q + 2) / 2;
  double fm[28];
  disk_square(cu, cv, d2 > 0.0 ? sqrt(d2) : 0.0, B.inside, q, gl, fm);
  for (int k = 0; k < K2; ++k) out[t * K2 + k] = fm[k];
}

// a face next to a covered cell closes (3-D)
__global__ void k_geo_close_faces3(const uint8_t* __restrict__ cflag, int N, int dir, int64_t n, uint8_t* fflag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || fflag[i] == 0) return;
  const int m0 = N + (dir == 0), m1 = N + (dir == 1);
  int c[3] = {(int)(i % m0), (int)((i / m0) % m1), (int)(i / ((int64_t)m0 * m1))};
  bool cov = false;
  if (c[dir] < N) cov |= cflag[c[0] + (int64_t)N * (c[1] + (int64_t)N * c[2])] == 0;
  c[dir] -= 1;
  if (c[dir] >= 0) cov |= cflag[c[0] + (int64_t)N * (c[1] + (int64_t)N * c[2])] == 0;
  if (cov) fflag[i] = 0;
}

// ---------------------------------------------------------------- 3-D shape derivatives
//
// The formulas at the 2-D derivative kernels above with the sphere's patch quadrature (k_sphere_patch)
// and, for the edge terms, the arcs the sphere cuts from the cell's six face planes: on the face plane
// xi_d = e the circle has radius rho = (R^2 - (e - c_d)^2)^(1/2), N . n_p = sign(e) (e - c_d) / R is
// constant along it, and V_e dl = -V (N . n_p) R dt in the arc angle t.

// The derivative tables of the cut cells with one warp per cell: the lanes own the monomials (k = lane
// and lane + 32), the quadrature nodes (the patch rule of sphere_patch_quad; 20-point Gauss-Legendre on
// pieces of at most pi/4 of the edge arcs) are computed 32 at a time, one per lane with its speed and the speed's surface gradient, and broadcast to
// the warp, which accumulates the five tables at once: each node's position, weight and sines serve
// all tables and monomials.
__device__ __forceinline__ double ipow_small(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// f = x^e0 y^e1 z^e2 and grad f . N for the exponents e
__device__ __forceinline__ void mono_grad(const int* e, double x, double y, double z, double n0, double n1, double n2,
                                          double* f, double* gN) {
  const double px = e[0] > 0 ? ipow_small(x, e[0] - 1) : 0.0, py = e[1] > 0 ? ipow_small(y, e[1] - 1) : 0.0;
  const double pz = e[2] > 0 ? ipow_small(z, e[2] - 1) : 0.0;
  const double fx = e[0] > 0 ? px * x : 1.0, fy = e[1] > 0 ? py * y : 1.0, fz = e[2] > 0 ? pz * z : 1.0;
  *f = fx * fy * fz;
  double g = 0.0;
  if (e[0] > 0) g = fma(e[0] * px * fy * fz, n0, g);
  if (e[1] > 0) g = fma(e[1] * fx * py * fz, n1, g);
  if (e[2] > 0) g = fma(e[2] * fx * fy * pz, n2, g);
  *gN = g;
}

template <int Q>
__global__ void __launch_bounds__(128) k_sphere_cells_dw(Spheres B, GlRule gl, GlRuleT glt, int N, double h,
                                                         ShapeVel sv, const int32_t* __restrict__ cells, int64_t n,
                                                         const int32_t* __restrict__ cbody, double* dvol,
                                                         double* deb, double* debn) {
  constexpr int K = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // warp-uniform
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const int c = cells[t];
  const int b = cbody[c];
  const bool own1 = lane + 32 < K;
  int e0[3] = {0, 0, 0}, e1[3] = {0, 0, 0};
  if (lane < K) {
    const int pk = mon3_packed(lane);
    e0[0] = pk & 15;
    e0[1] = (pk >> 4) & 15;
    e0[2] = pk >> 8;
  }
  if (own1) {
    const int pk = mon3_packed(lane + 32);
    e1[0] = pk & 15;
    e1[1] = (pk >> 4) & 15;
    e1[2] = pk >> 8;
  }
  double a0[5] = {0, 0, 0, 0, 0}, a1[5] = {0, 0, 0, 0, 0};
  if (shape_moves(sv, b)) {
    const int ix = c % N, iy = (c / N) % N, iz = c / (N * N);
    const double* C = B.c[b];
    const double cx = (C[0] - (ix + 0.5) * h) / h, cy = (C[1] - (iy + 0.5) * h) / h;
    const double cz = (C[2] - (iz + 0.5) * h) / h, R = B.r[b] / h;
    const double sgn = B.inside ? 1.0 : -1.0, c2 = 2.0 / R;
    // patch node (broadcast): position, normal, w V, w grad_G V (h-scaled)
    auto patch_node = [&](double x, double y, double z, double n0, double n1, double n2, double wv, double g0,
                          double g1, double g2, const int* e, double* a) {
      double f, gN;
      mono_grad(e, x, y, z, n0, n1, n2, &f, &gN);
      const double u = wv * fma(c2, f, gN);
      a[0] = fma(sgn * wv, f, a[0]);
      a[1] += u;
      a[2] = fma(sgn, fma(u, n0, -g0 * f), a[2]);
      a[3] = fma(sgn, fma(u, n1, -g1 * f), a[3]);
      a[4] = fma(sgn, fma(u, n2, -g2 * f), a[4]);
    };
    // the patch: theta panels as in sphere_patch_quad, the phi nodes of each arc 32 at a time
    const double zl = fmax(-0.5, cz - R), zh = fmin(0.5, cz + R);
    double br[20];
    int nb = 0;
    br[nb++] = zl;
    br[nb++] = zh;
    for (int e = -1; e <= 1; e += 2) {
      const double dd[2] = {(0.5 * e - cx) * (0.5 * e - cx), (0.5 * e - cy) * (0.5 * e - cy)};
      for (int j = 0; j < 2; ++j) {
        const double qq = R * R - dd[j];
        if (qq > 0.0)
          for (int sg = -1; sg <= 1; sg += 2) {
            const double zz = cz + sg * sqrt(qq);
            if (zz > zl && zz < zh) br[nb++] = zz;
          }
      }
      for (int e2 = -1; e2 <= 1; e2 += 2) {
        const double qq = R * R - (0.5 * e - cx) * (0.5 * e - cx) - (0.5 * e2 - cy) * (0.5 * e2 - cy);
        if (qq > 0.0)
          for (int sg = -1; sg <= 1; sg += 2) {
            const double zz = cz + sg * sqrt(qq);
            if (zz > zl && zz < zh) br[nb++] = zz;
          }
      }
    }
    for (int i = 0; i < nb; ++i) br[i] = acos(fmin(1.0, fmax(-1.0, (br[i] - cz) / R)));
    sort_small(br, nb);
    for (int pnl = 0; pnl + 1 < nb; ++pnl) {
      if (br[pnl + 1] <= br[pnl]) continue;
      for (int gz = 0; gz < GEO_GLT; ++gz) {
        double th, wth;
        sin2_node(glt, gz, br[pnl], br[pnl + 1], &th, &wth);
        const double z = cz + R * cos(th), rho = R * sin(th);
        const double wz = wth * rho;
        if (rho <= 0.0) continue;
        double aa0[4], aa1[4];
        const int narc = square_arcs(cx, cy, rho, aa0, aa1);
        for (int a = 0; a < narc; ++a) {
          const int npc = (int)ceil((aa1[a] - aa0[a]) / (0.25 * M_PI));
          const double span = (aa1[a] - aa0[a]) / npc, hw = 0.5 * span;
          const int M = npc * GEO_GL;
          for (int base = 0; base < M; base += 32) {
            const int j = base + lane;
            double x = 0, y = 0, n0 = 0, n1 = 0, n2 = 0, wv = 0, g0 = 0, g1 = 0, g2 = 0;
            if (j < M) {
              const int pc = j / GEO_GL, g = j % GEO_GL;
              const double ph = aa0[a] + (pc + 0.5) * span + hw * gl.x[g];
              const double w = wz * gl.w[g] * hw * R;
              const double cp = cos(ph), sp = sin(ph);
              const double ex = rho * cp, ey = rho * sp, ez = z - cz;
              x = cx + ex;
              y = cy + ey;
              n0 = ex / R;
              n1 = ey / R;
              n2 = ez / R;
              const double X[3] = {C[0] + h * ex, C[1] + h * ey, C[2] + h * ez};
              double gv[3];
              const double V = shape_speed(sv, B.inside, b, X, 3, gv);
              const double gn = gv[0] * n0 + gv[1] * n1 + gv[2] * n2;
              wv = w * V;
              g0 = w * h * (gv[0] - gn * n0);
              g1 = w * h * (gv[1] - gn * n1);
              g2 = w * h * (gv[2] - gn * n2);
            }
            const int cnt = min(32, M - base);
            for (int q = 0; q < cnt; ++q) {
              const double qx = __shfl_sync(0xffffffffu, x, q), qy = __shfl_sync(0xffffffffu, y, q);
              const double q0 = __shfl_sync(0xffffffffu, n0, q), q1 = __shfl_sync(0xffffffffu, n1, q);
              const double q2 = __shfl_sync(0xffffffffu, n2, q), qw = __shfl_sync(0xffffffffu, wv, q);
              const double r0 = __shfl_sync(0xffffffffu, g0, q), r1 = __shfl_sync(0xffffffffu, g1, q);
              const double r2 = __shfl_sync(0xffffffffu, g2, q);
              patch_node(qx, qy, z, q0, q1, q2, qw, r0, r1, r2, e0, a0);
              if (own1) patch_node(qx, qy, z, q0, q1, q2, qw, r0, r1, r2, e1, a1);
            }
          }
        }
      }
    }
    // the edges: the arcs of the circles on the cell's face planes inside the faces; V_e dl / h = V wl,
    // wl = -(N . n_p) R dt
    const double cc[3] = {cx, cy, cz};
    for (int dd = 0; dd < 3; ++dd) {
      const int u = dd == 0 ? 1 : 0, v = dd == 2 ? 1 : 2;
      for (int s = -1; s <= 1; s += 2) {
        const double e = 0.5 * s, dn = e - cc[dd], r2 = R * R - dn * dn;
        if (!(r2 > 0.0)) continue;
        const double rho = sqrt(r2), en = s * dn / R;
        double aa0[4], aa1[4];
        const int narc = square_arcs(cc[u], cc[v], rho, aa0, aa1);
        for (int a = 0; a < narc; ++a) {
          const int npc = (int)ceil((aa1[a] - aa0[a]) / (0.25 * M_PI));
          const double span = (aa1[a] - aa0[a]) / npc, hw = 0.5 * span;
          const int M = npc * GEO_GL;
          for (int base = 0; base < M; base += 32) {
            const int j = base + lane;
            double p[3] = {0, 0, 0}, nv[3] = {0, 0, 0}, we = 0;
            if (j < M) {
              const int pc = j / GEO_GL, g = j % GEO_GL;
              const double tt = aa0[a] + (pc + 0.5) * span + hw * gl.x[g];
              p[dd] = e;
              p[u] = cc[u] + rho * cos(tt);
              p[v] = cc[v] + rho * sin(tt);
              for (int k = 0; k < 3; ++k) nv[k] = (p[k] - cc[k]) / R;
              const double X[3] = {C[0] + h * R * nv[0], C[1] + h * R * nv[1], C[2] + h * R * nv[2]};
              double gv[3];
              we = shape_speed(sv, B.inside, b, X, 3, gv) * (-en * R * gl.w[g] * hw);
            }
            const int cnt = min(32, M - base);
            for (int q = 0; q < cnt; ++q) {
              const double px = __shfl_sync(0xffffffffu, p[0], q), py = __shfl_sync(0xffffffffu, p[1], q);
              const double pz = __shfl_sync(0xffffffffu, p[2], q), q0 = __shfl_sync(0xffffffffu, nv[0], q);
              const double q1 = __shfl_sync(0xffffffffu, nv[1], q), q2 = __shfl_sync(0xffffffffu, nv[2], q);
              const double qw = __shfl_sync(0xffffffffu, we, q);
              double f, gN;
              mono_grad(e0, px, py, pz, q0, q1, q2, &f, &gN);
              a0[1] = fma(qw, f, a0[1]);
              a0[2] = fma(sgn * qw * q0, f, a0[2]);
              a0[3] = fma(sgn * qw * q1, f, a0[3]);
              a0[4] = fma(sgn * qw * q2, f, a0[4]);
              if (own1) {
                mono_grad(e1, px, py, pz, q0, q1, q2, &f, &gN);
                a1[1] = fma(qw, f, a1[1]);
                a1[2] = fma(sgn * qw * q0, f, a1[2]);
                a1[3] = fma(sgn * qw * q1, f, a1[3]);
                a1[4] = fma(sgn * qw * q2, f, a1[4]);
              }
            }
          }
        }
      }
    }
    for (int k = 0; k < 5; ++k) {
      a0[k] /= h;
      a1[k] /= h;
    }
  }
  if (lane < K) {
    dvol[t * K + lane] = a0[0];
    deb[t * K + lane] = a0[1];
    for (int d = 0; d < 3; ++d) debn[(t * 3 + d) * K + lane] = a0[2 + d];
  }
  if (own1) {
    dvol[t * K + lane + 32] = a1[0];
    deb[t * K + lane + 32] = a1[1];
    for (int d = 0; d < 3; ++d) debn[(t * 3 + d) * K + lane + 32] = a1[2 + d];
  }
}

// derivative of the tangential moments of the cut faces normal to dir (thread per face)
__global__ void k_sphere_faces_dv(Spheres B, GlRule gl, int N, int dir, double h, ShapeVel sv,
                                  const int32_t* __restrict__ faces, int64_t n, const int32_t* __restrict__ fbody,
                                  int q, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int f = faces[t];
  const int b = fbody[f];
  const int K2 = (q + 1) * (q + 2) / 2;
  double acc[28];
  for (int k = 0; k < K2; ++k) acc[k] = 0.0;
  if (shape_moves(sv, b)) {
    const int m0 = N + (dir == 0), m1 = N + (dir == 1);
    const int i3[3] = {f % m0, (f / m0) % m1, f / (m0 * m1)};
    const int u = dir == 0 ? 1 : 0, v = dir == 2 ? 1 : 2;
    const double dn = (i3[dir] * h - B.c[b][dir]) / h;
    const double cu = (B.c[b][u] - (i3[u] + 0.5) * h) / h, cv = (B.c[b][v] - (i3[v] + 0.5) * h) / h;
    const double R = B.r[b] / h, r2 = R * R - dn * dn;
    if (r2 > 0.0) {
      const double rho = sqrt(r2), sg = B.inside ? 1.0 : -1.0;
      double a0[4], a1[4];
      const int narc = square_arcs(cu, cv, rho, a0, a1);
      for (int a = 0; a < narc; ++a) {
        const int npc = (int)ceil((a1[a] - a0[a]) / (0.25 * M_PI));
        const double span = (a1[a] - a0[a]) / npc;
        for (int pc = 0; pc < npc; ++pc) {
          const double mm = a0[a] + (pc + 0.5) * span, hw = 0.5 * span;
          for (int g = 0; g < GEO_GL; ++g) {
            const double tt = mm + hw * gl.x[g];
            const double uu = cu + rho * cos(tt), vv = cv + rho * sin(tt);
            double X[3], gv[3];
            X[dir] = i3[dir] * h;
            X[u] = (i3[u] + 0.5) * h + h * uu;
            X[v] = (i3[v] + 0.5) * h + h * vv;
            // the rim moves with V R / rho; dl / h = rho dt
            const double c0 = sg * shape_speed(sv, B.inside, b, X, 3, gv) * R * gl.w[g] * hw;
            double up[GEO_MAXQ + 1], vp[GEO_MAXQ + 1];
            up[0] = vp[0] = 1.0;
            for (int k = 1; k <= q; ++k) {
              up[k] = up[k - 1] * uu;
              vp[k] = vp[k - 1] * vv;
            }
            for (int k = 0; k < K2; ++k) {
              int pa, pb;
              mon2(k, &pa, &pb);
              acc[k] += c0 * up[pa] * vp[pb];
            }
          }
        }
      }
    }
    for (int k = 0; k < K2; ++k) acc[k] /= h;
  }
  for (int k = 0; k < K2; ++k) out[t * K2 + k] = acc[k];
}

}  // namespace eb

using namespace eb;

namespace eb {
int geometry_bodies(const eb_geometry* g) { return g->n_body; }
int64_t geometry_cutfaces(const eb_geometry* g, int d) { return g->desc.n_cutface[d]; }
bool geometry_matches(const eb_geometry* g, int dim, const int* n, int n_cut) {
  const eb_geom& d = g->desc;
  return d.dim == dim && d.n[0] == n[0] && d.n[1] == n[1] && (dim < 3 || d.n[2] == n[2]) && d.n_cut == n_cut;
}

// derivatives of the moment tables of a device geometry for the boundary velocity sv, into caller arrays
// laid out like the tables (dface[d]: [n_cutface[d]][K_F]); stream-ordered
cudaError_t geometry_shape_derivative(const eb_geometry* g, const ShapeVel& sv, double* dvol, double* deb,
                                      double* debn, double* const* dface, cudaStream_t s) {
  static const GlRule gl = gl_rule<GEO_GL>();
  static const GlRuleT glt = gl_rule<GEO_GLT>();
  const eb_geom& d = g->desc;
  if ((sv.kind == 0 && (sv.body < 0 || sv.body >= g->n_body)) || sv.kind < 0 || sv.kind > 1)
    return cudaErrorInvalidValue;
  const int q = d.moment_degree;
  const int N = d.n[0];
  const double h = d.h;
  if (d.dim == 2) {
    Circles B;
    B.n = g->n_body;
    B.inside = g->inside;
    for (int b = 0; b < g->n_body; ++b) {
      B.c[b][0] = g->centers[b][0];
      B.c[b][1] = g->centers[b][1];
      B.r[b] = g->radii[b];
    }
    const int K = (q + 1) * (q + 2) / 2;
    if (d.n_cut > 0) {
      k_circle_cells_dv<<<(unsigned)((d.n_cut + 127) / 128), 128, 0, s>>>(B, gl, N, h, sv, d.cut_cell, d.n_cut,
                                                                         g->cell_body, q, K, dvol, deb, debn);
      eb::count_launch();
    }
    for (int dir = 0; dir < 2; ++dir) {
      if (d.n_cutface[dir] == 0) continue;
      k_circle_faces_dv<<<(unsigned)((d.n_cutface[dir] + 127) / 128), 128, 0, s>>>(
          B, N, dir, h, sv, d.cutface[dir], d.n_cutface[dir], g->face_body[dir], q, dface[dir]);
      eb::count_launch();
    }
    return cudaGetLastError();
  }
  Spheres B;
  B.n = g->n_body;
  B.inside = g->inside;
  for (int b = 0; b < g->n_body; ++b) {
    for (int k = 0; k < 3; ++k) B.c[b][k] = g->centers[b][k];
    B.r[b] = g->radii[b];
  }
  if (d.n_cut > 0) {
    const unsigned nb = (unsigned)((32 * (int64_t)d.n_cut + 127) / 128);  // a warp per cut cell
    const int64_t nc = d.n_cut;
    switch (q) {
      case 0: k_sphere_cells_dw<0><<<nb, 128, 0, s>>>(B, gl, glt, N, h, sv, d.cut_cell, nc, g->cell_body, dvol, deb, debn); break;
      case 1: k_sphere_cells_dw<1><<<nb, 128, 0, s>>>(B, gl, glt, N, h, sv, d.cut_cell, nc, g->cell_body, dvol, deb, debn); break;
      case 2: k_sphere_cells_dw<2><<<nb, 128, 0, s>>>(B, gl, glt, N, h, sv, d.cut_cell, nc, g->cell_body, dvol, deb, debn); break;
      case 3: k_sphere_cells_dw<3><<<nb, 128, 0, s>>>(B, gl, glt, N, h, sv, d.cut_cell, nc, g->cell_body, dvol, deb, debn); break;
      default: k_sphere_cells_dw<4><<<nb, 128, 0, s>>>(B, gl, glt, N, h, sv, d.cut_cell, nc, g->cell_body, dvol, deb, debn); break;
    }
    eb::count_launch();
  }
  for (int dir = 0; dir < 3; ++dir) {
    if (d.n_cutface[dir] == 0) continue;
    k_sphere_faces_dv<<<(unsigned)((d.n_cutface[dir] + 127) / 128), 128, 0, s>>>(
        B, gl, N, dir, h, sv, d.cutface[dir], d.n_cutface[dir], g->face_body[dir], q, dface[dir]);
    eb::count_launch();
  }
  return cudaGetLastError();
}
}  // namespace eb

namespace {

unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

// device allocations of one call: the geometry's own arrays (kept) and temporaries (freed at the end)
struct GeoAlloc {
  cudaStream_t s;
  eb_geometry* g;
  std::vector<void*> tmp;
  ~GeoAlloc() {
    for (void* p : tmp) cudaFreeAsync(p, s);
  }
  template <typename T>
  cudaError_t keep(T** p, int64_t n) {
    cudaError_t e = cudaMallocAsync((void**)p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), s);
    if (e == cudaSuccess) g->allocs.push_back(*p);
    return e;
  }
  template <typename T>
  cudaError_t temp(T** p, int64_t n) {
    cudaError_t e = cudaMallocAsync((void**)p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), s);
    if (e == cudaSuccess) tmp.push_back(*p);
    return e;
  }
};

// exclusive scan of sel[0..n) into pos, returning the total (synchronises the stream)
cudaError_t geo_scan(const int32_t* sel, int64_t n, int64_t* pos, int64_t* total, GeoAlloc& A) {
  const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  *total = 0;
  if (nb == 0) return cudaSuccess;
  int64_t *sums, *dtot;
  cudaError_t e;
  if ((e = A.temp(&sums, nb)) || (e = A.temp(&dtot, 1))) return e;
  k_scan_block_sums<int32_t><<<(unsigned)nb, SCAN_BLOCK, 0, A.s>>>(sel, n, sums);
  k_scan_single<<<1, SCAN_BLOCK, 0, A.s>>>(sums, nb, dtot);
  k_scan_apply<int32_t><<<(unsigned)nb, SCAN_BLOCK, 0, A.s>>>(sel, n, sums, pos);
  eb::count_launch();
  eb::count_launch();
  eb::count_launch();
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(total, dtot, 8, cudaMemcpyDeviceToHost, A.s))) return e;
  return cudaStreamSynchronize(A.s);
}

// list of the indices i < n with flag[i] == v, ascending
cudaError_t geo_list(const uint8_t* flag, int64_t n, uint8_t v, int32_t** list, int64_t* count, GeoAlloc& A,
                     bool keep) {
  int32_t* sel;
  int64_t* pos;
  cudaError_t e;
  if ((e = A.temp(&sel, n)) || (e = A.temp(&pos, n))) return e;
  k_geo_is<<<nb256(n), 256, 0, A.s>>>(flag, n, v, sel);
  eb::count_launch();
  if ((e = geo_scan(sel, n, pos, count, A))) return e;
  if ((e = keep ? A.keep(list, *count) : A.temp(list, *count))) return e;
  k_geo_compact<<<nb256(n), 256, 0, A.s>>>(sel, pos, n, *list);
  eb::count_launch();
  return cudaGetLastError();
}

int mono_count(int dim, int q) {
  int n = 0;
  for (int d = 0; d <= q; ++d) n += dim == 1 ? 1 : (dim == 2 ? d + 1 : (d + 1) * (d + 2) / 2);
  return n;
}

}  // namespace

extern "C" eb_status eb_geometry_circles(int32_t N, int32_t n_body, const double* centers_host,
                                         const double* radii_host, int32_t inside, int32_t moment_degree,
                                         eb_geometry** out, eb_geom* desc, eb_stream_t stream) {
  if (!out || !desc) { set_error("eb_geometry_circles: out and desc are required"); return EB_ERR_INVALID; }
  *out = nullptr;
  if (N < 2 || n_body < 0 || n_body > GEO_MAXB || (n_body > 0 && (!centers_host || !radii_host)) ||
      moment_degree < 0 || moment_degree > GEO_MAXQ || (inside && n_body != 1)) {
    set_error("eb_geometry_circles: N >= 2, 0 <= n_body <= 64 (exactly 1 when inside), moment_degree in 0..6");
    return EB_ERR_INVALID;
  }
  Circles B;
  B.n = n_body;
  B.inside = inside ? 1 : 0;
  for (int b = 0; b < n_body; ++b) {
    B.c[b][0] = centers_host[2 * b];
    B.c[b][1] = centers_host[2 * b + 1];
    B.r[b] = radii_host[b];
    if (!(B.r[b] > 0.0)) { set_error("eb_geometry_circles: radii must be positive"); return EB_ERR_INVALID; }
  }
  static const GlRule gl = gl_rule<GEO_GL>();
  const double h = 1.0 / N;
  const int q = moment_degree, K = mono_count(2, q), KF = q + 1;
  cudaStream_t s = (cudaStream_t)stream;
  eb_geometry* G = new eb_geometry();
  eb_status st = EB_OK;
  cudaError_t e = cudaSuccess;
  {
    GeoAlloc A{s, G, {}};
    const int64_t ncell = (int64_t)N * N;
    uint8_t* cflag;
    int32_t *cbody, *err;
#define GEO_TRY(x)                                 \
  do {                                             \
    if ((e = (x)) != cudaSuccess) goto cuda_fail;  \
  } while (0)
    GEO_TRY(A.keep(&cflag, ncell));
    GEO_TRY(A.keep(&cbody, ncell));
    G->cell_body = cbody;
    GEO_TRY(A.temp(&err, 1));
    GEO_TRY(cudaMemsetAsync(err, 0, 4, s));
    k_geo_classify2<<<nb256(ncell), 256, 0, s>>>(B, N, N, h, -1, ncell, cflag, cbody, err);
    eb::count_launch();
    {
      // cut cells: moments, then the volume-fraction ends
      int32_t* cut0;
      int64_t nc0 = 0;
      GEO_TRY(geo_list(cflag, ncell, 2, &cut0, &nc0, A, false));
      int32_t herr = 0;
      GEO_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
      GEO_TRY(cudaStreamSynchronize(s));
      if (herr) {
        st = EB_ERR_MULTIVALUED;
        set_error("eb_geometry_circles: two circles reach into one cell or face");
        goto done;
      }
      GeoOut2 o0;
      o0.q = q;
      o0.K = K;
      GEO_TRY(A.temp(&o0.vol, nc0 * K));
      GEO_TRY(A.temp(&o0.eb, nc0 * K));
      GEO_TRY(A.temp(&o0.ebn, nc0 * 2 * K));
      if (nc0 > 0) {
        k_circle_cells<<<nb256(nc0), 256, 0, s>>>(B, gl, N, h, cut0, nc0, cbody, o0);
        eb::count_launch();
      }
      int32_t* keep;
      int64_t* pos;
      int64_t nc = 0;
      GEO_TRY(A.temp(&keep, nc0));
      GEO_TRY(A.temp(&pos, nc0));
      if (nc0 > 0) {
        k_geo_settle<<<nb256(nc0), 256, 0, s>>>(cut0, nc0, o0.vol, K, cflag, keep);
        eb::count_launch();
      }
      GEO_TRY(geo_scan(keep, nc0, pos, &nc, A));
      int32_t* cut;
      double *vol, *ebm, *ebn;
      GEO_TRY(A.keep(&cut, nc));
      GEO_TRY(A.keep(&vol, nc * K));
      GEO_TRY(A.keep(&ebm, nc * K));
      GEO_TRY(A.keep(&ebn, nc * 2 * K));
      if (nc0 > 0) {
        k_geo_pack_idx<<<nb256(nc0), 256, 0, s>>>(keep, pos, nc0, cut0, cut);
        k_geo_pack<<<nb256(nc0 * K), 256, 0, s>>>(keep, pos, nc0, K, o0.vol, vol);
        k_geo_pack<<<nb256(nc0 * K), 256, 0, s>>>(keep, pos, nc0, K, o0.eb, ebm);
        k_geo_pack<<<nb256(nc0 * 2 * K), 256, 0, s>>>(keep, pos, nc0, 2 * K, o0.ebn, ebn);
        for (int i = 0; i < 4; ++i) eb::count_launch();
      }
      memset(desc, 0, sizeof(*desc));
      desc->dim = 2;
      desc->n[0] = desc->n[1] = N;
      desc->n[2] = 1;
      desc->h = h;
      desc->moment_degree = q;
      desc->cell_flag = cflag;
      desc->n_cut = (int32_t)nc;
      desc->cut_cell = cut;
      desc->vol_mom = vol;
      desc->eb_mom = ebm;
      desc->eb_nmom = ebn;
      desc->eb_bc = nullptr;
    }
    // faces
    for (int d = 0; d < 2; ++d) {
      const int64_t nf = (int64_t)(N + (d == 0)) * (N + (d == 1));
      uint8_t* ff;
      int32_t* fbody;
      GEO_TRY(A.keep(&ff, nf));
      GEO_TRY(A.keep(&fbody, nf));
      G->face_body[d] = fbody;
      GEO_TRY(cudaMemsetAsync(err, 0, 4, s));
      k_geo_classify2<<<nb256(nf), 256, 0, s>>>(B, N, N, h, d, nf, ff, fbody, err);
      eb::count_launch();
      int32_t* cf0;
      int64_t nf0 = 0;
      GEO_TRY(geo_list(ff, nf, 2, &cf0, &nf0, A, false));
      int32_t herr = 0;
      GEO_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
      GEO_TRY(cudaStreamSynchronize(s));
      if (herr) {
        st = EB_ERR_MULTIVALUED;
        set_error("eb_geometry_circles: two circles reach into one cell or face");
        goto done;
      }
      double* fm0;
      GEO_TRY(A.temp(&fm0, nf0 * KF));
      int32_t* keep;
      int64_t* pos;
      int64_t nfc = 0;
      GEO_TRY(A.temp(&keep, nf0));
      GEO_TRY(A.temp(&pos, nf0));
      if (nf0 > 0) {
        k_circle_faces<<<nb256(nf0), 256, 0, s>>>(B, N, d, h, cf0, nf0, fbody, q, fm0);
        k_geo_settle<<<nb256(nf0), 256, 0, s>>>(cf0, nf0, fm0, KF, ff, keep);
        eb::count_launch();
        eb::count_launch();
      }
      k_geo_close_faces<<<nb256(nf), 256, 0, s>>>(cflag, N, N, d, nf, ff);
      eb::count_launch();
      if (nf0 > 0) {
        k_geo_keep_open<<<nb256(nf0), 256, 0, s>>>(cf0, nf0, ff, keep);
        eb::count_launch();
      }
      GEO_TRY(geo_scan(keep, nf0, pos, &nfc, A));
      int32_t* cf;
      double* fm;
      GEO_TRY(A.keep(&cf, nfc));
      GEO_TRY(A.keep(&fm, nfc * KF));
      if (nf0 > 0) {
        k_geo_pack_idx<<<nb256(nf0), 256, 0, s>>>(keep, pos, nf0, cf0, cf);
        k_geo_pack<<<nb256(nf0 * KF), 256, 0, s>>>(keep, pos, nf0, KF, fm0, fm);
        eb::count_launch();
        eb::count_launch();
      }
      desc->face_flag[d] = ff;
      desc->n_cutface[d] = (int32_t)nfc;
      desc->cutface[d] = cf;
      desc->face_mom[d] = fm;
    }
    GEO_TRY(cudaGetLastError());
    GEO_TRY(cudaStreamSynchronize(s));
    goto done;
  cuda_fail:
    st = e == cudaErrorMemoryAllocation ? EB_ERR_OOM : cuda_status(e, "eb_geometry_circles");
  done:;
#undef GEO_TRY
  }
  if (st != EB_OK) {
    eb_geometry_destroy(G);
    memset(desc, 0, sizeof(*desc));
    return st;
  }
  G->desc = *desc;
  G->n_body = n_body;
  G->inside = B.inside;
  for (int b = 0; b < n_body; ++b) {
    G->centers[b][0] = B.c[b][0];
    G->centers[b][1] = B.c[b][1];
    G->radii[b] = B.r[b];
  }
  *out = G;
  return EB_OK;
}

extern "C" eb_status eb_geometry_spheres(int32_t N, int32_t n_body, const double* centers_host,
                                         const double* radii_host, int32_t inside, int32_t moment_degree,
                                         eb_geometry** out, eb_geom* desc, eb_stream_t stream) {
  if (!out || !desc) { set_error("eb_geometry_spheres: out and desc are required"); return EB_ERR_INVALID; }
  *out = nullptr;
  if (N < 2 || N > 1290 || n_body < 0 || n_body > GEO_MAXB || (n_body > 0 && (!centers_host || !radii_host)) ||
      moment_degree < 0 || moment_degree > 4 || (inside && n_body != 1)) {
    set_error("eb_geometry_spheres: 2 <= N <= 1290, 0 <= n_body <= 64 (exactly 1 when inside), moment_degree in 0..4");
    return EB_ERR_INVALID;
  }
  Spheres B;
  B.n = n_body;
  B.inside = inside ? 1 : 0;
  for (int b = 0; b < n_body; ++b) {
    for (int d = 0; d < 3; ++d) B.c[b][d] = centers_host[3 * b + d];
    B.r[b] = radii_host[b];
    if (!(B.r[b] > 0.0)) { set_error("eb_geometry_spheres: radii must be positive"); return EB_ERR_INVALID; }
  }
  static const GlRule gl = gl_rule<GEO_GL>();
  static const GlRuleT glt = gl_rule<GEO_GLT>();
  const double h = 1.0 / N;
  const int q = moment_degree, K = mono_count(3, q), KF = mono_count(2, q);
  cudaStream_t s = (cudaStream_t)stream;
  eb_geometry* G = new eb_geometry();
  eb_status st = EB_OK;
  cudaError_t e = cudaSuccess;
  {
    GeoAlloc A{s, G, {}};
    const int64_t ncell = (int64_t)N * N * N;
    uint8_t* cflag;
    int32_t *cbody, *err;
#define GEO_TRY(x)                                 \
  do {                                             \
    if ((e = (x)) != cudaSuccess) goto cuda_fail;  \
  } while (0)
    GEO_TRY(A.keep(&cflag, ncell));
    GEO_TRY(A.keep(&cbody, ncell));
    G->cell_body = cbody;
    GEO_TRY(A.temp(&err, 1));
    GEO_TRY(cudaMemsetAsync(err, 0, 4, s));
    k_geo_classify3<<<nb256(ncell), 256, 0, s>>>(B, N, h, -1, ncell, cflag, cbody, err);
    eb::count_launch();
    {
      int32_t* cut0;
      int64_t nc0 = 0;
      GEO_TRY(geo_list(cflag, ncell, 2, &cut0, &nc0, A, false));
      int32_t herr = 0;
      GEO_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
      GEO_TRY(cudaStreamSynchronize(s));
      if (herr) {
        st = EB_ERR_MULTIVALUED;
        set_error("eb_geometry_spheres: two spheres reach into one cell or face");
        goto done;
      }
      double *vol0, *eb0, *ebn0, *volp;
      GEO_TRY(A.temp(&vol0, nc0 * K));
      GEO_TRY(A.temp(&eb0, nc0 * K));
      GEO_TRY(A.temp(&ebn0, nc0 * 3 * K));
      GEO_TRY(A.temp(&volp, nc0 * K));
      if (nc0 > 0) {
        switch (q) {
          case 0: k_sphere_patch<0><<<nb256(5 * nc0), 256, 0, s>>>(B, gl, glt, N, h, cut0, nc0, cbody, eb0, ebn0, volp); break;
          case 1: k_sphere_patch<1><<<nb256(5 * nc0), 256, 0, s>>>(B, gl, glt, N, h, cut0, nc0, cbody, eb0, ebn0, volp); break;
          case 2: k_sphere_patch<2><<<nb256(5 * nc0), 256, 0, s>>>(B, gl, glt, N, h, cut0, nc0, cbody, eb0, ebn0, volp); break;
          case 3: k_sphere_patch<3><<<nb256(5 * nc0), 256, 0, s>>>(B, gl, glt, N, h, cut0, nc0, cbody, eb0, ebn0, volp); break;
          default: k_sphere_patch<4><<<nb256(5 * nc0), 256, 0, s>>>(B, gl, glt, N, h, cut0, nc0, cbody, eb0, ebn0, volp); break;
        }
        k_sphere_vol<<<nb256(nc0), 256, 0, s>>>(B, glt, N, h, cut0, nc0, cbody, q, K, volp, vol0);
        eb::count_launch();
        eb::count_launch();
      }
      int32_t* keep;
      int64_t* pos;
      int64_t nc = 0;
      GEO_TRY(A.temp(&keep, nc0));
      GEO_TRY(A.temp(&pos, nc0));
      if (nc0 > 0) {
        k_geo_settle<<<nb256(nc0), 256, 0, s>>>(cut0, nc0, vol0, K, cflag, keep);
        eb::count_launch();
      }
      GEO_TRY(geo_scan(keep, nc0, pos, &nc, A));
      int32_t* cut;
      double *vol, *ebm, *ebn;
      GEO_TRY(A.keep(&cut, nc));
      GEO_TRY(A.keep(&vol, nc * K));
      GEO_TRY(A.keep(&ebm, nc * K));
      GEO_TRY(A.keep(&ebn, nc * 3 * K));
      if (nc0 > 0) {
        k_geo_pack_idx<<<nb256(nc0), 256, 0, s>>>(keep, pos, nc0, cut0, cut);
        k_geo_pack<<<nb256(nc0 * K), 256, 0, s>>>(keep, pos, nc0, K, vol0, vol);
        k_geo_pack<<<nb256(nc0 * K), 256, 0, s>>>(keep, pos, nc0, K, eb0, ebm);
        k_geo_pack<<<nb256(nc0 * 3 * K), 256, 0, s>>>(keep, pos, nc0, 3 * K, ebn0, ebn);
        for (int i = 0; i < 4; ++i) eb::count_launch();
      }
      memset(desc, 0, sizeof(*desc));
      desc->dim = 3;
      desc->n[0] = desc->n[1] = desc->n[2] = N;
      desc->h = h;
      desc->moment_degree = q;
      desc->cell_flag = cflag;
      desc->n_cut = (int32_t)nc;
      desc->cut_cell = cut;
      desc->vol_mom = vol;
      desc->eb_mom = ebm;
      desc->eb_nmom = ebn;
      desc->eb_bc = nullptr;
    }
    for (int d = 0; d < 3; ++d) {
      const int64_t nf = (int64_t)(N + (d == 0)) * (N + (d == 1)) * (N + (d == 2));
      uint8_t* ff;
      int32_t* fbody;
      GEO_TRY(A.keep(&ff, nf));
      GEO_TRY(A.keep(&fbody, nf));
      G->face_body[d] = fbody;
      GEO_TRY(cudaMemsetAsync(err, 0, 4, s));
      k_geo_classify3<<<nb256(nf), 256, 0, s>>>(B, N, h, d, nf, ff, fbody, err);
      eb::count_launch();
      int32_t* cf0;
      int64_t nf0 = 0;
      GEO_TRY(geo_list(ff, nf, 2, &cf0, &nf0, A, false));
      int32_t herr = 0;
      GEO_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
      GEO_TRY(cudaStreamSynchronize(s));
      if (herr) {
        st = EB_ERR_MULTIVALUED;
        set_error("eb_geometry_spheres: two spheres reach into one cell or face");
        goto done;
      }
      double* fm0;
      GEO_TRY(A.temp(&fm0, nf0 * KF));
      int32_t* keep;
      int64_t* pos;
      int64_t nfc = 0;
      GEO_TRY(A.temp(&keep, nf0));
      GEO_TRY(A.temp(&pos, nf0));
      if (nf0 > 0) {
        k_sphere_faces<<<nb256(nf0), 256, 0, s>>>(B, glt, N, d, h, cf0, nf0, fbody, q, fm0);
        k_geo_settle<<<nb256(nf0), 256, 0, s>>>(cf0, nf0, fm0, KF, ff, keep);
        eb::count_launch();
        eb::count_launch();
      }
      k_geo_close_faces3<<<nb256(nf), 256, 0, s>>>(cflag, N, d, nf, ff);
      eb::count_launch();
      if (nf0 > 0) {
        k_geo_keep_open<<<nb256(nf0), 256, 0, s>>>(cf0, nf0, ff, keep);
        eb::count_launch();
      }
      GEO_TRY(geo_scan(keep, nf0, pos, &nfc, A));
      int32_t* cf;
      double* fm;
      GEO_TRY(A.keep(&cf, nfc));
      GEO_TRY(A.keep(&fm, nfc * KF));
      if (nf0 > 0) {
        k_geo_pack_idx<<<nb256(nf0), 256, 0, s>>>(keep, pos, nf0, cf0, cf);
        k_geo_pack<<<nb256(nf0 * KF), 256, 0, s>>>(keep, pos, nf0, KF, fm0, fm);
        eb::count_launch();
        eb::count_launch();
      }
      desc->face_flag[d] = ff;
      desc->n_cutface[d] = (int32_t)nfc;
      desc->cutface[d] = cf;
      desc->face_mom[d] = fm;
    }
    GEO_TRY(cudaGetLastError());
    GEO_TRY(cudaStreamSynchronize(s));
    goto done;
  cuda_fail:
    st = e == cudaErrorMemoryAllocation ? EB_ERR_OOM : cuda_status(e, "eb_geometry_spheres");
  done:;
#undef GEO_TRY
  }
  if (st != EB_OK) {
    eb_geometry_destroy(G);
    memset(desc, 0, sizeof(*desc));
    return st;
  }
  G->desc = *desc;
  G->n_body = n_body;
  G->inside = B.inside;
  for (int b = 0; b < n_body; ++b) {
    for (int d = 0; d < 3; ++d) G->centers[b][d] = B.c[b][d];
    G->radii[b] = B.r[b];
  }
  *out = G;
  return EB_OK;
}

extern "C" void eb_geometry_destroy(eb_geometry* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  for (void* p : g->allocs) cudaFree(p);
  delete g;
}

extern "C" eb_status eb_geometry_table(const eb_geometry* g, int32_t which, int32_t dir, void* dst_host,
                                       int64_t cap_bytes, int64_t* bytes) {
  if (!g || !bytes) { set_error("eb_geometry_table: null argument"); return EB_ERR_INVALID; }
  const eb_geom& d = g->desc;
  const int D = d.dim;
  int64_t ncell = 1;
  for (int k = 0; k < D; ++k) ncell *= d.n[k];
  auto mons = [](int dim, int q) {
    int n = 0;
    for (int k = 0; k <= q; ++k) n += dim <= 1 ? 1 : (dim == 2 ? k + 1 : (k + 1) * (k + 2) / 2);
    return n;
  };
  const int KS = mons(D, d.moment_degree), KF = mons(D - 1, d.moment_degree);
  if ((which >= EB_TABLE_FACE_FLAG) && (dir < 0 || dir >= D)) { set_error("eb_geometry_table: dir"); return EB_ERR_INVALID; }
  const void* src = nullptr;
  int64_t nb = 0;
  switch (which) {
    case EB_TABLE_CELL_FLAG: src = d.cell_flag; nb = ncell; break;
    case EB_TABLE_CUT_CELL: src = d.cut_cell; nb = (int64_t)d.n_cut * 4; break;
    case EB_TABLE_VOL_MOM: src = d.vol_mom; nb = (int64_t)d.n_cut * KS * 8; break;
    case EB_TABLE_EB_MOM: src = d.eb_mom; nb = (int64_t)d.n_cut * KS * 8; break;
    case EB_TABLE_EB_NMOM: src = d.eb_nmom; nb = (int64_t)d.n_cut * D * KS * 8; break;
    case EB_TABLE_FACE_FLAG: {
      int64_t nf = 1;
      for (int k = 0; k < D; ++k) nf *= d.n[k] + (k == dir);
      src = d.face_flag[dir];
      nb = nf;
      break;
    }
    case EB_TABLE_CUTFACE: src = d.cutface[dir]; nb = (int64_t)d.n_cutface[dir] * 4; break;
    case EB_TABLE_FACE_MOM: src = d.face_mom[dir]; nb = (int64_t)d.n_cutface[dir] * KF * 8; break;
    default: set_error("eb_geometry_table: unknown table"); return EB_ERR_INVALID;
  }
  *bytes = nb;
  if (!dst_host) return EB_OK;
  if (cap_bytes < nb) { set_error("eb_geometry_table: destination too small"); return EB_ERR_INVALID; }
  if (nb > 0) EB_CUDA(cudaMemcpy(dst_host, src, (size_t)nb, cudaMemcpyDeviceToHost));
  return EB_OK;
}

extern "C" eb_status eb_geometry_shape_table(const eb_geometry* g, int32_t kind, int32_t body, const double* mode_host,
                                             int32_t which, int32_t dir, double* dst_host, int64_t cap_bytes,
                                             int64_t* bytes) {
  if (!g || !bytes) { set_error("eb_geometry_shape_table: null argument"); return EB_ERR_INVALID; }
  const eb_geom& d = g->desc;
  const int D = d.dim, q = d.moment_degree;
  const int KS = D == 2 ? (q + 1) * (q + 2) / 2 : (q + 1) * (q + 2) * (q + 3) / 6;
  const int KF = D == 2 ? q + 1 : (q + 1) * (q + 2) / 2;
  ShapeVel sv;
  memset(&sv, 0, sizeof(sv));
  sv.kind = kind;
  sv.body = body;
  if (kind == 1) {
    if (!mode_host) { set_error("eb_geometry_shape_table: the mode is required"); return EB_ERR_INVALID; }
    for (int k = 0; k < 3; ++k) sv.k[k] = mode_host[k];
    sv.theta = mode_host[3];
  } else if (kind != 0 || body < 0 || body >= g->n_body) {
    set_error("eb_geometry_shape_table: kind 0 (radius of a body) or 1 (level-set mode)");
    return EB_ERR_INVALID;
  }
  if (which == EB_TABLE_FACE_MOM && (dir < 0 || dir >= D)) { set_error("eb_geometry_shape_table: dir"); return EB_ERR_INVALID; }
  int64_t nb = 0;
  switch (which) {
    case EB_TABLE_VOL_MOM: case EB_TABLE_EB_MOM: nb = (int64_t)d.n_cut * KS * 8; break;
    case EB_TABLE_EB_NMOM: nb = (int64_t)d.n_cut * D * KS * 8; break;
    case EB_TABLE_FACE_MOM: nb = (int64_t)d.n_cutface[dir] * KF * 8; break;
    default: set_error("eb_geometry_shape_table: volume, EB, normal EB or face moments"); return EB_ERR_INVALID;
  }
  *bytes = nb;
  if (!dst_host) return EB_OK;
  if (cap_bytes < nb) { set_error("eb_geometry_shape_table: destination too small"); return EB_ERR_INVALID; }
  const int64_t nc = std::max<int64_t>(1, d.n_cut);
  std::vector<void*> tmp;
  auto get = [&](int64_t n) -> double* {
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)n * 8) != cudaSuccess) return nullptr;
    tmp.push_back(p);
    return (double*)p;
  };
  double* dv = get(nc * KS);
  double* de = get(nc * KS);
  double* dn = get(nc * D * KS);
  double* df[3] = {nullptr, nullptr, nullptr};
  bool ok = dv && de && dn;
  for (int k = 0; k < D && ok; ++k) ok = (df[k] = get(std::max<int64_t>(1, d.n_cutface[k]) * KF)) != nullptr;
  cudaError_t e = ok ? geometry_shape_derivative(g, sv, dv, de, dn, df, 0) : cudaErrorMemoryAllocation;
  if (e == cudaSuccess && nb > 0) {
    const double* src = which == EB_TABLE_VOL_MOM ? dv : (which == EB_TABLE_EB_MOM ? de : (which == EB_TABLE_EB_NMOM ? dn : df[dir]));
    e = cudaMemcpy(dst_host, src, (size_t)nb, cudaMemcpyDeviceToHost);
  }
  for (void* p : tmp) cudaFree(p);
  if (e != cudaSuccess) { set_error(std::string("eb_geometry_shape_table: ") + cudaGetErrorString(e)); return e == cudaErrorMemoryAllocation ? EB_ERR_OOM : EB_ERR_CUDA; }
  return EB_OK;
}
