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
//   volume moments  the divergence theorem with the x-derivative,
//                   int_V xi^p = 1/(p_0+1) oint xi^(p+e_0) n_0: the fluid parts
//                   of the two x edges in closed form and the arcs.
// Cells whose volume fraction is at most 1e-14 count as covered and those at
// least 1 - 1e-14 as full, faces likewise; a face next to a covered cell is
// closed.  The lists of cut cells and cut faces are ascending.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

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

struct GlRule {
  double x[GEO_GL], w[GEO_GL];  // nodes and weights on [-1, 1]
};

// Gauss-Legendre rule by Newton's method on P_n (three-term recurrence), from the Chebyshev guesses
static GlRule gl_rule() {
  GlRule g;
  const int n = GEO_GL;
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
  double arcx[28];                         // int xi^(p + e_0) n_0 ds over the arcs
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
        double xp[GEO_MAXQ + 2], yp[GEO_MAXQ + 1];
        xp[0] = yp[0] = 1.0;
        for (int k = 1; k <= q + 1; ++k) xp[k] = xp[k - 1] * x;
        for (int k = 1; k <= q; ++k) yp[k] = yp[k - 1] * y;
        for (int k = 0; k < K; ++k) {
          int p0, p1;
          mon2(k, &p0, &p1);
          const double v = wt * xp[p0] * yp[p1];
          eb[k] += v;
          ebn[0][k] += v * n0;
          ebn[1][k] += v * n1;
          arcx[k] += wt * xp[p0 + 1] * yp[p1] * n0;
        }
      }
    }
  }
  // ---- volume moments: x edges (fluid intervals, closed form) and the arcs
  for (int s = -1; s <= 1; s += 2) {
    const double e = 0.5 * s;
    double ia[2], ib[2];
    const int ni = fluid_intervals(e - cx, cy, R, inside, ia, ib);
    for (int j = 0; j < ni; ++j) {
      double sp[GEO_MAXQ + 1];
      seg_powers(ia[j], ib[j], q, sp);
      for (int k = 0; k < K; ++k) {
        int p0, p1;
        mon2(k, &p0, &p1);
        vol[k] += s * pow(e, p0 + 1) * sp[p1];  // n_0 = s on the edge x = s/2
      }
    }
  }
  for (int k = 0; k < K; ++k) {
    int p0, p1;
    mon2(k, &p0, &p1);
    vol[k] = (vol[k] + arcx[k]) / (p0 + 1);
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

// ---------------------------------------------------------------- shape derivatives (radius)
//
// d/dr of the moment tables of the cells and faces cut by circle b, the fluid outside the circle (the
// boundary moves with unit normal speed into the fluid as r grows); the cut sets are held fixed:
//   volume moments  d/dr int_V xi^p dV / h^2 = - int_patch xi^p ds / h^2 = - eb / h   (transport);
//   EB moments      the arc {c + r e(t)}: d/dr int f r dt = int (r grad f . e + f) dt
//                   + f(t_b) r t_b' - f(t_a) r t_a', the ends sliding along the cell edges they lie on
//                   (t' = cos t / (r sin t) on an x edge, -sin t / (r cos t) on a y edge); the normal
//                   at fixed t does not turn;
//   face moments    the covered chord |t - c_t| < s, s = (r^2 - d^2)^(1/2), grows at both ends with
//                   speed r / s.
__global__ void k_circle_cells_dr(Circles B, GlRule gl, int nx, double h, int body, const int32_t* __restrict__ cells,
                                  int64_t n, const int32_t* __restrict__ cbody, const double* __restrict__ eb_mom,
                                  int q, int K, double* dvol, double* deb, double* debn) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int c = cells[t];
  double dv[28], de[28], dn[2][28];
  for (int k = 0; k < K; ++k) dv[k] = de[k] = dn[0][k] = dn[1][k] = 0.0;
  if (cbody[c] == body) {
    const int ix = c % nx, iy = c / nx;
    const double cx = (B.c[body][0] - (ix + 0.5) * h) / h, cy = (B.c[body][1] - (iy + 0.5) * h) / h;
    const double R = B.r[body] / h;
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
    const double sgn = B.inside ? 1.0 : -1.0;  // normal out of the fluid
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
          const double th = mm + hw * gl.x[g], wt = gl.w[g] * hw;  // d theta
          const double ct = cos(th), st = sin(th);
          const double x = cx + R * ct, y = cy + R * st;
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
            // R grad_xi f . e (the h of grad_x and of R cancel)
            double ge = 0.0;
            if (p0 > 0) ge += p0 * xp[p0 - 1] * yp[p1] * ct;
            if (p1 > 0) ge += p1 * xp[p0] * yp[p1 - 1] * st;
            const double v = wt * (R * ge + f);
            de[k] += v;
            dn[0][k] += v * sgn * ct;
            dn[1][k] += v * sgn * st;
          }
        }
      }
      // ends: + f(t_b) R t_b' - f(t_a) R t_a'
      for (int end = 0; end < 2; ++end) {
        const double th = end ? e : a, dth = end ? dE : da, sg = end ? 1.0 : -1.0;
        const double ct = cos(th), st = sin(th);
        const double x = cx + R * ct, y = cy + R * st;
        for (int k = 0; k < K; ++k) {
          int p0, p1;
          mon2(k, &p0, &p1);
          const double v = sg * pow(x, p0) * pow(y, p1) * R * dth;
          de[k] += v;
          dn[0][k] += v * sgn * ct;
          dn[1][k] += v * sgn * st;
        }
      }
    }
    // d/dr with r = h R: the tables above are d/dR; d/dr = (1/h) d/dR.  Volume: -eb / h.
    for (int k = 0; k < K; ++k) {
      dv[k] = (B.inside ? 1.0 : -1.0) * eb_mom[t * K + k] / h;
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

__global__ void k_circle_faces_dr(Circles B, int nx, int dir, double h, int body, const int32_t* __restrict__ faces,
                                  int64_t n, const int32_t* __restrict__ fbody, int q, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int f = faces[t];
  double acc[GEO_MAXQ + 1];
  for (int k = 0; k <= q; ++k) acc[k] = 0.0;
  if (fbody[f] == body) {
    const int mx = nx + (dir == 0), ix = f % mx, iy = f / mx;
    const double fc[2] = {dir == 0 ? ix * h : (ix + 0.5) * h, dir == 1 ? iy * h : (iy + 0.5) * h};
    const double dn = (fc[dir] - B.c[body][dir]) / h, ct = (B.c[body][1 - dir] - fc[1 - dir]) / h;
    const double R = B.r[body] / h, s2 = R * R - dn * dn;
    if (s2 > 0.0) {
      const double s = sqrt(s2), speed = R / s;  // d(end)/dR for both chord ends
      // outside fluid loses length at both ends; inside fluid gains it
      const double sg = B.inside ? 1.0 : -1.0;
      for (int e = -1; e <= 1; e += 2) {
        const double end = ct + e * s;
        if (end > -0.5 && end < 0.5) {
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

}  // namespace eb

using namespace eb;

namespace eb {
int geometry_bodies(const eb_geometry* g) { return g->n_body; }
int64_t geometry_cutfaces(const eb_geometry* g, int d) { return g->desc.n_cutface[d]; }
bool geometry_matches(const eb_geometry* g, int dim, const int* n, int n_cut) {
  const eb_geom& d = g->desc;
  return d.dim == dim && d.n[0] == n[0] && d.n[1] == n[1] && (dim < 3 || d.n[2] == n[2]) && d.n_cut == n_cut;
}

// d/dr of the moment tables of a device geometry for the radius of circle `body` (2-D), into caller
// arrays laid out like the tables (dface[d]: [n_cutface[d]][K_F]); stream-ordered
cudaError_t geometry_radius_derivative(const eb_geometry* g, int body, double* dvol, double* deb, double* debn,
                                       double* const* dface, cudaStream_t s) {
  static const GlRule gl = gl_rule();
  const eb_geom& d = g->desc;
  if (d.dim != 2 || body < 0 || body >= g->n_body) return cudaErrorInvalidValue;
  Circles B;
  B.n = g->n_body;
  B.inside = g->inside;
  for (int b = 0; b < g->n_body; ++b) {
    B.c[b][0] = g->centers[b][0];
    B.c[b][1] = g->centers[b][1];
    B.r[b] = g->radii[b];
  }
  const int q = d.moment_degree, K = (q + 1) * (q + 2) / 2;
  const int N = d.n[0];
  const double h = d.h;
  if (d.n_cut > 0) {
    k_circle_cells_dr<<<(unsigned)((d.n_cut + 127) / 128), 128, 0, s>>>(B, gl, N, h, body, d.cut_cell, d.n_cut,
                                                                       g->cell_body, d.eb_mom, q, K, dvol, deb, debn);
    eb::count_launch();
  }
  for (int dir = 0; dir < 2; ++dir) {
    if (d.n_cutface[dir] == 0) continue;
    k_circle_faces_dr<<<(unsigned)((d.n_cutface[dir] + 127) / 128), 128, 0, s>>>(
        B, N, dir, h, body, d.cutface[dir], d.n_cutface[dir], g->face_body[dir], q, dface[dir]);
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
  static const GlRule gl = gl_rule();
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
