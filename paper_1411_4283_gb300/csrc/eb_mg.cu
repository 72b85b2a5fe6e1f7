// Geometric multigrid preconditioner for the Krylov solve of kappa L phi = f.
//
// The paper preconditions GMRES with algebraic multigrid (PETSc GAMG, Sec.
// 3.2).  Here a cell-centred geometric V-cycle approximates the inverse of a
// second-order, kappa-weighted, 7-point (5-point in 2-D) operator on the same
// cut-cell grid:
//   (M phi)_v = (1/h^2) [ sum_faces alpha_f (phi_nb - phi_v) - 2 sum_walls alpha_f phi_v ] - e_v phi_v
// with alpha_f the face area fractions (Dirichlet walls half a cell away) and,
// at cut cells, e_v >= 0 chosen so that M's diagonal equals the diagonal of
// the high-order operator (the small-cell stiffness the Krylov method must
// see).  Coarse levels average kappa and the face fractions of their
// children and sum the EB terms (Galerkin scaling for piecewise-constant
// transfers); smoothing is weighted Jacobi; restriction averages the children;
// prolongation is piecewise constant.
//
// A few cut cells have a high-order diagonal that is weak (below half of the
// 7-point one), zero or positive: the row is dominated by its neighbours, the
// 7-point model is wrong there, and BiCGStab preconditioned by the V-cycle
// alone goes through long near-breakdown phases (at 256^3, 169 FP64
// iterations instead of 17).  After the V-cycle the preconditioner therefore
// solves the high-order operator exactly on the 3x3(x3) block of cells around
// each such cell (a multiplicative Schwarz step: z += A_BB^-1 (r - A z)_B,
// blocks precomputed by Gauss-Jordan in FP64).  The whole map is fixed and
// linear, so it serves as a right preconditioner of BiCGStab.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "eb_internal.cuh"
#include "eb_mg.cuh"
#include "eb_tables.cuh"

namespace eb {

__device__ __forceinline__ void xyz_of(int64_t c, int nx, int ny, int* x) {
  x[0] = (int)(c % nx);
  int64_t r = c / nx;
  x[1] = (int)(r % ny);
  x[2] = (int)(r / ny);
}

// Fine-level coefficients.  cpl[d][c]: coupling (1/h^2) alpha of the face between c and c + e_d;
// diag[c]: diagonal (negative on volumes, 0 on covered cells).
__global__ void k_mg_fine(int dim, int nx, int ny, int nz, double h, const uint8_t* __restrict__ flag,
                          const uint8_t* ff0, const uint8_t* ff1, const uint8_t* ff2, const int32_t* cf0,
                          const int32_t* cf1, const int32_t* cf2, const double* fm0, const double* fm1,
                          const double* fm2, int KFS, const double* __restrict__ dinv_high, float* cp0, float* cp1,
                          float* cp2, float* diag, int32_t* weak, int32_t* nweak, int cap) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t ncell = (int64_t)nx * ny * nz;
  if (c >= ncell) return;
  int x[3];
  xyz_of(c, nx, ny, x);
  const uint8_t* ff[3] = {ff0, ff1, ff2};
  const int32_t* cfm[3] = {cf0, cf1, cf2};
  const double* fm[3] = {fm0, fm1, fm2};
  float* cp[3] = {cp0, cp1, cp2};
  int n[3] = {nx, ny, nz};
  double ih2 = 1.0 / (h * h);
  double sum = 0.0;
  for (int d = 0; d < dim; ++d) {
    for (int side = 0; side < 2; ++side) {
      int fx[3] = {x[0], x[1], x[2]};
      if (side) fx[d] += 1;
      int64_t m0 = nx + (d == 0), m1 = ny + (d == 1);
      int64_t fl = (int64_t)fx[0] + m0 * ((int64_t)fx[1] + m1 * fx[2]);
      double a = 0.0;
      if (flag[c] > 0 && ff[d][fl] > 0) a = ff[d][fl] == 1 ? 1.0 : fm[d][(int64_t)cfm[d][fl] * KFS];
      bool wall = side ? x[d] == n[d] - 1 : x[d] == 0;
      if (wall) sum += 2.0 * a;
      else sum += a;
      if (side) cp[d][c] = (float)(wall ? 0.0 : a * ih2);
    }
  }
  if (flag[c] == 0) { diag[c] = 0.0f; return; }
  double dg = -sum * ih2;
  if (flag[c] == 2) {
    const double dh = dinv_high[c] != 0.0 ? 1.0 / dinv_high[c] : 0.0;  // diagonal of the high-order operator
    if (dh > 0.5 * dg) {             // weaker than half the 7-point diagonal, zero or positive
      const int q = atomicAdd(nweak, 1);
      if (q < cap) weak[q] = (int32_t)c;
    }
    if (dh < dg) dg = dh;            // add a non-negative EB term e_v
  }
  diag[c] = (float)dg;
}

// Coarse level from the fine level (factor 2 per dimension).  The coarse
// coupling of a face averages its 2^(D-1) fine faces and is rescaled by
// (h/H)^2; walls likewise; the EB part of the diagonal sums the children's
// with the Galerkin factor 4 / 2^D.
__global__ void k_mg_coarsen(int dim, int nxf, int nyf, int nzf, int nxc, int nyc, int nzc, const float* __restrict__ cpf0,
                             const float* __restrict__ cpf1, const float* __restrict__ cpf2,
                             const float* __restrict__ dgf, float* cpc0, float* cpc1, float* cpc2, float* dgc) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t ncc = (int64_t)nxc * nyc * nzc;
  if (c >= ncc) return;
  int X[3];
  xyz_of(c, nxc, nyc, X);
  int nf[3] = {nxf, nyf, nzf};
  int nc[3] = {nxc, nyc, nzc};
  const float* cpf[3] = {cpf0, cpf1, cpf2};
  float* cpc[3] = {cpc0, cpc1, cpc2};
  const int nch = 1 << dim;
  const float nfaces = (float)(1 << (dim - 1));
  // per child: couplings to in-block neighbours are internal; external ones form the coarse faces
  float ext[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  float offd_f = 0.0f, dsum = 0.0f;
  int live = 0;
  for (int k = 0; k < nch; ++k) {
    int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
    int f[3];
    bool in = true;
    for (int d = 0; d < 3; ++d) {
      f[d] = d < dim ? 2 * X[d] + o[d] : 0;
      if (f[d] >= nf[d]) in = false;
    }
    if (!in) continue;
    int64_t fc = (int64_t)f[0] + (int64_t)nxf * ((int64_t)f[1] + (int64_t)nyf * f[2]);
    float dg = dgf[fc];
    if (dg == 0.0f) continue;  // covered child
    ++live;
    float offsum = 0.0f;
    for (int d = 0; d < dim; ++d) {
      // + face of the child
      float up = cpf[d][fc];
      // - face: the coupling stored on the lower neighbour
      float dn = 0.0f;
      if (f[d] > 0) {
        int g[3] = {f[0], f[1], f[2]};
        g[d] -= 1;
        dn = cpf[d][(int64_t)g[0] + (int64_t)nxf * ((int64_t)g[1] + (int64_t)nyf * g[2])];
      }
      offsum += up + dn;
      if (o[d] == 1) ext[d][1] += up;
      if (o[d] == 0) ext[d][0] += dn;
    }
    offd_f += offsum;
    dsum += dg;
  }
  if (!live) {
    dgc[c] = 0.0f;
    for (int d = 0; d < dim; ++d) cpc[d][c] = 0.0f;
    return;
  }
  // fine diagonal = -(sum of couplings + walls + EB) ; the part beyond the couplings is walls + EB
  float extra = -dsum - offd_f;       // >= 0: wall and EB terms of the children (1/h^2 units)
  const float r2 = 0.25f;             // (h/H)^2
  float cpl_sum = 0.0f;
  for (int d = 0; d < dim; ++d) {
    float up = X[d] + 1 < nc[d] ? ext[d][1] / nfaces * r2 : 0.0f;
    cpc[d][c] = up;
    float dn = X[d] > 0 ? ext[d][0] / nfaces * r2 : 0.0f;
    cpl_sum += up + dn;
    // faces on the domain boundary keep their Dirichlet weight inside `extra`
  }
  float eb = extra * 4.0f / (float)nch * r2;
  dgc[c] = -(cpl_sum + eb);
}

// y = M x on one level
template <typename T>
__device__ __forceinline__ T mg_apply_at(int dim, int nx, int ny, int nz, int64_t c, const int* x, const float* cp0,
                                         const float* cp1, const float* cp2, const float* dg, const T* v) {
  T s = (T)dg[c] * v[c];
  const float* cp[3] = {cp0, cp1, cp2};
  int64_t st[3] = {1, nx, (int64_t)nx * ny};
  int n[3] = {nx, ny, nz};
  for (int d = 0; d < dim; ++d) {
    if (x[d] + 1 < n[d]) s += (T)cp[d][c] * v[c + st[d]];
    if (x[d] > 0) s += (T)cp[d][c - st[d]] * v[c - st[d]];
  }
  return s;
}

// Level kernels run on a 3-D grid of (32 x 4)-thread blocks over (x, y) rows and z planes, so that a
// thread's cell coordinates need no integer division.
constexpr int MG_BX = 32, MG_BY = 4;

__device__ __forceinline__ bool mg_cell(int nx, int ny, int* p, int64_t* c) {
  p[0] = blockIdx.x * MG_BX + threadIdx.x;
  p[1] = blockIdx.y * MG_BY + threadIdx.y;
  p[2] = blockIdx.z;
  if (p[0] >= nx || p[1] >= ny) return false;
  *c = (int64_t)p[0] + (int64_t)nx * ((int64_t)p[1] + (int64_t)ny * p[2]);
  return true;
}

// weighted Jacobi: out = x + w (b - M x) / diag   (x == null: out = w b / diag)
template <typename T>
__global__ void __launch_bounds__(MG_BX * MG_BY) k_mg_jacobi(int dim, int nx, int ny, int nz, const float* cp0,
                                                             const float* cp1, const float* cp2, const float* dg,
                                                             const T* __restrict__ b, const T* x, T* out, float w) {
  int p[3];
  int64_t c;
  if (!mg_cell(nx, ny, p, &c)) return;
  float d = dg[c];
  if (d == 0.0f) { out[c] = (T)0; return; }
  if (!x) { out[c] = (T)w * b[c] / (T)d; return; }
  T r = b[c] - mg_apply_at<T>(dim, nx, ny, nz, c, p, cp0, cp1, cp2, dg, x);
  out[c] = x[c] + (T)w * r / (T)d;
}

// coarse right-hand side: average of the children's residuals b - M x
template <typename T>
__global__ void __launch_bounds__(MG_BX * MG_BY) k_mg_restrict(int dim, int nxf, int nyf, int nzf, int nxc, int nyc, int nzc, const float* cp0,
                              const float* cp1, const float* cp2, const float* dg, const T* __restrict__ b,
                              const T* __restrict__ x, T* bc) {
  int X[3];
  int64_t c;
  if (!mg_cell(nxc, nyc, X, &c)) return;
  int nf[3] = {nxf, nyf, nzf};
  const int nch = 1 << dim;
  T acc = (T)0;
  for (int k = 0; k < nch; ++k) {
    int f[3] = {0, 0, 0};
    bool in = true;
    for (int d = 0; d < dim; ++d) {
      f[d] = 2 * X[d] + ((k >> d) & 1);
      if (f[d] >= nf[d]) in = false;
    }
    if (!in) continue;
    int64_t fc = (int64_t)f[0] + (int64_t)nxf * ((int64_t)f[1] + (int64_t)nyf * f[2]);
    if (dg[fc] == 0.0f) continue;
    acc += b[fc] - mg_apply_at<T>(dim, nxf, nyf, nzf, fc, f, cp0, cp1, cp2, dg, x);
  }
  bc[c] = acc / (T)nch;
}

// x_f += x_c (piecewise constant) on volumes
template <typename T>
__global__ void __launch_bounds__(MG_BX * MG_BY) k_mg_prolong(int dim, int nxf, int nyf, int nzf, int nxc, int nyc, const float* dg, const T* __restrict__ xc,
                             T* xf) {
  int p[3];
  int64_t c;
  if (!mg_cell(nxf, nyf, p, &c)) return;
  if (dg[c] == 0.0f) return;
  int64_t cc = (int64_t)(p[0] >> 1) + (int64_t)nxc * ((int64_t)(p[1] >> 1) + (int64_t)nyc * (dim == 3 ? (p[2] >> 1) : 0));
  xf[c] += xc[cc];
}

// The levels from `l0` down, when small, in one CTA: the same V-cycle with
// block-wide barriers instead of kernel boundaries.
template <typename T>
struct MgDev {
  int n[3];
  const float* cp[3];
  const float* dg;
  T* b;
  T* x;
  T* w;
};

template <typename T>
__device__ void cta_jacobi(int dim, const MgDev<T>& L, const T* x, T* out, float om) {
  int64_t n = (int64_t)L.n[0] * L.n[1] * L.n[2];
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    float d = L.dg[c];
    if (d == 0.0f) { out[c] = (T)0; continue; }
    if (!x) { out[c] = (T)om * L.b[c] / (T)d; continue; }
    int p[3];
    xyz_of(c, L.n[0], L.n[1], p);
    T r = L.b[c] - mg_apply_at<T>(dim, L.n[0], L.n[1], L.n[2], c, p, L.cp[0], L.cp[1], L.cp[2], L.dg, x);
    out[c] = x[c] + (T)om * r / (T)d;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_mg_coarse(int dim, int nlev, const MgDev<T>* __restrict__ lev, float om,
                                                    int nu, int ncoarse) {
  // per-thread copies of the ping-pong pointers (identical in every thread)
  T* xs[MG_MAXLEV];
  T* ws[MG_MAXLEV];
  for (int l = 0; l < nlev; ++l) {
    xs[l] = lev[l].x;
    ws[l] = lev[l].w;
  }
  for (int l = 0; l < nlev; ++l) {  // descend
    MgDev<T> L = lev[l];
    const bool last = l == nlev - 1;
    const int sweeps = last ? ncoarse : nu;
    cta_jacobi<T>(dim, L, nullptr, xs[l], om);
    __syncthreads();
    for (int it = 1; it < sweeps; ++it) {
      cta_jacobi<T>(dim, L, xs[l], ws[l], om);
      __syncthreads();
      T* t = xs[l]; xs[l] = ws[l]; ws[l] = t;
    }
    if (!last) {
      MgDev<T> C = lev[l + 1];
      int64_t ncc = (int64_t)C.n[0] * C.n[1] * C.n[2];
      const int nch = 1 << dim;
      for (int64_t c = threadIdx.x; c < ncc; c += blockDim.x) {
        int X[3];
        xyz_of(c, C.n[0], C.n[1], X);
        T acc = (T)0;
        for (int k = 0; k < nch; ++k) {
          int f[3] = {0, 0, 0};
          bool in = true;
          for (int d = 0; d < dim; ++d) {
            f[d] = 2 * X[d] + ((k >> d) & 1);
            if (f[d] >= L.n[d]) in = false;
          }
          if (!in) continue;
          int64_t fc = (int64_t)f[0] + (int64_t)L.n[0] * ((int64_t)f[1] + (int64_t)L.n[1] * f[2]);
          if (L.dg[fc] == 0.0f) continue;
          acc += L.b[fc] - mg_apply_at<T>(dim, L.n[0], L.n[1], L.n[2], fc, f, L.cp[0], L.cp[1], L.cp[2], L.dg, xs[l]);
        }
        C.b[c] = acc / (T)nch;
      }
      __syncthreads();
    }
  }
  for (int l = nlev - 2; l >= 0; --l) {  // ascend
    MgDev<T> L = lev[l];
    MgDev<T> C = lev[l + 1];
    int64_t n = (int64_t)L.n[0] * L.n[1] * L.n[2];
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
      if (L.dg[c] == 0.0f) continue;
      int p[3];
      xyz_of(c, L.n[0], L.n[1], p);
      int64_t cc = (int64_t)(p[0] >> 1) + (int64_t)C.n[0] * ((int64_t)(p[1] >> 1) + (int64_t)C.n[1] * (dim == 3 ? (p[2] >> 1) : 0));
      xs[l][c] += xs[l + 1][cc];
    }
    __syncthreads();
    for (int it = 0; it < nu; ++it) {
      cta_jacobi<T>(dim, L, xs[l], ws[l], om);
      __syncthreads();
      T* t = xs[l]; xs[l] = ws[l]; ws[l] = t;
    }
  }
  // the group's result belongs in level 0's x buffer
  if (xs[0] != lev[0].x) {
    int64_t n = (int64_t)lev[0].n[0] * lev[0].n[1] * lev[0].n[2];
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) lev[0].x[c] = xs[0][c];
  }
}

static unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

// ---------------------------------------------------------------- local block solves
constexpr int BLK = 27;  // 3 x 3 x 3 cells around a weak-diagonal cut cell
constexpr int MAX_BLOCKS = 8192;

struct RowSrc {
  const int32_t* irr_cell;
  const int32_t* irr_row;
  int64_t n_irr;
  const uint8_t* kind;
  const double* tmpl64;
  const double* rows64;
  const float* tmpl32;
  const float* rows32;
  int64_t n_rows;
  int nfoot;
  const int32_t* foot_off;
  const int16_t* lut;
  int L, S, nx, ny, nz;
  int64_t ncell;
};

// canonical row of cell c (-1: the template row, -2: covered)
__device__ int64_t row_of_cell(const RowSrc& a, int64_t c) {
  if (a.kind[c] == 0) return -2;
  if (a.kind[c] == 1) return -1;
  int64_t lo = 0, hi = a.n_irr - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a.irr_cell[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return a.irr_row[lo];
}

template <typename T>
__device__ __forceinline__ T coef_at(const RowSrc& a, int64_t row, int f);
template <>
__device__ __forceinline__ double coef_at<double>(const RowSrc& a, int64_t row, int f) {
  return row == -1 ? a.tmpl64[f] : a.rows64[(int64_t)f * a.n_rows + row];
}
template <>
__device__ __forceinline__ float coef_at<float>(const RowSrc& a, int64_t row, int f) {
  return row == -1 ? a.tmpl32[f] : a.rows32[(int64_t)f * a.n_rows + row];
}

// A_BB of every block (FP64); padding entries get the identity
__global__ void k_blk_assemble(RowSrc a, int nblk, const int32_t* __restrict__ cells, double* __restrict__ M) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nblk * BLK * BLK) return;
  const int b = (int)(t / (BLK * BLK)), i = (int)(t / BLK % BLK), j = (int)(t % BLK);
  const int32_t ci = cells[b * BLK + i], cj = cells[b * BLK + j];
  double v = 0.0;
  if (ci < 0 || cj < 0) {
    v = i == j ? 1.0 : 0.0;
  } else {
    int xi[3], xj[3];
    xyz_of(ci, a.nx, a.ny, xi);
    xyz_of(cj, a.nx, a.ny, xj);
    const int dx = xj[0] - xi[0], dy = xj[1] - xi[1], dz = xj[2] - xi[2];
    const int f = a.lut[(dx + a.L) + a.S * ((dy + a.L) + a.S * (dz + a.L))];
    const int64_t row = row_of_cell(a, ci);
    if (f >= 0 && row != -2) v = coef_at<double>(a, row, f);
  }
  M[t] = v;
}

// in-place Gauss-Jordan inverse with partial pivoting, one thread per block
__global__ void k_blk_invert(int nblk, double* __restrict__ M, float* __restrict__ M32, int32_t* __restrict__ fail) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  double a[BLK][2 * BLK];
  const double* src = M + (int64_t)b * BLK * BLK;
  for (int i = 0; i < BLK; ++i)
    for (int j = 0; j < BLK; ++j) {
      a[i][j] = src[i * BLK + j];
      a[i][BLK + j] = i == j ? 1.0 : 0.0;
    }
  for (int k = 0; k < BLK; ++k) {
    int p = k;
    for (int i = k + 1; i < BLK; ++i)
      if (fabs(a[i][k]) > fabs(a[p][k])) p = i;
    if (a[p][k] == 0.0) { atomicExch(fail, 1); return; }
    if (p != k)
      for (int j = 0; j < 2 * BLK; ++j) { double t = a[k][j]; a[k][j] = a[p][j]; a[p][j] = t; }
    const double inv = 1.0 / a[k][k];
    for (int j = 0; j < 2 * BLK; ++j) a[k][j] *= inv;
    for (int i = 0; i < BLK; ++i) {
      if (i == k) continue;
      const double m = a[i][k];
      if (m == 0.0) continue;
      for (int j = 0; j < 2 * BLK; ++j) a[i][j] -= m * a[k][j];
    }
  }
  double* dst = M + (int64_t)b * BLK * BLK;
  for (int i = 0; i < BLK; ++i)
    for (int j = 0; j < BLK; ++j) {
      dst[i * BLK + j] = a[i][BLK + j];
      M32[(int64_t)b * BLK * BLK + i * BLK + j] = (float)a[i][BLK + j];
    }
}

// res_i = r_ci - (A z)_ci for the cells of every block; one warp per cell, the lanes splitting the
// footprint (few cells, long rows: a thread per cell leaves the GPU idle behind 637 dependent loads).
// TR: the transposed operator, (A^T z)_c = sum_f A(c - off_f, f) z_(c - off_f) (the rows that reach c;
// a linear offset that wraps across a grid line lands on a row whose entry there is zero)
template <typename T, bool TR>
__global__ void k_blk_res(RowSrc a, int nblk, const int32_t* __restrict__ cells, const T* __restrict__ r,
                          const T* __restrict__ z, T* __restrict__ res) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // warp-uniform
  const int lane = threadIdx.x & 31;
  if (t >= (int64_t)nblk * BLK) return;
  const int32_t c = cells[t];
  if (c < 0) {
    if (lane == 0) res[t] = (T)0;
    return;
  }
  const int64_t row = row_of_cell(a, c);
  if (row == -2) {
    if (lane == 0) res[t] = (T)0;
    return;
  }
  T acc = (T)0;
  const int64_t hi = a.ncell - 1;
  if (TR) {
    for (int f = lane; f < a.nfoot; f += 32) {
      const int64_t q = c - a.foot_off[f];
      if (q < 0 || q > hi) continue;
      const int64_t rq = row_of_cell(a, q);
      if (rq == -2) continue;
      acc = fma(coef_at<T>(a, rq, f), z[q], acc);
    }
  } else {
    for (int f = lane; f < a.nfoot; f += 32) {
      int64_t q = c + a.foot_off[f];
      q = q < 0 ? 0 : (q > hi ? hi : q);  // out-of-domain entries have zero coefficients
      acc = fma(coef_at<T>(a, row, f), z[q], acc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) res[t] = r[c] - acc;
}

// z_ci += sum_j inv(A_BB)_ij res_j (blocks may overlap: additive); TR: inv(A_BB^T) = inv(A_BB)^T
template <typename T, bool TR>
__global__ void k_blk_corr(int nblk, const int32_t* __restrict__ cells, const T* __restrict__ inv,
                           const T* __restrict__ res, T* z) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nblk * BLK) return;
  const int32_t c = cells[t];
  if (c < 0) return;
  const int64_t b = t / BLK, i = t % BLK;
  const T* rr = res + b * BLK;
  T d = (T)0;
  if (TR) {
    const T* m = inv + b * BLK * BLK + i;
    for (int j = 0; j < BLK; ++j) d = fma(m[j * BLK], rr[j], d);
  } else {
    const T* m = inv + (b * BLK + i) * BLK;
    for (int j = 0; j < BLK; ++j) d = fma(m[j], rr[j], d);
  }
  atomicAdd(z + c, d);
}

static RowSrc row_src(const Multigrid& mg) {
  RowSrc a;
  a.irr_cell = mg.irr_cell;
  a.irr_row = mg.irr_row;
  a.n_irr = mg.n_irr;
  a.kind = mg.kind;
  a.tmpl64 = mg.tmpl64;
  a.rows64 = mg.rows64;
  a.tmpl32 = mg.tmpl32;
  a.rows32 = mg.rows32;
  a.n_rows = mg.n_rows;
  a.nfoot = mg.nfoot;
  a.foot_off = mg.foot_off;
  a.lut = mg.foot_lut;
  a.L = mg.R + 1;
  a.S = 2 * mg.R + 3;
  a.nx = mg.lev[0].n[0];
  a.ny = mg.lev[0].n[1];
  a.nz = mg.lev[0].n[2];
  a.ncell = mg.lev[0].ncell;
  return a;
}

// blocks around the weak-diagonal cut cells (3 x 3 x 3, or 3 x 3 in 2-D with the other entries padding):
// cell lists on the host, A_BB and its inverse on the device
// cells of the block around weak cell list[b]: the 3x3x3 box (in the domain, not covered), -1 elsewhere
__global__ void k_blk_cells(const int32_t* __restrict__ list, int nb, int nx, int ny, int nz,
                            const uint8_t* __restrict__ flag, int32_t* __restrict__ cells) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nb * BLK) return;
  const int b = (int)(t / BLK), k = (int)(t % BLK);
  int p[3];
  xyz_of(list[b], nx, ny, p);
  const int X = p[0] + k % 3 - 1, Y = p[1] + k / 3 % 3 - 1, Z = p[2] + k / 9 - 1;
  int32_t v = -1;
  if (X >= 0 && X < nx && Y >= 0 && Y < ny && Z >= 0 && Z < nz) {
    const int64_t q = X + (int64_t)nx * (Y + (int64_t)ny * Z);
    if (flag[q]) v = (int32_t)q;
  }
  cells[t] = v;
}

static cudaError_t blocks_setup(const MgFineInput& in, Multigrid* mg, const int32_t* weak_d, const int32_t* nweak_d,
                                cudaStream_t s) {
  if (!in.irr_cell || in.n_irr == 0) return cudaSuccess;
  const int nx = in.n[0], ny = in.n[1], nz = in.n[2];
  cudaError_t e;
  int32_t nw = 0;
  if ((e = cudaMemcpyAsync(&nw, nweak_d, 4, cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  const int nb = nw < MAX_BLOCKS ? nw : MAX_BLOCKS;
  std::vector<int32_t> list(nb > 0 ? nb : 1);
  if (nb > 0) {
    if ((e = cudaMemcpyAsync(list.data(), weak_d, (size_t)nb * 4, cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    std::sort(list.begin(), list.begin() + nb);  // appended in any order: make the blocks deterministic
  }
  // row lookup data
  mg->irr_cell = in.irr_cell;
  mg->irr_row = in.irr_row;
  mg->n_irr = in.n_irr;
  mg->kind = in.kind;
  mg->tmpl64 = in.tmpl64;
  mg->tmpl32 = in.tmpl32;
  mg->rows64 = in.rows64;
  mg->rows32 = in.rows32;
  mg->n_rows = in.n_rows;
  mg->nfoot = in.nfoot;
  mg->foot_off = in.foot_off;
  mg->R = in.R;
  if (nb == 0) return cudaSuccess;
  const int L = in.R + 1, S = 2 * L + 1;
  std::vector<int16_t> lut(S * S * S, -1);
  int nf = 0;
  const int zr = in.dim == 3 ? L : 0;
  for (int z = -zr; z <= zr; ++z)
    for (int y = -L; y <= L; ++y)
      for (int x = -L; x <= L; ++x)
        if (in_footprint(x, y, z, in.R, in.box)) lut[(x + L) + S * ((y + L) + S * (z + L))] = (int16_t)nf++;
  if (nf != in.nfoot) return cudaErrorInvalidValue;
  if ((e = cudaMalloc(&mg->foot_lut, lut.size() * 2))) return e;
  if ((e = cudaMalloc(&mg->blk_cells, (size_t)nb * BLK * 4))) return e;
  if ((e = cudaMalloc(&mg->blk_inv64, (size_t)nb * BLK * BLK * 8))) return e;
  if ((e = cudaMalloc(&mg->blk_inv32, (size_t)nb * BLK * BLK * 4))) return e;
  if ((e = cudaMalloc(&mg->blk_res, (size_t)nb * BLK * 8))) return e;
  if ((e = cudaMemcpyAsync(mg->foot_lut, lut.data(), lut.size() * 2, cudaMemcpyHostToDevice, s))) return e;
  int32_t* dl;
  if ((e = cudaMalloc(&dl, (size_t)nb * 4))) return e;
  if ((e = cudaMemcpyAsync(dl, list.data(), (size_t)nb * 4, cudaMemcpyHostToDevice, s))) { cudaFree(dl); return e; }
  k_blk_cells<<<nb256((int64_t)nb * BLK), 256, 0, s>>>(dl, nb, nx, ny, nz, in.flag, mg->blk_cells);
  eb::count_launch();
  mg->nblk = nb;
  RowSrc a = row_src(*mg);
  const int64_t nm = (int64_t)nb * BLK * BLK;
  k_blk_assemble<<<nb256(nm), 256, 0, s>>>(a, nb, mg->blk_cells, mg->blk_inv64);
  int32_t* fail;
  if ((e = cudaMalloc(&fail, 4))) return e;
  cudaMemsetAsync(fail, 0, 4, s);
  k_blk_invert<<<(nb + 31) / 32, 32, 0, s>>>(nb, mg->blk_inv64, mg->blk_inv32, fail);
  eb::count_launches(2);
  int32_t hf = 0;
  cudaMemcpyAsync(&hf, fail, 4, cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  cudaFree(fail);
  cudaFree(dl);
  if (e) return e;
  if (hf) mg->nblk = 0;  // a singular block: no local solves
  return cudaGetLastError();
}

cudaError_t mg_setup(const MgFineInput& in, Multigrid* mg, cudaStream_t s) {
  mg->dim = in.dim;
  mg->nlev = 0;
  int32_t* weak = nullptr;  // fine-level cut cells with a weak high-order diagonal (list, count after it)
  int n[3] = {in.n[0], in.n[1], in.n[2]};
  cudaError_t e;
  for (int l = 0; l < MG_MAXLEV; ++l) {
    MgLevel& L = mg->lev[l];
    for (int d = 0; d < 3; ++d) L.n[d] = n[d];
    int64_t nc = (int64_t)n[0] * n[1] * n[2];
    L.ncell = nc;
    for (int d = 0; d < 3; ++d) {
      if ((e = cudaMalloc(&L.cp[d], nc * 4))) return e;
      if ((e = cudaMemsetAsync(L.cp[d], 0, nc * 4, s))) return e;
    }
    if ((e = cudaMalloc(&L.dg, nc * 4))) return e;
    for (int k = 0; k < 3; ++k)
      if ((e = cudaMalloc(&L.v32[k], nc * 4))) return e;
    for (int k = 0; k < 3; ++k)
      if ((e = cudaMalloc(&L.v64[k], nc * 8))) return e;
    mg->nlev = l + 1;
    if (l == 0) {
      if ((e = cudaMalloc(&weak, (MAX_BLOCKS + 1) * 4))) return e;
      if ((e = cudaMemsetAsync(weak + MAX_BLOCKS, 0, 4, s))) return e;
      k_mg_fine<<<nb256(nc), 256, 0, s>>>(in.dim, n[0], n[1], n[2], in.h, in.flag, in.ff[0], in.ff[1], in.ff[2],
                                          in.cf[0], in.cf[1], in.cf[2], in.fm[0], in.fm[1], in.fm[2], in.KFS,
                                          in.dinv_high, L.cp[0], L.cp[1], L.cp[2], L.dg, weak, weak + MAX_BLOCKS,
                                          MAX_BLOCKS);
      eb::count_launch();
    } else {
      MgLevel& F = mg->lev[l - 1];
      k_mg_coarsen<<<nb256(nc), 256, 0, s>>>(in.dim, F.n[0], F.n[1], F.n[2], n[0], n[1], n[2], F.cp[0], F.cp[1], F.cp[2],
                                             F.dg, L.cp[0], L.cp[1], L.cp[2], L.dg);
      eb::count_launch();
    }
    if ((e = cudaGetLastError())) return e;
    int mn = n[0] < n[1] ? n[0] : n[1];
    if (in.dim == 3 && n[2] < mn) mn = n[2];
    if (mn <= 4) break;
    for (int d = 0; d < in.dim; ++d) n[d] = (n[d] + 1) / 2;
  }
  if (weak) {
    e = blocks_setup(in, mg, weak, weak + MAX_BLOCKS, s);
    cudaFree(weak);
    if (e) return e;
  }
  // device descriptors of every level for the single-CTA coarse cycle
  MgDev<float> h32[MG_MAXLEV];
  MgDev<double> h64[MG_MAXLEV];
  for (int l = 0; l < mg->nlev; ++l) {
    MgLevel& L = mg->lev[l];
    for (int d = 0; d < 3; ++d) { h32[l].n[d] = L.n[d]; h64[l].n[d] = L.n[d]; h32[l].cp[d] = L.cp[d]; h64[l].cp[d] = L.cp[d]; }
    h32[l].dg = L.dg; h64[l].dg = L.dg;
    h32[l].b = L.v32[0]; h32[l].x = L.v32[1]; h32[l].w = L.v32[2];
    h64[l].b = L.v64[0]; h64[l].x = L.v64[1]; h64[l].w = L.v64[2];
  }
  if ((e = cudaMalloc(&mg->dev32, sizeof(h32)))) return e;
  if ((e = cudaMalloc(&mg->dev64, sizeof(h64)))) return e;
  if ((e = cudaMemcpyAsync(mg->dev32, h32, sizeof(h32), cudaMemcpyHostToDevice, s))) return e;
  if ((e = cudaMemcpyAsync(mg->dev64, h64, sizeof(h64), cudaMemcpyHostToDevice, s))) return e;
  return cudaStreamSynchronize(s);
}

void mg_free(Multigrid* mg) {
  cudaFree(mg->blk_cells);
  cudaFree(mg->blk_inv64);
  cudaFree(mg->blk_inv32);
  cudaFree(mg->blk_res);
  cudaFree(mg->foot_lut);
  mg->blk_cells = nullptr;
  mg->blk_inv64 = nullptr;
  mg->blk_inv32 = nullptr;
  mg->blk_res = nullptr;
  mg->foot_lut = nullptr;
  mg->nblk = 0;
  if (mg->dev32) cudaFree(mg->dev32);
  if (mg->dev64) cudaFree(mg->dev64);
  mg->dev32 = mg->dev64 = nullptr;
  for (int k = 0; k < 2; ++k)
    if (mg->exec[k]) { cudaGraphExecDestroy(mg->exec[k]); mg->exec[k] = nullptr; }
  for (int l = 0; l < mg->nlev; ++l) {
    MgLevel& L = mg->lev[l];
    for (int d = 0; d < 3; ++d) cudaFree(L.cp[d]);
    cudaFree(L.dg);
    for (int k = 0; k < 3; ++k) {
      cudaFree(L.v32[k]);
      cudaFree(L.v64[k]);
    }
  }
  mg->nlev = 0;
}

template <typename T>
static T* vbuf(MgLevel& L, int k);
template <>
float* vbuf<float>(MgLevel& L, int k) { return L.v32[k]; }
template <>
double* vbuf<double>(MgLevel& L, int k) { return L.v64[k]; }

// z = V(b) on level l; b and z live in the level's buffers (0: b, 1: x, 2: work)
constexpr int64_t MG_CTA_CELLS = 4096;  // levels at most this large run inside one CTA

static dim3 mg_grid(const int* n) {
  return dim3((unsigned)((n[0] + MG_BX - 1) / MG_BX), (unsigned)((n[1] + MG_BY - 1) / MG_BY), (unsigned)n[2]);
}

template <typename T>
static cudaError_t vcycle(const Multigrid& mgc, int l, cudaStream_t s) {
  Multigrid& mg = const_cast<Multigrid&>(mgc);
  MgLevel& L = mg.lev[l];
  if (L.ncell <= MG_CTA_CELLS) {
    const int D = mg.dim;
    MgDev<T>* dev = sizeof(T) == 4 ? (MgDev<T>*)mg.dev32 : (MgDev<T>*)mg.dev64;
    k_mg_coarse<T><<<1, 1024, 0, s>>>(D, mg.nlev - l, dev + l, 0.8f, MG_NU, 24);
    eb::count_launch();
    return cudaGetLastError();
  }
  T* b = vbuf<T>(L, 0);
  const int D = mg.dim;
  const float om = 0.8f;
  const bool coarsest = l == mg.nlev - 1;
  const int pre = coarsest ? 24 : MG_NU;
  const int post = coarsest ? 0 : MG_NU;
  // the level's result ends in buffer 1: the first smoothing step writes buffer 1 or 2 by the parity
  // of the sweeps that follow it
  T* x = vbuf<T>(L, (pre - 1 + post) % 2 == 0 ? 1 : 2);
  T* w = vbuf<T>(L, (pre - 1 + post) % 2 == 0 ? 2 : 1);
  const dim3 blk(MG_BX, MG_BY), grd = mg_grid(L.n);
  // smoothing: x = w b / d, then sweeps ping-ponging x <-> w
  k_mg_jacobi<T><<<grd, blk, 0, s>>>(D, L.n[0], L.n[1], L.n[2], L.cp[0], L.cp[1], L.cp[2], L.dg, b, nullptr, x, om);
  eb::count_launch();
  for (int it = 1; it < pre; ++it) {
    k_mg_jacobi<T><<<grd, blk, 0, s>>>(D, L.n[0], L.n[1], L.n[2], L.cp[0], L.cp[1], L.cp[2], L.dg, b, x, w, om);
    eb::count_launch();
    T* t = x; x = w; w = t;
  }
  if (!coarsest) {
    MgLevel& C = mg.lev[l + 1];
    k_mg_restrict<T><<<mg_grid(C.n), blk, 0, s>>>(D, L.n[0], L.n[1], L.n[2], C.n[0], C.n[1], C.n[2], L.cp[0], L.cp[1],
                                                 L.cp[2], L.dg, b, x, vbuf<T>(C, 0));
    eb::count_launch();
    cudaError_t e = vcycle<T>(mg, l + 1, s);
    if (e) return e;
    k_mg_prolong<T><<<grd, blk, 0, s>>>(D, L.n[0], L.n[1], L.n[2], C.n[0], C.n[1], L.dg, vbuf<T>(C, 1), x);
    eb::count_launch();
    for (int it = 0; it < post; ++it) {
      k_mg_jacobi<T><<<grd, blk, 0, s>>>(D, L.n[0], L.n[1], L.n[2], L.cp[0], L.cp[1], L.cp[2], L.dg, b, x, w, om);
      eb::count_launch();
      T* t = x; x = w; w = t;
    }
  }
  if (x != vbuf<T>(L, 1)) return cudaErrorUnknown;  // parity bookkeeping above
  return cudaGetLastError();
}

// The V-cycle works on the levels' fixed buffers, so it is captured once per
// precision as a CUDA graph (on a private stream) and replayed; the input and
// output copies stay outside the graph.
template <typename T>
cudaError_t mg_precond(const Multigrid& mgc, const T* r, T* z, cudaStream_t s) {
  Multigrid& mg = const_cast<Multigrid&>(mgc);
  MgLevel& L = mg.lev[0];
  const int k = sizeof(T) == 4 ? 0 : 1;
  cudaError_t e;
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(s, &cst))) return e;
  const bool capturing = cst == cudaStreamCaptureStatusActive;  // inside a graph being captured: the cycle's kernels
  if (!capturing && !mg.exec[k]) {
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) return e;
    long long before = eb::launches_so_far();
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal))) { cudaStreamDestroy(cap); return e; }
    cudaError_t ev = vcycle<T>(mg, 0, cap);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (ev) return ev;
    if (e) return e;
    mg.nodes[k] = eb::launches_so_far() - before;
    eb::uncount_launches(mg.nodes[k]);  // capture issued no work
    e = cudaGraphInstantiate(&mg.exec[k], graph, 0);
    cudaGraphDestroy(graph);
    if (e) return e;
  }
  if ((e = cudaMemcpyAsync(vbuf<T>(L, 0), r, L.ncell * sizeof(T), cudaMemcpyDeviceToDevice, s))) return e;
  if (capturing) {
    if ((e = vcycle<T>(mg, 0, s))) return e;
  } else {
    if ((e = cudaGraphLaunch(mg.exec[k], s))) return e;
    eb::count_launches(mg.nodes[k]);
  }
  if ((e = cudaMemcpyAsync(z, vbuf<T>(L, 1), L.ncell * sizeof(T), cudaMemcpyDeviceToDevice, s))) return e;
  if (mg.nblk > 0) {
    RowSrc a = row_src(mg);
    const int64_t nt = (int64_t)mg.nblk * BLK;
    const T* inv;
    if constexpr (sizeof(T) == 4) inv = mg.blk_inv32;
    else inv = mg.blk_inv64;
    if (mg.transpose) {
      k_blk_res<T, true><<<nb256(nt * 32), 256, 0, s>>>(a, mg.nblk, mg.blk_cells, r, z, (T*)mg.blk_res);
      k_blk_corr<T, true><<<nb256(nt), 256, 0, s>>>(mg.nblk, mg.blk_cells, inv, (const T*)mg.blk_res, z);
    } else {
      k_blk_res<T, false><<<nb256(nt * 32), 256, 0, s>>>(a, mg.nblk, mg.blk_cells, r, z, (T*)mg.blk_res);
      k_blk_corr<T, false><<<nb256(nt), 256, 0, s>>>(mg.nblk, mg.blk_cells, inv, (const T*)mg.blk_res, z);
    }
    eb::count_launches(2);
  }
  return cudaGetLastError();
}

template cudaError_t mg_precond<float>(const Multigrid&, const float*, float*, cudaStream_t);
template cudaError_t mg_precond<double>(const Multigrid&, const double*, double*, cudaStream_t);

}  // namespace eb
