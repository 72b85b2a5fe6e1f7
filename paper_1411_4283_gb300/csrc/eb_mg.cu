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
// prolongation is piecewise constant.  The V-cycle is a fixed linear map, so
// it serves as a right preconditioner of BiCGStab.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "eb_internal.cuh"
#include "eb_mg.cuh"

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
                          float* cp2, float* diag) {
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
  if (flag[c] == 2 && dinv_high[c] != 0.0) {
    double dh = 1.0 / dinv_high[c];  // diagonal of the high-order kappa-weighted operator
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

// weighted Jacobi: out = x + w (b - M x) / diag   (x == null: out = w b / diag)
template <typename T>
__global__ void k_mg_jacobi(int dim, int nx, int ny, int nz, const float* cp0, const float* cp1, const float* cp2,
                            const float* dg, const T* __restrict__ b, const T* x, T* out, float w) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)nx * ny * nz;
  if (c >= n) return;
  float d = dg[c];
  if (d == 0.0f) { out[c] = (T)0; return; }
  if (!x) { out[c] = (T)w * b[c] / (T)d; return; }
  int p[3];
  xyz_of(c, nx, ny, p);
  T r = b[c] - mg_apply_at<T>(dim, nx, ny, nz, c, p, cp0, cp1, cp2, dg, x);
  out[c] = x[c] + (T)w * r / (T)d;
}

// coarse right-hand side: average of the children's residuals b - M x
template <typename T>
__global__ void k_mg_restrict(int dim, int nxf, int nyf, int nzf, int nxc, int nyc, int nzc, const float* cp0,
                              const float* cp1, const float* cp2, const float* dg, const T* __restrict__ b,
                              const T* __restrict__ x, T* bc) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t ncc = (int64_t)nxc * nyc * nzc;
  if (c >= ncc) return;
  int X[3];
  xyz_of(c, nxc, nyc, X);
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
__global__ void k_mg_prolong(int dim, int nxf, int nyf, int nzf, int nxc, int nyc, const float* dg, const T* __restrict__ xc,
                             T* xf) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)nxf * nyf * nzf;
  if (c >= n) return;
  if (dg[c] == 0.0f) return;
  int p[3];
  xyz_of(c, nxf, nyf, p);
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

cudaError_t mg_setup(const MgFineInput& in, Multigrid* mg, cudaStream_t s) {
  mg->dim = in.dim;
  mg->nlev = 0;
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
      k_mg_fine<<<nb256(nc), 256, 0, s>>>(in.dim, n[0], n[1], n[2], in.h, in.flag, in.ff[0], in.ff[1], in.ff[2],
                                          in.cf[0], in.cf[1], in.cf[2], in.fm[0], in.fm[1], in.fm[2], in.KFS,
                                          in.dinv_high, L.cp[0], L.cp[1], L.cp[2], L.dg);
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

template <typename T>
static cudaError_t vcycle(const Multigrid& mgc, int l, cudaStream_t s) {
  Multigrid& mg = const_cast<Multigrid&>(mgc);
  MgLevel& L = mg.lev[l];
  const int D = mg.dim;
  if (L.ncell <= MG_CTA_CELLS) {
    MgDev<T>* dev = sizeof(T) == 4 ? (MgDev<T>*)mg.dev32 : (MgDev<T>*)mg.dev64;
    k_mg_coarse<T><<<1, 1024, 0, s>>>(D, mg.nlev - l, dev + l, 0.8f, MG_NU, 24);
    eb::count_launch();
    return cudaGetLastError();
  }
  T* b = vbuf<T>(L, 0);
  T* x = vbuf<T>(L, 1);
  T* w = vbuf<T>(L, 2);
  const int64_t n = L.ncell;
  const float om = D == 3 ? 0.8f : 0.8f;
  const bool coarsest = l == mg.nlev - 1;
  const int pre = coarsest ? 24 : MG_NU;
  // smoothing: x = w b / d, then sweeps ping-ponging x <-> w
  k_mg_jacobi<T><<<nb256(n), 256, 0, s>>>(D, L.n[0], L.n[1], L.n[2], L.cp[0], L.cp[1], L.cp[2], L.dg, b, nullptr, x, om);
  eb::count_launch();
  for (int it = 1; it < pre; ++it) {
    k_mg_jacobi<T><<<nb256(n), 256, 0, s>>>(D, L.n[0], L.n[1], L.n[2], L.cp[0], L.cp[1], L.cp[2], L.dg, b, x, w, om);
    eb::count_launch();
    T* t = x; x = w; w = t;
  }
  if (!coarsest) {
    MgLevel& C = mg.lev[l + 1];
    k_mg_restrict<T><<<nb256(C.ncell), 256, 0, s>>>(D, L.n[0], L.n[1], L.n[2], C.n[0], C.n[1], C.n[2], L.cp[0], L.cp[1],
                                                   L.cp[2], L.dg, b, x, vbuf<T>(C, 0));
    eb::count_launch();
    cudaError_t e = vcycle<T>(mg, l + 1, s);
    if (e) return e;
    k_mg_prolong<T><<<nb256(n), 256, 0, s>>>(D, L.n[0], L.n[1], L.n[2], C.n[0], C.n[1], L.dg, vbuf<T>(C, 1), x);
    eb::count_launch();
    for (int it = 0; it < MG_NU; ++it) {
      k_mg_jacobi<T><<<nb256(n), 256, 0, s>>>(D, L.n[0], L.n[1], L.n[2], L.cp[0], L.cp[1], L.cp[2], L.dg, b, x, w, om);
      eb::count_launch();
      T* t = x; x = w; w = t;
    }
  }
  // the level's result must end in buffer 1
  if (x != vbuf<T>(L, 1)) {
    cudaError_t e = cudaMemcpyAsync(vbuf<T>(L, 1), x, n * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e) return e;
  }
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
  if (!mg.exec[k]) {
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
  if ((e = cudaGraphLaunch(mg.exec[k], s))) return e;
  eb::count_launches(mg.nodes[k]);
  return cudaMemcpyAsync(z, vbuf<T>(L, 1), L.ncell * sizeof(T), cudaMemcpyDeviceToDevice, s);
}

template cudaError_t mg_precond<float>(const Multigrid&, const float*, float*, cudaStream_t);
template cudaError_t mg_precond<double>(const Multigrid&, const double*, double*, cudaStream_t);

}  // namespace eb
