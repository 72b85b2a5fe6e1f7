// Operator apply: y = kappa .* (L phi) (or L phi), the homogeneous part of the
// flux-divergence Laplacian of Sec. 2.3.  Two passes:
//   K4  template cells: the translation-invariant cell stencil of the interior
//       (every face stencil there is the same weighted-LS template);
//   K5  irregular cells (near the EB or a domain wall): footprint-dense rows,
//       stored footprint-major so that consecutive rows load coalesced.
// Covered cells get y = 0.
#include <cuda_runtime.h>
#include <algorithm>
#include <stdint.h>

#include "eb_apply.cuh"
#include "eb_internal.cuh"
#include "eb_apply_tma.cuh"
#include "eb_apply_quad.cuh"
#include "eb_apply_wall.cuh"
#include "eb_apply_brick.cuh"
#include "eb_apply_fold.cuh"

#include <cuda.h>

namespace eb {

// footprint offsets of the template stencil, staged in shared memory
template <typename T, int TILE_X>
__global__ void __launch_bounds__(256) k_apply_template(ApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  int32_t* off = reinterpret_cast<int32_t*>(sm_raw);
  T* coef = reinterpret_cast<T*>(sm_raw + ((a.nfoot * 4 + 15) / 16) * 16);
  for (int i = threadIdx.x; i < a.nfoot; i += blockDim.x) {
    off[i] = a.foot_off[i];
    coef[i] = a.tmpl[i];
  }
  __syncthreads();
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.ncell) return;
  uint8_t kind = a.kind[c];
  if (kind == 2) return;  // written by the irregular pass
  T acc = 0;
  if (kind == 1) {
    const T* p = a.phi + c;
#pragma unroll 8
    for (int i = 0; i < a.nfoot; ++i) acc += coef[i] * __ldg(p + off[i]);
    if (!a.kappa_weighted) acc *= (T)a.inv_kappa[c];
  }
  a.y[c] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_apply_irregular(ApplyArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  int32_t* off = reinterpret_cast<int32_t*>(sm_raw);
  for (int i = threadIdx.x; i < a.nfoot; i += blockDim.x) off[i] = a.foot_off[i];
  __syncthreads();
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_irr) return;
  int64_t c = a.irr_cell[t];
  int64_t row = a.irr_row[t];
  const T* rows = a.rows + row;
  T acc = 0;
  const int64_t hi = a.ncell - 1;
  for (int i = 0; i < a.nfoot; ++i) {
    int64_t q = c + off[i];
    q = q < 0 ? 0 : (q > hi ? hi : q);  // out-of-domain offsets carry zero coefficients
    acc += __ldg(rows + (int64_t)i * a.n_rows) * __ldg(a.phi + q);
  }
  if (!a.kappa_weighted) acc *= (T)a.inv_kappa[c];
  a.y[c] = acc;
}

// Irregular rows for box neighbourhoods of radius R in D dimensions: the
// footprint is a union of x-contiguous segments (dz, dy, dx in [-X, X]) whose
// coefficients are consecutive in footprint order.  One thread per row walks
// the segments (a rolled loop keeps the code small); a segment whose
// (y + dy, z + dz) leaves the grid has zero coefficients and is skipped, and
// only the x-ends of the first and last grid rows need an address clamp.
template <typename T, int R, int D>
__global__ void __launch_bounds__(256) k_apply_irregular_seg(ApplyArgs<T> a, int nx, int ny, int nz) {
  constexpr int L = R + 1;
  constexpr int NZ = D == 3 ? 2 * L + 1 : 1;
  constexpr int NY = 2 * L + 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_irr) return;
  const int64_t c = a.irr_cell[t];
  const int cx = (int)(c % nx);
  const int64_t cr = c / nx;
  const int cy = (int)(cr % ny), cz = (int)(cr / ny);
  const int64_t stride = a.n_rows;
  const T* cf = a.rows + a.irr_row[t];
  const int64_t ncell = a.ncell;
  T acc0 = 0, acc1 = 0;
#pragma unroll 1
  for (int sgi = 0; sgi < NZ * NY; ++sgi) {
    const int dz = D == 3 ? sgi / NY - L : 0;
    const int dy = sgi % NY - L;
    const int az = dz < 0 ? -dz : dz, ay = dy < 0 ? -dy : dy;
    if (az > R && ay > R) continue;
    const bool wide = !(az > R || ay > R);  // x extent L (wide) or R
    const int X = wide ? L : R;
    const int zz = cz + dz, yy = cy + dy;
    if (zz >= 0 && zz < nz && yy >= 0 && yy < ny) {
      const int64_t base = (int64_t)nx * ((int64_t)yy + (int64_t)ny * zz) + cx;
      if (base - X >= 0 && base + X < ncell) {
        const T* ph = a.phi + base;
        if (wide) {
#pragma unroll
          for (int dx = -L; dx <= L; ++dx) {
            if (dx & 1) acc1 = fma(__ldg(cf), __ldg(ph + dx), acc1);
            else acc0 = fma(__ldg(cf), __ldg(ph + dx), acc0);
            cf += stride;
          }
        } else {
#pragma unroll
          for (int dx = -R; dx <= R; ++dx) {
            if (dx & 1) acc1 = fma(__ldg(cf), __ldg(ph + dx), acc1);
            else acc0 = fma(__ldg(cf), __ldg(ph + dx), acc0);
            cf += stride;
          }
        }
        continue;
      }
      for (int dx = -X; dx <= X; ++dx) {
        int64_t q = base + dx;
        q = q < 0 ? 0 : (q >= ncell ? ncell - 1 : q);
        acc0 = fma(__ldg(cf), __ldg(a.phi + q), acc0);
        cf += stride;
      }
    } else {
      cf += (int64_t)(2 * X + 1) * stride;
    }
  }
  T acc = acc0 + acc1;
  if (!a.kappa_weighted) acc *= (T)a.inv_kappa[c];
  a.y[c] = acc;
}

// wall-layer x-runs need 16-byte aligned phi for their vector loads
template <typename T>
static bool use_runs(const ApplyArgs<T>& a) {
  const ApplyPlan* pl = a.plan;
  return pl && pl->quad && pl->nG > 0 && ((uintptr_t)a.phi & 15u) == 0;
}

template <typename T>
static cudaError_t launch_runs(const ApplyArgs<T>& a, cudaStream_t st) {
  const ApplyPlan* pl = a.plan;
  XqArgs<T> x;
  x.nG = pl->nG;
  x.cellG = pl->cellG;
  x.classG = pl->classG;
  if constexpr (sizeof(T) == 4) x.rowsK = pl->rowsK32;
  else x.rowsK = pl->rowsK64;
  x.nfoot = a.nfoot;
  x.phi = a.phi;
  x.y = a.y;
  x.inv_kappa = a.inv_kappa;
  x.kappa_weighted = a.kappa_weighted;
  x.nx = pl->nx;
  x.ny = pl->ny;
  x.nz = pl->nz;
  const unsigned nb = (unsigned)((pl->nG + 127) / 128);
  if (pl->R == 3) k_class_xquad<T, 3><<<nb, 128, 0, st>>>(x);
  else k_class_xquad<T, 2><<<nb, 128, 0, st>>>(x);
  eb::count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_brick(const ApplyArgs<T>& a, cudaStream_t st) {
  const ApplyPlan* pl = a.plan;
  BrickArgs<T> b;
  b.nx = pl->nx;
  b.ny = pl->ny;
  b.nz = pl->nz;
  b.nyb = pl->nyb;
  b.nzb = pl->nzb;
  b.y_org = pl->y_org;
  b.z_org = pl->z_org;
  b.y_hi = pl->y_hi;
  b.z_hi = pl->z_hi;
  b.unit_class = pl->unit_class;
  if constexpr (sizeof(T) == 4) b.rowsK = pl->rowsK32;
  else b.rowsK = pl->rowsK64;
  b.nfoot = a.nfoot;
  b.phi = a.phi;
  b.y = a.y;
  b.inv_kappa = a.inv_kappa;
  b.kappa_weighted = a.kappa_weighted;
  const unsigned grid = (unsigned)(2 * b.nyb * b.nzb);
  cudaError_t e;
  if (pl->R == 3) {
    constexpr size_t sm = brick_smem<T, 3>();
    if ((e = cudaFuncSetAttribute(k_wall_brick<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    k_wall_brick<T, 3><<<grid, BR_W * 32, sm, st>>>(b);
  } else {
    constexpr size_t sm = brick_smem<T, 2>();
    if ((e = cudaFuncSetAttribute(k_wall_brick<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    k_wall_brick<T, 2><<<grid, BR_W * 32, sm, st>>>(b);
  }
  eb::count_launch();
  return cudaGetLastError();
}

#ifndef EB_QUAD_PER_SM
#define EB_QUAD_PER_SM 8  // CTAs per SM of the unique-row stream (0: one CTA per 128 rows)
#endif

// class cells outside the runs and the slab bricks: per-cell segment walk over the canonical rows
template <typename T>
static cudaError_t launch_seg_rest(const ApplyArgs<T>& a, cudaStream_t st) {
  const ApplyPlan* pl = a.plan;
  ApplyArgs<T> c = a;
  c.n_irr = pl->nL;
  c.irr_cell = pl->cellL;
  c.irr_row = pl->classL;
  const unsigned bc = (unsigned)((pl->nL + 255) / 256);
  if (pl->R == 3) k_apply_irregular_seg<T, 3, 3><<<bc, 256, 0, st>>>(c, pl->nx, pl->ny, pl->nz);
  else k_apply_irregular_seg<T, 2, 3><<<bc, 256, 0, st>>>(c, pl->nx, pl->ny, pl->nz);
  eb::count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_irregular(const ApplyArgs<T>& a, cudaStream_t st) {
  const ApplyPlan* pl = a.plan;
  int64_t nb = (a.n_irr + 255) / 256;
  if (pl && pl->quad) {
    // unique rows (HBM stream) in the quad layout; without the x-runs (phi not 16-byte aligned) the class
    // rows (L2-resident, shared by the wall-layer cells) follow by the segment walk over the canonical rows
    const QuadArgs<T> q = quad_args<T>(*pl);
    int64_t bu = (pl->nU + 127) / 128;
    if (EB_QUAD_PER_SM > 0) bu = std::min<int64_t>(bu, (int64_t)pl->nsm * EB_QUAD_PER_SM);
    if (bu > 0) {
      if (pl->R == 3) k_irr_quad<T, 3, ApplyEpi><<<(unsigned)bu, 128, 0, st>>>(a, q, ApplyEpi());
      else k_irr_quad<T, 2, ApplyEpi><<<(unsigned)bu, 128, 0, st>>>(a, q, ApplyEpi());
      eb::count_launch();
    }
    if (use_runs(a)) return cudaGetLastError();  // the class cells go on the template pass's stream
    const int64_t nrest = pl->nC;
    if (nrest > 0) {
      ApplyArgs<T> c = a;
      c.n_irr = nrest;
      c.irr_cell = pl->cellC;
      c.irr_row = pl->classC;
      const int64_t bc = (nrest + 255) / 256;
      if (pl->R == 3) k_apply_irregular_seg<T, 3, 3><<<(unsigned)bc, 256, 0, st>>>(c, pl->nx, pl->ny, pl->nz);
      else k_apply_irregular_seg<T, 2, 3><<<(unsigned)bc, 256, 0, st>>>(c, pl->nx, pl->ny, pl->nz);
      eb::count_launch();
    }
    return cudaGetLastError();
  }
  if (pl && pl->seg) {
    if (pl->dim == 3 && pl->R == 3) k_apply_irregular_seg<T, 3, 3><<<(unsigned)nb, 256, 0, st>>>(a, pl->nx, pl->ny, pl->nz);
    else if (pl->dim == 3 && pl->R == 2) k_apply_irregular_seg<T, 2, 3><<<(unsigned)nb, 256, 0, st>>>(a, pl->nx, pl->ny, pl->nz);
    else if (pl->dim == 2 && pl->R == 3) k_apply_irregular_seg<T, 3, 2><<<(unsigned)nb, 256, 0, st>>>(a, pl->nx, pl->ny, pl->nz);
    else k_apply_irregular_seg<T, 2, 2><<<(unsigned)nb, 256, 0, st>>>(a, pl->nx, pl->ny, pl->nz);
  } else {
    k_apply_irregular<T><<<(unsigned)nb, 256, a.nfoot * 4, st>>>(a);
  }
  eb::count_launch();
  return cudaGetLastError();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static const EncodeTiledFn fn = [] {  // looked up once (thread-safe static initialisation)
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

template <typename T, int R, int D, bool ZSYM>
static cudaError_t launch_tma(const ApplyArgs<T>& a, const ApplyPlan& pl, cudaStream_t s) {
  constexpr int L = R + 1;
  constexpr int S = 2 * L + 1;
  constexpr int NP = D == 3 ? S + 1 : 1;
  constexpr int PX = TT_OX + 2 * TT_XH, PY = TT_OY + 2 * L;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  cuuint64_t gdim[3] = {(cuuint64_t)pl.nx, (cuuint64_t)pl.ny, (cuuint64_t)pl.nz};
  cuuint64_t gstr[2] = {(cuuint64_t)pl.nx * sizeof(T), (cuuint64_t)pl.nx * pl.ny * sizeof(T)};
  cuuint32_t box[3] = {PX, PY, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(&map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                   (void*)a.phi, gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  TmplCoef<T, R> cf;
  const T* cube;
  if constexpr (sizeof(T) == 4) cube = ZSYM ? pl.zcube32.data() : pl.cube32.data();
  else cube = ZSYM ? pl.zcube64.data() : pl.cube64.data();
  for (int i = 0; i < S * S * S; ++i) cf.c[i] = cube[i];
  TmplArgs<T> ta;
  ta.nx = pl.nx;
  ta.ny = pl.ny;
  ta.nz = pl.nz;
  ta.ntx = (pl.nx + TT_OX - 1) / TT_OX;
  ta.nty = (pl.ny + TT_OY - 1) / TT_OY;
  ta.zchunk = D == 3 ? 8 : 1;
  ta.nzc = (pl.nz + ta.zchunk - 1) / ta.zchunk;
  ta.items = (int64_t)ta.ntx * ta.nty * ta.nzc;
  ta.kind = a.kind;
  ta.inv_kappa = a.inv_kappa;
  ta.y = a.y;
  ta.kappa_weighted = a.kappa_weighted;
  ta.err = pl.err;
  constexpr size_t SLOT = ((PX * PY * sizeof(T) + 127) / 128) * 128;  // ring slot bytes (128-byte aligned TMA writes)
  size_t smem = (size_t)NP * SLOT + NP * 8;
  auto kern = k_apply_tma<T, R, D, ZSYM>;
  // attribute and occupancy are per device; kept for the last device seen
  static int cached_dev = -1, cached_per_sm = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev != cached_dev) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached_per_sm, kern, TT_THREADS, smem);
    if (e != cudaSuccess) return e;
    cached_dev = dev;
  }
  int per_sm = cached_per_sm;
  int64_t grid = (int64_t)pl.nsm * (per_sm > 0 ? per_sm : 1);
  if (grid > ta.items) grid = ta.items;
  kern<<<(unsigned)grid, TT_THREADS, smem, s>>>(map, cf, ta); eb::count_launch();
  return cudaGetLastError();
}

// tensor map of phi for the staged planes (TT_OX + 2 TT_XH) x (TT_OY + 2L) of the template passes
template <typename T, int L>
static cudaError_t phi_map(const ApplyArgs<T>& a, const ApplyPlan& pl, CUtensorMap* map) {
  constexpr int PX = TT_OX + 2 * TT_XH, PY = TT_OY + 2 * L;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t gdim[3] = {(cuuint64_t)pl.nx, (cuuint64_t)pl.ny, (cuuint64_t)pl.nz};
  cuuint64_t gstr[2] = {(cuuint64_t)pl.nx * sizeof(T), (cuuint64_t)pl.nx * pl.ny * sizeof(T)};
  cuuint32_t box[3] = {PX, PY, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                   (void*)a.phi, gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

#ifndef EB_FOLD_PER_SM
#define EB_FOLD_PER_SM 1  // persistent CTAs per SM of the folded template pass (0: as many as fit)
#endif

template <typename T, int R>
static cudaError_t launch_fold(const ApplyArgs<T>& a, const ApplyPlan& pl, cudaStream_t s) {
  constexpr int L = R + 1, F = L + 1;
  static_assert(FD_OX == TT_OX && FD_PX == TT_OX + 2 * TT_XH, "staged plane of the tensor map");
  CUtensorMap map;
  cudaError_t e = phi_map<T, L>(a, pl, &map);
  if (e != cudaSuccess) return e;
  FoldCoef<T, R> cf;
  for (int i = 0; i < F * F * F; ++i) cf.c[i] = sizeof(T) == 4 ? (T)pl.fold32[i] : (T)pl.fold64[i];
  TmplArgs<T> ta;
  ta.nx = pl.nx;
  ta.ny = pl.ny;
  ta.nz = pl.nz;
  ta.ntx = (pl.nx + FD_OX - 1) / FD_OX;
  ta.nty = (pl.ny + FD_OY - 1) / FD_OY;
  ta.zchunk = 8;
  ta.nzc = (pl.nz + ta.zchunk - 1) / ta.zchunk;
  ta.items = (int64_t)ta.ntx * ta.nty * ta.nzc;
  ta.kind = a.kind;
  ta.inv_kappa = a.inv_kappa;
  ta.y = a.y;
  ta.kappa_weighted = a.kappa_weighted;
  ta.err = pl.err;
  constexpr size_t smem = fold_smem<T, R>();
  auto kern = k_apply_fold<T, R>;
  static int cached_dev = -1, cached_per_sm = 0;  // per device: attribute set, occupancy
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev != cached_dev) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached_per_sm, kern, FD_THREADS, smem))) return e;
    cached_dev = dev;
  }
  int per_sm = cached_per_sm > 0 ? cached_per_sm : 1;
  if (EB_FOLD_PER_SM > 0 && per_sm > EB_FOLD_PER_SM) per_sm = EB_FOLD_PER_SM;
  int64_t grid = (int64_t)pl.nsm * per_sm;
  if (grid > ta.items) grid = ta.items;
  kern<<<(unsigned)grid, FD_THREADS, smem, s>>>(map, cf, ta);
  eb::count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_template_pass(const ApplyArgs<T>& a, cudaStream_t s) {
  const ApplyPlan* pl = a.plan;
  bool tma = pl && (sizeof(T) == 4 ? pl->tma32 : pl->tma64);
  if (tma && pl->dim == 3 && pl->fsym) {
    if (pl->R == 3) return launch_fold<T, 3>(a, *pl, s);
    if (pl->R == 2) return launch_fold<T, 2>(a, *pl, s);
  }
  if (tma) {
    if (pl->dim == 3 && pl->R == 3)
      return pl->zsym ? launch_tma<T, 3, 3, true>(a, *pl, s) : launch_tma<T, 3, 3, false>(a, *pl, s);
    if (pl->dim == 3 && pl->R == 2)
      return pl->zsym ? launch_tma<T, 2, 3, true>(a, *pl, s) : launch_tma<T, 2, 3, false>(a, *pl, s);
    if (pl->dim == 2 && pl->R == 3) return launch_tma<T, 3, 2, false>(a, *pl, s);
    if (pl->dim == 2 && pl->R == 2) return launch_tma<T, 2, 2, false>(a, *pl, s);
  }
  size_t sm = ((a.nfoot * 4 + 15) / 16) * 16 + a.nfoot * sizeof(T);
  int64_t nb = (a.ncell + 255) / 256;
  k_apply_template<T, 32><<<(unsigned)nb, 256, sm, s>>>(a); eb::count_launch();
  return cudaGetLastError();
}

// y_j = sum_i M_ij phi_i over the cells i whose footprint holds j (M = kappa L, or L when not
// kappa-weighted: phi_i / kappa_i): the rows read in transposed order, one thread per output cell, no
// atomics.  Covered cells get 0.
template <typename T>
__global__ void __launch_bounds__(256) k_apply_transpose(ApplyArgs<T> a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.ncell) return;
  if (a.kind[j] == 0) {
    a.y[j] = (T)0;
    return;
  }
  const int jx = (int)(j % a.nx), jy = (int)((j / a.nx) % a.ny), jz = (int)(j / ((int64_t)a.nx * a.ny));
  T acc = 0;
  for (int k = 0; k < a.nfoot; ++k) {
    const int ix = jx - a.foot_d[3 * k], iy = jy - a.foot_d[3 * k + 1], iz = jz - a.foot_d[3 * k + 2];
    if ((unsigned)ix >= (unsigned)a.nx || (unsigned)iy >= (unsigned)a.ny || (unsigned)iz >= (unsigned)a.nz) continue;
    const int64_t i = ix + (int64_t)a.nx * (iy + (int64_t)a.ny * iz);
    const uint8_t ki = a.kind[i];
    if (ki == 0) continue;
    const T m = ki == 1 ? a.tmpl[k] : a.rows[(int64_t)k * a.n_rows + a.row_of_cell[i]];
    const T p = a.kappa_weighted ? a.phi[i] : a.phi[i] * (T)a.inv_kappa[i];
    acc = fma(m, p, acc);
  }
  a.y[j] = acc;
}

template <typename T>
cudaError_t launch_apply(const ApplyArgs<T>& a, cudaStream_t s) {
  if (a.transpose) {
    k_apply_transpose<T><<<(unsigned)((a.ncell + 255) / 256), 256, 0, s>>>(a);
    eb::count_launch();
    return cudaGetLastError();
  }
  const ApplyPlan* pl = a.plan;
  cudaError_t e;
  bool fork = pl && pl->side && a.n_irr > 0;
  if (fork) {
    // the irregular rows run on the side stream, overlapped with the template pass (disjoint cells).
    // The template pass is launched first: its persistent grid takes a few CTAs per SM and the
    // HBM-bound row stream fills the rest of each SM, so the two run at the same time.
    if ((e = cudaEventRecord(pl->fork, s))) return e;
    if ((e = cudaStreamWaitEvent(pl->side, pl->fork, 0))) return e;
  }
  if ((e = launch_template_pass<T>(a, s))) return e;
  if (a.n_irr > 0) {
    if ((e = launch_irregular<T>(a, fork ? pl->side : s))) return e;
  }
  if (a.n_irr > 0 && use_runs(a)) {
    // the wall-layer class cells (FMA-bound, rows L2-resident) follow the template pass on the main
    // stream while the HBM-bound unique-row stream runs on the side stream
    if ((e = launch_runs<T>(a, s))) return e;
    if (pl->brick && (e = launch_brick<T>(a, s))) return e;
    if (pl->nL > 0 && (e = launch_seg_rest<T>(a, s))) return e;
  }
  if (fork) {
    if ((e = cudaEventRecord(pl->join, pl->side))) return e;
    if ((e = cudaStreamWaitEvent(s, pl->join, 0))) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_apply<float>(const ApplyArgs<float>&, cudaStream_t);
template cudaError_t launch_apply<double>(const ApplyArgs<double>&, cudaStream_t);

}  // namespace eb
