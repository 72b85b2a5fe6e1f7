// Wall-slab pass of the operator apply (Sec. 2.3) for box neighbourhoods in
// 3-D: the class cells (rows shared by translation, away from the EB) in the
// five x layers next to each x wall (the wall layers of R <= 3).  There a cell's class changes with x
// but, away from the y and z walls, not with y or z, so the pass is laid out
// across y.  A unit is 32 consecutive y by BZ consecutive z cells of one x
// layer (blocks start L + 1 cells in from the low y and z walls, where the
// y and z wall layers end); the plan marks the units whose class cells all
// share one class (the others stay with the per-cell walk).  A CTA stages a
// brick of phi (16 x planes, 32 + 2L rows of y, BZ + 2L planes of z; zero
// outside the grid) in shared memory with y contiguous; warp w takes the unit
// of x layer w, copies its class row into shared memory, and lane i computes
// the BZ cells (y0 + i, z0 .. z0 + BZ - 1).  For each footprint column (dx, dy)
// a thread loads the BZ + 2L staged values along z once (consecutive lanes
// read consecutive words) and feeds every coefficient of the column (one
// broadcast shared-memory load) to BZ FMAs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "eb_apply_tma.cuh"  // fp_box

namespace eb {

constexpr int BR_W = 5;                      // x layers of a slab (one warp each): the L + 1 <= 5 wall layers
constexpr int BR_XH = 4;                     // staged x halo (>= L for R <= 3)
constexpr int BR_PX = BR_W + 2 * BR_XH;      // staged x planes
constexpr int BR_PY = 32 + 2 * BR_XH + 1;    // staged y pitch (odd: the staging writes spread over banks)
constexpr int BR_BZ = 8;                     // cells per thread along z

// canonical (z-major, then y, then x) index of the offset (dx, dy, dz) in the box footprint of radius R:
// planes |dz| = L hold (2R+1)^2 entries (|dx|, |dy| <= R); planes |dz| <= R hold a row of 2R+1 at
// dy = -L, rows of 2L+1 for |dy| <= R, and a row of 2R+1 at dy = L
template <int R>
__host__ __device__ constexpr int canon_idx(int dx, int dy, int dz) {
  constexpr int L = R + 1;
  constexpr int W = 2 * R + 1, WL = 2 * L + 1;
  constexpr int PA = W * W, PF = W + W * WL + W;
  if (dz == -L) return (dy + R) * W + (dx + R);
  const int base = PA + (dz + R) * PF;
  if (dz == L) return base + (dy + R) * W + (dx + R);
  if (dy == -L) return base + (dx + R);
  if (dy <= R) return base + W + (dy + R) * WL + (dx + L);
  return base + W + W * WL + (dx + R);
}

template <typename T>
struct BrickArgs {
  int nx, ny, nz;
  int nyb, nzb;                // y blocks of 32, z blocks of BR_BZ
  int y_org, z_org;            // blocks cover [y_org, y_hi) x [z_org, z_hi): the cells away from the y
  int y_hi, z_hi;              // and z wall layers
  const int32_t* unit_class;   // [2][BR_W][nzb][nyb]: the class of a uniform unit, -1 otherwise
  const T* rowsK;              // [n_class][nfoot] class rows, class-major, canonical order
  int nfoot;
  const T* phi;
  T* y;
  const double* inv_kappa;
  int kappa_weighted;
};

template <typename T, int R>
__global__ void __launch_bounds__(BR_W * 32) k_wall_brick(BrickArgs<T> a) {
  constexpr int L = R + 1;
  constexpr int BZ = BR_BZ;
  constexpr int PZ = BZ + 2 * L;
  constexpr int SY = 32 + 2 * L;  // staged rows of y
  constexpr int NF = (2 * R + 1) * (2 * R + 1) * (2 * R + 1) + 6 * (2 * R + 1) * (2 * R + 1);  // footprint
  static_assert(L <= BR_XH, "x halo");
  extern __shared__ __align__(16) unsigned char sm_brick[];
  T* S = reinterpret_cast<T*>(sm_brick);   // [PZ][BR_PX][BR_PY]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* Cw = S + (size_t)PZ * BR_PX * BR_PY + (size_t)warp * NF;  // this warp's class row
  int item = blockIdx.x;
  const int side = item & 1;
  item >>= 1;
  const int yblk = item % a.nyb, zblk = item / a.nyb;
  const int yb = a.y_org + 32 * yblk, zb = a.z_org + BZ * zblk;
  const int xs = side ? a.nx - BR_W : 0;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  for (int i = threadIdx.x; i < PZ * SY * BR_PX; i += blockDim.x) {
    const int xx = i % BR_PX, r = i / BR_PX, yy = r % SY, zz = r / SY;
    const int gx = xs - BR_XH + xx, gy = yb - L + yy, gz = zb - L + zz;
    T v = (T)0;
    if ((unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny && (unsigned)gz < (unsigned)nz)
      v = __ldg(a.phi + (gx + (int64_t)nx * (gy + (int64_t)ny * gz)));
    S[(zz * BR_PX + xx) * BR_PY + yy] = v;
  }
  const int ucls = a.unit_class[(((int64_t)side * BR_W + warp) * a.nzb + zblk) * a.nyb + yblk];
  if (ucls >= 0) {
    const T* __restrict__ row = a.rowsK + (int64_t)ucls * a.nfoot;
    for (int i = lane; i < NF; i += 32) Cw[i] = __ldg(row + i);
  }
  __syncthreads();
  const int y = yb + lane;
  if (ucls < 0 || y >= a.y_hi) return;
  const int x = xs + warp;
  const int sx = warp + BR_XH, sy = lane + L;
  T acc[BZ];
#pragma unroll
  for (int j = 0; j < BZ; ++j) acc[j] = (T)0;
  // dx is a runtime loop (one body for |dx| <= R, one for the arms |dx| = L, so that the code stays
  // small); the row of the canonical order that holds (dx, dy, dz) is contiguous in dx, so the
  // coefficient is Cw[canon_idx(0, dy, dz) + dx], a compile-time offset from Cw + dx
#pragma unroll 1
  for (int dx = -L; dx <= L; ++dx) {
    const T* cx = Cw + dx;
    const T* sc = S + (sx + dx) * BR_PY + sy;
    if (dx >= -R && dx <= R) {
#pragma unroll
      for (int dy = -L; dy <= L; ++dy) {
        T v[PZ];
#pragma unroll
        for (int q = 0; q < PZ; ++q) v[q] = sc[q * BR_PX * BR_PY + dy];
#pragma unroll
        for (int dz = -L; dz <= L; ++dz) {
          if (!fp_box(0, dy, dz, R)) continue;
          const T k = cx[canon_idx<R>(0, dy, dz)];
#pragma unroll
          for (int j = 0; j < BZ; ++j) acc[j] = fma(k, v[j + dz + L], acc[j]);
        }
      }
    } else {
#pragma unroll
      for (int dy = -R; dy <= R; ++dy) {
        T v[PZ];
#pragma unroll
        for (int q = 1; q < PZ - 1; ++q) v[q] = sc[q * BR_PX * BR_PY + dy];
#pragma unroll
        for (int dz = -R; dz <= R; ++dz) {
          const T k = cx[canon_idx<R>(0, dy, dz)];
#pragma unroll
          for (int j = 0; j < BZ; ++j) acc[j] = fma(k, v[j + dz + L], acc[j]);
        }
      }
    }
  }
  const int64_t c0 = x + (int64_t)nx * (y + (int64_t)ny * zb);
  const int64_t zs = (int64_t)nx * ny;
#pragma unroll
  for (int j = 0; j < BZ; ++j) {
    if (zb + j >= a.z_hi) break;
    const int64_t c = c0 + j * zs;
    a.y[c] = a.kappa_weighted ? acc[j] : acc[j] * (T)a.inv_kappa[c];
  }
}

// the class of each unit (side, x layer, z block, y block): the one class of all its cells inside the
// grid when they are all slab class cells of one class, else -1
__global__ void k_brick_units(const int32_t* __restrict__ slab, int ny, int nz, int nyb, int nzb, int y_org,
                              int z_org, int y_hi, int z_hi, int32_t* __restrict__ unit_class);

template <typename T, int R>
constexpr size_t brick_smem() {
  constexpr int NF = (2 * R + 1) * (2 * R + 1) * (2 * R + 1) + 6 * (2 * R + 1) * (2 * R + 1);
  return ((size_t)(BR_BZ + 2 * (R + 1)) * BR_PX * BR_PY + (size_t)BR_W * NF) * sizeof(T);
}

}  // namespace eb
