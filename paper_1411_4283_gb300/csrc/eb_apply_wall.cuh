// Wall-layer pass of the operator apply (Sec. 2.3) for box neighbourhoods in
// 3-D.  Cells within R+1 of the domain walls and away from the EB carry one of
// the shared "class" rows (the row depends only on the cell's position relative
// to the walls).  Along x, away from the x walls, four consecutive cells of a
// grid row have the same class, so one thread computes such a run of four:
// each segment of the footprint (a fixed (dy, dz), x-contiguous) is loaded once
// as 12 consecutive phi values by aligned vector loads, and every coefficient
// of the class row (one load, the same address across the warp) feeds four
// FMAs.  Against one thread per cell this takes the loads per cell from about
// 2 x 637 to about 450 / 4, which is what bounds the per-cell walk (L1
// wavefronts, not FMAs).
//
// Runs are aligned (first x a multiple of 4, nx a multiple of 4), and the
// loaded window x-4 .. x+7 stays inside the grid row; class cells that are not
// in such a run keep the per-cell segment walk of eb_apply.cu.  Segments whose
// (y, z) row leaves the grid have zero coefficients and are skipped.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eb {

template <typename T>
struct XqArgs {
  int64_t nG;              // runs
  const int32_t* cellG;    // [nG] first cell of the run
  const int32_t* classG;   // [nG] its class row
  const T* rowsK;          // [n_class][nfoot] class rows, class-major, canonical footprint order
  int nfoot;
  const T* phi;
  T* y;
  const double* inv_kappa;
  int kappa_weighted;
  int nx, ny, nz;
};

template <typename T, int N>
__device__ __forceinline__ void load_run(const T* p, T* v);
template <>
__device__ __forceinline__ void load_run<float, 12>(const float* p, float* v) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float4 w = __ldg(reinterpret_cast<const float4*>(p) + q);
    v[4 * q] = w.x;
    v[4 * q + 1] = w.y;
    v[4 * q + 2] = w.z;
    v[4 * q + 3] = w.w;
  }
}
template <>
__device__ __forceinline__ void load_run<double, 12>(const double* p, double* v) {
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const double2 w = __ldg(reinterpret_cast<const double2*>(p) + q);
    v[2 * q] = w.x;
    v[2 * q + 1] = w.y;
  }
}

constexpr int XQ_HALO = 4;  // x halo of a loaded run (>= L for R <= 3, a multiple of 4: aligned loads)

template <typename T, int R>
__global__ void __launch_bounds__(128) k_class_xquad(XqArgs<T> a) {
  constexpr int L = R + 1;
  constexpr int H = XQ_HALO;
  static_assert(L <= H, "x halo");
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.nG) return;
  const int64_t c = a.cellG[t];
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int64_t cr = c / nx;
  const int cy = (int)(cr % ny), cz = (int)(cr / ny);
  const int64_t nxy = (int64_t)nx * ny;
  const T* __restrict__ cf = a.rowsK + (int64_t)a.classG[t] * a.nfoot;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
  int idx = 0;  // canonical footprint index of the segment's first entry (a constant after unrolling)
#pragma unroll
  for (int dz = -L; dz <= L; ++dz) {
#pragma unroll
    for (int dy = -L; dy <= L; ++dy) {
      const int ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
      if (ay > R && az > R) continue;
      const int X = (ay > R || az > R) ? R : L;
      if ((unsigned)(cy + dy) < (unsigned)ny && (unsigned)(cz + dz) < (unsigned)nz) {
        T v[4 + 2 * H];
        load_run<T, 4 + 2 * H>(a.phi + (c - H + (int64_t)dy * nx + (int64_t)dz * nxy), v);
#pragma unroll
        for (int dx = -X; dx <= X; ++dx) {
          const T k = __ldg(cf + idx + dx + X);
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j] = fma(k, v[H + j + dx], acc[j]);
        }
      }
      idx += 2 * X + 1;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) a.y[c + j] = a.kappa_weighted ? acc[j] : acc[j] * (T)a.inv_kappa[c + j];
}

}  // namespace eb
