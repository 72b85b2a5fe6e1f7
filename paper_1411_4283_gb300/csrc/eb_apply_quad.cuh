// Irregular-row pass of the operator apply (Sec. 2.3) for box neighbourhoods
// in 3-D, with the row coefficients in an apply-specific "quad" layout.
//
// Footprint walk.  The footprint {|d|_inf <= R} plus the one-coordinate arms
// at |d_k| = L = R+1 is a union of x-contiguous segments: (2R+1)^2 "wide"
// segments (|dy|, |dz| <= R, dx in [-L, L]) and 4(2R+1) "narrow" ones (one of
// |dy|, |dz| = L, dx in [-R, R]).  The apply order lists the wide segments in
// groups of four (z-major), then the narrow ones in groups of four, then the
// one wide segment left over, so that every group spans a whole number of
// 4-coefficient quads; the tail is padded with zeros to a quad boundary.
//
// Coefficient layout (T = float or double, nq quads per row) of the unique
// rows (one per irregular cell near the EB), warp-interleaved:
//     qU[((u / 32) * nq + k) * 32 + u % 32][0..3]
// so that a warp loads 32 consecutive quads of one index k with one coalesced
// 16- or 32-byte load per lane.  The quad index of a group is a compile-time
// offset from one base pointer, so the inner loop issues one vector load per
// four coefficients, one phi load and one FMA per coefficient, and the
// coefficient stream (the bulk of the apply's bytes) runs near the HBM rate.
// Rows shared by the wall-layer cells (class rows, L2-resident) keep the
// canonical footprint-major layout and the segment walk of eb_apply.cu.  Segments whose (y, z) row leaves the
// grid have zero coefficients and read a zero buffer instead of phi; the few
// cells next to the first or last grid row (where a segment's x ends could
// leave the linear cell range) take a clamped per-entry path over the
// canonical footprint-major rows.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "eb_apply.cuh"

namespace eb {

__device__ __align__(16) static double g_zero_seg[16];  // zero phi for segments outside the grid

template <int R>
struct QuadShape {
  static constexpr int L = R + 1;
  static constexpr int W = 2 * R + 1;
  static constexpr int NW = W * W;            // wide segments
  static constexpr int NN = 4 * W;            // narrow segments
  static constexpr int EW = 2 * L + 1;        // entries of a wide segment
  static constexpr int EN = 2 * R + 1;        // entries of a narrow segment
  static constexpr int GW = NW / 4;           // full groups of wide segments (one wide segment is left over)
  static constexpr int GN = NN / 4;           // groups of narrow segments
  static constexpr int QW = EW;               // quads per wide group (4 * EW / 4)
  static constexpr int QN = EN;               // quads per narrow group
  static constexpr int QT = (EW + 3) / 4;     // quads of the left-over wide segment
  static constexpr int NQ = GW * QW + GN * QN + QT;
};

template <typename T>
__device__ __forceinline__ void load_quad(const T* p, T* out);
template <>
__device__ __forceinline__ void load_quad<float>(const float* p, float* out) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  out[0] = v.x;
  out[1] = v.y;
  out[2] = v.z;
  out[3] = v.w;
}
template <>
__device__ __forceinline__ void load_quad<double>(const double* p, double* out) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  out[0] = a.x;
  out[1] = a.y;
  out[2] = b.x;
  out[3] = b.y;
}

// phi pointer of the segment (dy, dz) of cell (cy, cz); a zero buffer when the row leaves the grid
template <typename T, int L>
__device__ __forceinline__ const T* seg_ptr(const T* __restrict__ phi, int64_t c, int cy, int cz, int dy, int dz, int nx,
                                            int ny, int nz) {
  const int yy = cy + dy, zz = cz + dz;
  if ((unsigned)yy < (unsigned)ny && (unsigned)zz < (unsigned)nz)
    return phi + (c + (int64_t)dy * nx + (int64_t)dz * nx * ny);
  return reinterpret_cast<const T*>(g_zero_seg) + L;
}

// NSEG segments of half-width X whose 4-coefficient quads start at gq (quad stride QS elements)
template <typename T, int X, int NSEG, int QS>
__device__ __forceinline__ void quad_group(const T* __restrict__ gq, const T* const* ph, T& acc0, T& acc1) {
  constexpr int E = 2 * X + 1;
  constexpr int NQ = (NSEG * E + 3) / 4;
  T cf[NQ * 4];
#pragma unroll
  for (int k = 0; k < NQ; ++k) load_quad<T>(gq + (size_t)k * QS, cf + 4 * k);
#pragma unroll
  for (int i = 0; i < NSEG; ++i) {
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const T v = __ldg(ph[i] + (j - X));
      if (j & 1) acc1 = fma(cf[i * E + j], v, acc1);
      else acc0 = fma(cf[i * E + j], v, acc0);
    }
  }
}

// Sum over the footprint of one cell; q: the row's first quad, QS: quad stride (elements)
template <typename T, int R, int QS>
__device__ __forceinline__ T quad_row(const T* __restrict__ q, const T* __restrict__ phi, int64_t c, int cy, int cz,
                                      int nx, int ny, int nz) {
  using S = QuadShape<R>;
  constexpr int L = S::L;
  T acc0 = 0, acc1 = 0;
  const T* gq = q;
#pragma unroll 1
  for (int g = 0; g < S::GW; ++g) {
    const T* ph[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int w = 4 * g + i;
      ph[i] = seg_ptr<T, L>(phi, c, cy, cz, w % S::W - R, w / S::W - R, nx, ny, nz);
    }
    quad_group<T, L, 4, QS>(gq, ph, acc0, acc1);
    gq += (size_t)S::QW * QS;
  }
#pragma unroll 1
  for (int g = 0; g < S::GN; ++g) {
    const T* ph[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int v = 4 * g + i, arm = v / S::W, j = v % S::W - R;
      const int dy = arm < 2 ? (arm == 0 ? -L : L) : j;
      const int dz = arm < 2 ? j : (arm == 2 ? -L : L);
      ph[i] = seg_ptr<T, L>(phi, c, cy, cz, dy, dz, nx, ny, nz);
    }
    quad_group<T, R, 4, QS>(gq, ph, acc0, acc1);
    gq += (size_t)S::QN * QS;
  }
  {
    const T* ph[1];
    ph[0] = seg_ptr<T, L>(phi, c, cy, cz, R, R, nx, ny, nz);  // the left-over wide segment (dy = dz = R)
    quad_group<T, L, 1, QS>(gq, ph, acc0, acc1);
  }
  return acc0 + acc1;
}

template <typename T>
struct QuadArgs {
  int64_t nU;                // cells with a unique row
  const int32_t* cellU;      // [nU] cell of unique row u (ascending)
  int64_t n_class;           // canonical row of unique row u is n_class + u
  const T* qU;
  int nx, ny, nz;
};

// Clamped footprint-major walk over the canonical rows (cells next to the first or last grid row)
template <typename T>
__device__ T canonical_row(const ApplyArgs<T>& a, int64_t c, int64_t row) {
  T acc = 0;
  const int64_t hi = a.ncell - 1;
  for (int i = 0; i < a.nfoot; ++i) {
    int64_t p = c + a.foot_off[i];
    p = p < 0 ? 0 : (p > hi ? hi : p);
    acc = fma(__ldg(a.rows + (int64_t)i * a.n_rows + row), __ldg(a.phi + p), acc);
  }
  return acc;
}

// Row sums (A x)_c over the unique-row cells; the epilogue decides what is stored.
// Grid-stride over the rows (the stride is a multiple of 32, so a warp keeps 32 consecutive rows):
// launched with a bounded grid, the pass leaves room on every SM for the template pass that runs
// beside it.
template <typename T, int R, class Epi>
__global__ void __launch_bounds__(128) k_irr_quad(ApplyArgs<T> a, QuadArgs<T> qa, Epi epi) {
  using S = QuadShape<R>;
  constexpr int L = S::L;
  const int nx = qa.nx, ny = qa.ny, nz = qa.nz;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < qa.nU; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = qa.cellU[t];
    const int cx = (int)(c % nx);
    const int64_t cr = c / nx;
    const int cy = (int)(cr % ny), cz = (int)(cr / ny);
    T acc;
    const bool edge = (cy <= L && cz <= L && cx < L) || (cy >= ny - 1 - L && cz >= nz - 1 - L && cx > nx - 1 - L);
    if (edge) {
      acc = canonical_row<T>(a, c, qa.n_class + t);
    } else {
      const T* q = qa.qU + (((t >> 5) * S::NQ) * 32 + (t & 31)) * 4;
      acc = quad_row<T, R, 128>(q, a.phi, c, cy, cz, nx, ny, nz);
    }
    epi(a, t, c, acc);
  }
}

template <typename T>
inline QuadArgs<T> quad_args(const ApplyPlan& pl) {
  QuadArgs<T> q;
  q.nU = pl.nU;
  q.cellU = pl.cellU;
  q.n_class = pl.n_class;
  if constexpr (sizeof(T) == 4) q.qU = pl.qU32;
  else q.qU = pl.qU64;
  q.nx = pl.nx;
  q.ny = pl.ny;
  q.nz = pl.nz;
  return q;
}

// the operator apply: y_c = (kappa L phi)_c, or (L phi)_c
struct ApplyEpi {
  template <typename T>
  __device__ __forceinline__ void operator()(const ApplyArgs<T>& a, int64_t, int64_t c, T acc) const {
    if (!a.kappa_weighted) acc *= (T)a.inv_kappa[c];
    a.y[c] = acc;
  }
};

}  // namespace eb
