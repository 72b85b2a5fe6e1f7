// Operator apply: y = kappa .* (L phi) (or L phi), the homogeneous part of the
// flux-divergence Laplacian of Sec. 2.3.  Two passes:
//   K4  template cells: the translation-invariant cell stencil of the interior
//       (every face stencil there is the same weighted-LS template);
//   K5  irregular cells (near the EB or a domain wall): footprint-dense rows,
//       stored footprint-major so that consecutive rows load coalesced.
// Covered cells get y = 0.
#include <cuda_runtime.h>
#include <stdint.h>

#include "eb_apply.cuh"
#include "eb_internal.cuh"

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

template <typename T>
cudaError_t launch_apply(const ApplyArgs<T>& a, cudaStream_t s) {
  size_t sm = ((a.nfoot * 4 + 15) / 16) * 16 + a.nfoot * sizeof(T);
  int64_t nb = (a.ncell + 255) / 256;
  k_apply_template<T, 32><<<(unsigned)nb, 256, sm, s>>>(a); eb::count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.n_irr > 0) {
    int64_t nb2 = (a.n_irr + 255) / 256;
    k_apply_irregular<T><<<(unsigned)nb2, 256, a.nfoot * 4, s>>>(a); eb::count_launch();
    e = cudaGetLastError();
  }
  return e;
}

template cudaError_t launch_apply<float>(const ApplyArgs<float>&, cudaStream_t);
template cudaError_t launch_apply<double>(const ApplyArgs<double>&, cudaStream_t);

}  // namespace eb
