#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eb {

template <typename T>
struct ApplyArgs {
  int64_t ncell;
  int nfoot;
  const int32_t* foot_off;  // [nfoot] linear offsets
  const T* tmpl;            // [nfoot] kappa-weighted template row
  const uint8_t* kind;      // [ncell] 0 covered, 1 template, 2 irregular
  const double* inv_kappa;  // [ncell]
  int64_t n_irr;
  const int32_t* irr_cell;
  const int32_t* irr_row;
  int64_t n_rows;
  const T* rows;            // [nfoot][n_rows]
  const T* phi;
  T* y;
  int kappa_weighted;
};

template <typename T>
cudaError_t launch_apply(const ApplyArgs<T>& a, cudaStream_t s);

}  // namespace eb
