#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace eb {

struct ApplyPlan;

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
  // fast template path (TMA tiles); null plan = generic kernels only
  const ApplyPlan* plan;
  // transposed apply y = (kappa L)^T phi (or L^T phi) in gather form, for the adjoint solve: the row
  // of every irregular cell (-1 elsewhere), the footprint offsets [nfoot][3] and the grid
  int transpose = 0;
  const int32_t* row_of_cell = nullptr;
  const int8_t* foot_d = nullptr;
  int nx = 0, ny = 0, nz = 0;
};

// Host-side launch plan of the apply, owned by eb_stencils.
struct ApplyPlan {
  int nx, ny, nz, dim, R;
  int tma32, tma64;              // template pass by TMA tiles possible (box metric, aligned rows)
  int seg;                       // box footprint: irregular rows by x-contiguous segments
  // irregular rows in the quad layout (3-D box neighbourhoods, R = 2 or 3; see eb_apply_quad.cuh)
  int quad = 0;
  int64_t nU = 0, nC = 0, n_class = 0;
  int32_t* cellU = nullptr;      // [nU] cells with a unique row, ascending (unique row u = canonical n_class + u)
  int32_t* cellC = nullptr;      // [nC] cells with a class row, ascending
  int32_t* classC = nullptr;     // [nC] their class row
  float* qU32 = nullptr;         // unique rows in the quad layout
  double* qU64 = nullptr;
  // class cells split into aligned x-runs of four with one class (eb_apply_wall.cuh) and the rest
  int64_t nG = 0, nL = 0;
  int32_t* cellG = nullptr;      // [nG] first cell of each run
  int32_t* classG = nullptr;     // [nG] class row of the run
  int32_t* cellL = nullptr;      // [nL] class cells outside the runs, ascending
  int32_t* classL = nullptr;     // [nL] their class row
  float* rowsK32 = nullptr;      // [n_class][nfoot] class rows, class-major
  double* rowsK64 = nullptr;
  // the class cells outside the runs that lie in the 5 x layers next to each x wall, by x-slab brick
  // (eb_apply_brick.cuh); cellL/classL then hold only the others
  int brick = 0;
  int32_t* slab_class = nullptr; // [2][5][nz][ny] class row of a slab cell, -1 otherwise
  int32_t* unit_class = nullptr; // [2][5][nzb][nyb] class of a uniform brick unit, -1 otherwise
  int nyb = 0, nzb = 0, y_org = 0, z_org = 0, y_hi = 0, z_hi = 0;
  std::vector<float> cube32;     // dense (2R+3)^3 template coefficients
  std::vector<double> cube64;
  int zsym = 0;                  // template symmetric in z (to a few ulps): z-folded template pass
  std::vector<float> zcube32;    // the cube with c(., ., a) = c(., ., -a) averaged (entries a >= 0 used)
  std::vector<double> zcube64;
  int fsym = 0;                  // template even in x, y and z (to a few ulps): fully folded pass (3-D)
  std::vector<float> fold32;     // T(a, b, c), a, b, c in 0..R+1: the mean of the cube's eight sign images
  std::vector<double> fold64;
  int32_t* err;                  // device error word (bounded waits)
  cudaStream_t side;             // irregular pass runs here, overlapped with the template pass
  cudaEvent_t fork, join;
  int nsm;
};

template <typename T>
cudaError_t launch_apply(const ApplyArgs<T>& a, cudaStream_t s);

}  // namespace eb
