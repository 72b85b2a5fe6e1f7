// Geometric multigrid preconditioner (see eb_mg.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>


namespace eb {

constexpr int MG_MAXLEV = 10;
constexpr int MG_NU = 2;  // pre- and post-smoothing sweeps

struct MgLevel {
  int n[3];
  int64_t ncell;
  float* cp[3] = {nullptr, nullptr, nullptr};  // coupling to the +d neighbour (1/h^2 alpha)
  float* dg = nullptr;                         // diagonal (0: covered)
  float* v32[3] = {nullptr, nullptr, nullptr};  // b, x, work (FP32 cycles)
  double* v64[3] = {nullptr, nullptr, nullptr};  // b, x, work (FP64 cycles)
};

struct Multigrid {
  int dim = 0;
  int nlev = 0;
  MgLevel lev[MG_MAXLEV];
  void* dev32 = nullptr;  // device descriptors of the levels (single-CTA coarse cycle)
  void* dev64 = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // captured V-cycle (FP32, FP64)
  long long nodes[2] = {0, 0};                    // kernels per replay
  // exact local solves of the high-order operator on 3x3x3 blocks around the cut cells whose
  // diagonal is weak or positive (multiplicative Schwarz step after the V-cycle)
  int nblk = 0;
  int32_t* blk_cells = nullptr;  // [nblk][27] cells (-1: none)
  double* blk_inv64 = nullptr;   // [nblk][27][27]
  float* blk_inv32 = nullptr;
  void* blk_res = nullptr;       // [nblk][27] doubles
  // row lookup of the high-order operator for the block kernels
  const int32_t* irr_cell = nullptr;
  const int32_t* irr_row = nullptr;
  int64_t n_irr = 0;
  const uint8_t* kind = nullptr;
  const double* tmpl64 = nullptr;
  const double* rows64 = nullptr;
  const float* rows32 = nullptr;
  const float* tmpl32 = nullptr;
  int64_t n_rows = 0;
  int nfoot = 0;
  const int32_t* foot_off = nullptr;
  int16_t* foot_lut = nullptr;    // [(2R+3)^3] footprint index of an offset (-1 outside)
  int R = 0;
  // 1: precondition the transposed operator (the adjoint solve): the V-cycle (on a symmetric
  // approximation) as it is, the block solves with A_BB^T
  int transpose = 0;
};

struct MgFineInput {
  int dim;
  int n[3];
  double h;
  const uint8_t* flag;
  const uint8_t* ff[3];
  const int32_t* cf[3];
  const double* fm[3];
  int KFS;
  const double* dinv_high;  // inverse diagonal of the high-order kappa-weighted operator
  // high-order rows for the local block solves
  const double* rows64;      // canonical rows [nfoot][n_rows]
  const float* rows32;
  int64_t n_rows;
  int nfoot, center;         // footprint size, index of the zero offset
  const int32_t* irr_cell;   // irregular cells (ascending) and their canonical rows
  const int32_t* irr_row;
  int64_t n_irr;
  const uint8_t* kind;       // 0 covered, 1 template, 2 irregular
  const double* tmpl64;      // template row
  const float* tmpl32;
  const int32_t* foot_off;   // linear offsets of the footprint entries
  int R, box;
};

cudaError_t mg_setup(const MgFineInput& in, Multigrid* mg, cudaStream_t s);
void mg_free(Multigrid* mg);
// z = V-cycle(r), then the local block solves of the high-order operator (multiplicative)
template <typename T>
cudaError_t mg_precond(const Multigrid& mg, const T* r, T* z, cudaStream_t s);

}  // namespace eb
