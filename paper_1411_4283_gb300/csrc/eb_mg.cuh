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
};

cudaError_t mg_setup(const MgFineInput& in, Multigrid* mg, cudaStream_t s);
void mg_free(Multigrid* mg);
template <typename T>
cudaError_t mg_precond(const Multigrid& mg, const T* r, T* z, cudaStream_t s);

}  // namespace eb
