#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "eb_apply.cuh"
#include "eb_mg.cuh"

namespace eb {

cudaError_t vec_fill64(int64_t n, double* x, double v, cudaStream_t s);
cudaError_t compute_rhs(int64_t n, const uint8_t* flag, const double* kappa, const double* rho, const double* bg,
                        double* out, cudaStream_t s);
cudaError_t launch_bg(int64_t n_irr, const int32_t* irr_cell, const int64_t* bptr, const int64_t* bcol,
                      const double* bval, int64_t n_grid_faces, const int64_t* wall_pos, const double* g_eb,
                      const double* g_wall, const double* inv_kappa, int kw, double* out, cudaStream_t s);
cudaError_t launch_norms(int64_t n, const uint8_t* flag, const double* kappa, const double* e, double* out,
                         cudaStream_t s);
template <typename T>
cudaError_t bicgstab(const ApplyArgs<T>& A, const T* b, T* x, const T* dinv, T* work, int64_t n, double tol,
                     int maxit, double* dscr, int* iters, double* relres, cudaStream_t s, const Multigrid* mg);
cudaError_t resid64(int64_t n, const double* b, const double* y, double* r, cudaStream_t s);
cudaError_t to32(int64_t n, const double* a, double scale, float* o, cudaStream_t s);
cudaError_t add32(int64_t n, double* x, double scale, const float* d, cudaStream_t s);
cudaError_t fill32(int64_t n, float* x, float v, cudaStream_t s);
cudaError_t norm2_64(int64_t n, const double* a, double* dscr, double* out, cudaStream_t s);
cudaError_t any_nonzero64(int64_t n, const double* a, int32_t* dflag, bool* out, cudaStream_t s);
// Device-resident BiCGStab scalars (FP64): slots of the running dot products; alpha and omega follow
enum { SC_RHO0 = 0, SC_RHO1 = 1, SC_RV = 2, SC_TS = 3, SC_TT = 4, SC_RR = 5, SC_BB = 6, SC_N = 8 };

// ---- batched refined solve (eb_solve.cu): one CUDA graph for several independent systems
// Device control block of one system: parameters, loop state and the loops' condition handles.
struct BatchCtl {
  double tol, inner_tol;
  int32_t max_outer, max_inner, max_iters;
  int32_t status;        // 0 running, 1 converged, 2 iteration caps reached, 3 FP32 breakdown or non-finite residual
  double bnorm2;         // ||rhs||^2
  double rn2;            // ||rhs - kappa L phi||^2 of the current sweep (FP64)
  double rn, scale;      // its norm and 1 / norm
  double rel_residual;   // rn / ||rhs||
  double inner_relres;   // the inner solve's recurrence residual
  int32_t sweeps, it, total, active, n_hist, runs;  // runs: sweep bodies executed
  double hist[64];
  cudaGraphConditionalHandle ho, hi;  // outer (sweeps) and inner (BiCGStab) loop conditions
};
// One system of the batch: its operators, preconditioner and vectors (device, owned by the caller)
struct BatchSys {
  ApplyArgs<double> A64;
  ApplyArgs<float> A32;
  const Multigrid* mg;  // null: Jacobi with dinv32
  const float* dinv32;
  int64_t n;
  double *rhs, *phi, *y64, *r64;
  float *b32, *x32, *w32;  // w32: 8 n
  double* sc;              // SC_N + 2 BiCGStab scalars
  BatchCtl* ctl;
  cudaGraphConditionalHandle ctl_hi_host;  // the inner loop's handle (set by batch_graph)
  long long k_sweep, k_iter;               // kernels per sweep body and per inner iteration (set by batch_graph)
};
// Builds and instantiates the graph; writes the loop handles into each ctl (H2D, stream s) and each
// system's kernel counts per sweep body and per inner iteration (launch accounting).
cudaError_t batch_graph(std::vector<BatchSys>& sys, cudaGraph_t* graph, cudaGraphExec_t* exec, cudaStream_t s);
cudaError_t batch_dots(int64_t n, const double* a, double* out, cudaStream_t s);  // out = a . a (accumulated)

void set_apply_timer(void* t);
void* new_apply_timer();
void free_apply_timer(void* p, double* ms, long long* n);

}  // namespace eb
