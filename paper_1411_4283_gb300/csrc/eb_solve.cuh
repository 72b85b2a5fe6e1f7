#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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
void set_apply_timer(void* t);
void* new_apply_timer();
void free_apply_timer(void* p, double* ms, long long* n);

}  // namespace eb
