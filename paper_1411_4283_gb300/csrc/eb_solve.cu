// Linear solve of the kappa-weighted system kappa L phi = kappa (rho - B g)
// (the paper uses PETSc GMRES + algebraic multigrid, Sec. 3.2; here a
// BiCGStab written for the GPU, preconditioned by a geometric multigrid
// V-cycle (eb_mg.cu) or by Jacobi):
//   mixed: FP32 BiCGStab inner solves on the FP32 operator copy, wrapped in
//          FP64 iterative refinement whose residual uses the FP64 operator;
//   plain: FP64 BiCGStab throughout.
// Dot products are summed across threads in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string.h>

#include <vector>

#include "eb_apply.cuh"
#include "eb_internal.cuh"
#include "eb_solve.cuh"
#include "eb_mg.cuh"

namespace eb {

constexpr int VB = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// out[k] += sum_i a_k[i] * b_k[i] for up to 3 pairs (FP64 accumulation)
template <typename T>
__global__ void k_dots(int64_t n, const T* a0, const T* b0, const T* a1, const T* b1, const T* a2, const T* b2,
                       double* out) {
  __shared__ double sh[32];
  double s0 = 0, s1 = 0, s2 = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    s0 += (double)a0[i] * (double)b0[i];
    if (a1) s1 += (double)a1[i] * (double)b1[i];
    if (a2) s2 += (double)a2[i] * (double)b2[i];
  }
  s0 = block_sum(s0, sh);
  __syncthreads();
  if (a1) { s1 = block_sum(s1, sh); __syncthreads(); }
  if (a2) { s2 = block_sum(s2, sh); __syncthreads(); }
  if (threadIdx.x == 0) {
    atomicAdd(out, s0);
    if (a1) atomicAdd(out + 1, s1);
    if (a2) atomicAdd(out + 2, s2);
  }
}




// r = b - y (FP64), on volumes only
__global__ void k_resid64(int64_t n, const double* b, const double* y, double* r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - y[i];
}

// r32 = scale * r64
__global__ void k_to32(int64_t n, const double* a, double scale, float* o) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = (float)(scale * a[i]);
}

// x64 += scale * d32
__global__ void k_add32(int64_t n, double* x, double scale, const float* d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += scale * (double)d[i];
}

template <typename T>
__global__ void k_fill(int64_t n, T* x, T v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

template <typename T>
__global__ void k_copy(int64_t n, const T* a, T* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = a[i];
}

// rhs = kappa rho - Bg_kw on volumes, 0 on covered cells
__global__ void k_rhs(int64_t n, const uint8_t* flag, const double* kappa, const double* rho, const double* bg,
                      double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = flag[i] ? kappa[i] * rho[i] - bg[i] : 0.0;
}

// norms of Sec. 3.3: [sum |e| kappa, sum e^2 kappa, sum kappa, max |e|] over volumes
__global__ void k_norms(int64_t n, const uint8_t* flag, const double* kappa, const double* e, double* out) {
  __shared__ double sh[32];
  double a = 0, b = 0, c = 0, m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!flag[i]) continue;
    double v = fabs(e[i]), k = kappa[i];
    a += v * k;
    b += v * v * k;
    c += k;
    m = fmax(m, v);
  }
  a = block_sum(a, sh); __syncthreads();
  b = block_sum(b, sh); __syncthreads();
  c = block_sum(c, sh); __syncthreads();
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  __shared__ double mx[32];
  if ((threadIdx.x & 31) == 0) mx[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, mx[w]);
    atomicAdd(out, a);
    atomicAdd(out + 1, b);
    atomicAdd(out + 2, c);
    atomicMax((unsigned long long*)(out + 3), (unsigned long long)__double_as_longlong(m));
  }
}

// B g (kappa-weighted B, CSR over irregular cells)
__global__ void k_bg(int64_t n_irr, const int32_t* irr_cell, const int64_t* bptr, const int64_t* bcol,
                     const double* bval, int64_t n_grid_faces, const int64_t* wall_pos, const double* g_eb,
                     const double* g_wall, const double* inv_kappa, int kw, double* out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_irr) return;
  double acc = 0.0;
  for (int64_t k = bptr[t]; k < bptr[t + 1]; ++k) {
    int64_t col = bcol[k];
    double g = col >= n_grid_faces ? g_eb[col - n_grid_faces] : g_wall[wall_pos[k]];
    acc += bval[k] * g;
  }
  int64_t c = irr_cell[t];
  out[c] = kw ? acc : acc * inv_kappa[c];
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + VB - 1) / VB;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

// ----------------------------------------------------------------- host drivers

cudaError_t vec_fill64(int64_t n, double* x, double v, cudaStream_t s) {
  k_fill<double><<<grid_for(n), VB, 0, s>>>(n, x, v); eb::count_launch();
  return cudaGetLastError();
}

cudaError_t compute_rhs(int64_t n, const uint8_t* flag, const double* kappa, const double* rho, const double* bg,
                        double* out, cudaStream_t s) {
  k_rhs<<<grid_for(n), VB, 0, s>>>(n, flag, kappa, rho, bg, out); eb::count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bg(int64_t n_irr, const int32_t* irr_cell, const int64_t* bptr, const int64_t* bcol,
                      const double* bval, int64_t n_grid_faces, const int64_t* wall_pos, const double* g_eb,
                      const double* g_wall, const double* inv_kappa, int kw, double* out, cudaStream_t s) {
  if (n_irr == 0) return cudaSuccess;
  k_bg<<<(unsigned)((n_irr + 255) / 256), 256, 0, s>>>(n_irr, irr_cell, bptr, bcol, bval, n_grid_faces, wall_pos,
                                                       g_eb, g_wall, inv_kappa, kw, out); eb::count_launch();
  return cudaGetLastError();
}

cudaError_t launch_norms(int64_t n, const uint8_t* flag, const double* kappa, const double* e, double* out,
                         cudaStream_t s) {
  k_norms<<<grid_for(n), VB, 0, s>>>(n, flag, kappa, e, out); eb::count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t dots(int64_t n, const T* a0, const T* b0, const T* a1, const T* b1, const T* a2, const T* b2,
                        double* dev, double* host, int cnt, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(dev, 0, 3 * sizeof(double), s);
  if (e) return e;
  k_dots<T><<<grid_for(n), VB, 0, s>>>(n, a0, b0, a1, b1, a2, b2, dev); eb::count_launch();
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(host, dev, cnt * sizeof(double), cudaMemcpyDeviceToHost, s))) return e;
  return cudaStreamSynchronize(s);
}

// Device time of every operator apply issued by the solver, from CUDA events
// on the solve stream.  Event pairs are read back lazily (at the next use of
// the same pair, by which time the solver's per-iteration synchronisation has
// completed them), so timing adds no synchronisation of its own.
struct ApplyTimer {
  cudaEvent_t e0[4] = {}, e1[4] = {};
  bool pending[4] = {false, false, false, false};
  int next = 0;
  double ms = 0.0;
  long long n = 0;
  void collect(int k) {
    if (!pending[k]) return;
    cudaEventSynchronize(e1[k]);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0[k], e1[k]);
    ms += t;
    n += 1;
    pending[k] = false;
  }
};
static ApplyTimer* g_timer = nullptr;
void set_apply_timer(void* t) { g_timer = (ApplyTimer*)t; }
void* new_apply_timer() {
  ApplyTimer* t = new ApplyTimer();
  for (int k = 0; k < 4; ++k) {
    cudaEventCreate(&t->e0[k]);
    cudaEventCreate(&t->e1[k]);
  }
  return t;
}
void free_apply_timer(void* p, double* ms, long long* n) {
  ApplyTimer* t = (ApplyTimer*)p;
  if (!t) return;
  for (int k = 0; k < 4; ++k) t->collect(k);
  *ms = t->ms;
  *n = t->n;
  for (int k = 0; k < 4; ++k) {
    cudaEventDestroy(t->e0[k]);
    cudaEventDestroy(t->e1[k]);
  }
  delete t;
}

template <typename T>
static cudaError_t timed_apply(const ApplyArgs<T>& A, cudaStream_t s) {
  if (!g_timer) return launch_apply<T>(A, s);
  int k = g_timer->next;
  g_timer->next = (k + 1) & 3;
  g_timer->collect(k);
  cudaEventRecord(g_timer->e0[k], s);
  cudaError_t e = launch_apply<T>(A, s);
  cudaEventRecord(g_timer->e1[k], s);
  g_timer->pending[k] = true;
  return e;
}

// The iteration kernels' dot products: per-thread partial sums accumulate in the vector precision
// (a thread handles at most a few dozen elements), the block and grid sums in FP64.  FP64
// arithmetic is slow on this GPU, so FP32 vectors keep their per-element work in FP32.


__device__ __forceinline__ void block_accumulate(double v, double* dst, double* sh) {
  v = block_sum(v, sh);
  if (threadIdx.x == 0) atomicAdd(dst, v);
}

// p = r + beta (p - omega v), beta = (rho_i / rho_{i-1}) (alpha / omega); phat = dinv p.
// Also clears the slot of (rhat, v) for this iteration.
// itp (batched solve): the iteration count on the device; q and first follow from it
template <typename T>
__global__ void k_bs_p(int64_t n, const T* r, const T* v, T* p, T* ph, const T* dinv, double* sc, int q, int first,
                       const double* ao, const int32_t* itp) {
  if (itp) {
    q = *itp & 1;
    first = *itp == 0;
  }
  double beta = 0.0, omega = 0.0;
  if (!first) {
    double rho = sc[q], rho_old = sc[1 - q];
    omega = ao[1];
    beta = (rho_old != 0.0 && omega != 0.0) ? (rho / rho_old) * (ao[0] / omega) : 0.0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T pi = first ? r[i] : r[i] + (T)beta * (p[i] - (T)omega * v[i]);
    p[i] = pi;
    if (dinv) ph[i] = dinv[i] * pi;  // Jacobi; the multigrid preconditioner writes ph itself
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[SC_RV] = 0.0;
}

// (rhat, v) -> sc[SC_RV]
template <typename T>
__global__ void k_bs_dot_rv(int64_t n, const T* rh, const T* v, double* sc) {
  __shared__ double sh[32];
  T a = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a = fma(rh[i], v[i], a);
  block_accumulate((double)a, sc + SC_RV, sh);
}

// alpha = rho_i / (rhat, v); s = r - alpha v; shat = dinv s.  Clears the slots filled later this iteration.
template <typename T>
__global__ void k_bs_s(int64_t n, const T* r, const T* v, T* s, T* shv, const T* dinv, double* sc, int q, double* ao,
                       const int32_t* itp) {
  if (itp) q = *itp & 1;
  double rv = sc[SC_RV];
  double alpha = rv != 0.0 ? sc[q] / rv : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T si = r[i] - (T)alpha * v[i];
    s[i] = si;
    if (dinv) shv[i] = dinv[i] * si;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ao[0] = alpha;
    sc[SC_TS] = 0.0;
    sc[SC_TT] = 0.0;
    sc[1 - q] = 0.0;
    sc[SC_RR] = 0.0;
  }
}

// (t, s) -> TS, (t, t) -> TT
template <typename T>
__global__ void k_bs_dot_ts(int64_t n, const T* t, const T* s, double* sc) {
  __shared__ double sh[32];
  T a = 0, b = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T ti = t[i];
    a = fma(ti, s[i], a);
    b = fma(ti, ti, b);
  }
  block_accumulate((double)a, sc + SC_TS, sh);
  __syncthreads();
  block_accumulate((double)b, sc + SC_TT, sh);
}

// omega = (t,s)/(t,t); x += alpha phat + omega shat; r = s - omega t; rho_{i+1} = (rhat, r); (r, r)
template <typename T>
__global__ void k_bs_x(int64_t n, T* x, const T* ph, const T* shv, T* r, const T* s, const T* t, const T* rh,
                       double* sc, int q, double* ao, const int32_t* itp) {
  __shared__ double sh[32];
  if (itp) q = *itp & 1;
  double alpha = ao[0];
  double omega = sc[SC_TT] > 0.0 ? sc[SC_TS] / sc[SC_TT] : 0.0;
  T a = 0, b = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += (T)alpha * ph[i] + (T)omega * shv[i];
    T ri = s[i] - (T)omega * t[i];
    r[i] = ri;
    a = fma(rh[i], ri, a);
    b = fma(ri, ri, b);
  }
  block_accumulate((double)a, sc + (1 - q), sh);
  __syncthreads();
  block_accumulate((double)b, sc + SC_RR, sh);
  if (blockIdx.x == 0 && threadIdx.x == 0) ao[1] = omega;
}

// r = b - r (in place, r holds A x); rhat = r; p = v = 0; rho_0 = (r, r) -> sc[0]; (b, b) -> sc[SC_BB]
template <typename T>
__global__ void k_bs_init(int64_t n, const T* bvec, T* r, T* rh, T* p, T* v, double* sc) {
  __shared__ double sh[32];
  double a = 0.0, bb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T ri = bvec[i] - r[i];
    r[i] = ri;
    rh[i] = ri;
    p[i] = (T)0;
    v[i] = (T)0;
    a += (double)ri * (double)ri;
    bb += (double)bvec[i] * (double)bvec[i];
  }
  block_accumulate(a, sc + SC_RHO0, sh);
  __syncthreads();
  block_accumulate(bb, sc + SC_BB, sh);
}

// Jacobi-preconditioned BiCGStab on A x = b (x in/out), scalars kept on the
// device; the host reads ||r||^2 once per iteration.  Returns iterations used
// and the recurrence's relative residual.
template <typename T>
cudaError_t bicgstab(const ApplyArgs<T>& A0, const T* b, T* x, const T* dinv, T* work, int64_t n, double tol,
                     int maxit, double* dscr, int* iters, double* relres, cudaStream_t s, const Multigrid* mg) {
  T* r = work;
  T* rh = work + n;
  T* p = work + 2 * n;
  T* v = work + 3 * n;
  T* ph = work + 4 * n;
  T* sv = work + 5 * n;
  T* shv = work + 6 * n;
  T* t = work + 7 * n;
  double* sc = dscr;        // SC_N slots
  double* ao = dscr + SC_N;  // alpha, omega
  ApplyArgs<T> A = A0;
  cudaError_t e;
  const unsigned G = grid_for(n);
  if ((e = cudaMemsetAsync(dscr, 0, (SC_N + 2) * sizeof(double), s))) return e;
  A.phi = x;
  A.y = r;
  if ((e = timed_apply<T>(A, s))) return e;
  k_bs_init<T><<<G, VB, 0, s>>>(n, b, r, rh, p, v, sc); eb::count_launch();
  double h[SC_N];
  if ((e = cudaMemcpyAsync(h, sc, SC_N * sizeof(double), cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  double bn = sqrt(h[SC_BB]);
  if (bn == 0.0) bn = 1.0;
  *relres = sqrt(h[SC_RHO0]) / bn;
  int it = 0;
  if (*relres <= tol) { *iters = 0; return cudaSuccess; }
  for (it = 1; it <= maxit; ++it) {
    int q = (it - 1) & 1;
    k_bs_p<T><<<G, VB, 0, s>>>(n, r, v, p, ph, mg ? nullptr : dinv, sc, q, it == 1, ao, nullptr); eb::count_launch();
    if (mg && (e = mg_precond<T>(*mg, p, ph, s))) return e;  // phat = V-cycle(p) instead of Jacobi
    A.phi = ph;
    A.y = v;
    if ((e = timed_apply<T>(A, s))) return e;
    k_bs_dot_rv<T><<<G, VB, 0, s>>>(n, rh, v, sc); eb::count_launch();
    k_bs_s<T><<<G, VB, 0, s>>>(n, r, v, sv, shv, mg ? nullptr : dinv, sc, q, ao, nullptr); eb::count_launch();
    if (mg && (e = mg_precond<T>(*mg, sv, shv, s))) return e;
    A.phi = shv;
    A.y = t;
    if ((e = timed_apply<T>(A, s))) return e;
    k_bs_dot_ts<T><<<G, VB, 0, s>>>(n, t, sv, sc); eb::count_launch();
    k_bs_x<T><<<G, VB, 0, s>>>(n, x, ph, shv, r, sv, t, rh, sc, q, ao, nullptr); eb::count_launch();
    if ((e = cudaMemcpyAsync(h, sc, SC_N * sizeof(double), cudaMemcpyDeviceToHost, s))) return e;
    if ((e = cudaStreamSynchronize(s))) return e;
    *relres = sqrt(h[SC_RR]) / bn;
    if (!(*relres > tol)) break;                                    // converged (or NaN: stop)
    if (h[1 - q] == 0.0 || h[SC_TT] == 0.0 || h[SC_RV] == 0.0) break;  // breakdown
  }
  *iters = it > maxit ? maxit : it;
  return cudaGetLastError();
}

template cudaError_t bicgstab<float>(const ApplyArgs<float>&, const float*, float*, const float*, float*, int64_t,
                                     double, int, double*, int*, double*, cudaStream_t, const Multigrid*);
template cudaError_t bicgstab<double>(const ApplyArgs<double>&, const double*, double*, const double*, double*,
                                      int64_t, double, int, double*, int*, double*, cudaStream_t, const Multigrid*);

cudaError_t resid64(int64_t n, const double* b, const double* y, double* r, cudaStream_t s) {
  k_resid64<<<grid_for(n), VB, 0, s>>>(n, b, y, r); eb::count_launch();
  return cudaGetLastError();
}
cudaError_t to32(int64_t n, const double* a, double scale, float* o, cudaStream_t s) {
  k_to32<<<grid_for(n), VB, 0, s>>>(n, a, scale, o); eb::count_launch();
  return cudaGetLastError();
}
cudaError_t add32(int64_t n, double* x, double scale, const float* d, cudaStream_t s) {
  k_add32<<<grid_for(n), VB, 0, s>>>(n, x, scale, d); eb::count_launch();
  return cudaGetLastError();
}
cudaError_t fill32(int64_t n, float* x, float v, cudaStream_t s) {
  k_fill<float><<<grid_for(n), VB, 0, s>>>(n, x, v); eb::count_launch();
  return cudaGetLastError();
}
// *nz = 1 when some a[i] != 0 (exact test, no reduction arithmetic)
__global__ void k_any_nonzero(int64_t n, const double* __restrict__ a, int32_t* nz) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (a[i] != 0.0) {
      *nz = 1;
      return;
    }
}

cudaError_t any_nonzero64(int64_t n, const double* a, int32_t* dflag, bool* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(dflag, 0, 4, s);
  if (e) return e;
  k_any_nonzero<<<grid_for(n), VB, 0, s>>>(n, a, dflag); eb::count_launch();
  int32_t h = 0;
  if ((e = cudaMemcpyAsync(&h, dflag, 4, cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  *out = h != 0;
  return cudaGetLastError();
}

cudaError_t norm2_64(int64_t n, const double* a, double* dscr, double* out, cudaStream_t s) {
  double h[3];
  cudaError_t e = dots<double>(n, a, a, nullptr, nullptr, nullptr, nullptr, dscr, h, 1, s);
  *out = sqrt(h[0]);
  return e;
}


// ----------------------------------------------------------------- batched refined solve
//
// Several independent systems (one per geometry) go through the refinement of eb_solve in one CUDA
// graph: per system a conditional WHILE node runs the refinement sweeps (the FP64 residual with the
// FP64 operator, the inner FP32 BiCGStab as a nested WHILE node, phi += its correction); one-thread
// control kernels set the loop conditions on the device from the device-resident scalars, so the
// systems' loops run side by side in one graph launch with no host synchronisation.  Every loop ends
// at its iteration cap: the control kernels count the iterations and clear the condition there.

cudaError_t batch_dots(int64_t n, const double* a, double* out, cudaStream_t s) {
  k_dots<double><<<grid_for(n), VB, 0, s>>>(n, a, a, nullptr, nullptr, nullptr, nullptr, out); eb::count_launch();
  return cudaGetLastError();
}

// after the FP64 residual of a sweep: stop (converged, caps, non-finite) or start an inner solve
__global__ void k_bt_outer(BatchCtl* c) {
  const double bn = c->bnorm2 > 0.0 ? sqrt(c->bnorm2) : 1.0;
  c->rn = sqrt(c->rn2);
  const double rel = c->rn / bn;
  c->runs += 1;
  c->rel_residual = rel;
  if (c->n_hist < 64) c->hist[c->n_hist++] = rel;
  int go = 0;
  if (c->status == 3) go = 0;  // the last inner solve broke down: phi is unchanged, stop
  else if (rel <= c->tol) c->status = 1;
  else if (!isfinite(rel)) c->status = 3;
  else if (c->sweeps >= c->max_outer || c->total >= c->max_iters) c->status = 2;
  else go = 1;
  c->active = go;
  if (go) {
    c->sweeps += 1;
    c->it = 0;
    c->scale = 1.0 / c->rn;
  }
  cudaGraphSetConditional(c->ho, go);
  cudaGraphSetConditional(c->hi, go);
}

// b32 = r64 / ||r64||, x32 = 0, r32 = 0 (A x for the zero guess)
__global__ void k_bt_prep(int64_t n, const BatchCtl* c, const double* r64, float* b32, float* x32, float* r32) {
  if (!c->active) return;
  const double sc = c->scale;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    b32[i] = (float)(sc * r64[i]);
    x32[i] = 0.0f;
    r32[i] = 0.0f;
  }
}

// the inner solve's initial residual: skip the loop when it already meets inner_tol
__global__ void k_bt_inner0(BatchCtl* c, const double* sc) {
  if (!c->active) return;
  const double bn = sc[SC_BB] > 0.0 ? sqrt(sc[SC_BB]) : 1.0;
  const double rel = sqrt(sc[SC_RHO0]) / bn;
  c->inner_relres = rel;
  if (!(rel > c->inner_tol)) cudaGraphSetConditional(c->hi, 0);
}

// after an inner iteration: the recurrence residual, breakdown and the caps decide whether to go on
__global__ void k_bt_inner(BatchCtl* c, const double* sc) {
  const int q = c->it & 1;
  const double bn = sc[SC_BB] > 0.0 ? sqrt(sc[SC_BB]) : 1.0;
  const double rr = sqrt(sc[SC_RR]) / bn;
  c->it += 1;
  c->total += 1;
  c->inner_relres = rr;
  int more = rr > c->inner_tol;
  if (sc[1 - q] == 0.0 || sc[SC_TT] == 0.0 || sc[SC_RV] == 0.0) more = 0;  // breakdown
  if (c->it >= c->max_inner || c->total >= c->max_iters) more = 0;
  if (!isfinite(rr)) {  // no usable correction: phi stays unchanged and the next sweep's control stops
    c->status = 3;
    c->active = 0;
    more = 0;
  }
  cudaGraphSetConditional(c->hi, more);
}

// phi += ||r|| x32
__global__ void k_bt_corr(int64_t n, const BatchCtl* c, double* phi, const float* x32) {
  if (!c->active) return;
  const double sc = c->rn;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    phi[i] += sc * (double)x32[i];
}

namespace {

// a WHILE node on the stream's capture, after its current dependencies; returns its body graph
cudaError_t add_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
  if (e) return e;
  if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp))) return e;
  *body = cp.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// one inner BiCGStab iteration of system y (the loop of bicgstab with the parity from the device)
cudaError_t capture_iteration(const BatchSys& y, cudaStream_t s) {
  const int64_t n = y.n;
  float* w = y.w32;
  float *r = w, *rh = w + n, *p = w + 2 * n, *v = w + 3 * n, *ph = w + 4 * n, *sv = w + 5 * n, *shv = w + 6 * n,
        *t = w + 7 * n;
  double* sc = y.sc;
  double* ao = y.sc + SC_N;
  const int32_t* itp = &y.ctl->it;
  const float* dinv = y.mg ? nullptr : y.dinv32;
  const unsigned G = grid_for(n);
  cudaError_t e;
  ApplyArgs<float> A = y.A32;
  k_bs_p<float><<<G, VB, 0, s>>>(n, r, v, p, ph, dinv, sc, 0, 0, ao, itp); eb::count_launch();
  if (y.mg && (e = mg_precond<float>(*y.mg, p, ph, s))) return e;
  A.phi = ph;
  A.y = v;
  if ((e = launch_apply<float>(A, s))) return e;
  k_bs_dot_rv<float><<<G, VB, 0, s>>>(n, rh, v, sc); eb::count_launch();
  k_bs_s<float><<<G, VB, 0, s>>>(n, r, v, sv, shv, dinv, sc, 0, ao, itp); eb::count_launch();
  if (y.mg && (e = mg_precond<float>(*y.mg, sv, shv, s))) return e;
  A.phi = shv;
  A.y = t;
  if ((e = launch_apply<float>(A, s))) return e;
  k_bs_dot_ts<float><<<G, VB, 0, s>>>(n, t, sv, sc); eb::count_launch();
  k_bs_x<float><<<G, VB, 0, s>>>(n, y.x32, ph, shv, r, sv, t, rh, sc, 0, ao, itp); eb::count_launch();
  k_bt_inner<<<1, 1, 0, s>>>(y.ctl, sc); eb::count_launch();
  return cudaGetLastError();
}

// one refinement sweep of system y: FP64 residual, control, inner solve (nested loop), correction
cudaError_t capture_sweep(BatchSys& y, cudaStream_t s, cudaStream_t s2) {
  const int64_t n = y.n;
  const unsigned G = grid_for(n);
  cudaError_t e;
  const long long c0 = eb::launches_so_far();
  ApplyArgs<double> A = y.A64;
  A.phi = y.phi;
  A.y = y.y64;
  if ((e = launch_apply<double>(A, s))) return e;
  k_resid64<<<G, VB, 0, s>>>(n, y.rhs, y.y64, y.r64); eb::count_launch();
  if ((e = cudaMemsetAsync(&y.ctl->rn2, 0, sizeof(double), s))) return e;
  if ((e = batch_dots(n, y.r64, &y.ctl->rn2, s))) return e;
  k_bt_outer<<<1, 1, 0, s>>>(y.ctl); eb::count_launch();
  float* r32 = y.w32;
  k_bt_prep<<<G, VB, 0, s>>>(n, y.ctl, y.r64, y.b32, y.x32, r32); eb::count_launch();
  if ((e = cudaMemsetAsync(y.sc, 0, (SC_N + 2) * sizeof(double), s))) return e;
  float* w = y.w32;
  k_bs_init<float><<<G, VB, 0, s>>>(n, y.b32, w, w + n, w + 2 * n, w + 3 * n, y.sc); eb::count_launch();
  k_bt_inner0<<<1, 1, 0, s>>>(y.ctl, y.sc); eb::count_launch();
  cudaGraph_t ib = nullptr;
  if ((e = add_while(s, y.ctl_hi_host, &ib))) return e;
  const long long c1 = eb::launches_so_far();
  if ((e = cudaStreamBeginCaptureToGraph(s2, ib, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) return e;
  cudaError_t ce = capture_iteration(y, s2);
  cudaGraph_t done = nullptr;
  e = cudaStreamEndCapture(s2, &done);
  if (ce) return ce;
  if (e) return e;
  const long long c2 = eb::launches_so_far();
  k_bt_corr<<<G, VB, 0, s>>>(n, y.ctl, y.phi, y.x32); eb::count_launch();
  y.k_iter = c2 - c1;
  y.k_sweep = (eb::launches_so_far() - c0) - y.k_iter;
  return cudaGetLastError();
}

}  // namespace

cudaError_t batch_graph(std::vector<BatchSys>& sys, cudaGraph_t* graph, cudaGraphExec_t* exec, cudaStream_t s) {
  *graph = nullptr;
  *exec = nullptr;
  cudaStream_t cs = nullptr, cs2 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (!e) e = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking);
  cudaGraph_t top = nullptr;
  if (!e) e = cudaGraphCreate(&top, 0);
  const long long before = eb::launches_so_far();
  for (size_t k = 0; k < sys.size() && !e; ++k) {
    BatchSys& y = sys[k];
    cudaGraphConditionalHandle ho, hi;
    if ((e = cudaGraphConditionalHandleCreate(&ho, top, 1, cudaGraphCondAssignDefault))) break;
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = ho;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, top, nullptr, nullptr, 0, &cp))) break;
    cudaGraph_t ob = cp.conditional.phGraph_out[0];
    if ((e = cudaGraphConditionalHandleCreate(&hi, ob, 0, 0))) break;
    y.ctl_hi_host = hi;
    if ((e = cudaMemcpyAsync(&y.ctl->ho, &ho, sizeof(ho), cudaMemcpyHostToDevice, s))) break;
    if ((e = cudaMemcpyAsync(&y.ctl->hi, &hi, sizeof(hi), cudaMemcpyHostToDevice, s))) break;
    if ((e = cudaStreamSynchronize(s))) break;
    if ((e = cudaStreamBeginCaptureToGraph(cs, ob, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
    cudaError_t ce = capture_sweep(y, cs, cs2);
    cudaGraph_t done = nullptr;
    e = cudaStreamEndCapture(cs, &done);
    if (ce) e = ce;
  }
  eb::uncount_launches(eb::launches_so_far() - before);  // capture issued no work
  if (!e) e = cudaGraphInstantiate(exec, top, 0);
  if (cs) cudaStreamDestroy(cs);
  if (cs2) cudaStreamDestroy(cs2);
  if (e) {
    if (top) cudaGraphDestroy(top);
    *exec = nullptr;
    return e;
  }
  *graph = top;
  return cudaSuccess;
}

}  // namespace eb
