// Batched weighted minimum-norm least squares that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code running inside a memory pool or arena that owns all of the
// device memory it may touch, real-time or embedded hosts whose allocation
// happens once at start-up, and plugin hosts that forbid allocation in their
// callbacks.  eb_lsq_batch_noalloc serves them: the caller passes the inputs
// and outputs, and the per-warp working storage the solve needs lives in one
// fixed array compiled into this library (NA_SCRATCH_BYTES, held by every GPU
// that loads the library until the process exits).  Nothing else is
// allocated: no cudaMalloc, no cudaFree, no allocating library routine.
//
// The solve is the same as the one in the stencil build (a row-streamed
// Householder QR of B = W A followed by corrected semi-normal equations for
// the least-||t|| solution of B^T t = F, returning s = W t), applied to rows
// the caller has already formed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "eb_internal.cuh"

namespace eb {

constexpr int NA_CTAS = 32;                  // persistent grid: 32 CTAs of 4 warps
constexpr int NA_WARPS_PER_CTA = 4;
constexpr int NA_WARPS = NA_CTAS * NA_WARPS_PER_CTA;
constexpr int NA_MAXROWS = 256;              // rows per system accepted by this entry point
constexpr int NA_MAXK = 35;                  // unknowns per system (monomials of degree <= 4 in 3-D)
constexpr int NA_RPL = 4;
constexpr int NA_CH = 32 * NA_RPL;
constexpr int NA_KST = NA_MAXK;
constexpr int64_t NA_HEAD = 32;              // doubles reserved in front: work counter
constexpr int64_t NA_PER_WARP = (int64_t)NA_MAXROWS * (NA_MAXK + 1);  // B column-major + t1
constexpr int64_t NA_SCRATCH_DOUBLES = NA_HEAD + NA_WARPS * NA_PER_WARP;
constexpr int64_t NA_SCRATCH_BYTES = NA_SCRATCH_DOUBLES * 8;  // 9.4 MB

// The fixed scratch.  Host code must not pass this symbol to a kernel: on the
// host it names a stand-in, not the device address, which is obtained with
// cudaGetSymbolAddress once per device (na_scratch_ptr below).
static __device__ __align__(256) double g_na_scratch[NA_SCRATCH_DOUBLES];

struct NaSmem {
  double R[NA_MAXK * NA_MAXK];
  double C[NA_CH * NA_KST];
  double P[32 * NA_KST];
  double vec[5 * NA_MAXK];
};
static_assert(NA_WARPS_PER_CTA * sizeof(NaSmem) <= 232448, "dynamic shared memory of one CTA exceeds 227 KB");

__device__ __forceinline__ double na_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// column sums of P[0..32)[c0 .. c0 + mm), one result per column in the group's first lane
__device__ __forceinline__ double na_column_sums(const double* P, int c0, int mm, int lane, int* col) {
  int g = 1;
  while (g * 2 * mm <= 32) g *= 2;
  int cl = lane / g, part = lane % g, L = 32 / g;
  double acc = 0.0;
  if (cl < mm)
    for (int l = part * L; l < part * L + L; ++l) acc += P[l * NA_KST + c0 + cl];
  for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  *col = (cl < mm && part == 0) ? cl : -1;
  return acc;
}

// B: [nnz][K] row-major weighted rows; w: [nnz]; F: [n_sys][K]; s: [nnz]; status: [n_sys]
__global__ void __launch_bounds__(NA_WARPS_PER_CTA * 32, 1)
    k_lsq_rows_noalloc(const double* __restrict__ B, const double* __restrict__ w, const double* __restrict__ F,
                       const int64_t* __restrict__ row_ptr, int32_t n_sys, int K, double* __restrict__ s,
                       int32_t* __restrict__ status, double* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char na_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  NaSmem& S = reinterpret_cast<NaSmem*>(na_smem)[warp];
  int* counter = reinterpret_cast<int*>(scratch);
  double* scr = scratch + NA_HEAD + (int64_t)(blockIdx.x * NA_WARPS_PER_CTA + warp) * NA_PER_WARP;
  double* scr_t = scr + (int64_t)NA_MAXROWS * NA_MAXK;
  double* Fv = S.vec;
  double* y = S.vec + NA_MAXK;
  double* z = S.vec + 2 * NA_MAXK;
  double* tau = S.vec + 3 * NA_MAXK;
  double* rinv = S.vec + 4 * NA_MAXK;
  while (true) {
    int q = 0;
    if (lane == 0) q = atomicAdd(counter, 1);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= n_sys) break;
    const int64_t p0 = row_ptr[q];
    const int n = (int)(row_ptr[q + 1] - p0);
    if (n > NA_MAXROWS || n < K) {
      if (lane == 0) status[q] = n > NA_MAXROWS ? 3 : 1;
      for (int i = lane; i < n; i += 32) s[p0 + i] = 0.0;
      __syncwarp();
      continue;
    }
    for (int i = lane; i < K * K; i += 32) S.R[i] = 0.0;
    __syncwarp();
    for (int c0 = 0; c0 < n; c0 += NA_CH) {
      for (int r = 0; r < NA_RPL; ++r) {
        int li = lane + 32 * r, i = c0 + li;
        double* dst = S.C + li * NA_KST;
        for (int k = 0; k < K; ++k) {
          double v = i < n ? B[(p0 + i) * K + k] : 0.0;
          dst[k] = v;
          if (i < n) scr[(int64_t)k * NA_MAXROWS + i] = v;
        }
      }
      __syncwarp();
      for (int k = 0; k < K; ++k) {
        double ck[NA_RPL];
        double ss = 0.0;
#pragma unroll
        for (int r = 0; r < NA_RPL; ++r) {
          ck[r] = S.C[(lane + 32 * r) * NA_KST + k];
          ss = fma(ck[r], ck[r], ss);
        }
        ss = na_warp_sum(ss);
        if (ss == 0.0) continue;
        const double alpha = S.R[k * K + k];
        const double sigma = sqrt(fma(alpha, alpha, ss));
        const double beta = alpha > 0.0 ? -sigma : sigma;
        const double v0 = alpha - beta;
        const double gamma = -1.0 / (beta * v0);
        const int m = K - k - 1;
        for (int jj = 0; jj < m; ++jj) {
          double p = 0.0;
#pragma unroll
          for (int r = 0; r < NA_RPL; ++r) p = fma(ck[r], S.C[(lane + 32 * r) * NA_KST + k + 1 + jj], p);
          S.P[lane * NA_KST + jj] = p;
        }
        __syncwarp();
        for (int c1 = 0; c1 < m; c1 += 32) {
          int mm = m - c1 < 32 ? m - c1 : 32, col;
          double sum = na_column_sums(S.P, c1, mm, lane, &col);
          if (col >= 0) {
            int jc = c1 + col, j = k + 1 + jc;
            double rkj = S.R[k * K + j];
            double t = gamma * fma(v0, rkj, sum);
            S.R[k * K + j] = fma(-t, v0, rkj);
            tau[jc] = t;
          }
        }
        __syncwarp();
        for (int jj = 0; jj < m; ++jj) {
          double t = tau[jj];
#pragma unroll
          for (int r = 0; r < NA_RPL; ++r) {
            double* c = S.C + (lane + 32 * r) * NA_KST + k + 1 + jj;
            *c = fma(-t, ck[r], *c);
          }
        }
        if (lane == 0) S.R[k * K + k] = beta;
        __syncwarp();
      }
    }
    double dmax = 0.0, dmin = INFINITY;
    for (int k = 0; k < K; ++k) {
      double v = fabs(S.R[k * K + k]);
      dmax = fmax(dmax, v);
      dmin = fmin(dmin, v);
    }
    if (!(dmin > 1e-12 * dmax)) {
      if (lane == 0) status[q] = 1;
      for (int i = lane; i < n; i += 32) s[p0 + i] = 0.0;
      __syncwarp();
      continue;
    }
    for (int k = lane; k < K; k += 32) {
      rinv[k] = 1.0 / S.R[k * K + k];
      Fv[k] = F[(int64_t)q * K + k];
    }
    __syncwarp();
    auto solve_rtr = [&](const double* rhs, double* outz) {
      for (int j = lane; j < K; j += 32) y[j] = rhs[j];
      __syncwarp();
      for (int k = 0; k < K; ++k) {
        double yk = y[k] * rinv[k];
        __syncwarp();
        for (int j = k + 1 + lane; j < K; j += 32) y[j] = fma(-S.R[k * K + j], yk, y[j]);
        if (lane == 0) y[k] = yk;
        __syncwarp();
      }
      for (int j = lane; j < K; j += 32) outz[j] = y[j];
      __syncwarp();
      for (int k = K - 1; k >= 0; --k) {
        double zk = outz[k] * rinv[k];
        __syncwarp();
        for (int j = lane; j < k; j += 32) outz[j] = fma(-S.R[j * K + k], zk, outz[j]);
        if (lane == 0) outz[k] = zk;
        __syncwarp();
      }
    };
    solve_rtr(Fv, z);
    for (int k = 0; k < K; ++k) S.P[lane * NA_KST + k] = 0.0;
    for (int i = lane; i < n; i += 32) {
      double t1 = 0.0;
      for (int k = 0; k < K; ++k) t1 = fma(scr[(int64_t)k * NA_MAXROWS + i], z[k], t1);
      scr_t[i] = t1;
      for (int k = 0; k < K; ++k)
        S.P[lane * NA_KST + k] = fma(scr[(int64_t)k * NA_MAXROWS + i], t1, S.P[lane * NA_KST + k]);
    }
    __syncwarp();
    for (int c1 = 0; c1 < K; c1 += 32) {
      int mm = K - c1 < 32 ? K - c1 : 32, col;
      double sum = na_column_sums(S.P, c1, mm, lane, &col);
      if (col >= 0) tau[c1 + col] = Fv[c1 + col] - sum;
    }
    __syncwarp();
    double* z2 = S.C;
    solve_rtr(tau, z2);
    for (int i = lane; i < n; i += 32) {
      double t = scr_t[i];
      for (int k = 0; k < K; ++k) t = fma(scr[(int64_t)k * NA_MAXROWS + i], z2[k], t);
      s[p0 + i] = w[p0 + i] * t;
    }
    if (lane == 0) status[q] = 0;
    __syncwarp();
  }
}

// Device address of the fixed scratch, looked up once per device with that
// device current (the symbol itself is only a host-side stand-in).  The
// address and the kernel attribute are cached for the life of the process: a
// cudaDeviceReset (or any other teardown of the device's primary context)
// invalidates them, so a process that resets a device must not call this
// entry point on that device again.
static std::mutex g_na_mutex;
static void* g_na_ptr[128];
static bool g_na_ready[128];

static eb_status na_setup(int dev, double** ptr) {
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (dev < 0 || dev >= 128) { set_error("device ordinal out of range"); return EB_ERR_INVALID; }
  if (!g_na_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_na_scratch)");
    e = cudaFuncSetAttribute(k_lsq_rows_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(NA_WARPS_PER_CTA * sizeof(NaSmem)));
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_lsq_rows_noalloc)");
    g_na_ptr[dev] = p;
    g_na_ready[dev] = true;
  }
  *ptr = (double*)g_na_ptr[dev];
  return EB_OK;
}

}  // namespace eb

using namespace eb;

extern "C" eb_status eb_lsq_batch_noalloc(const double* B, const double* w, const double* F, const int64_t* row_ptr,
                                          int32_t n_sys, int32_t K, int32_t max_rows, double* s, int32_t* status,
                                          eb_stream_t stream) {
  if (n_sys < 0 || K < 1 || K > NA_MAXK) {
    set_error("eb_lsq_batch_noalloc: K must be in 1..35 and n_sys >= 0");
    return EB_ERR_INVALID;
  }
  if (max_rows > NA_MAXROWS) {
    set_error("eb_lsq_batch_noalloc: systems may have at most 256 rows (max_rows exceeds the fixed scratch)");
    return EB_ERR_CAPACITY;
  }
  if (n_sys == 0) return EB_OK;
  if (!B || !w || !F || !row_ptr || !s || !status) {
    set_error("eb_lsq_batch_noalloc: null argument");
    return EB_ERR_INVALID;
  }
  int dev = 0;
  EB_CUDA(cudaGetDevice(&dev));
  double* scratch = nullptr;
  eb_status st = na_setup(dev, &scratch);
  if (st != EB_OK) return st;
  cudaStream_t s_ = (cudaStream_t)stream;
  // the work counter at the head of the scratch must start at zero for every call
  EB_CUDA(cudaMemsetAsync(scratch, 0, sizeof(int), s_));
  k_lsq_rows_noalloc<<<NA_CTAS, NA_WARPS_PER_CTA * 32, NA_WARPS_PER_CTA * sizeof(NaSmem), s_>>>(
      B, w, F, row_ptr, n_sys, K, s, status, scratch);
  eb::count_launch();
  EB_CUDA(cudaGetLastError());
  return EB_OK;
}
