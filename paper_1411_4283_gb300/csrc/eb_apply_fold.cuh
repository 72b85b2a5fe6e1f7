// Template pass of the operator apply (Sec. 2.3) for the interior cells in
// 3-D, with the template row folded by its reflection symmetry.
//
// The interior cell row is the sum of the six interior face stencils, so it is
// even in each of dx, dy, dz (to rounding in the LS solves; the plan averages
// the eight sign images and checks that they agree).  With
// T(a, b, c) = c(+-a, +-b, +-c) and the folds S_z^c f = f(z+c) + f(z-c)
// (S^0 f = f), the apply is
//     y(x, y, z) = sum_{a,b,c >= 0} T(a,b,c) S_x^a S_y^b S_z^c phi,
// evaluated in two passes per output plane z (the a-sum last):
//   stage 1: for every staged x (tile plus halo) and the tile's y,
//            U_a(x, y) = sum_{b,c} T(a,b,c) S_y^b S_z^c phi(x, ., .)
//            -- a thread owns one staged x column and four consecutive y:
//            it folds the planes z+-c (P_c), then the rows y+-b of P_c,
//            and accumulates the five U_a, which go to shared memory;
//   stage 2: y(x, y) = U_0(x) + sum_{a >= 1} (U_a(x+a) + U_a(x-a)).
// Against the z-folded pass (357 FMAs per cell for R = 3) this takes about
// 126 FMAs and 36 adds per cell: one FMA per term of the folded footprint
// (112 terms T(a, b, c) for R = 3) per staged column (72 staged columns per
// 64 cells), the fold adds, and in stage 2 nine loads and eight adds.
//
// Data movement is that of the z-folded pass: a ring of 2L+2 staged planes
// (64 + 8 by 16 + 2L) filled by TMA one plane ahead, bounded mbarrier waits,
// and every CTA leaves its item loop together when a wait gives up.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "eb_apply_tma.cuh"

namespace eb {

constexpr int FD_OX = 64;                    // tile width (x)
constexpr int FD_OY = 16;                    // tile height (y)
constexpr int FD_PX = FD_OX + 2 * TT_XH;     // staged x (halo TT_XH, 16-byte aligned TMA boxes)
constexpr int FD_YB = 4;                     // outputs per thread along y in stage 1
constexpr int FD_T1 = FD_PX * (FD_OY / FD_YB);  // stage-1 tasks: one per (staged x, y group) = 288
constexpr int FD_THREADS = FD_T1;

template <typename T, int R>
struct FoldCoef {
  static constexpr int L = R + 1;
  T c[(L + 1) * (L + 1) * (L + 1)];  // T(a, b, c) at a + (L+1) (b + (L+1) c)
};

template <typename T, int R>
__global__ void __launch_bounds__(FD_THREADS) k_apply_fold(const __grid_constant__ CUtensorMap tmap,
                                                          const __grid_constant__ FoldCoef<T, R> cf, TmplArgs<T> a) {
  constexpr int L = R + 1;
  constexpr int S = 2 * L + 1;
  constexpr int NP = S + 1;  // ring: planes z-L .. z+L and the one requested ahead
  constexpr int PY = FD_OY + 2 * L;
  constexpr uint32_t PBYTES = FD_PX * PY * sizeof(T);
  constexpr int PLANE = (int)(((PBYTES + 127) / 128) * 128 / sizeof(T));
  constexpr int NR = FD_YB + 2 * L;      // staged rows a stage-1 thread reads
  constexpr int UPL = FD_OY * FD_PX;     // one U_a plane
  static_assert(L <= TT_XH, "x halo");
  extern __shared__ __align__(128) unsigned char sm_fold[];
  T* ring = reinterpret_cast<T*>(sm_fold);
  T* U = ring + (size_t)NP * PLANE;      // [L+1][FD_OY][FD_PX]
  uint64_t* bars = reinterpret_cast<uint64_t*>(U + (size_t)(L + 1) * UPL);
  const int tid = threadIdx.x;
  // stage 1: staged column xs, rows yg .. yg + FD_YB - 1 of the tile
  const int xs = tid % FD_PX, yg = (tid / FD_PX) * FD_YB;
  if (tid == 0) {
    for (int p = 0; p < NP; ++p) mbar_init(&bars[p], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t parity = 0, pending = 0;
  bool failed = false;
  for (int64_t item = blockIdx.x; item < a.items; item += gridDim.x) {
    const int zc = (int)(item % a.nzc);
    const int64_t t2 = item / a.nzc;
    const int tyl = (int)(t2 % a.nty), txl = (int)(t2 / a.nty);
    const int x0 = txl * FD_OX, y0 = tyl * FD_OY;
    const int z0 = zc * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.nz);
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int q = 0; q < S; ++q) {
        const int zz = z0 - L + q, slot = ((zz % NP) + NP) % NP;
        mbar_expect_tx(&bars[slot], PBYTES);
        tma_load_3d(ring + (size_t)slot * PLANE, &tmap, &bars[slot], x0 - TT_XH, y0 - L, zz);
      }
    }
    for (int q = 0; q < S; ++q) pending |= 1u << (((z0 - L + q) % NP + NP) % NP);
    for (int q = 0; q < S; ++q) {
      const int slot = (((z0 - L + q) % NP) + NP) % NP;
      if (!mbar_wait(&bars[slot], (parity >> slot) & 1u)) { failed = true; break; }
      parity ^= 1u << slot;
      pending &= ~(1u << slot);
    }
    if (__syncthreads_or(failed)) { failed = true; break; }
    for (int z = z0; z < z1; ++z) {
      if (z + 1 < z1) {
        const int zz = z + L + 1, slot = (zz % NP + NP) % NP;
        if (tid == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(&bars[slot], PBYTES);
          tma_load_3d(ring + (size_t)slot * PLANE, &tmap, &bars[slot], x0 - TT_XH, y0 - L, zz);
        }
        pending |= 1u << slot;
      }
      if (z > z0) {
        const int slot = ((z + L) % NP + NP) % NP;
        if (mbar_wait(&bars[slot], (parity >> slot) & 1u)) {
          parity ^= 1u << slot;
          pending &= ~(1u << slot);
        } else {
          failed = true;  // acted on at the barrier that ends this step, uniformly
        }
      }
      // kinds of this thread's stage-2 cells, loaded now so that their latency hides behind stage 1
      uint8_t kd[FD_OY / 4];
      if (tid < FD_OX * 4) {
        const int xg = x0 + tid % FD_OX;
#pragma unroll
        for (int m = 0; m < FD_OY / 4; ++m) {
          const int yg2 = y0 + tid / FD_OX + 4 * m;
          kd[m] = (xg < a.nx && yg2 < a.ny) ? a.kind[xg + (int64_t)a.nx * ((int64_t)yg2 + (int64_t)a.ny * z)] : 2;
        }
      }
      // ring slot of plane z - L (one modulo per step; the others follow by a wrapped increment)
      const int s0 = ((z - L) % NP + NP) % NP;
      // ---- stage 1: U_a(xs, yg + j) for j < FD_YB
      {
        T u[L + 1][FD_YB];
#pragma unroll
        for (int q = 0; q <= L; ++q)
#pragma unroll
          for (int j = 0; j < FD_YB; ++j) u[q][j] = (T)0;
#pragma unroll
        for (int c = 0; c <= L; ++c) {
          int sp = s0 + L + c, sm = s0 + L - c;
          sp -= sp >= NP ? NP : 0;
          sm -= sm >= NP ? NP : 0;
          const T* pp = ring + (size_t)sp * PLANE + yg * FD_PX + xs;
          const T* pm = ring + (size_t)sm * PLANE + yg * FD_PX + xs;
          T p[NR];
#pragma unroll
          for (int r = 0; r < NR; ++r) p[r] = c == 0 ? pp[r * FD_PX] : pp[r * FD_PX] + pm[r * FD_PX];
#pragma unroll
          for (int b = 0; b <= L; ++b) {
#pragma unroll
            for (int j = 0; j < FD_YB; ++j) {
              const T q = b == 0 ? p[j + L] : p[j + L + b] + p[j + L - b];
#pragma unroll
              for (int aa = 0; aa <= L; ++aa) {
                if (!fp_box(aa, b, c, R)) continue;
                u[aa][j] = fma(cf.c[aa + (L + 1) * (b + (L + 1) * c)], q, u[aa][j]);
              }
            }
          }
        }
#pragma unroll
        for (int aa = 0; aa <= L; ++aa)
#pragma unroll
          for (int j = 0; j < FD_YB; ++j) U[aa * UPL + (yg + j) * FD_PX + xs] = u[aa][j];
      }
      __syncthreads();
      // ---- stage 2: x fold and the epilogue; thread: x = tid % FD_OX, rows (tid / FD_OX) + 4 m
      if (tid < FD_OX * 4) {
        const int ox = tid % FD_OX, oy0 = tid / FD_OX;
        const int xg = x0 + ox;
#pragma unroll
        for (int m = 0; m < FD_OY / 4; ++m) {
          const int oy = oy0 + 4 * m;
          const T* ur = U + oy * FD_PX + ox + TT_XH;
          T acc = ur[0];
#pragma unroll
          for (int aa = 1; aa <= L; ++aa) acc += ur[aa * UPL + aa] + ur[aa * UPL - aa];
          const int yg2 = y0 + oy;
          const uint8_t k = kd[m];  // 2 (leave alone) outside the grid
          if (k < 2) {
            const int64_t c = xg + (int64_t)a.nx * ((int64_t)yg2 + (int64_t)a.ny * z);
            if (k == 1) a.y[c] = a.kappa_weighted ? acc : acc * (T)a.inv_kappa[c];
            else a.y[c] = (T)0;
          }
        }
      }
      // every thread is done with plane z - L and with U; a wait that gave up on any thread ends the CTA's work
      if (__syncthreads_or(failed)) { failed = true; break; }
    }
    if (failed) break;
  }
  if (failed) {
    for (int p = 0; p < NP; ++p)
      if ((pending >> p) & 1u) mbar_wait(&bars[p], (parity >> p) & 1u);
    if (tid == 0) atomicExch(a.err, 1);
  }
}

template <typename T, int R>
constexpr size_t fold_smem() {
  constexpr int L = R + 1;
  constexpr int NP = 2 * L + 2;
  constexpr size_t SLOT = ((FD_PX * (FD_OY + 2 * L) * sizeof(T) + 127) / 128) * 128;
  return NP * SLOT + (size_t)(L + 1) * FD_OY * FD_PX * sizeof(T) + NP * 8;
}

}  // namespace eb
