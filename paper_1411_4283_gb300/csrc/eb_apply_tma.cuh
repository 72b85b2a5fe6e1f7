// Template pass of the operator apply for the interior cells (Sec. 2.3): the
// cell stencil there is one translation-invariant row (sum of the interior
// face stencils).  Box neighbourhoods of radius R give the footprint
// {|d|_inf <= R} plus one-coordinate arms at |d_k| = R+1, stored densely in a
// (2R+3)^3 coefficient cube passed as a kernel parameter so that every
// coefficient is a compile-time constant-bank operand of its FMA.
//
// Data movement: each CTA owns an OX x OY tile of (x, y) and a chunk of z.
// phi planes (OX+2L) x (OY+2L), L = R+1, are brought into a ring of 2L+2
// shared-memory planes by TMA (cp.async.bulk.tensor.3d with zero fill
// outside the grid), one mbarrier per ring slot: the plane needed one step
// ahead is requested at the start of each step, so its copy overlaps the
// step's arithmetic.  Waits are bounded and set an error word instead of
// hanging.  Each thread computes 4 consecutive x by 2 consecutive y outputs,
// reusing every loaded row for both outputs.  When the template is symmetric
// in z (ZSYM; the interior template of a box neighbourhood is, to rounding),
// rows of the planes z+a and z-a are added first and multiplied once by the
// common coefficient, which takes the FMAs per output from 637 to 357 (R=3).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace eb {

constexpr int TT_OX = 64;   // tile width (x)
constexpr int TT_OY = 16;   // tile height (y)
constexpr int TT_THREADS = 128;
// x halo of the staged planes: 4 >= L for R <= 3, and a multiple of 4 so that the first x coordinate of
// every TMA box (x0 - TT_XH, x0 a multiple of TT_OX) is 16-byte aligned for 4- and 8-byte elements
constexpr int TT_XH = 4;

template <typename T, int R>
struct TmplCoef {
  static constexpr int L = R + 1;
  static constexpr int S = 2 * L + 1;
  T c[S * S * S];
};

__host__ __device__ constexpr bool fp_box(int dx, int dy, int dz, int R) {
  int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
  int over = (ax > R) + (ay > R) + (az > R);
  int mx = ax > ay ? (ax > az ? ax : az) : (ay > az ? ay : az);
  return mx <= R + 1 && over <= 1;
}

}  // namespace eb

namespace eb {

template <typename T>
struct TmplArgs {
  int nx, ny, nz;
  int ntx, nty, nzc, zchunk;
  int64_t items;
  const uint8_t* kind;
  const double* inv_kappa;
  T* y;
  int kappa_weighted;
  int32_t* err;  // set when a bounded wait gives up
};

constexpr uint32_t TMA_WAIT_LIMIT = 4000000u;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait on the phase with the given parity; false when the limit is reached
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < TMA_WAIT_LIMIT; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using V = float4;
  static constexpr int N = 4;
};
template <>
struct Vec2<double> {
  using V = double2;
  static constexpr int N = 2;
};

template <typename T, int R, int D, bool ZSYM>
__global__ void __launch_bounds__(TT_THREADS) k_apply_tma(const __grid_constant__ CUtensorMap tmap,
                                                         const __grid_constant__ TmplCoef<T, R> cf, TmplArgs<T> a) {
  constexpr int L = R + 1;
  constexpr int S = 2 * L + 1;
  constexpr int NP = D == 3 ? S + 1 : 1;  // ring planes: z-L .. z+L and the one requested ahead
  static_assert(L <= TT_XH, "x halo");
  constexpr int PX = TT_OX + 2 * TT_XH, PY = TT_OY + 2 * L;
  constexpr uint32_t PBYTES = PX * PY * sizeof(T);         // bytes of one staged plane
  constexpr int PLANE = (int)(((PBYTES + 127) / 128) * 128 / sizeof(T));  // slot stride: TMA writes 128-byte aligned
  constexpr int VW = Vec2<T>::N;
  constexpr int NV = (4 + 2 * TT_XH + VW - 1) / VW;  // vectors covering 4 outputs + the x halo
  extern __shared__ __align__(128) unsigned char sm_tma[];
  T* ring = reinterpret_cast<T*>(sm_tma);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm_tma + (size_t)NP * PLANE * sizeof(T));
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int ox0 = 4 * tx, oy0 = 2 * ty;
  if (tid == 0) {
    for (int p = 0; p < NP; ++p) mbar_init(&bars[p], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t parity = 0;   // bit p: parity of the next phase of slot p
  uint32_t pending = 0;  // bit p: slot p has a copy requested and not yet waited for
  bool failed = false;
  for (int64_t item = blockIdx.x; item < a.items; item += gridDim.x) {
    const int zc = (int)(item % a.nzc);
    const int64_t t2 = item / a.nzc;
    const int tyl = (int)(t2 % a.nty), txl = (int)(t2 / a.nty);
    const int x0 = txl * TT_OX, y0 = tyl * TT_OY;
    const int z0 = zc * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.nz);
    constexpr int NPRO = D == 3 ? S : 1;  // prologue planes: z0-L .. z0+L (3-D) or the single plane (2-D)
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int q = 0; q < NPRO; ++q) {
        int zz = D == 3 ? z0 - L + q : 0;
        int slot = D == 3 ? ((zz % NP) + NP) % NP : 0;
        mbar_expect_tx(&bars[slot], PBYTES);
        tma_load_3d(ring + (size_t)slot * PLANE, &tmap, &bars[slot], x0 - TT_XH, y0 - L, zz);
      }
    }
    for (int q = 0; q < NPRO; ++q) {
      int zz = D == 3 ? z0 - L + q : 0;
      int slot = D == 3 ? ((zz % NP) + NP) % NP : 0;
      pending |= 1u << slot;
    }
    for (int q = 0; q < NPRO; ++q) {
      int zz = D == 3 ? z0 - L + q : 0;
      int slot = D == 3 ? ((zz % NP) + NP) % NP : 0;
      if (!mbar_wait(&bars[slot], (parity >> slot) & 1u)) { failed = true; break; }
      parity ^= 1u << slot;
      pending &= ~(1u << slot);
    }
    // every thread leaves together: a wait that gave up on any thread ends the CTA's work
    if (__syncthreads_or(failed)) { failed = true; break; }
    for (int z = z0; z < z1; ++z) {
      if (D == 3) {
        // request plane z+L+1 for the next step into the slot of plane z-L-1 (released by the
        // barrier that ended the previous step), then wait for plane z+L (requested one step ago)
        if (z + 1 < z1) {
          int zz = z + L + 1;
          int slot = (zz % NP + NP) % NP;
          if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&bars[slot], PBYTES);
            tma_load_3d(ring + (size_t)slot * PLANE, &tmap, &bars[slot], x0 - TT_XH, y0 - L, zz);
          }
          pending |= 1u << slot;
        }
        if (z > z0) {
          int slot = ((z + L) % NP + NP) % NP;
          if (mbar_wait(&bars[slot], (parity >> slot) & 1u)) {
            parity ^= 1u << slot;
            pending &= ~(1u << slot);
          } else {
            failed = true;  // acted on at the barrier that ends this step, uniformly
          }
        }
      }
      T acc[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
#pragma unroll
      for (int dz = (D == 3 ? (ZSYM ? 0 : -L) : 0); dz <= (D == 3 ? L : 0); ++dz) {
        const int slot = D == 3 ? ((z + dz) % NP + NP) % NP : 0;
        const T* pl = ring + (size_t)slot * PLANE;
        const T* plm = ring + (size_t)(D == 3 ? ((z - dz) % NP + NP) % NP : 0) * PLANE;  // plane z-dz (ZSYM)
#pragma unroll
        for (int yy = -L; yy <= L + 1; ++yy) {
          const T* rp = pl + (oy0 + yy + L) * PX + ox0;
          T v[NV * VW];
#pragma unroll
          for (int q = 0; q < NV; ++q) {
            typename Vec2<T>::V w = reinterpret_cast<const typename Vec2<T>::V*>(rp)[q];
            reinterpret_cast<typename Vec2<T>::V*>(v)[q] = w;
          }
          if (ZSYM && D == 3 && dz > 0) {
            const T* rm = plm + (oy0 + yy + L) * PX + ox0;
            T u[NV * VW];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
              typename Vec2<T>::V w = reinterpret_cast<const typename Vec2<T>::V*>(rm)[q];
              reinterpret_cast<typename Vec2<T>::V*>(u)[q] = w;
            }
#pragma unroll
            for (int q = 0; q < NV * VW; ++q) v[q] += u[q];
          }
#pragma unroll
          for (int oy = 0; oy < 2; ++oy) {
            const int dy = yy - oy;
            if (dy < -L || dy > L) continue;
#pragma unroll
            for (int dx = -L; dx <= L; ++dx) {
              if (!fp_box(dx, dy, D == 3 ? dz : 0, R)) continue;
              const T c = cf.c[(dx + L) + S * ((dy + L) + S * (dz + L))];
#pragma unroll
              for (int ox = 0; ox < 4; ++ox) acc[oy][ox] = fma(c, v[ox + dx + TT_XH], acc[oy][ox]);
            }
          }
        }
      }
      // outputs: template cells get the stencil, covered cells 0, irregular cells are left alone
#pragma unroll
      for (int oy = 0; oy < 2; ++oy) {
        const int yg = y0 + oy0 + oy;
        if (yg >= a.ny) continue;
        const int64_t rowbase = (int64_t)a.nx * ((int64_t)yg + (int64_t)a.ny * z);
#pragma unroll
        for (int ox = 0; ox < 4; ++ox) {
          const int xg = x0 + ox0 + ox;
          if (xg >= a.nx) continue;
          const int64_t c = rowbase + xg;
          const uint8_t k = a.kind[c];
          if (k == 1) a.y[c] = a.kappa_weighted ? acc[oy][ox] : acc[oy][ox] * (T)a.inv_kappa[c];
          else if (k == 0) a.y[c] = (T)0;
        }
      }
      // every thread is done with plane z - L; a wait that gave up on any thread ends the CTA's work
      if (__syncthreads_or(failed)) { failed = true; break; }
    }
    if (failed) break;
  }
  if (failed) {
    // failed is uniform across the CTA here.  Before the CTA exits, wait (bounded) for the copies
    // still in flight into its shared memory, then report.
    for (int p = 0; p < NP; ++p)
      if ((pending >> p) & 1u) mbar_wait(&bars[p], (parity >> p) & 1u);
    if (tid == 0) atomicExch(a.err, 1);
  }
}

}  // namespace eb
