// Build phase of the cut-cell Poisson discretisation (arXiv:1411.4283, Sec. 2):
//   1. classify faces: EB-affected faces get their own least-squares (LS)
//      system; faces whose neighbourhood sees only full cells and domain walls
//      share one stencil per translation class (the interior template is the
//      class far from every wall);
//   2. neighbourhood of each volume: the cells of its box (or L1 ball) of
//      radius R_n reached through open faces (Sec. 2.4, "R_n cells away");
//   3. gather the canonical row list of every solved face: volumes, then wall
//      faces, then EB faces touched by those volumes (Sec. 2.4);
//   4. FP64 weighted LS: s = W (A^T W)^+ F, the least-||W^-1 s|| solution of
//      A^T s = F (Sec. 2.2.1), by a row-streamed Householder QR of W A and
//      corrected semi-normal equations;
//   5. assemble the kappa-weighted operator rows kappa_v L_v =
//      (1/h^2) sum_f sigma s_hat_f (Sec. 2.3) and the boundary matrix B.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "eb_internal.cuh"
#include "eb_tables.cuh"
#include "eb_build.cuh"

namespace eb {

// ============================================================ geometry helpers

__device__ __forceinline__ void cell_xyz(const Dims& dm, int64_t c, int* x) {
  x[0] = (int)(c % dm.n[0]);
  int64_t r = c / dm.n[0];
  x[1] = (int)(r % dm.n[1]);
  x[2] = (int)(r / dm.n[1]);
}
__device__ __forceinline__ int64_t cell_id(const Dims& dm, const int* x) {
  return (int64_t)x[0] + (int64_t)dm.n[0] * ((int64_t)x[1] + (int64_t)dm.n[1] * x[2]);
}
__device__ __forceinline__ bool in_domain(const Dims& dm, const int* x) {
  for (int d = 0; d < 3; ++d)
    if (x[d] < 0 || x[d] >= dm.n[d]) return false;
  return true;
}
// local index of the face normal to d whose coordinates are x (x[d] in 0..n_d)
__device__ __forceinline__ int64_t face_local(const Dims& dm, int d, const int* x) {
  int64_t m0 = dm.n[0] + (d == 0), m1 = dm.n[1] + (d == 1);
  return (int64_t)x[0] + m0 * ((int64_t)x[1] + m1 * x[2]);
}
__device__ __forceinline__ void face_xyz(const Dims& dm, int d, int64_t f, int* x) {
  int64_t m0 = dm.n[0] + (d == 0), m1 = dm.n[1] + (d == 1);
  x[0] = (int)(f % m0);
  int64_t r = f / m0;
  x[1] = (int)(r % m1);
  x[2] = (int)(r / m1);
}

// ============================================================ 1. masks and classes

// bit 0: non-full cell (covered or cut); bit 1: non-full or touching the domain boundary
__global__ void k_mark(Dims dm, const uint8_t* __restrict__ flag, uint8_t* __restrict__ mark) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= dm.ncell) return;
  int x[3];
  cell_xyz(dm, c, x);
  uint8_t nf = flag[c] != 1;
  bool bd = false;
  for (int d = 0; d < dm.dim; ++d) bd |= (x[d] == 0) || (x[d] == dm.n[d] - 1);
  mark[c] = nf | ((nf || bd) ? 2 : 0);
}

// dilation by R along one axis; outside the domain counts as bit 1 set (walls), bit 0 clear
__global__ void k_dilate(Dims dm, int axis, int R, const uint8_t* __restrict__ in, uint8_t* __restrict__ out) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= dm.ncell) return;
  int x[3];
  cell_xyz(dm, c, x);
  uint8_t acc = 0;
  for (int t = -R; t <= R; ++t) {
    int y = x[axis] + t;
    if (y < 0 || y >= dm.n[axis]) { acc |= 2; continue; }
    int z[3] = {x[0], x[1], x[2]};
    z[axis] = y;
    acc |= in[cell_id(dm, z)];
  }
  out[c] = acc;
}

// class key of a wall-only grid face: d and, per dimension, clamped distances to both walls
__device__ __forceinline__ int class_key(const Dims& dm, int d, const int* x) {
  int M = dm.R + 3;
  int key = 0;
  for (int k = dm.dim - 1; k >= 0; --k) {
    int lo, hi;
    if (k == d) { lo = x[k]; hi = dm.n[k] - x[k]; }
    else { lo = x[k]; hi = dm.n[k] - 1 - x[k]; }
    lo = lo < M - 1 ? lo : M - 1;
    hi = hi < M - 1 ? hi : M - 1;
    key = (key * M + lo) * M + hi;
  }
  return key * 3 + d;
}

// face state: -1 closed, -2 EB-affected (own system), >= 0 class key
__global__ void k_classify_faces(Dims dm, int d, const uint8_t* __restrict__ fflag, const uint8_t* __restrict__ dil,
                                 int32_t* __restrict__ state, int64_t* __restrict__ class_rep,
                                 int32_t* __restrict__ is_unique) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= dm.nface[d]) return;
  int x[3];
  face_xyz(dm, d, f, x);
  int32_t st;
  if (fflag[f] == 0) st = -1;
  else {
    bool eb = false;
    if (x[d] > 0) { int lo[3] = {x[0], x[1], x[2]}; lo[d] -= 1; eb |= (dil[cell_id(dm, lo)] & 1) != 0; }
    if (x[d] < dm.n[d]) eb |= (dil[cell_id(dm, x)] & 1) != 0;
    if (eb) st = -2;
    else {
      st = class_key(dm, d, x);
      atomicMin((unsigned long long*)&class_rep[st], (unsigned long long)(dm.face_base[d] + f));
    }
  }
  state[f] = st;
  is_unique[f] = st == -2;
}

// slot of every grid face: unique faces -> their position; class faces -> class slot
__global__ void k_face_slots(Dims dm, int d, const int32_t* __restrict__ state, const int64_t* __restrict__ upos,
                             int64_t ubase, const int32_t* __restrict__ class_slot, int32_t* __restrict__ slot,
                             int64_t* __restrict__ slot_face) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= dm.nface[d]) return;
  int32_t st = state[f];
  int32_t s;
  if (st == -1) s = -1;
  else if (st == -2) {
    s = (int32_t)(ubase + upos[f]);
    slot_face[s] = dm.face_base[d] + f;
  } else s = class_slot[st];
  slot[f] = s;
}

// ============================================================ 2. reach masks


__device__ __forceinline__ void mset(Mask& m, int b) { m.w[b >> 6] |= 1ull << (b & 63); }
__device__ __forceinline__ bool mtest(const Mask& m, int b) { return (m.w[b >> 6] >> (b & 63)) & 1ull; }
__device__ __forceinline__ Mask mshl(const Mask& m, int s) {
  Mask o;
  int ws = s >> 6, bs = s & 63;
  for (int i = RW - 1; i >= 0; --i) {
    uint64_t v = 0;
    int j = i - ws;
    if (j >= 0) v = m.w[j] << bs;
    if (bs && j - 1 >= 0) v |= m.w[j - 1] >> (64 - bs);
    o.w[i] = v;
  }
  return o;
}
__device__ __forceinline__ Mask mshr(const Mask& m, int s) {
  Mask o;
  int ws = s >> 6, bs = s & 63;
  for (int i = 0; i < RW; ++i) {
    uint64_t v = 0;
    int j = i + ws;
    if (j < RW) v = m.w[j] >> bs;
    if (bs && j + 1 < RW) v |= m.w[j + 1] << (64 - bs);
    o.w[i] = v;
  }
  return o;
}

// Volumes of the box (box metric) or L1 ball (path metric) of radius R around
// cell c that are reached from c through open faces inside the box.
// Bit b = bx + S*(by + S*bz), S = 2R+1, b? = offset + R.
__global__ void k_reach(Dims dm, const int32_t* __restrict__ cells, int64_t ncells, const uint8_t* __restrict__ flag,
                        const uint8_t* __restrict__ ff0, const uint8_t* __restrict__ ff1,
                        const uint8_t* __restrict__ ff2, Mask* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells) return;
  const int R = dm.R, S = 2 * R + 1;
  const int SZ = dm.dim == 3 ? S : 1;
  int x[3];
  cell_xyz(dm, cells[t], x);
  const uint8_t* ff[3] = {ff0, ff1, ff2};
  Mask vol = {}, open[3] = {};
  for (int bz = 0; bz < SZ; ++bz)
    for (int by = 0; by < S; ++by)
      for (int bx = 0; bx < S; ++bx) {
        int y[3] = {x[0] + bx - R, x[1] + by - R, dm.dim == 3 ? x[2] + bz - R : 0};
        if (!in_domain(dm, y)) continue;
        int b = bx + S * (by + S * bz);
        if (flag[cell_id(dm, y)] > 0) mset(vol, b);
        int bb[3] = {bx, by, bz};
        for (int d = 0; d < dm.dim; ++d) {
          if (bb[d] == S - 1 || y[d] == dm.n[d] - 1) continue;  // face to +d stays in the box and domain
          int fy[3] = {y[0], y[1], y[2]};
          fy[d] += 1;
          if (ff[d][face_local(dm, d, fy)] > 0) mset(open[d], b);
        }
      }
  Mask m = {};
  int center = R + S * (R + (dm.dim == 3 ? S * R : 0));
  mset(m, center);
  int stride[3] = {1, S, S * S};
  int maxit = dm.nbr_box ? S * S * SZ : R;
  for (int it = 0; it < maxit; ++it) {
    Mask nm = m;
    for (int d = 0; d < dm.dim; ++d) {
      Mask a, up, dn;
      for (int i = 0; i < RW; ++i) a.w[i] = m.w[i] & open[d].w[i];
      up = mshl(a, stride[d]);          // b -> b + e_d through the face above b
      Mask shifted = mshr(m, stride[d]);  // b + e_d -> b through the face above b
      for (int i = 0; i < RW; ++i) dn.w[i] = shifted.w[i] & open[d].w[i];
      for (int i = 0; i < RW; ++i) nm.w[i] |= (up.w[i] | dn.w[i]) & vol.w[i];
    }
    bool same = true;
    for (int i = 0; i < RW; ++i) same &= nm.w[i] == m.w[i];
    m = nm;
    if (same) break;
  }
  out[t] = m;
}

// ============================================================ 3. gather


__device__ __forceinline__ bool reached(const GatherArgs& a, int64_t v, int dx, int dy, int dz) {
  const Dims& dm = a.dm;
  int R = dm.R;
  int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
  if (dm.nbr_box) { if (ax > R || ay > R || az > R) return false; }
  else if (ax + ay + az > R) return false;
  int32_t ri = a.reach_idx[v];
  if (ri < 0) return true;  // clean neighbourhood: every in-domain cell of the box is reached
  int S = 2 * R + 1;
  int b = (dx + R) + S * ((dy + R) + S * (dm.dim == 3 ? dz + R : 0));
  return mtest(a.masks[ri], b);
}

// Rows of slot s, in canonical order: volumes (ascending cell index), wall
// faces (ascending global face id), EB faces (ascending cut index).
__device__ int gather_rows(const GatherArgs& a, int64_t s, uint32_t* out) {
  const Dims& dm = a.dm;
  int64_t gf = a.slot_face[s];
  int R = dm.R;
  int base[3], lo_ok = 0, hi_ok = 0, dface = -1;
  int64_t vlo = -1, vhi = -1;
  int rng_lo[3], rng_hi[3];
  if (gf >= dm.n_grid_faces) return -1;  // EB slots are handled by the caller (base cell passed separately)
  for (int d = 0; d < dm.dim; ++d)
    if (gf >= dm.face_base[d]) dface = d;
  int64_t f = gf - dm.face_base[dface];
  face_xyz(dm, dface, f, base);
  if (base[dface] < dm.n[dface]) { hi_ok = 1; vhi = cell_id(dm, base); hi_ok = a.flag[vhi] > 0; }
  if (base[dface] > 0) {
    int lo[3] = {base[0], base[1], base[2]};
    lo[dface] -= 1;
    vlo = cell_id(dm, lo);
    lo_ok = a.flag[vlo] > 0;
  }
  for (int k = 0; k < 3; ++k) {
    rng_lo[k] = k < dm.dim ? -R : 0;
    rng_hi[k] = k < dm.dim ? R : 0;
  }
  rng_lo[dface] = -R - 1;
  int n = 0;
  for (int pass = 0; pass < 2 + dm.dim; ++pass) {
    for (int dz = rng_lo[2]; dz <= rng_hi[2]; ++dz)
      for (int dy = rng_lo[1]; dy <= rng_hi[1]; ++dy)
        for (int dx = rng_lo[0]; dx <= rng_hi[0]; ++dx) {
          int c[3] = {base[0] + dx, base[1] + dy, base[2] + dz};
          if (!in_domain(dm, c)) continue;
          int64_t cid = cell_id(dm, c);
          if (a.flag[cid] == 0) continue;
          int dd[3] = {dx, dy, dz};
          bool in = false;
          if (hi_ok) in = reached(a, vhi, dx, dy, dz);
          if (!in && lo_ok) {
            int e[3] = {dx, dy, dz};
            e[dface] += 1;
            in = reached(a, vlo, e[0], e[1], e[2]);
          }
          if (!in) continue;
          if (pass == 0) {
            if (out) out[n] = rd_pack(0, 0, 0, dd[0], dd[1], dd[2]);
            ++n;
          } else if (pass == 1 + dm.dim) {
            if (a.flag[cid] == 2) {
              if (out) out[n] = rd_pack(1, 0, 0, dd[0], dd[1], dd[2]);
              ++n;
            }
          } else {
            int wd = pass - 1;
            if (c[wd] == 0) {
              int fx[3] = {c[0], c[1], c[2]};
              if (a.ff[wd][face_local(dm, wd, fx)] > 0) {
                if (out) out[n] = rd_pack(2, wd, 0, dd[0], dd[1], dd[2]);
                ++n;
              }
            }
            if (c[wd] == dm.n[wd] - 1) {
              int fx[3] = {c[0], c[1], c[2]};
              fx[wd] += 1;
              if (a.ff[wd][face_local(dm, wd, fx)] > 0) {
                if (out) out[n] = rd_pack(2, wd, 1, dd[0], dd[1], dd[2]);
                ++n;
              }
            }
          }
        }
  }
  return n;
}

// EB faces: neighbourhood of the cut cell itself
__device__ int gather_rows_eb(const GatherArgs& a, int64_t v, uint32_t* out) {
  const Dims& dm = a.dm;
  int R = dm.R;
  int base[3];
  cell_xyz(dm, v, base);
  int zr = dm.dim == 3 ? R : 0;
  int n = 0;
  for (int pass = 0; pass < 2 + dm.dim; ++pass)
    for (int dz = -zr; dz <= zr; ++dz)
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          int c[3] = {base[0] + dx, base[1] + dy, base[2] + dz};
          if (!in_domain(dm, c)) continue;
          int64_t cid = cell_id(dm, c);
          if (a.flag[cid] == 0) continue;
          if (!reached(a, v, dx, dy, dz)) continue;
          if (pass == 0) {
            if (out) out[n] = rd_pack(0, 0, 0, dx, dy, dz);
            ++n;
          } else if (pass == 1 + dm.dim) {
            if (a.flag[cid] == 2) {
              if (out) out[n] = rd_pack(1, 0, 0, dx, dy, dz);
              ++n;
            }
          } else {
            int wd = pass - 1;
            if (c[wd] == 0) {
              if (a.ff[wd][face_local(dm, wd, c)] > 0) {
                if (out) out[n] = rd_pack(2, wd, 0, dx, dy, dz);
                ++n;
              }
            }
            if (c[wd] == dm.n[wd] - 1) {
              int fx[3] = {c[0], c[1], c[2]};
              fx[wd] += 1;
              if (a.ff[wd][face_local(dm, wd, fx)] > 0) {
                if (out) out[n] = rd_pack(2, wd, 1, dx, dy, dz);
                ++n;
              }
            }
          }
        }
  return n;
}

__global__ void k_gather(GatherArgs a, int64_t n_slots, const int32_t* __restrict__ cut_cell) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  int64_t gf = a.slot_face[s];
  uint32_t* out = a.row_ptr ? a.row_desc + a.row_ptr[s] : nullptr;
  int n;
  if (gf >= a.dm.n_grid_faces) n = gather_rows_eb(a, cut_cell[gf - a.dm.n_grid_faces], out);
  else n = gather_rows(a, s, out);
  if (!a.row_ptr) {
    a.count[s] = n;
    if (n > MAXROWS) atomicExch(a.too_many, 1);
  }
}

// ============================================================ 4. weighted LS (FP64)

__device__ __forceinline__ int tab_index(const double* delta) {
  int i0 = (int)lrint(2.0 * delta[0]) + 11, i1 = (int)lrint(2.0 * delta[1]) + 11, i2 = (int)lrint(2.0 * delta[2]) + 11;
  if (i0 < 0 || i0 >= TAB_S || i1 < 0 || i1 >= TAB_S || i2 < 0 || i2 >= TAB_S) return -1;
  return i0 + TAB_S * (i1 + TAB_S * i2);
}

__device__ __forceinline__ double weight_of(const Dims& dm, double r2) {
  // Sec. 2.4: W_ii = 1 if r < 1/2, else (2r)^-5, r = |x_i - x0| / h
  if (!dm.weighted || r2 < dm.w_threshold * dm.w_threshold) return 1.0;
  return pow(4.0 * r2, -0.5 * dm.w_power);
}

// Rows of full cells depend only on the offset delta = (cell centre - x0)/h:
// the average of prod_d xi_d^{p_d} over the unit cell centred at delta is
// prod_d ((delta_d + 1/2)^{p_d+1} - (delta_d - 1/2)^{p_d+1}) / (p_d + 1).
__global__ void k_full_rows(Dims dm, const Tables* __restrict__ T, double* __restrict__ ftab,
                            double* __restrict__ wtab) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= TAB_N) return;
  double delta[3] = {0.5 * (t % TAB_S - 11), 0.5 * ((t / TAB_S) % TAB_S - 11), 0.5 * (t / (TAB_S * TAB_S) - 11)};
  double oned[3][8];
  for (int d = 0; d < 3; ++d) {
    double a = delta[d] - 0.5, b = delta[d] + 0.5, pa = a, pb = b;
    for (int p = 0; p < 8; ++p) {
      oned[d][p] = d < dm.dim ? (pb - pa) / (p + 1) : (p == 0 ? 1.0 : 0.0);
      pa *= a;
      pb *= b;
    }
  }
  double r2 = 0.0;
  for (int d = 0; d < dm.dim; ++d) r2 += delta[d] * delta[d];
  double w = weight_of(dm, r2);
  wtab[t] = w;
  for (int i = 0; i < T->K; ++i) {
    double v = 1.0;
    for (int d = 0; d < dm.dim; ++d) v *= oned[d][T->mon[i][d]];
    ftab[(int64_t)t * MAXK + i] = w * v;
  }
}

// Moments of (x + delta)^p from the moments of x^p, one dimension at a time.  Along a line of
// monomials (exponents 0..N-1 in dimension d, the others fixed) the new moments are
// m'_p = sum_{j <= p} C(p, j) delta^(p-j) m_j; N-1 sweeps of m_j += delta m_{j-1} (j descending)
// build the binomial sums without forming binomials or powers (Horner's scheme for the Taylor
// shift of a polynomial), N(N-1)/2 FMAs per line.
template <int N>
__device__ __forceinline__ void shift_line(double* out, const uint8_t* idx, double dl) {
  double a[N];
#pragma unroll
  for (int p = 0; p < N; ++p) a[p] = out[idx[p]];
#pragma unroll
  for (int i = 1; i < N; ++i)
#pragma unroll
    for (int j = N - 1; j >= i; --j) a[j] = fma(dl, a[j - 1], a[j]);
#pragma unroll
  for (int p = 1; p < N; ++p) out[idx[p]] = a[p];
}

__device__ void shift_moments(const Tables& T, const double* __restrict__ in, const double* delta, double* out) {
  const int K = T.K;
  if (in != out)
    for (int i = 0; i < K; ++i) out[i] = in[i];
  for (int d = 0; d < T.dim; ++d) {
    const double dl = delta[d];
    if (dl == 0.0) continue;
    for (int l = 0; l < T.nln[d]; ++l) {
      const uint8_t* ix = T.ln_idx[d][l];
      switch (T.ln_len[d][l]) {
        case 2: shift_line<2>(out, ix, dl); break;
        case 3: shift_line<3>(out, ix, dl); break;
        case 4: shift_line<4>(out, ix, dl); break;
        case 5: shift_line<5>(out, ix, dl); break;
        default: break;
      }
    }
  }
}

// One weighted LS row (Sec. 2.2.1 rows, Sec. 2.4 weights) in row[]; x0s: x0 offset from the base cell
// centre in units of h.  Returns the weight.  Rows of full cells come from the offset table; a row
// whose moments must be shifted to x0 is left pending (*pend = 1) with its source pointer, offset
// and weight recorded in row[0..4], so that the warp can shift all pending rows of a chunk with
// every lane busy (row_finish).  Wall rows over a cut face are shifted here.
__device__ double row_prepare(const LsArgs& a, const Tables& T, uint32_t desc, const int* base, const double* x0s,
                              double* row, int* bad, int* pend) {
  const Dims& dm = a.dm;
  const int K = T.K;
  *pend = 0;
  int kind = rd_kind(desc);
  int c[3], dl[3];
  for (int d = 0; d < 3; ++d) {
    dl[d] = d < dm.dim ? rd_off(desc, d) : 0;
    c[d] = base[d] + dl[d];
  }
  int64_t cid = cell_id(dm, c);
  double delta[3];
  for (int d = 0; d < 3; ++d) delta[d] = (double)dl[d] - x0s[d];
  const double* src;
  double w;
  if (kind == 2) {
    int wd = rd_wdir(desc), ws = rd_wside(desc);
    delta[wd] += ws ? 0.5 : -0.5;
    int fx[3] = {c[0], c[1], c[2]};
    if (ws) fx[wd] += 1;
    int32_t cf = a.cutface_of[wd][face_local(dm, wd, fx)];
    double r2 = 0.0;
    for (int d = 0; d < dm.dim; ++d) r2 += delta[d] * delta[d];
    w = weight_of(dm, r2);
    if (cf >= 0) {
      const double* fm = a.face_mom[wd] + (int64_t)cf * dm.KFS;
      for (int i = 0; i < K; ++i) row[i] = T.tang[wd][i] >= 0 ? fm[T.tang[wd][i]] : 0.0;
      shift_moments(T, row, delta, row);
      double sc = w / row[0];
      for (int i = 0; i < K; ++i) row[i] *= sc;
      return w;
    }
    src = T.full_face[wd];
  } else {
    int ti = tab_index(delta);
    if (ti >= 0) w = a.wtab[ti];
    else {
      double r2 = 0.0;
      for (int d = 0; d < dm.dim; ++d) r2 += delta[d] * delta[d];
      w = weight_of(dm, r2);
    }
    int32_t cut = a.cut_of_cell[cid];
    if (kind == 0 && cut < 0 && ti >= 0) {
      const double* fr = a.ftab + (int64_t)ti * MAXK;
      for (int i = 0; i < K; ++i) row[i] = fr[i];
      return w;
    }
    if (kind == 1 && a.eb_bc && a.eb_bc[cut] != 0) {
      // Neumann row (Sec. 2.2.1): (1/m^0) sum_d p_d m^{p - e_d}_d, from the EB moments weighted by
      // the normal components, shifted to x0.  It is a derivative in xi = (x - x0)/h, so its
      // coefficient is h^(D-1) s_hat and the physical minimum-norm problem weighs it with W_ii / h.
      const double wn = w / dm.h;
      double sh[MAXK];
      for (int i = 0; i < K; ++i) row[i] = 0.0;
      for (int d = 0; d < dm.dim; ++d) {
        shift_moments(T, a.eb_nmom + ((int64_t)cut * dm.dim + d) * dm.KS, delta, sh);
        for (int i = 0; i < K; ++i) {
          const int lo = T.lower[d][i];
          if (lo >= 0) row[i] = fma((double)T.mon[i][d], sh[lo], row[i]);
        }
      }
      const double sc = wn / a.eb_mom[(int64_t)cut * dm.KS];
      for (int i = 0; i < K; ++i) row[i] *= sc;
      return wn;
    }
    if (kind == 1) src = a.eb_mom + (int64_t)cut * dm.KS;
    else src = cut >= 0 ? a.vol_mom + (int64_t)cut * dm.KS : T.full_vol;
  }
  row[0] = __longlong_as_double((long long)(uintptr_t)src);
  row[1] = delta[0];
  row[2] = delta[1];
  row[3] = delta[2];
  row[4] = w;
  *pend = 1;
  return w;
}

// the moment shift and weighting of a pending row (record in row[0..4])
__device__ void row_finish(const Tables& T, double* row) {
  const double* src = reinterpret_cast<const double*>((uintptr_t)__double_as_longlong(row[0]));
  const double delta[3] = {row[1], row[2], row[3]};
  const double w = row[4];
  shift_moments(T, src, delta, row);
  const double sc = w / row[0];
  for (int i = 0; i < T.K; ++i) row[i] *= sc;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Column sums of P[0..32)[c0 + STR*c] for c < mm (mm <= 32/G columns): G lanes per column each sum
// 32/G partials with independent accumulators, then a shuffle tree.  Returns the sum in the first
// lane of each group; *col is the column number c (or -1).  The accumulators start from the first
// partials (no additions of zero: the FP64 pipe is the kernel's bound, and an add costs it as much
// as an FMA).
template <int G, int STR, typename T>
__device__ __forceinline__ T colsum_g(const T* P, int c0, int mm, int lane, int* col) {
  constexpr int L = 32 / G;
  const int cl = lane / G, part = lane % G;
  T s = 0;
  if (cl < mm) {
    const T* p = P + (part * L) * KST + c0 + STR * cl;
    if constexpr (L >= 4) {
      T a0 = p[0], a1 = p[KST], a2 = p[2 * KST], a3 = p[3 * KST];
#pragma unroll
      for (int l = 4; l < L; l += 4) {
        a0 += p[l * KST];
        a1 += p[(l + 1) * KST];
        a2 += p[(l + 2) * KST];
        a3 += p[(l + 3) * KST];
      }
      s = (a0 + a1) + (a2 + a3);
    } else if constexpr (L == 2) {
      s = p[0] + p[KST];
    } else {
      s = p[0];
    }
  }
#pragma unroll
  for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  *col = (cl < mm && part == 0) ? cl : -1;
  return s;
}

template <int STR, typename T>
__device__ __forceinline__ T column_sums(const T* P, int c0, int mm, int lane, int* col) {
  if (mm > 16) return colsum_g<1, STR>(P, c0, mm, lane, col);
  if (mm > 8) return colsum_g<2, STR>(P, c0, mm, lane, col);
  if (mm > 4) return colsum_g<4, STR>(P, c0, mm, lane, col);
  if (mm > 2) return colsum_g<8, STR>(P, c0, mm, lane, col);
  if (mm > 1) return colsum_g<16, STR>(P, c0, mm, lane, col);
  return colsum_g<32, STR>(P, c0, mm, lane, col);
}

// sign and zero tests on the bit patterns (integer pipe)
__device__ __forceinline__ bool bits_nonzero(double v) { return __double_as_longlong(v) != 0; }
__device__ __forceinline__ bool bits_nonzero(float v) { return __float_as_int(v) != 0; }
__device__ __forceinline__ bool bits_positive(double v) { return __double_as_longlong(v) > 0; }
__device__ __forceinline__ bool bits_positive(float v) { return __float_as_int(v) > 0; }

constexpr uint32_t PAIR_WAIT_LIMIT = 1000000u;
constexpr int LS_MAX_CORR = 8;             // corrections of the FP32-factorisation path
constexpr double LS_CORR_TOL = 1e-14;      // converged: the last correction moved t by at most this (2-norm, relative)
constexpr double LS_CORR_FLOOR = 1e-11;    // ... or by at most this and less than half the one before (rounding floor)
constexpr float LS_F32_MIN_DIAG = 2e-5f;   // FP32 factor with min |R_kk| below this times the largest: FP64 path

// Barrier of the two warps of one system: every lane arrives on the system's mbarrier (64 arrivals
// complete a phase; arrive releases, the wait acquires), then waits for the phase.  The wait is
// bounded: when it gives up it sets the error word and returns false, and the caller leaves the
// kernel (its partner then gives up at its next barrier), so the kernel cannot hang on it.
__device__ __forceinline__ bool pair_sync(unsigned long long* bar, uint32_t& phase, int32_t* err) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
  bool ok = false;
  for (uint32_t i = 0; i < PAIR_WAIT_LIMIT; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(phase)
        : "memory");
    if (done) { ok = true; break; }
  }
  if (!ok) atomicExch(err, 1);
  phase ^= 1u;
  return __all_sync(0xffffffffu, ok);
}

#define PAIR_SYNC()                                    \
  do {                                                 \
    if (!pair_sync(&S.bar, phase, a0.err)) return;     \
  } while (0)

// One system (face) per group of LS_NW warps.  Every warp holds the chunk's rows (lane l: rows
// l + 32 r) and the current Householder vector; warp h owns the columns j with j % LS_NW == h: their
// partial dots, column sums, taus, R entries and updates.  Per Householder step the exchanges are
// column k+1 (the next vector, updated by its owner and read by the others after a group barrier)
// and its scalars (posted by the owner with a sequence flag and read at the start of the next step).
//
// QT = double: the FP64 factorisation, the rank test |R_kk| <= 1e-12 max |R_jj| and one correction of
// the semi-normal equations (t = B z, z = R^-1 R^-T F; t += B R^-1 R^-T (F - B^T t)).
// QT = float: the rows are built in FP64 (kept for the corrections) and factorised in FP32; the FP32
// factor preconditions FP64 corrections of the semi-normal equations, repeated until a correction moves
// t by at most LS_CORR_TOL, or stops shrinking at the rounding floor (B R^-1 has singular values within
// 1 +- cond(B) eps_32 of one, so each correction gains about that factor; the corrections end at the
// same rounding floor as the FP64 path).  A
// system whose FP32 factor is too ill-conditioned for that, or whose corrections do not settle within
// LS_MAX_CORR, gets status 3 and is solved again by the FP64 kernel (which also makes the rank test).
//
// BATCH: the systems of several geometries (same dimension and order) in one launch; the work counter,
// the total system count, the scratch and the error word come from a0, each system's geometry data
// from batch[g] with g found from the prefix sums of the systems per geometry (slot_base).
template <bool BATCH, typename QT>
__global__ void __launch_bounds__(ls_sys<QT>() * LS_NW * 32, 1)
    k_lsq(const __grid_constant__ LsArgs a0, const __grid_constant__ Tables T, const LsArgs* __restrict__ batch,
          const int64_t* __restrict__ slot_base, int n_geom) {
  constexpr bool F32 = sizeof(QT) == 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sys = warp / LS_NW, h = warp % LS_NW;
  LsSysSmem<QT>& S = reinterpret_cast<LsSysSmem<QT>*>(smem_raw)[sys];
  const int K = T.K;
  const int gs = blockIdx.x * ls_sys<QT>() + sys;
  double* scr = a0.scratch + (int64_t)gs * LS_SCRATCH;  // column-major: scr[k * MAXROWS + i]
  double* scr_w = scr + (int64_t)MAXROWS * MAXK;
  double* scr_t = scr_w + MAXROWS;
  double* stage = scr_t + MAXROWS;  // FP64 rows of the chunk (FP32 factorisation), row stride KST
  double* F = S.vec;
  double* y = S.vec + MAXK;
  double* z = S.vec + 2 * MAXK;
  double* tau = S.vec + 3 * MAXK;
  double* rinv = S.vec + 4 * MAXK;
  if (h == 0 && lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(&S.bar)),
                 "r"(32 * LS_NW)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    S.hs_seq[0] = S.hs_seq[1] = -1;
  }
  __syncthreads();
  uint32_t phase = 0;
  int32_t stepno = 0;  // Householder steps taken by this pair (same count in both warps)
  while (true) {
    if (h == 0 && lane == 0) S.slot = atomicAdd(a0.next, 1);
    PAIR_SYNC();
    int s = S.slot;
    if (s >= a0.n_slots) break;
    if (a0.slot_list) s = a0.slot_list[s];
    int g = 0;
    if constexpr (BATCH) {  // the geometry of system s: last g with slot_base[g] <= s
      int lo = 0, hi = n_geom - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (slot_base[mid] <= s) lo = mid;
        else hi = mid - 1;
      }
      g = lo;
      s -= (int)slot_base[g];
    }
    const LsArgs& a = BATCH ? batch[g] : a0;
    const Dims& dm = a.dm;
    const int64_t p0 = a.row_ptr[s];
    const int n = (int)(a.row_ptr[s + 1] - p0);
    const int64_t gf = a.slot_face[s];
    // base cell and x0 (Sec. 2.4: face centre for grid faces, cell centre for EB faces)
    int base[3] = {0, 0, 0};
    double x0s[3] = {0.0, 0.0, 0.0};
    int dface = -1;
    int64_t cut_self = -1, flocal = -1;
    if (gf >= dm.n_grid_faces) {
      cut_self = gf - dm.n_grid_faces;
      cell_xyz(dm, a.cut_cell[cut_self], base);
    } else {
      for (int d = 0; d < dm.dim; ++d)
        if (gf >= dm.face_base[d]) dface = d;
      flocal = gf - dm.face_base[dface];
      face_xyz(dm, dface, flocal, base);
      x0s[dface] = -0.5;
    }
    int bad = 0;
    for (int i = lane + 32 * h; i < K * K; i += 32 * LS_NW) S.R[i] = (QT)0;
    // ---- row-streamed Householder QR of B = W A: R accumulates the triangular factor
    for (int c0 = 0; c0 < n; c0 += CH) {
      // rows of the chunk (warp h builds the row slots r with r % LS_NW == h): table rows directly,
      // shifted rows queued (one ballot mask per row slot) and shifted with every lane busy.  FP64
      // factorisation: built in the chunk buffer; FP32: built in the FP64 staging rows, then rounded
      // into the chunk buffer
      constexpr int NSLOT = (RPL + LS_NW - 1) / LS_NW;
      unsigned pend[NSLOT];
      int npend = 0;
      auto row_at = [&](int li) -> double* {
        if constexpr (F32) return stage + li * KST;
        else return reinterpret_cast<double*>(S.C) + li * KST;
      };
#pragma unroll
      for (int rr = 0; rr < NSLOT; ++rr) {
        const int r = h + LS_NW * rr;
        pend[rr] = 0u;
        if (r >= RPL) continue;
        const int li = lane + 32 * r, i = c0 + li;
        double* dst = row_at(li);
        int pd = 0;
        if (i < n) {
          scr_w[i] = row_prepare(a, T, a.row_desc[p0 + i], base, x0s, dst, &bad, &pd);
        } else {
          for (int k = 0; k < K; ++k) dst[k] = 0.0;
        }
        pend[rr] = __ballot_sync(0xffffffffu, pd);
        npend += __popc(pend[rr]);
      }
      __syncwarp();
      for (int q0 = 0; q0 < npend; q0 += 32) {
        int q = q0 + lane;
        if (q < npend) {
          int rr = 0;
          while (q >= __popc(pend[rr])) {
            q -= __popc(pend[rr]);
            ++rr;
          }
          unsigned mk = pend[rr];
          for (int t = 0; t < q; ++t) mk &= mk - 1;  // drop the q lowest set bits
          const int l = __ffs(mk) - 1;
          row_finish(T, row_at(l + 32 * (h + LS_NW * rr)));
        }
      }
      __syncwarp();
#pragma unroll
      for (int rr = 0; rr < NSLOT; ++rr) {
        const int r = h + LS_NW * rr;
        if (r >= RPL) continue;
        const int li = lane + 32 * r, i = c0 + li;
        const double* src = row_at(li);
        if (i < n) {
          for (int k = 0; k < K; ++k) {
            const double v = src[k];
            scr[(int64_t)k * MAXROWS + i] = v;
            if constexpr (F32) S.C[li * KST + k] = (QT)v;
          }
        } else if constexpr (F32) {
          for (int k = 0; k < K; ++k) S.C[li * KST + k] = (QT)0;
        }
      }
      PAIR_SYNC();  // the chunk's rows are complete
      // rows of this chunk per lane (the last chunk is short: skip its empty row slots)
      const int nr = (min(CH, n - c0) + 31) >> 5;
      // Householder steps k = 0..K-1 on [R; C].  The update of step k and the partial dot products of
      // step k+1 share one pass: column k+1 is updated first by its owner (it is step k+1's Householder
      // vector), then each warp loads, updates, stores and dots its own later columns.
      QT ck[RPL];
#pragma unroll
      for (int r = 0; r < RPL; ++r) ck[r] = r < nr ? S.C[(lane + 32 * r) * KST] : (QT)0;
      QT* Pl = S.P + lane * KST;
      {  // partial dots of column 0 with the own columns j >= 1
        const QT* Cl = S.C + lane * KST;
        for (int j = 1 + (h + LS_NW - 1) % LS_NW; j < K; j += LS_NW) {
          QT pp = 0;
#pragma unroll
          for (int r = 0; r < RPL; ++r)
            if (r < nr) pp = fma(ck[r], Cl[32 * r * KST + j], pp);
          Pl[j] = pp;
        }
      }
      // Householder scalars of step k from its vector (chunk part c, R part alpha = R_kk)
      auto hscalars = [&](const QT* c, int k, QT* out) {
        QT ss = c[0] * c[0];
#pragma unroll
        for (int r = 1; r < RPL; ++r) ss = fma(c[r], c[r], ss);
        ss = warp_sum(ss);
        // a zero chunk column needs no reflection
        const bool refl = bits_nonzero(ss);
        const QT alpha = S.R[k * K + k];
        const QT sigma = refl ? sqrt(fma(alpha, alpha, ss)) : (QT)0;
        out[0] = bits_positive(alpha) ? -sigma : sigma;  // beta
        out[1] = alpha - out[0];                          // v0
        out[2] = refl ? (QT)-1 / (out[0] * out[1]) : (QT)0;  // gamma
        out[3] = refl ? (QT)1 : (QT)0;
      };
      QT hk[4], hnext[4] = {0, 0, 0, 0};
      hscalars(ck, 0, hk);  // step 0: both warps (the vector is column 0)
      for (int k = 0; k < K; ++k, ++stepno) {
        if (k > 0 && h != k % LS_NW) {
          // step k's scalars, computed once by the owner of column k during step k-1 and posted with the
          // step number after the values (bounded wait; giving up sets the error word and leaves)
          volatile int32_t* seq = &S.hs_seq[k & 1];
          uint32_t it = 0;
          while (*seq != stepno && ++it < PAIR_WAIT_LIMIT) {
          }
          if (it >= PAIR_WAIT_LIMIT) {
            atomicExch(a0.err, 1);
            return;
          }
          __threadfence_block();
#pragma unroll
          for (int q = 0; q < 4; ++q) hk[q] = S.hs[k & 1][q];
        } else if (k > 0) {
#pragma unroll
          for (int q = 0; q < 4; ++q) hk[q] = hnext[q];  // this warp computed them in step k-1
        }
        const QT beta = hk[0], v0 = hk[1], gamma = hk[2];
        const bool refl = bits_nonzero(hk[3]);  // 1 or 0
        __syncwarp();  // P holds the partial dots of column k with the own later columns
        const int jf = k + 1 + (h + LS_NW - (k + 1) % LS_NW) % LS_NW;  // first own column after k
        const int mown = jf < K ? (K - 1 - jf) / LS_NW + 1 : 0;
        for (int c1 = 0; c1 < mown; c1 += 32) {
          const int mm = mown - c1 < 32 ? mown - c1 : 32;
          int col;
          const QT sum = column_sums<LS_NW>(S.P, jf + LS_NW * c1, mm, lane, &col);
          if (col >= 0) {
            const int j = jf + LS_NW * (c1 + col);
            const QT rkj = S.R[k * K + j];
            const QT t = gamma * fma(v0, rkj, sum);
            if (refl) S.R[k * K + j] = fma(-t, v0, rkj);
            tau[j] = (double)t;
          }
        }
        __syncwarp();
        if (k + 1 < K) {
          const int owner = (k + 1) % LS_NW;
          QT ck1[RPL];
          if (h == owner) {  // column k+1: update, keep as the next Householder vector
            const QT t1 = (QT)tau[k + 1];
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
              QT* c = S.C + (lane + 32 * r) * KST + k + 1;
              ck1[r] = 0;
              if (r < nr) {
                ck1[r] = fma(-t1, ck[r], *c);
                *c = ck1[r];
              }
            }
          }
          PAIR_SYNC();
          if (h != owner) {
#pragma unroll
            for (int r = 0; r < RPL; ++r) ck1[r] = r < nr ? S.C[(lane + 32 * r) * KST + k + 1] : (QT)0;
          } else {
            // step k+1's scalars, off the other warp's path: it picks them up at the start of step k+1
            QT hn[4];
            hscalars(ck1, k + 1, hn);  // R_{k+1,k+1} is not touched by step k
            if (lane == 0) {
#pragma unroll
              for (int q = 0; q < 4; ++q) S.hs[(k + 1) & 1][q] = hn[q];
              __threadfence_block();
              *(volatile int32_t*)&S.hs_seq[(k + 1) & 1] = stepno + 1;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) hnext[q] = hn[q];
          }
          // own columns j >= k+2: update and dot with column k+1 (four columns per pass)
          constexpr int W = LS_NW;
          int j = k + 2 + (h + W - (k + 2) % W) % W;
          for (; j + 3 * W < K; j += 4 * W) {
            const QT t0 = (QT)tau[j], tt1 = (QT)tau[j + W], t2 = (QT)tau[j + 2 * W], t3 = (QT)tau[j + 3 * W];
            QT q0 = 0, q1 = 0, q2 = 0, q3 = 0;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
              if (r < nr) {
                QT* c = S.C + (lane + 32 * r) * KST + j;
                const QT e0 = fma(-t0, ck[r], c[0]), e1 = fma(-tt1, ck[r], c[W]);
                const QT e2 = fma(-t2, ck[r], c[2 * W]), e3 = fma(-t3, ck[r], c[3 * W]);
                c[0] = e0;
                c[W] = e1;
                c[2 * W] = e2;
                c[3 * W] = e3;
                q0 = fma(ck1[r], e0, q0);
                q1 = fma(ck1[r], e1, q1);
                q2 = fma(ck1[r], e2, q2);
                q3 = fma(ck1[r], e3, q3);
              }
            }
            Pl[j] = q0;
            Pl[j + W] = q1;
            Pl[j + 2 * W] = q2;
            Pl[j + 3 * W] = q3;
          }
          for (; j < K; j += W) {
            const QT t0 = (QT)tau[j];
            QT q0 = 0;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
              if (r < nr) {
                QT* c = S.C + (lane + 32 * r) * KST + j;
                const QT e0 = fma(-t0, ck[r], c[0]);
                c[0] = e0;
                q0 = fma(ck1[r], e0, q0);
              }
            }
            Pl[j] = q0;
          }
#pragma unroll
          for (int r = 0; r < RPL; ++r) ck[r] = ck1[r];
        }
        if (h == 0 && lane == 0 && refl) S.R[k * K + k] = beta;
        __syncwarp();
      }
      PAIR_SYNC();  // both warps are done with the chunk and with R
    }
    // ---- rank check (FP64: |R_kk| <= 1e-12 max |R_jj| counts as rank deficient; FP32: a factor that
    // ill-conditioned leaves the system to the FP64 kernel)
    const int anyb = __any_sync(0xffffffffu, bad);
    if (lane == 0) S.bad[h] = anyb;
    PAIR_SYNC();
    {
      int any = 0;
      for (int q = 0; q < LS_NW; ++q) any |= S.bad[q];
      bad = any ? 2 : 0;
    }
    double dmax = 0.0, dmin = INFINITY;
    for (int k = 0; k < K; ++k) {
      double v = fabs((double)S.R[k * K + k]);
      dmax = fmax(dmax, v);
      dmin = fmin(dmin, v);
    }
    if (!bad && !(dmin > (F32 ? (double)LS_F32_MIN_DIAG : 1e-12) * dmax)) bad = F32 ? 3 : 1;
    if (bad) {
      if (h == 0 && lane == 0) a.status[s] = bad;
      if (bad != 3)
        for (int i = lane + 32 * h; i < n; i += 32 * LS_NW) a.row_val[p0 + i] = 0.0;
      PAIR_SYNC();
      continue;
    }
    // ---- z = R^-1 R^-T rhs (two triangular solves, lanes own columns), by warp 0, in FP64
    auto solve_rtr = [&](const double* rhs, double* outz) {
      for (int j = lane; j < K; j += 32) y[j] = rhs[j];
      __syncwarp();
      for (int k = 0; k < K; ++k) {  // R^T y = rhs (forward)
        double yk = y[k] * rinv[k];
        __syncwarp();
        for (int j = k + 1 + lane; j < K; j += 32) y[j] = fma(-(double)S.R[k * K + j], yk, y[j]);
        if (lane == 0) y[k] = yk;
        __syncwarp();
      }
      for (int j = lane; j < K; j += 32) outz[j] = y[j];
      __syncwarp();
      for (int k = K - 1; k >= 0; --k) {  // R z = y (backward)
        double zk = outz[k] * rinv[k];
        __syncwarp();
        for (int j = lane; j < k; j += 32) outz[j] = fma(-(double)S.R[j * K + k], zk, outz[j]);
        if (lane == 0) outz[k] = zk;
        __syncwarp();
      }
    };
    if (h == 0) {
      for (int k = lane; k < K; k += 32) rinv[k] = 1.0 / (double)S.R[k * K + k];
      // ---- F_hat (Sec. 2.2.1): grid face: p_d m_f^{p-e_d}; EB face: sum_d p_d m_{d,f}^{p-e_d}
      for (int i = lane; i < K; i += 32) {
        double f = 0.0;
        if (cut_self >= 0) {
          for (int d = 0; d < dm.dim; ++d) {
            const double* nm = a.eb_nmom + ((int64_t)cut_self * dm.dim + d) * dm.KS;
            if (T.lower[d][i] >= 0) f += (double)T.mon[i][d] * nm[T.lower[d][i]];
          }
        } else {
          int q = T.lower[dface][i];
          if (q >= 0) {
            int32_t cf = a.cutface_of[dface][flocal];
            double mq;
            if (cf >= 0) mq = T.tang[dface][q] >= 0 ? a.face_mom[dface][(int64_t)cf * dm.KFS + T.tang[dface][q]] : 0.0;
            else mq = T.full_face[dface][q];
            f = (double)T.mon[i][dface] * mq;
          }
        }
        F[i] = f;
      }
      __syncwarp();
      solve_rtr(F, z);
    }
    PAIR_SYNC();
    // ---- corrected semi-normal equations: t = B z, then corrections t += B R^-1 R^-T (F - B^T t).
    // FP64 factorisation: one correction, B^T t from per-lane partials over the rows (warps h > 0 in the
    // free chunk buffer) and column sums.  FP32: lanes own columns and each warp sums half of the rows
    // (the chunk buffer is too small for the partials in FP64)
    for (int i = lane + 32 * h; i < n; i += 32 * LS_NW) {
      double t1 = 0.0;
      for (int k = 0; k < K; ++k) t1 = fma(scr[(int64_t)k * MAXROWS + i], z[k], t1);
      scr_t[i] = t1;
    }
    double* z2 = reinterpret_cast<double*>(S.C) + (CH * KST * sizeof(QT)) / 8 - 2 * MAXK;  // the chunk buffer's tail
    bool settled = false;
    double prev_sd = INFINITY;  // the previous correction's squared norm
    int ncorr = 0;
    for (int corr = 0; corr < (F32 ? LS_MAX_CORR : 1) && !settled; ++corr) {
      ++ncorr;
      if constexpr (F32) {
        PAIR_SYNC();  // t is complete
        const int i0 = h * ((n + 1) >> 1), i1 = h ? n : (n + 1) >> 1;
        double s0 = 0.0, s1 = 0.0;
        const double* c0p = scr + (int64_t)lane * MAXROWS;
        const double* c1p = scr + (int64_t)(lane + 32) * MAXROWS;
        for (int i = i0; i < i1; ++i) {
          const double t1 = scr_t[i];
          if (lane < K) s0 = fma(c0p[i], t1, s0);
          if (lane + 32 < K) s1 = fma(c1p[i], t1, s1);
        }
        if (lane < K) S.xch[h * MAXK + lane] = s0;
        if (lane + 32 < K) S.xch[h * MAXK + lane + 32] = s1;
      } else {
        double* Pw = h == 0 ? reinterpret_cast<double*>(S.P) : reinterpret_cast<double*>(S.C) + (h - 1) * 32 * KST;
        for (int k = 0; k < K; ++k) Pw[lane * KST + k] = 0.0;
        for (int i = lane + 32 * h; i < n; i += 32 * LS_NW) {
          const double t1 = scr_t[i];
          for (int k = 0; k < K; ++k) Pw[lane * KST + k] = fma(scr[(int64_t)k * MAXROWS + i], t1, Pw[lane * KST + k]);
        }
        __syncwarp();
        for (int c1 = 0; c1 < K; c1 += 32) {
          int mm = K - c1 < 32 ? K - c1 : 32;
          int col;
          double sum = column_sums<1>(Pw, c1, mm, lane, &col);
          if (col >= 0) S.xch[h * MAXK + c1 + col] = sum;
        }
      }
      PAIR_SYNC();
      if (h == 0) {
        for (int c = lane; c < K; c += 32) {
          double sx = 0.0;
          for (int q = 0; q < LS_NW; ++q) sx += S.xch[q * MAXK + c];
          tau[c] = F[c] - sx;
        }
        __syncwarp();
        solve_rtr(tau, z2);
      }
      PAIR_SYNC();
      if constexpr (F32) {
        double dd = 0.0, tt = 0.0;  // the correction's and the result's squared norms (this warp's rows)
        for (int i = lane + 32 * h; i < n; i += 32 * LS_NW) {
          double dt = 0.0;
          for (int k = 0; k < K; ++k) dt = fma(scr[(int64_t)k * MAXROWS + i], z2[k], dt);
          const double t = scr_t[i] + dt;
          scr_t[i] = t;
          dd = fma(dt, dt, dd);
          tt = fma(t, t, tt);
        }
        dd = warp_sum(dd);
        tt = warp_sum(tt);
        __syncwarp();
        if (lane == 0) {
          S.xch[h * MAXK] = dd;
          S.xch[h * MAXK + 1] = tt;
        }
        PAIR_SYNC();
        double sd = 0.0, st = 0.0;
        for (int q = 0; q < LS_NW; ++q) {
          sd += S.xch[q * MAXK];
          st += S.xch[q * MAXK + 1];
        }
        settled = sd <= LS_CORR_TOL * LS_CORR_TOL * st ||
                  (sd <= LS_CORR_FLOOR * LS_CORR_FLOOR * st && sd > 0.25 * prev_sd);
        prev_sd = sd;
      } else {
        for (int i = lane + 32 * h; i < n; i += 32 * LS_NW) {
          double t = scr_t[i];
          for (int k = 0; k < K; ++k) t = fma(scr[(int64_t)k * MAXROWS + i], z2[k], t);
          scr_t[i] = t;
        }
        settled = true;
      }
    }
    if (h == 0 && lane == 0 && a0.flops) {  // executed flops of this system (the row construction not counted)
      const double nn = n, kk = K;
      const double fact = 2.0 * nn * kk * kk - 2.0 / 3.0 * kk * kk * kk;  // Householder QR of n x K
      const double semi = 2.0 * nn * kk + 2.0 * kk * kk + ncorr * (4.0 * nn * kk + 2.0 * kk * kk);
      atomicAdd(a0.flops + 0, F32 ? semi : fact + semi);
      if (F32) atomicAdd(a0.flops + 1, fact);
    }
    if (!settled) {  // FP32 factor: the corrections did not settle; the FP64 kernel takes the system
      if (h == 0 && lane == 0) a.status[s] = 3;
      PAIR_SYNC();
      continue;
    }
    for (int i = lane + 32 * h; i < n; i += 32 * LS_NW) a.row_val[p0 + i] = scr_w[i] * scr_t[i];  // s_hat = W t
    if (h == 0 && lane == 0) a.status[s] = a0.slot_list ? 4 : 0;  // 4: solved by the FP64 pass after the FP32 one
    PAIR_SYNC();  // xch and the chunk buffer are free for the next system
  }
}

// ============================================================ 5. operator assembly


// flux faces of cell c: grid faces (sigma = +1 on the high face whose +e_d normal points out)
// and the EB face (sigma = +1); returns count, fills slot, sigma, base cell
__device__ int cell_faces(const AsmArgs& a, const int* x, int64_t c, int32_t* slots, double* sig, int (*bases)[3]) {
  const Dims& dm = a.dm;
  int nf = 0;
  for (int d = 0; d < dm.dim; ++d) {
    for (int side = 0; side < 2; ++side) {
      int fx[3] = {x[0], x[1], x[2]};
      if (side) fx[d] += 1;
      int32_t sl = a.face_slot[d][face_local(dm, d, fx)];
      if (sl < 0) continue;
      slots[nf] = sl;
      sig[nf] = side ? 1.0 : -1.0;
      bases[nf][0] = fx[0]; bases[nf][1] = fx[1]; bases[nf][2] = fx[2];
      ++nf;
    }
  }
  if (a.flag[c] == 2) {
    int32_t cut = a.cut_of_cell[c];
    slots[nf] = a.eb_slot[cut];
    sig[nf] = 1.0;
    bases[nf][0] = x[0]; bases[nf][1] = x[1]; bases[nf][2] = x[2];
    ++nf;
  }
  return nf;
}

// the cell is cut and its EB face carries Neumann data (the EB face is the last of cell_faces)
__device__ __forceinline__ bool neumann_eb(const AsmArgs& a, int64_t c) {
  return a.flag[c] == 2 && a.eb_bc[a.cut_of_cell[c]] != 0;
}

__device__ __forceinline__ int foot_index(const AsmArgs& a, int dx, int dy, int dz) {
  int L = a.dm.R + 1, S = 2 * L + 1;
  if (dx < -L || dx > L || dy < -L || dy > L || dz < -L || dz > L) return -1;
  return a.foot_lut[(dx + L) + S * ((dy + L) + S * (dz + L))];
}

// one warp per operator row: rows[r] from representative cell rep_cell[r]
__global__ void k_assemble_rows(AsmArgs a, const int32_t* __restrict__ rep_cell, int64_t nrep, int64_t row0,
                                int32_t* __restrict__ err) {
  extern __shared__ double acc_all[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (r >= nrep) return;
  double* acc = acc_all + warp * a.nfoot;
  for (int i = lane; i < a.nfoot; i += 32) acc[i] = 0.0;
  __syncwarp();
  int64_t c = rep_cell[r];
  int x[3];
  cell_xyz(a.dm, c, x);
  int32_t slots[8];
  double sig[8];
  int bases[8][3];
  int nf = cell_faces(a, x, c, slots, sig, bases);
  // the flux through a Neumann EB face is its datum (a column of B), not a stencil
  if (neumann_eb(a, c)) --nf;
  for (int q = 0; q < nf; ++q) {
    int64_t p0 = a.row_ptr[slots[q]], p1 = a.row_ptr[slots[q] + 1];
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      uint32_t ds = a.row_desc[p];
      if (rd_kind(ds) != 0) continue;
      int dx = rd_off(ds, 0) + bases[q][0] - x[0];
      int dy = rd_off(ds, 1) + bases[q][1] - x[1];
      int dz = a.dm.dim == 3 ? rd_off(ds, 2) + bases[q][2] - x[2] : 0;
      int fi = foot_index(a, dx, dy, dz);
      if (fi < 0) { atomicExch(err, 1); continue; }
      acc[fi] += sig[q] * a.row_val[p] * a.inv_h2;
    }
    __syncwarp();
  }
  for (int i = lane; i < a.nfoot; i += 32) {
    a.rows64[(int64_t)i * a.n_rows + row0 + r] = acc[i];
    a.rows32[(int64_t)i * a.n_rows + row0 + r] = (float)acc[i];
  }
}

// boundary entries of irregular cell rows: count (vals == null) or write
__global__ void k_assemble_b(AsmArgs a, const int32_t* __restrict__ cells, int64_t ncells, int64_t* __restrict__ cnt,
                             const int64_t* __restrict__ bptr, int64_t* __restrict__ bcol, double* __restrict__ bval,
                             const int32_t* __restrict__ cut_cell_unused) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells) return;
  const Dims& dm = a.dm;
  int64_t c = cells[t];
  int x[3];
  cell_xyz(dm, c, x);
  int32_t slots[8];
  double sig[8];
  int bases[8][3];
  int nf = cell_faces(a, x, c, slots, sig, bases);
  int64_t k = bptr ? bptr[t] : 0;
  int64_t n = 0;
  if (neumann_eb(a, c)) {
    // Neumann EB face: the flux is the datum, |A_f| <g>_f (sigma = +1, kappa-weighted scale 1/h^2)
    --nf;
    if (bptr) {
      const int32_t cut = a.cut_of_cell[c];
      bcol[k + n] = dm.n_grid_faces + cut;
      bval[k + n] = a.eb_mom[(int64_t)cut * dm.KS] * dm.h * a.inv_h2;
    }
    ++n;
  }
  for (int q = 0; q < nf; ++q) {
    int64_t p0 = a.row_ptr[slots[q]], p1 = a.row_ptr[slots[q] + 1];
    for (int64_t p = p0; p < p1; ++p) {
      uint32_t ds = a.row_desc[p];
      int kind = rd_kind(ds);
      if (kind == 0) continue;
      if (bptr) {
        int y[3];
        for (int d = 0; d < 3; ++d) y[d] = bases[q][d] + (d < dm.dim ? rd_off(ds, d) : 0);
        int64_t col;
        double sc = 1.0;
        if (kind == 1) {
          const int32_t cut = a.cut_of_cell[cell_id(dm, y)];
          col = dm.n_grid_faces + cut;
          if (a.eb_bc[cut] != 0) sc = dm.h;  // a Neumann row's datum enters as h <g> (derivative in xi)
        } else {
          int wd = rd_wdir(ds);
          if (rd_wside(ds)) y[wd] += 1;
          col = dm.face_base[wd] + face_local(dm, wd, y);
        }
        bcol[k + n] = col;
        bval[k + n] = sig[q] * a.row_val[p] * a.inv_h2 * sc;
      }
      ++n;
    }
  }
  if (!bptr) cnt[t] = n;
}

}  // namespace eb

namespace eb {

size_t lsq_smem(bool fp32) {
  return fp32 ? (size_t)LS_SYS_F * sizeof(LsSysSmem<float>) : (size_t)LS_SYS * sizeof(LsSysSmem<double>);
}

cudaError_t lsq_prepare() {
  const int sd = (int)lsq_smem(false), sf = (int)lsq_smem(true);
  cudaError_t e = cudaFuncSetAttribute(k_lsq<false, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sd);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lsq<true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sd);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lsq<false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sf);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lsq<true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sf);
  return e;
}

// ============================================================ 4c. adjoint of the stencil solves
//
// For J(s) with s_hat = W t, t the least-||t|| solution of B^T t = F, B = W A (Sec. 2.2.1), and sbar =
// dJ/ds_hat, the reverse-mode derivative with respect to B and F is (y = G^-1 F, G = B^T B,
// tbar = W sbar, z = G^-1 B^T tbar)
//     Fbar = z,   Bbar = tbar y^T - B (z y^T + y z^T),
// so a tangent (dB, dF) of the system changes J by
//     sum_i [(tbar_i - b_i . z)(y . db_i) - (b_i . y)(z . db_i)] + z . dF.
// Here J is the Lagrangian term -lam^T (kappa L) phi of the adjoint method: kappa L phi sums
// (1/h^2) sigma s_hat_f . Phi over the faces of each volume (Sec. 2.3), so for face f with volume
// columns c_i, sbar_i = -(sum_v sigma_v lam_v) phi_(c_i) / h^2 (boundary columns carry zero data).
// The tangent rows come from the moment tables' derivatives through the same row construction (the
// shift to x0 is linear; the row is normalised by its zeroth moment: d(m / m0) = (dm - m dm0 / m0) / m0).
// One warp per system; G by lanes over its upper-triangle entries, its Cholesky factor in shared memory
// (the adjoint needs about eight digits, which the normal equations keep for these systems).

// Several parameters share one pass: the rows, G's factor, y and z do not depend on the parameter, and
// each parameter adds its tangent's contraction (dJ[p]).  Systems without a cut cell, cut face or EB
// face among their rows and right-hand side do not move and are skipped.

// source of a row's moments: none (a full cell or face), a cut cell's volume or EB moments, or a cut face
enum : int { ROW_SRC_NONE = 0, ROW_SRC_VOL = 1, ROW_SRC_EB = 2, ROW_SRC_FACE = 3 };  // + wall direction

// weighted row b of one LS row (Dirichlet rows); returns the weight.  *col: the cell of a volume row, -1
// for a boundary row; *sc: w / m0 (b = sc m, m the moments shifted to x0); delta: the shift; *src: the
// table and entry its moments come from (kind << 56 | entry, kind ROW_SRC_*, 0 for full rows)
__device__ double row_build(const LsArgs& a, const Tables& T, uint32_t desc, const int* base, const double* x0s,
                            double* b, double* sc, double* delta, int64_t* col, int64_t* src) {
  const Dims& dm = a.dm;
  const int K = T.K;
  const int kind = rd_kind(desc);
  int c[3], dl[3];
  for (int d = 0; d < 3; ++d) {
    dl[d] = d < dm.dim ? rd_off(desc, d) : 0;
    c[d] = base[d] + dl[d];
  }
  const int64_t cid = cell_id(dm, c);
  for (int d = 0; d < 3; ++d) delta[d] = (double)dl[d] - x0s[d];
  *col = kind == 0 ? cid : -1;
  *src = 0;
  double m[MAXK];
  const double* mp = nullptr;
  double w;
  if (kind == 2) {
    const int wd = rd_wdir(desc), ws = rd_wside(desc);
    delta[wd] += ws ? 0.5 : -0.5;
    int fx[3] = {c[0], c[1], c[2]};
    if (ws) fx[wd] += 1;
    const int32_t cf = a.cutface_of[wd][face_local(dm, wd, fx)];
    double r2 = 0.0;
    for (int d = 0; d < dm.dim; ++d) r2 += delta[d] * delta[d];
    w = weight_of(dm, r2);
    if (cf >= 0) {
      const double* fm = a.face_mom[wd] + (int64_t)cf * dm.KFS;
      for (int i = 0; i < K; ++i) m[i] = T.tang[wd][i] >= 0 ? fm[T.tang[wd][i]] : 0.0;
      mp = m;
      *src = ((int64_t)(ROW_SRC_FACE + wd) << 56) | cf;
    } else {
      mp = T.full_face[wd];
    }
  } else {
    double r2 = 0.0;
    for (int d = 0; d < dm.dim; ++d) r2 += delta[d] * delta[d];
    w = weight_of(dm, r2);
    const int32_t cut = a.cut_of_cell[cid];
    if (kind == 1) {
      mp = a.eb_mom + (int64_t)cut * dm.KS;
      *src = ((int64_t)ROW_SRC_EB << 56) | cut;
    } else if (cut >= 0) {
      mp = a.vol_mom + (int64_t)cut * dm.KS;
      *src = ((int64_t)ROW_SRC_VOL << 56) | cut;
    } else {
      mp = T.full_vol;
    }
  }
  double sm[MAXK];
  shift_moments(T, mp, delta, sm);
  *sc = w / sm[0];
  for (int i = 0; i < K; ++i) b[i] = *sc * sm[i];
  return w;
}

// tangent db of a row built by row_build (b at stride MAXROWS) for parameter p
__device__ void row_dtangent(const LsArgs& a, const Tables& T, const AdjArgs& g, int p, int64_t src,
                             const double* delta, double sc, double w, const double* b, double* db) {
  const Dims& dm = a.dm;
  const int K = T.K;
  const int kind = (int)(src >> 56);
  const int64_t e = src & ((1ll << 56) - 1);
  double m[MAXK];
  const double* dp;
  if (kind >= ROW_SRC_FACE) {
    const int wd = kind - ROW_SRC_FACE;
    const double* dfm = g.dface[wd] + p * g.s_face[wd] + e * dm.KFS;
    for (int i = 0; i < K; ++i) m[i] = T.tang[wd][i] >= 0 ? dfm[T.tang[wd][i]] : 0.0;
    dp = m;
  } else {
    dp = (kind == ROW_SRC_EB ? g.deb : g.dvol) + p * g.s_vol + e * dm.KS;
  }
  double sd[MAXK];
  shift_moments(T, dp, delta, sd);
  const double r0 = sd[0] * sc / w;  // dm0 / m0
  for (int i = 0; i < K; ++i) db[i] = sc * sd[i] - r0 * b[(int64_t)i * MAXROWS];
}

__global__ void __launch_bounds__(ADJ_WARPS * 32)
    k_stencil_adjoint(const __grid_constant__ LsArgs a, const __grid_constant__ Tables T, AdjArgs g) {
  __shared__ double Gs[ADJ_WARPS][MAXK * MAXK];
  __shared__ double vs[ADJ_WARPS][5 * MAXK];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* G = Gs[warp];
  double* F = vs[warp];
  double* y = F + MAXK;
  double* z = F + 2 * MAXK;
  double* u = F + 3 * MAXK;
  double* rinv = F + 4 * MAXK;
  const Dims& dm = a.dm;
  const int K = T.K;
  const int E = K * (K + 1) / 2;
  const int gw = blockIdx.x * ADJ_WARPS + warp;
  double* sb = g.scratch + (int64_t)gw * MAXROWS * ADJ_SCRATCH;  // rows b, column-major
  double* sw = sb + (int64_t)MAXROWS * MAXK;                     // weights
  double* ssc = sw + MAXROWS;                                    // w / m0
  double* sby = ssc + MAXROWS;                                   // b_i . y
  double* sbz = sby + MAXROWS;                                   // b_i . z
  double* stb = sbz + MAXROWS;                                   // tbar_i
  double* sdl = stb + MAXROWS;                                   // shifts, [3][MAXROWS]
  int64_t* scol = reinterpret_cast<int64_t*>(sdl + 3 * MAXROWS);  // columns
  int64_t* ssrc = scol + MAXROWS;                                 // moment sources
  while (true) {
    int s = 0;
    if (lane == 0) s = atomicAdd(g.next, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= g.n_slots) break;
    const int64_t p0 = a.row_ptr[s];
    const int n = (int)(a.row_ptr[s + 1] - p0);
    const int64_t gf = a.slot_face[s];
    int base[3] = {0, 0, 0};
    double x0s[3] = {0.0, 0.0, 0.0};
    int dface = -1;
    int64_t cut_self = -1, flocal = -1;
    if (gf >= dm.n_grid_faces) {
      cut_self = gf - dm.n_grid_faces;
      cell_xyz(dm, a.cut_cell[cut_self], base);
    } else {
      for (int d = 0; d < dm.dim; ++d)
        if (gf >= dm.face_base[d]) dface = d;
      flocal = gf - dm.face_base[dface];
      face_xyz(dm, dface, flocal, base);
      x0s[dface] = -0.5;
    }
    if (n < K) continue;
    // rows, weights, columns and moment sources
    int moving = 0;
    for (int i = lane; i < n; i += 32) {
      double b[MAXK], dl[3], sc;
      int64_t col, src;
      sw[i] = row_build(a, T, a.row_desc[p0 + i], base, x0s, b, &sc, dl, &col, &src);
      ssc[i] = sc;
      scol[i] = col;
      ssrc[i] = src;
      for (int d = 0; d < 3; ++d) sdl[d * MAXROWS + i] = dl[d];
      for (int k = 0; k < K; ++k) sb[(int64_t)k * MAXROWS + i] = b[k];
      moving |= src != 0;
    }
    // F (Sec. 2.2.1): grid face p_d m_f^{p-e_d}; EB face sum_d p_d m_{d,f}^{p-e_d}
    int32_t cf_self = -1;
    if (cut_self < 0) cf_self = a.cutface_of[dface][flocal];
    moving |= cut_self >= 0 || cf_self >= 0;
    for (int i = lane; i < K; i += 32) {
      double f = 0.0;
      if (cut_self >= 0) {
        for (int d = 0; d < dm.dim; ++d) {
          const int lo = T.lower[d][i];
          if (lo >= 0) f += (double)T.mon[i][d] * a.eb_nmom[((int64_t)cut_self * dm.dim + d) * dm.KS + lo];
        }
      } else {
        const int q = T.lower[dface][i];
        if (q >= 0) {
          if (cf_self >= 0) {
            if (T.tang[dface][q] >= 0)
              f = (double)T.mon[i][dface] * a.face_mom[dface][(int64_t)cf_self * dm.KFS + T.tang[dface][q]];
          } else {
            f = (double)T.mon[i][dface] * T.full_face[dface][q];
          }
        }
      }
      F[i] = f;
    }
    if (!__any_sync(0xffffffffu, moving)) continue;  // this system does not move with the geometry
    __syncwarp();
    // G = B^T B (upper triangle, lanes over entries), then its Cholesky factor in place
    for (int e = lane; e < E; e += 32) {
      int j = 0, rem = e;
      while (rem >= K - j) {
        rem -= K - j;
        ++j;
      }
      const int k = j + rem;
      double acc = 0.0;
      for (int i = 0; i < n; ++i) acc = fma(sb[(int64_t)j * MAXROWS + i], sb[(int64_t)k * MAXROWS + i], acc);
      G[j * K + k] = acc;
    }
    __syncwarp();
    bool ok = true;
    for (int k = 0; k < K; ++k) {
      const double piv = G[k * K + k];
      if (!(piv > 0.0)) {
        ok = false;
        break;
      }
      const double rk = sqrt(piv), ik = 1.0 / rk;
      __syncwarp();
      if (lane == 0) {
        G[k * K + k] = rk;
        rinv[k] = ik;
      }
      for (int j = k + 1 + lane; j < K; j += 32) G[k * K + j] *= ik;
      __syncwarp();
      for (int j = k + 1 + lane; j < K; j += 32) {
        const double rkj = G[k * K + j];
        for (int i = k + 1; i <= j; ++i) G[i * K + j] = fma(-G[k * K + i], rkj, G[i * K + j]);
      }
      __syncwarp();
    }
    if (!ok) {
      if (lane == 0) atomicExch(a.err, 1);  // a system the forward build solved cannot be singular here
      continue;
    }
    // y = G^-1 F and z = G^-1 B^T tbar, by one lane each (K <= 35: serial triangular solves)
    double lam_face = 0.0;  // sum over the face's volumes of sigma lam
    if (cut_self >= 0) {
      lam_face = g.lam[a.cut_cell[cut_self]];
    } else {
      int lo[3] = {base[0], base[1], base[2]};
      lo[dface] -= 1;
      if (lo[dface] >= 0) {
        const int64_t cl = cell_id(dm, lo);
        if (a.flag[cl]) lam_face += g.lam[cl];
      }
      if (base[dface] < dm.n[dface]) {
        const int64_t ch = cell_id(dm, base);
        if (a.flag[ch]) lam_face -= g.lam[ch];
      }
    }
    const double ih2 = 1.0 / (dm.h * dm.h);
    for (int i = lane; i < n; i += 32) {
      const int64_t col = scol[i];
      stb[i] = col >= 0 ? sw[i] * (-lam_face * g.phi[col] * ih2) : 0.0;
    }
    __syncwarp();
    for (int k = lane; k < K; k += 32) {  // u = B^T tbar, tbar_i = w_i sbar_i
      double acc = 0.0;
      for (int i = 0; i < n; ++i) acc = fma(sb[(int64_t)k * MAXROWS + i], stb[i], acc);
      u[k] = acc;
    }
    __syncwarp();
    if (lane == 0) {
      for (int pass = 0; pass < 2; ++pass) {
        double* v = pass ? z : y;
        const double* rhs = pass ? u : F;
        for (int k = 0; k < K; ++k) {  // R^T w = rhs
          double acc = rhs[k];
          for (int j = 0; j < k; ++j) acc = fma(-G[j * K + k], v[j], acc);
          v[k] = acc * rinv[k];
        }
        for (int k = K - 1; k >= 0; --k) {  // R v = w
          double acc = v[k];
          for (int j = k + 1; j < K; ++j) acc = fma(-G[k * K + j], v[j], acc);
          v[k] = acc * rinv[k];
        }
      }
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
      double by = 0.0, bz = 0.0;
      for (int k = 0; k < K; ++k) {
        const double bk = sb[(int64_t)k * MAXROWS + i];
        by = fma(bk, y[k], by);
        bz = fma(bk, z[k], bz);
      }
      sby[i] = by;
      sbz[i] = bz;
    }
    __syncwarp();
    for (int p = 0; p < g.n_par; ++p) {
      double dj = 0.0;
      for (int i = lane; i < n; i += 32) {
        if (ssrc[i] == 0) continue;
        double dl[3], db[MAXK];
        for (int d = 0; d < 3; ++d) dl[d] = sdl[d * MAXROWS + i];
        row_dtangent(a, T, g, p, ssrc[i], dl, ssc[i], sw[i], sb + i, db);
        double ydb = 0.0, zdb = 0.0;
        for (int k = 0; k < K; ++k) {
          ydb = fma(y[k], db[k], ydb);
          zdb = fma(z[k], db[k], zdb);
        }
        dj += (stb[i] - sbz[i]) * ydb - sby[i] * zdb;
      }
      // + z . dF
      for (int i = lane; i < K; i += 32) {
        double df = 0.0;
        if (cut_self >= 0) {
          for (int d = 0; d < dm.dim; ++d) {
            const int lo = T.lower[d][i];
            if (lo >= 0)
              df += (double)T.mon[i][d] * g.debn[p * g.s_ebn + ((int64_t)cut_self * dm.dim + d) * dm.KS + lo];
          }
        } else if (cf_self >= 0) {
          const int q = T.lower[dface][i];
          if (q >= 0 && T.tang[dface][q] >= 0)
            df = (double)T.mon[i][dface] *
                 g.dface[dface][p * g.s_face[dface] + (int64_t)cf_self * dm.KFS + T.tang[dface][q]];
        }
        dj = fma(z[i], df, dj);
      }
      dj = warp_sum(dj);
      if (lane == 0 && dj != 0.0) atomicAdd(g.dJ + p, dj);
    }
    __syncwarp();
  }
}

cudaError_t stencil_adjoint_launch(unsigned blocks, cudaStream_t s, const LsArgs& a, const Tables& T,
                                   const AdjArgs& g) {
  k_stencil_adjoint<<<blocks, ADJ_WARPS * 32, 0, s>>>(a, T, g);
  return cudaGetLastError();
}

cudaError_t lsq_launch(bool fp32, unsigned blocks, cudaStream_t s, const LsArgs& a0, const Tables& T,
                       const LsArgs* batch, const int64_t* slot_base, int n_geom) {
  const size_t smem = lsq_smem(fp32);
  if (fp32) {
    constexpr unsigned nt = LS_SYS_F * LS_NW * 32;
    if (batch) k_lsq<true, float><<<blocks, nt, smem, s>>>(a0, T, batch, slot_base, n_geom);
    else k_lsq<false, float><<<blocks, nt, smem, s>>>(a0, T, nullptr, nullptr, 1);
  } else {
    constexpr unsigned nt = LS_SYS * LS_NW * 32;
    if (batch) k_lsq<true, double><<<blocks, nt, smem, s>>>(a0, T, batch, slot_base, n_geom);
    else k_lsq<false, double><<<blocks, nt, smem, s>>>(a0, T, nullptr, nullptr, 1);
  }
  return cudaGetLastError();
}

// the systems with status 3 (global numbers: + base) appended to list[*count]
__global__ void k_ls_fallback(const int32_t* __restrict__ status, int64_t n, int64_t base, int32_t* list,
                              int32_t* count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && status[i] == 3) list[atomicAdd(count, 1)] = (int32_t)(base + i);
}

cudaError_t lsq_fallback_list(const int32_t* status, int64_t n, int64_t base, int32_t* list, int32_t* count,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_ls_fallback<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(status, n, base, list, count);
  return cudaGetLastError();
}

}  // namespace eb
