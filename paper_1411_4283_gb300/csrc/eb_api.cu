// C ABI of the library (include/eb.h): host orchestration of the build,
// apply and solve phases.  Every arithmetic step of the method runs in the
// kernels of eb_build.cu, eb_apply.cu and eb_solve.cu; this file validates
// arguments, allocates library-owned device memory and launches them.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "eb_apply.cuh"
#include "eb_apply_quad.cuh"
#include "eb_apply_brick.cuh"
#include "eb_internal.cuh"
#include "eb_scan.cuh"
#include "eb_solve.cuh"
#include "eb_tables.cuh"
#include "eb_build.cuh"

namespace eb {


// ------------------------------------------------------------------ errors

static thread_local std::string g_err;
static thread_local std::vector<int64_t> g_bad_faces;

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launches(long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(); }
void set_error(const std::string& msg) { g_err = msg; }
eb_status cuda_status(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? EB_ERR_OOM : EB_ERR_CUDA;
}

std::vector<std::vector<int>> monomials(int dim, int q) {
  std::vector<std::vector<int>> out;
  for (int deg = 0; deg <= q; ++deg) {
    if (dim == 1) { out.push_back({deg}); continue; }
    if (dim == 2) {
      for (int p0 = deg; p0 >= 0; --p0) out.push_back({p0, deg - p0});
      continue;
    }
    for (int p0 = deg; p0 >= 0; --p0)
      for (int p1 = deg - p0; p1 >= 0; --p1) out.push_back({p0, p1, deg - p0 - p1});
  }
  return out;
}

static double full1d(int q) { return (q & 1) ? 0.0 : pow(0.5, q) / (q + 1); }

bool make_tables(int dim, int order, int mdeg, Tables* t) {
  memset(t, 0, sizeof(*t));
  auto mon = monomials(dim, order);
  t->dim = dim;
  t->K = (int)mon.size();
  t->KS = (int)monomials(dim, mdeg).size();
  t->KFS = dim > 1 ? (int)monomials(dim - 1, mdeg).size() : 1;
  if (t->K > MAXK) return false;
  std::map<std::vector<int>, int> idx;
  for (int i = 0; i < t->K; ++i) {
    idx[mon[i]] = i;
    for (int d = 0; d < 3; ++d) t->mon[i][d] = d < dim ? (int8_t)mon[i][d] : 0;
  }
  for (int d = 0; d < dim; ++d) {
    // lines of the shift along d: start from each monomial with exponent 0 along d
    int nl = 0;
    for (int i = 0; i < t->K; ++i) {
      if (mon[i][d] != 0) continue;
      int len = 0;
      std::vector<int> q = mon[i];
      while (true) {
        auto it = idx.find(q);
        if (it == idx.end()) break;
        if (len >= MAXLN) return false;
        t->ln_idx[d][nl][len++] = (uint8_t)it->second;
        q[d] += 1;
      }
      t->ln_len[d][nl++] = (uint8_t)len;
    }
    t->nln[d] = nl;
    for (int i = 0; i < t->K; ++i) {
      if (mon[i][d] == 0) { t->lower[d][i] = -1; continue; }
      std::vector<int> q = mon[i];
      q[d] -= 1;
      t->lower[d][i] = (int8_t)idx[q];
    }
    // tangential monomials of faces normal to d
    std::vector<std::vector<int>> fm = dim > 1 ? monomials(dim - 1, mdeg) : std::vector<std::vector<int>>{{}};
    std::map<std::vector<int>, int> fidx;
    for (size_t i = 0; i < fm.size(); ++i) fidx[fm[i]] = (int)i;
    for (int i = 0; i < t->K; ++i) {
      if (mon[i][d] != 0) { t->tang[d][i] = -1; t->full_face[d][i] = 0.0; continue; }
      std::vector<int> pt;
      double ff = 1.0;
      for (int k = 0; k < dim; ++k)
        if (k != d) { pt.push_back(mon[i][k]); ff *= full1d(mon[i][k]); }
      t->tang[d][i] = dim > 1 ? (int16_t)fidx[pt] : 0;
      t->full_face[d][i] = ff;
    }
  }
  for (int i = 0; i < t->K; ++i) {
    double f = 1.0;
    for (int d = 0; d < dim; ++d) f *= full1d(mon[i][d]);
    t->full_vol[i] = f;
  }
  return true;
}

static unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Device memory of builds and solves comes from a library-owned stream-ordered pool per device that
// keeps freed memory cached (no release threshold), so that the dozens of allocations of a build and
// the temporaries of every solve cost neither a driver allocation nor a device-wide synchronisation.
static cudaMemPool_t eb_pool() {
  static std::mutex m;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(m);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    (void)cudaGetLastError();
    pools[dev] = nullptr;
    return nullptr;
  }
  uint64_t thr = UINT64_MAX;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  // memory freed in one stream is reused by another only once the free has completed (or an event
  // orders the two): never by making the allocating stream wait, which would serialise the streams of
  // a batch's worker threads
  int no = 0;
  cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  pools[dev] = pool;
  return pool;
}

static cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = eb_pool();
  if (pool) return cudaMallocFromPoolAsync(p, bytes, pool, s);
  return cudaMalloc(p, bytes);
}

// Bump allocation from chunks of pooled memory that grow geometrically (1 MB, 2 MB, ... 64 MB): a
// build makes dozens of small arrays, and one pool allocation costs tens of microseconds of host time
// when several threads allocate at once.  Arrays of 4 MB or more get their own allocation.  Blocks
// are 256-byte aligned; the chunks and large arrays are recorded in `owned` for their release.
static cudaError_t arena_alloc(Arena& a, void** p, size_t bytes, cudaStream_t s, std::vector<void*>& owned) {
  constexpr size_t LARGE = (size_t)4 << 20, MAX_CHUNK = (size_t)64 << 20;
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes >= LARGE) {
    cudaError_t e = pool_alloc(p, bytes, s);
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
  }
  if (bytes > a.left) {
    void* c = nullptr;
    const size_t sz = std::max(a.next, bytes);  // the chunk holds at least this request
    cudaError_t e = pool_alloc(&c, sz, s);
    if (e != cudaSuccess) return e;
    owned.push_back(c);
    a.cur = (char*)c;
    a.left = sz;
    if (a.next < MAX_CHUNK) a.next *= 2;
  }
  if (bytes > a.left) return cudaErrorMemoryAllocation;  // unreachable: the chunk was sized for it
  *p = a.cur;
  a.cur += bytes;
  a.left -= bytes;
  return cudaSuccess;
}

template <typename T>
static eb_status dalloc(eb_stencils* st, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = arena_alloc(st->arena, (void**)p, count * sizeof(T), st->build_stream, st->allocs);
  if (e != cudaSuccess) return cuda_status(e, "device allocation");
  return EB_OK;
}

// temporary allocations, freed in stream order at scope exit
struct Tmp {
  cudaStream_t s = nullptr;
  Arena arena;
  std::vector<void*> ptrs;
  ~Tmp() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  eb_status get(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = arena_alloc(arena, (void**)p, count * sizeof(T), s, ptrs);
    if (e != cudaSuccess) return cuda_status(e, "device allocation");
    return EB_OK;
  }
};

#define EB_TRY(x)                  \
  do {                             \
    eb_status _s = (x);            \
    if (_s != EB_OK) return _s;    \
  } while (0)

// exclusive scan of in[0..n) into out[0..n); returns the total
template <typename T>
static eb_status scan(const T* in, int64_t n, int64_t* out, int64_t* total, cudaStream_t s, Tmp& tmp) {
  int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  if (nb == 0) { *total = 0; return EB_OK; }
  int64_t* sums;
  int64_t* dtot;
  EB_TRY(tmp.get(&sums, nb));
  EB_TRY(tmp.get(&dtot, 1));
  k_scan_block_sums<T><<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, n, sums); eb::count_launch();
  k_scan_single<<<1, SCAN_BLOCK, 0, s>>>(sums, nb, dtot); eb::count_launch();
  k_scan_apply<T><<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, n, sums, out); eb::count_launch();
  EB_CUDA(cudaGetLastError());
  EB_CUDA(cudaMemcpyAsync(total, dtot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  return EB_OK;
}

// ------------------------------------------------------------------ small kernels

__global__ void k_scatter_index(const int32_t* idx, int64_t n, int32_t* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[idx[i]] = (int32_t)i;
}

__global__ void k_kappa(int64_t ncell, const uint8_t* flag, const int32_t* cut_of, const double* vol_mom, int KS,
                        double* kappa, double* invk) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  double k = flag[c] == 0 ? 0.0 : (flag[c] == 1 ? 1.0 : vol_mom[(int64_t)cut_of[c] * KS]);
  kappa[c] = k;
  invk[c] = k > 0 ? 1.0 / k : 0.0;
}

__global__ void k_flag_list(const uint8_t* dil, const uint8_t* flag, int64_t ncell, int32_t* sel) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell) sel[c] = (dil[c] & 1) && flag[c] > 0;
}

__global__ void k_compact(const int32_t* sel, const int64_t* pos, int64_t n, int32_t* out, int32_t* map) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  if (sel[c]) {
    out[pos[c]] = (int32_t)c;
    if (map) map[c] = (int32_t)pos[c];
  } else if (map) map[c] = -1;
}

__global__ void k_eb_slots(int64_t n_cut, int64_t base, int64_t n_grid, int64_t* slot_face, int32_t* eb_slot) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cut) return;
  slot_face[base + i] = n_grid + i;
  eb_slot[i] = (int32_t)(base + i);
}

// cell kind and row key: 0 covered, 1 template, 2 irregular.  rowkey: -2 unique, >= 0 class key
__global__ void k_cell_kind(Dims dm, const uint8_t* flag, const int32_t* fs0, const int32_t* fs1, const int32_t* fs2,
                            int64_t n_unique_slots, const int32_t* tmpl_slot, uint8_t* kind, int32_t* rowkey,
                            int64_t* row_rep, int32_t* is_unique) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= dm.ncell) return;
  is_unique[c] = 0;
  if (flag[c] == 0) { kind[c] = 0; rowkey[c] = -1; return; }
  int x[3];
  x[0] = (int)(c % dm.n[0]);
  int64_t r = c / dm.n[0];
  x[1] = (int)(r % dm.n[1]);
  x[2] = (int)(r / dm.n[1]);
  const int32_t* fs[3] = {fs0, fs1, fs2};
  bool uniq = flag[c] == 2, tmpl = flag[c] == 1;
  for (int d = 0; d < dm.dim; ++d)
    for (int side = 0; side < 2; ++side) {
      int fx[3] = {x[0], x[1], x[2]};
      if (side) fx[d] += 1;
      int64_t m0 = dm.n[0] + (d == 0), m1 = dm.n[1] + (d == 1);
      int64_t fl = (int64_t)fx[0] + m0 * ((int64_t)fx[1] + m1 * fx[2]);
      int32_t sl = fs[d][fl];
      if (sl < 0) { tmpl = false; continue; }
      if (sl < n_unique_slots) uniq = true;
      if (sl != tmpl_slot[d]) tmpl = false;
    }
  if (uniq) { kind[c] = 2; rowkey[c] = -2; is_unique[c] = 1; return; }
  if (tmpl) { kind[c] = 1; rowkey[c] = 0; atomicMin((unsigned long long*)&row_rep[0], (unsigned long long)c); return; }
  kind[c] = 2;
  int M = dm.R + 3, key = 0;
  for (int k = dm.dim - 1; k >= 0; --k) {
    int lo = x[k] < M - 1 ? x[k] : M - 1;
    int hi = dm.n[k] - 1 - x[k];
    hi = hi < M - 1 ? hi : M - 1;
    key = (key * M + lo) * M + hi;
  }
  key += 1;  // 0 is the template
  rowkey[c] = key;
  atomicMin((unsigned long long*)&row_rep[key], (unsigned long long)c);
}

__global__ void k_irr_list(int64_t ncell, const uint8_t* kind, const int64_t* pos, const int32_t* rowkey,
                           const int32_t* key_row, const int64_t* upos, int64_t ubase, int32_t* irr_cell,
                           int32_t* irr_row, int32_t* rep_of_row) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell || kind[c] != 2) return;
  int64_t p = pos[c];
  irr_cell[p] = (int32_t)c;
  int32_t row;
  if (rowkey[c] == -2) {
    row = (int32_t)(ubase + upos[c]);
    rep_of_row[row] = (int32_t)c;
  } else row = key_row[rowkey[c]];
  irr_row[p] = row;
}

__global__ void k_is_kind2(int64_t n, const uint8_t* kind, int32_t* sel) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) sel[c] = kind[c] == 2;
}

__global__ void k_wall_pos(int64_t nnz, const int64_t* bcol, int64_t n_grid, const int64_t* walls, int64_t nwall,
                           int64_t* pos) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  int64_t c = bcol[k];
  if (c >= n_grid) { pos[k] = -1; return; }
  int64_t lo = 0, hi = nwall - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (walls[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  pos[k] = lo;
}

// irregular list -> cells with a unique row (by unique row) and cells with a class row (ascending)
__global__ void k_flag_class(int64_t n_irr, const int32_t* irr_row, int64_t n_class, int32_t* flag) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_irr) flag[t] = irr_row[t] < n_class;
}

__global__ void k_split_irr(int64_t n_irr, const int32_t* irr_cell, const int32_t* irr_row, int64_t n_class,
                            const int64_t* posC, int32_t* cellU, int32_t* cellC, int32_t* classC) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_irr) return;
  const int32_t r = irr_row[t];
  if (r >= n_class) {
    cellU[r - n_class] = irr_cell[t];
  } else {
    cellC[posC[t]] = irr_cell[t];
    classC[posC[t]] = r;
  }
}

// canonical footprint-major unique rows -> quad layout (see eb_apply_quad.cuh); perm[e]: canonical
// footprint index of apply-order entry e (-1: padding)
template <typename T>
__global__ void k_pack_quads(const T* __restrict__ rows, int64_t n_rows, const int16_t* __restrict__ perm, int nq,
                             int64_t n_class, T* __restrict__ qU) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + n_class;
  const int e = blockIdx.y;
  if (r >= n_rows) return;
  const int f = perm[e];
  const T v = f >= 0 ? rows[(int64_t)f * n_rows + r] : (T)0;
  const int64_t u = r - n_class;
  qU[(((u >> 5) * nq + (e >> 2)) * 32 + (u & 31)) * 4 + (e & 3)] = v;
}

// start of an aligned x-run of four class cells of one class: x a multiple of 4 (nx is), and the
// loaded window x-4 .. x+7 inside the grid row
__global__ void k_run_mark(int64_t nC, const int32_t* cellC, const int32_t* classC, int nx, int32_t* gs) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nC) return;
  const int32_t c = cellC[t];
  const int x = c % nx;
  bool ok = (nx & 3) == 0 && (x & 3) == 0 && x >= 4 && x + 8 <= nx && t + 3 < nC && cellC[t + 3] == c + 3;
  if (ok) ok = classC[t + 1] == classC[t] && classC[t + 2] == classC[t] && classC[t + 3] == classC[t];
  gs[t] = ok;
}

__global__ void k_run_rest(int64_t nC, const int32_t* gs, int32_t* rest) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nC) return;
  bool in = gs[t] || (t >= 1 && gs[t - 1]) || (t >= 2 && gs[t - 2]) || (t >= 3 && gs[t - 3]);
  rest[t] = !in;
}

__global__ void k_run_split(int64_t nC, const int32_t* cellC, const int32_t* classC, const int32_t* gs,
                            const int32_t* rest, const int64_t* gpos, const int64_t* lpos, int32_t* cellG,
                            int32_t* classG, int32_t* cellL, int32_t* classL) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nC) return;
  if (gs[t]) {
    cellG[gpos[t]] = cellC[t];
    classG[gpos[t]] = classC[t];
  }
  if (rest[t]) {
    cellL[lpos[t]] = cellC[t];
    classL[lpos[t]] = classC[t];
  }
}

// class cells outside the runs: those in the x slabs (x < BR_W or x >= nx - BR_W) go to the slab map of the
// brick pass, the others stay in the per-cell list (keep = 1)
__global__ void k_slab_scatter(int64_t nL, const int32_t* cellL, const int32_t* classL, int nx, int ny, int nz,
                               int32_t* slab, int32_t* keep) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nL) return;
  const int32_t c = cellL[t];
  const int x = c % nx, y = (c / nx) % ny, z = c / nx / ny;
  int side, xl;
  if (x < BR_W) { side = 0; xl = x; }
  else if (x >= nx - BR_W) { side = 1; xl = x - (nx - BR_W); }
  else { keep[t] = 1; return; }
  keep[t] = 0;
  slab[((int64_t)(side * BR_W + xl) * nz + z) * ny + y] = classL[t];
}

// the unit of a slab cell (side, x layer, z block, y block), or -1 outside the units
__device__ __forceinline__ int64_t brick_unit(int side, int xl, int y, int z, int nyb, int nzb, int y_org, int z_org,
                                              int y_hi, int z_hi) {
  if (y < y_org || y >= y_hi || z < z_org || z >= z_hi) return -1;
  return (((int64_t)side * BR_W + xl) * nzb + (z - z_org) / BR_BZ) * nyb + (y - y_org) / 32;
}

}  // namespace eb

__global__ void eb::k_brick_units(const int32_t* __restrict__ slab, int ny, int nz, int nyb, int nzb, int y_org,
                                  int z_org, int y_hi, int z_hi, int32_t* __restrict__ unit_class) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= (int64_t)2 * BR_W * nzb * nyb) return;
  const int yblk = (int)(u % nyb), zblk = (int)((u / nyb) % nzb), sx = (int)(u / ((int64_t)nyb * nzb));
  const int y0 = y_org + 32 * yblk, z0 = z_org + BR_BZ * zblk;
  const int y1 = min(y0 + 32, y_hi), z1 = min(z0 + BR_BZ, z_hi);
  int cls = -2;
  for (int z = z0; z < z1 && cls != -1; ++z)
    for (int y = y0; y < y1; ++y) {
      const int v = slab[((int64_t)sx * nz + z) * ny + y];
      if (v < 0 || (cls != -2 && v != cls)) { cls = -1; break; }
      cls = v;
    }
  unit_class[u] = cls < 0 ? -1 : cls;
}

namespace eb {

// class cells of the slab list that a uniform brick unit covers leave the per-cell list (keep = 0)
__global__ void k_brick_keep(int64_t nL, const int32_t* cellL, int nx, int ny, int nz, int nyb, int nzb, int y_org,
                             int z_org, int y_hi, int z_hi, const int32_t* unit_class, int32_t* keep) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nL) return;
  const int32_t c = cellL[t];
  const int x = c % nx, y = (c / nx) % ny, z = c / nx / ny;
  int side, xl;
  if (x < BR_W) { side = 0; xl = x; }
  else if (x >= nx - BR_W) { side = 1; xl = x - (nx - BR_W); }
  else { keep[t] = 1; return; }
  const int64_t u = brick_unit(side, xl, y, z, nyb, nzb, y_org, z_org, y_hi, z_hi);
  keep[t] = (u < 0 || unit_class[u] < 0) ? 1 : 0;
}

__global__ void k_compact_pair(int64_t n, const int32_t* keep, const int64_t* pos, const int32_t* a,
                               const int32_t* b, int32_t* a2, int32_t* b2) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n || !keep[t]) return;
  a2[pos[t]] = a[t];
  b2[pos[t]] = b[t];
}

// class rows, class-major: out[k * nfoot + i] = rows[i][k]
template <typename T>
__global__ void k_class_major(const T* __restrict__ rows, int64_t n_rows, int64_t n_class, int nfoot,
                              T* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_class * nfoot) return;
  const int64_t k = t / nfoot, i = t % nfoot;
  out[t] = rows[i * n_rows + k];
}

__global__ void k_diag_inv(int64_t ncell, const uint8_t* kind, const int32_t* irr_map_unused, const double* tmpl,
                           int center, double* dinv64, float* dinv32) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  double d = kind[c] == 1 ? tmpl[center] : 0.0;
  double v = d != 0.0 ? 1.0 / d : 0.0;
  dinv64[c] = v;
  dinv32[c] = (float)v;
}

__global__ void k_diag_irr(int64_t n_irr, const int32_t* irr_cell, const int32_t* irr_row, const double* rows64,
                           int64_t n_rows, int center, double* dinv64, float* dinv32) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_irr) return;
  double d = rows64[(int64_t)center * n_rows + irr_row[t]];
  double v = d != 0.0 ? 1.0 / d : 0.0;
  dinv64[irr_cell[t]] = v;
  dinv32[irr_cell[t]] = (float)v;
}

__global__ void k_gather_flags(const uint8_t* ff, const int64_t* ids, int64_t n, uint8_t* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = ff[ids[i]];
}

__global__ void k_zero_f64(int64_t n, double* x) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = 0.0;
}

}  // namespace eb

using namespace eb;

// ====================================================================== ABI

extern "C" {

const char* eb_status_string(eb_status s) {
  switch (s) {
    case EB_OK: return "ok";
    case EB_ERR_INVALID: return "invalid argument";
    case EB_ERR_RANK_DEFICIENT: return "rank-deficient least-squares system";
    case EB_ERR_MULTIVALUED: return "multi-valued cell";
    case EB_ERR_NOT_CONVERGED: return "not converged";
    case EB_ERR_TIMEOUT: return "timeout";
    case EB_ERR_CUDA: return "CUDA error";
    case EB_ERR_OOM: return "out of device memory";
    case EB_ERR_CAPACITY: return "LS system larger than supported";
  }
  return "unknown";
}

const char* eb_last_error_message(void) { return g_err.c_str(); }
int32_t eb_abi_version(void) { return 3; }
int64_t eb_kernel_launches(void) { return (int64_t)g_launches.load(); }

void eb_stencils_destroy(eb_stencils* st) {
  if (!st) return;
  if (st->plan) {
    if (st->plan->side) {
      cudaStreamSynchronize(st->plan->side);
      cudaStreamDestroy(st->plan->side);
    }
    if (st->plan->fork) cudaEventDestroy(st->plan->fork);
    if (st->plan->join) cudaEventDestroy(st->plan->join);
    delete st->plan;
  }
  if (st->mg) {
    mg_free(st->mg);
    delete st->mg;
  }
  // pooled memory is freed without an implicit synchronisation: wait for work still using it
  cudaDeviceSynchronize();
  for (void* p : st->allocs) cudaFree(p);
  delete st;
}

eb_status eb_last_error_faces(int64_t* ids_host, int32_t cap, int32_t* n) {
  if (!n) return EB_ERR_INVALID;
  *n = (int32_t)g_bad_faces.size();
  for (int32_t i = 0; i < cap && i < *n && ids_host; ++i) ids_host[i] = g_bad_faces[i];
  return EB_OK;
}

// State of one build between its phases: before the least-squares launch (classification, gather,
// LS inputs), the launch itself (one geometry, or several sharing one launch), and after it
// (status check, operator rows, boundary matrix, apply plan, info).
struct BuildCtx {
  const eb_geom* g = nullptr;
  const eb_params* prm = nullptr;
  eb_stencils* st = nullptr;
  eb_build_info* info = nullptr;
  cudaStream_t s = nullptr;
  eb_params P;
  int R = 0, D = 0, nsm = 0;
  int64_t N = 0, n_slots = 0, n_unique = 0;
  Tables T;
  Tables* dT = nullptr;
  Tmp tmp;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int n_ev = 0;
  int32_t tmpl_slot_h[3] = {-1, -1, -1};
  double* invk = nullptr;
  LsArgs la;            // least-squares inputs (scratch, work counter and error word set per launch)
  int32_t* status = nullptr;
  double ls_flops[2] = {0.0, 0.0};  // executed FP64 and FP32 flops of the LS launches
  eb_status rc = EB_OK;  // a phase's failure in a batch worker thread, with its message and faces
  std::string err;
  std::vector<int64_t> bad;
  ~BuildCtx() {
    for (int i = 0; i < n_ev; ++i) cudaEventDestroy(ev[i]);
  }
};

static eb_status build_pre(BuildCtx& c);
static eb_status build_ls(BuildCtx* const* cs, int n, cudaStream_t s);
static eb_status build_post(BuildCtx& c);

eb_status eb_build_stencils(const eb_geom* geom, const eb_params* params, eb_stencils** out, eb_build_info* info,
                            eb_stream_t stream) {
  if (!out) { set_error("out is NULL"); return EB_ERR_INVALID; }
  *out = nullptr;
  g_bad_faces.clear();
  eb_stencils* st = new eb_stencils();
  eb_build_info local;
  memset(&local, 0, sizeof(local));
  eb_status r;
  {
    BuildCtx c;
    c.g = geom;
    c.prm = params;
    c.st = st;
    c.info = info ? info : &local;
    c.s = (cudaStream_t)stream;
    BuildCtx* cp = &c;
    r = build_pre(c);
    if (r == EB_OK) r = build_ls(&cp, 1, c.s);
    if (r == EB_OK) r = build_post(c);
  }
  if (r != EB_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    eb_stencils_destroy(st);
    return r;
  }
  *out = st;
  return EB_OK;
}

// The per-geometry phases of a batch run on several host threads, each with its own stream, so that
// their launches, small host reads and allocations overlap; the least-squares launch of all the
// geometries runs on the caller's stream between the two phases.
static constexpr int BATCH_MAX_THREADS = 8;

eb_status eb_build_stencils_batch(const eb_geom* geoms, int32_t n_geom, const eb_params* params, eb_stencils** out,
                                  eb_build_info* infos, eb_stream_t stream) {
  if (!out || !geoms || n_geom < 1) { set_error("bad batch arguments"); return EB_ERR_INVALID; }
  for (int32_t i = 0; i < n_geom; ++i) out[i] = nullptr;
  g_bad_faces.clear();
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  EB_CUDA(cudaGetDevice(&dev));
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nthr = (int)std::min<int64_t>(n_geom, std::min<unsigned>(BATCH_MAX_THREADS, hw));
  std::vector<cudaStream_t> ws(nthr, nullptr);
  std::vector<cudaEvent_t> wev(nthr, nullptr);
  cudaEvent_t sev = nullptr;
  std::vector<BuildCtx*> cs(n_geom, nullptr);
  std::vector<eb_build_info> local(n_geom);
  eb_status r = EB_OK;
  auto cleanup = [&](eb_status rr) {
    if (rr != EB_OK) cudaStreamSynchronize(s);
    for (int t = 0; t < nthr; ++t)
      if (ws[t]) cudaStreamSynchronize(ws[t]);
    for (int32_t i = 0; i < n_geom; ++i) {
      if (!cs[i]) continue;
      if (rr == EB_OK) out[i] = cs[i]->st;
      else eb_stencils_destroy(cs[i]->st);
      delete cs[i];  // returns its temporaries in its worker stream's order
    }
    for (int t = 0; t < nthr; ++t) {
      if (wev[t]) cudaEventDestroy(wev[t]);
      if (ws[t]) cudaStreamDestroy(ws[t]);
    }
    if (sev) cudaEventDestroy(sev);
    return rr;
  };
  for (int t = 0; t < nthr; ++t) {
    cudaError_t e = cudaStreamCreateWithFlags(&ws[t], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&wev[t], cudaEventDisableTiming);
    if (e != cudaSuccess) return cleanup(cuda_status(e, "batch worker streams"));
  }
  {
    cudaError_t e = cudaEventCreateWithFlags(&sev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cleanup(cuda_status(e, "batch events"));
  }
  for (int32_t i = 0; i < n_geom; ++i) {
    cs[i] = new BuildCtx();
    BuildCtx& c = *cs[i];
    c.g = &geoms[i];
    c.prm = params;
    c.st = new eb_stencils();
    memset(&local[i], 0, sizeof(eb_build_info));
    c.info = infos ? &infos[i] : &local[i];
    c.s = ws[i % nthr];
  }
  // worker streams start after the caller's stream (the geometry may come from it) and after the
  // least-squares launch; the caller's stream waits for the workers before that launch and at the end
  auto fork = [&]() -> cudaError_t {
    cudaError_t e = cudaEventRecord(sev, s);
    for (int t = 0; t < nthr && e == cudaSuccess; ++t) e = cudaStreamWaitEvent(ws[t], sev, 0);
    return e;
  };
  auto join = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < nthr && e == cudaSuccess; ++t) {
      e = cudaEventRecord(wev[t], ws[t]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, wev[t], 0);
    }
    return e;
  };
  auto phase = [&](bool post) -> eb_status {
    std::atomic<bool> failed(false);
    auto work = [&](int t) {
      if (cudaSetDevice(dev) != cudaSuccess) {
        failed = true;
        return;
      }
      for (int32_t i = t; i < n_geom && !failed; i += nthr) {
        BuildCtx& c = *cs[i];
        g_err.clear();
        g_bad_faces.clear();
        const eb_status ri = post ? build_post(c) : build_pre(c);
        if (ri != EB_OK) {
          c.rc = ri;
          c.err = g_err;
          c.bad = g_bad_faces;
          failed = true;
        }
      }
    };
    std::vector<std::thread> th;
    std::vector<int> inline_t;  // workers whose thread could not be started run on this thread
    for (int t = 1; t < nthr; ++t) {
      try {
        th.emplace_back(work, t);
      } catch (...) {
        inline_t.push_back(t);
      }
    }
    work(0);
    for (int t : inline_t) work(t);
    for (auto& x : th) x.join();
    for (int32_t i = 0; i < n_geom; ++i)
      if (cs[i]->rc != EB_OK) {
        set_error(cs[i]->err);
        g_bad_faces = cs[i]->bad;
        return cs[i]->rc;
      }
    if (failed) {
      set_error("a batch worker thread could not select the device");
      return EB_ERR_CUDA;
    }
    return EB_OK;
  };
  cudaError_t e = fork();
  if (e != cudaSuccess) return cleanup(cuda_status(e, "batch fork"));
  r = phase(false);
  if (r != EB_OK) return cleanup(r);
  if ((e = join()) != cudaSuccess) return cleanup(cuda_status(e, "batch join"));
  r = build_ls(cs.data(), n_geom, s);
  if (r != EB_OK) return cleanup(r);
  if ((e = fork()) != cudaSuccess) return cleanup(cuda_status(e, "batch fork"));
  r = phase(true);
  if (r != EB_OK) return cleanup(r);
  if ((e = join()) != cudaSuccess) return cleanup(cuda_status(e, "batch join"));
  return cleanup(EB_OK);
}

// apply order of the footprint for the quad layout (eb_apply_quad.cuh): groups of four wide segments,
// groups of four narrow segments, the left-over wide segment, zero padding to a whole quad
static std::vector<int16_t> quad_perm(int R, int box) {
  const int L = R + 1, S = 2 * L + 1, W = 2 * R + 1;
  std::vector<int16_t> lut(S * S * S, -1);
  int n = 0;
  for (int z = -L; z <= L; ++z)
    for (int y = -L; y <= L; ++y)
      for (int x = -L; x <= L; ++x)
        if (in_footprint(x, y, z, R, box)) lut[(x + L) + S * ((y + L) + S * (z + L))] = (int16_t)n++;
  std::vector<int16_t> perm;
  auto seg = [&](int dy, int dz, int X) {
    for (int dx = -X; dx <= X; ++dx) perm.push_back(lut[(dx + L) + S * ((dy + L) + S * (dz + L))]);
  };
  const int GW = W * W / 4;
  for (int w = 0; w < 4 * GW; ++w) seg(w % W - R, w / W - R, L);
  for (int v = 0; v < 4 * W; ++v) {
    const int arm = v / W, j = v % W - R;
    seg(arm < 2 ? (arm == 0 ? -L : L) : j, arm < 2 ? j : (arm == 2 ? -L : L), R);
  }
  seg(R, R, L);
  while (perm.size() % 4) perm.push_back(-1);
  return perm;
}

static eb_status build_quad_plan(eb_stencils* st, ApplyPlan* pl, int R, cudaStream_t s, Tmp& tmp) {
  std::vector<int16_t> perm = quad_perm(R, 1);
  const int nq = (int)(perm.size() / 4);
  if (nq != (R == 3 ? QuadShape<3>::NQ : QuadShape<2>::NQ)) { set_error("quad layout mismatch"); return EB_ERR_INVALID; }
  int64_t cnt = 0;
  for (int16_t v : perm) cnt += v >= 0;
  if (cnt != st->nfoot) { set_error("quad layout does not cover the footprint"); return EB_ERR_INVALID; }
  const int64_t n_irr = st->n_irr, n_class = st->n_row_classes, nU = st->n_rows - n_class;
  int32_t* flag;
  int64_t* posC;
  int64_t nC = 0;
  EB_TRY(tmp.get(&flag, n_irr));
  EB_TRY(tmp.get(&posC, n_irr));
  k_flag_class<<<nblk(n_irr, 256), 256, 0, s>>>(n_irr, st->irr_row, n_class, flag); eb::count_launch();
  EB_TRY(scan<int32_t>(flag, n_irr, posC, &nC, s, tmp));
  if (nU + nC != n_irr) { set_error("irregular rows are not one per cell"); return EB_ERR_INVALID; }
  pl->nU = nU;
  pl->nC = nC;
  pl->n_class = n_class;
  EB_TRY(dalloc(st, &pl->cellU, std::max<int64_t>(nU, 1)));
  EB_TRY(dalloc(st, &pl->cellC, std::max<int64_t>(nC, 1)));
  EB_TRY(dalloc(st, &pl->classC, std::max<int64_t>(nC, 1)));
  k_split_irr<<<nblk(n_irr, 256), 256, 0, s>>>(n_irr, st->irr_cell, st->irr_row, n_class, posC, pl->cellU, pl->cellC,
                                               pl->classC); eb::count_launch();
  const size_t nUp = (size_t)((nU + 31) / 32) * 32;
  const size_t szU = std::max<size_t>(nUp * nq * 4, 4);
  EB_TRY(dalloc(st, &pl->qU32, szU));
  EB_TRY(dalloc(st, &pl->qU64, szU));
  EB_CUDA(cudaMemsetAsync(pl->qU32, 0, szU * 4, s));
  EB_CUDA(cudaMemsetAsync(pl->qU64, 0, szU * 8, s));
  int16_t* dperm;
  EB_TRY(tmp.get(&dperm, perm.size()));
  EB_CUDA(cudaMemcpyAsync(dperm, perm.data(), perm.size() * 2, cudaMemcpyHostToDevice, s));
  if (nU > 0) {
    dim3 grid(nblk(nU, 256), (unsigned)(4 * nq));
    k_pack_quads<float><<<grid, 256, 0, s>>>(st->rows32, st->n_rows, dperm, nq, n_class, pl->qU32);
    eb::count_launch();
    k_pack_quads<double><<<grid, 256, 0, s>>>(st->rows64, st->n_rows, dperm, nq, n_class, pl->qU64);
    eb::count_launch();
  }
  if (nC > 0) {
    // wall-layer class cells: aligned x-runs of four with one class, and the rest per cell
    int32_t *gs, *rest;
    int64_t *gpos, *lpos;
    int64_t nG = 0, nL = 0;
    EB_TRY(tmp.get(&gs, nC));
    EB_TRY(tmp.get(&rest, nC));
    EB_TRY(tmp.get(&gpos, nC));
    EB_TRY(tmp.get(&lpos, nC));
    k_run_mark<<<nblk(nC, 256), 256, 0, s>>>(nC, pl->cellC, pl->classC, pl->nx, gs); eb::count_launch();
    k_run_rest<<<nblk(nC, 256), 256, 0, s>>>(nC, gs, rest); eb::count_launch();
    EB_TRY(scan<int32_t>(gs, nC, gpos, &nG, s, tmp));
    EB_TRY(scan<int32_t>(rest, nC, lpos, &nL, s, tmp));
    if (4 * nG + nL != nC) { set_error("wall-layer runs do not partition the class cells"); return EB_ERR_INVALID; }
    pl->nG = nG;
    pl->nL = nL;
    EB_TRY(dalloc(st, &pl->cellG, std::max<int64_t>(nG, 1)));
    EB_TRY(dalloc(st, &pl->classG, std::max<int64_t>(nG, 1)));
    EB_TRY(dalloc(st, &pl->cellL, std::max<int64_t>(nL, 1)));
    EB_TRY(dalloc(st, &pl->classL, std::max<int64_t>(nL, 1)));
    k_run_split<<<nblk(nC, 256), 256, 0, s>>>(nC, pl->cellC, pl->classC, gs, rest, gpos, lpos, pl->cellG, pl->classG,
                                              pl->cellL, pl->classL); eb::count_launch();
    if (nL > 0 && pl->nx >= 2 * BR_W && pl->dim == 3) {
      const int64_t ns = (int64_t)2 * BR_W * pl->nz * pl->ny;
      EB_TRY(dalloc(st, &pl->slab_class, ns));
      EB_CUDA(cudaMemsetAsync(pl->slab_class, 0xFF, ns * 4, s));
      int32_t* keep;
      int64_t* kpos;
      int64_t nK = 0;
      EB_TRY(tmp.get(&keep, nL));
      EB_TRY(tmp.get(&kpos, nL));
      k_slab_scatter<<<nblk(nL, 256), 256, 0, s>>>(nL, pl->cellL, pl->classL, pl->nx, pl->ny, pl->nz, pl->slab_class,
                                                   keep); eb::count_launch();
      // uniform units: 32 y by BR_BZ z cells of one x layer, away from the y and z wall layers
      const int org = R + 2;
      pl->y_org = pl->z_org = org;
      pl->y_hi = std::max(org, pl->ny - org);
      pl->z_hi = std::max(org, pl->nz - org);
      pl->nyb = std::max(1, (pl->y_hi - org + 31) / 32);
      pl->nzb = std::max(1, (pl->z_hi - org + BR_BZ - 1) / BR_BZ);
      const int64_t nu = (int64_t)2 * BR_W * pl->nzb * pl->nyb;
      EB_TRY(dalloc(st, &pl->unit_class, nu));
      k_brick_units<<<nblk(nu, 128), 128, 0, s>>>(pl->slab_class, pl->ny, pl->nz, pl->nyb, pl->nzb, pl->y_org,
                                                  pl->z_org, pl->y_hi, pl->z_hi, pl->unit_class);
      eb::count_launch();
      k_brick_keep<<<nblk(nL, 256), 256, 0, s>>>(nL, pl->cellL, pl->nx, pl->ny, pl->nz, pl->nyb, pl->nzb, pl->y_org,
                                                 pl->z_org, pl->y_hi, pl->z_hi, pl->unit_class, keep);
      eb::count_launch();
      EB_TRY(scan<int32_t>(keep, nL, kpos, &nK, s, tmp));
      int32_t *cellK, *classK;
      EB_TRY(dalloc(st, &cellK, std::max<int64_t>(nK, 1)));
      EB_TRY(dalloc(st, &classK, std::max<int64_t>(nK, 1)));
      k_compact_pair<<<nblk(nL, 256), 256, 0, s>>>(nL, keep, kpos, pl->cellL, pl->classL, cellK, classK);
      eb::count_launch();
      pl->cellL = cellK;
      pl->classL = classK;
      pl->nL = nK;
      pl->brick = 1;
    }
    const int64_t nk = n_class * (int64_t)st->nfoot;
    EB_TRY(dalloc(st, &pl->rowsK32, nk));
    EB_TRY(dalloc(st, &pl->rowsK64, nk));
    k_class_major<float><<<nblk(nk, 256), 256, 0, s>>>(st->rows32, st->n_rows, n_class, st->nfoot, pl->rowsK32);
    eb::count_launch();
    k_class_major<double><<<nblk(nk, 256), 256, 0, s>>>(st->rows64, st->n_rows, n_class, st->nfoot, pl->rowsK64);
    eb::count_launch();
  }
  EB_CUDA(cudaGetLastError());
  pl->quad = 1;
  return EB_OK;
}

static eb_status build_pre(BuildCtx& c) {
  const eb_geom* g = c.g;
  const eb_params* prm = c.prm;
  eb_stencils* st = c.st;
  cudaStream_t s = c.s;
  c.tmp.s = s;
  st->build_stream = s;
  if (!g) { set_error("geometry descriptor is NULL"); return EB_ERR_INVALID; }
  eb_params P = {4, 0, EB_NBR_BOX, 1, 0.5, 5.0, EB_LS_MIXED};
  if (prm) P = *prm;
  if (P.ls_precision != EB_LS_MIXED && P.ls_precision != EB_LS_FP64) { set_error("bad ls_precision"); return EB_ERR_INVALID; }
  if (g->dim != 2 && g->dim != 3) { set_error("dim must be 2 or 3"); return EB_ERR_INVALID; }
  if (P.order != 2 && P.order != 4) { set_error("order must be 2 or 4"); return EB_ERR_INVALID; }
  if (g->moment_degree < P.order) { set_error("moment tables shallower than the order"); return EB_ERR_INVALID; }
  if (P.nbr_metric != EB_NBR_BOX && P.nbr_metric != EB_NBR_PATH) { set_error("bad nbr_metric"); return EB_ERR_INVALID; }
  int R = P.path_radius > 0 ? P.path_radius : (P.order == 2 ? 2 : 3);
  if (R > 3) { set_error("path radius > 3 not supported"); return EB_ERR_INVALID; }
  Dims& dm = st->dm;
  memset(&dm, 0, sizeof(dm));
  dm.dim = g->dim;
  for (int d = 0; d < 3; ++d) dm.n[d] = d < g->dim ? g->n[d] : 1;
  for (int d = 0; d < g->dim; ++d)
    if (dm.n[d] < 1) { set_error("bad grid size"); return EB_ERR_INVALID; }
  dm.ncell = (int64_t)dm.n[0] * dm.n[1] * dm.n[2];
  if (dm.ncell >= (1ll << 31)) { set_error("grid too large for int32 cell indices"); return EB_ERR_INVALID; }
  int64_t fb = 0;
  for (int d = 0; d < 3; ++d) {
    dm.nface[d] = d < g->dim ? (int64_t)(dm.n[0] + (d == 0)) * (dm.n[1] + (d == 1)) * (dm.n[2] + (d == 2)) : 0;
    dm.face_base[d] = fb;
    fb += dm.nface[d];
  }
  dm.n_grid_faces = fb;
  dm.order = P.order;
  dm.R = R;
  dm.nbr_box = P.nbr_metric == EB_NBR_BOX;
  dm.weighted = P.weighted;
  dm.w_threshold = P.w_threshold;
  dm.w_power = P.w_power;
  dm.mdeg = g->moment_degree;
  dm.h = g->h;
  dm.n_cut = g->n_cut;
  if (!(g->h > 0)) { set_error("h must be positive"); return EB_ERR_INVALID; }
  if (!g->cell_flag || (g->n_cut > 0 && (!g->cut_cell || !g->vol_mom || !g->eb_mom || !g->eb_nmom))) {
    set_error("missing geometry arrays");
    return EB_ERR_INVALID;
  }
  Tables& T = c.T;
  if (!make_tables(g->dim, P.order, g->moment_degree, &T)) { set_error("table construction failed"); return EB_ERR_INVALID; }
  dm.K = T.K;
  dm.KS = T.KS;
  dm.KFS = T.KFS;
  const int D = g->dim;
  const int64_t N = dm.ncell;
  Tmp& tmp = c.tmp;
  cudaEvent_t* ev = c.ev;
  for (int i = 0; i < 5; ++i) {
    EB_CUDA(cudaEventCreate(&ev[i]));
    c.n_ev = i + 1;
  }
  EB_CUDA(cudaEventRecord(ev[0], s));

  // ---- library-owned copies of the geometry
  Tables*& dT = c.dT;
  EB_TRY(dalloc(st, &dT, 1));
  EB_CUDA(cudaMemcpyAsync(dT, &T, sizeof(T), cudaMemcpyHostToDevice, s));
  EB_TRY(dalloc(st, &st->flag, N));
  EB_CUDA(cudaMemcpyAsync(st->flag, g->cell_flag, N, cudaMemcpyDeviceToDevice, s));
  const int64_t nc = g->n_cut;
  EB_TRY(dalloc(st, &st->cut_cell, nc));
  EB_TRY(dalloc(st, &st->vol_mom, nc * T.KS));
  EB_TRY(dalloc(st, &st->eb_mom, nc * T.KS));
  EB_TRY(dalloc(st, &st->eb_nmom, nc * D * T.KS));
  EB_TRY(dalloc(st, &st->eb_bc, nc));
  if (nc > 0) {
    EB_CUDA(cudaMemcpyAsync(st->cut_cell, g->cut_cell, nc * 4, cudaMemcpyDeviceToDevice, s));
    EB_CUDA(cudaMemcpyAsync(st->vol_mom, g->vol_mom, nc * T.KS * 8, cudaMemcpyDeviceToDevice, s));
    EB_CUDA(cudaMemcpyAsync(st->eb_mom, g->eb_mom, nc * T.KS * 8, cudaMemcpyDeviceToDevice, s));
    EB_CUDA(cudaMemcpyAsync(st->eb_nmom, g->eb_nmom, nc * D * T.KS * 8, cudaMemcpyDeviceToDevice, s));
    if (g->eb_bc) EB_CUDA(cudaMemcpyAsync(st->eb_bc, g->eb_bc, nc, cudaMemcpyDeviceToDevice, s));
    else EB_CUDA(cudaMemsetAsync(st->eb_bc, 0, nc, s));
  }
  EB_TRY(dalloc(st, &st->cut_of_cell, N));
  EB_CUDA(cudaMemsetAsync(st->cut_of_cell, 0xFF, N * 4, s));
  if (nc > 0) k_scatter_index<<<nblk(nc, 256), 256, 0, s>>>(st->cut_cell, nc, st->cut_of_cell); eb::count_launch();
  for (int d = 0; d < D; ++d) {
    if (!g->face_flag[d]) { set_error("missing face flags"); return EB_ERR_INVALID; }
    EB_TRY(dalloc(st, &st->face_flag[d], dm.nface[d]));
    EB_CUDA(cudaMemcpyAsync(st->face_flag[d], g->face_flag[d], dm.nface[d], cudaMemcpyDeviceToDevice, s));
    int64_t ncf = g->n_cutface[d];
    EB_TRY(dalloc(st, &st->cutface_of[d], dm.nface[d]));
    EB_CUDA(cudaMemsetAsync(st->cutface_of[d], 0xFF, dm.nface[d] * 4, s));
    EB_TRY(dalloc(st, &st->face_mom[d], ncf * T.KFS));
    if (ncf > 0) {
      if (!g->cutface[d] || !g->face_mom[d]) { set_error("missing cut-face arrays"); return EB_ERR_INVALID; }
      EB_CUDA(cudaMemcpyAsync(st->face_mom[d], g->face_mom[d], ncf * T.KFS * 8, cudaMemcpyDeviceToDevice, s));
      k_scatter_index<<<nblk(ncf, 256), 256, 0, s>>>(g->cutface[d], ncf, st->cutface_of[d]); eb::count_launch();
    }
  }
  EB_TRY(dalloc(st, &st->kappa, N));
  double*& invk = c.invk;
  EB_TRY(dalloc(st, &invk, N));
  k_kappa<<<nblk(N, 256), 256, 0, s>>>(N, st->flag, st->cut_of_cell, st->vol_mom, T.KS, st->kappa, invk); eb::count_launch();
  EB_CUDA(cudaGetLastError());

  // ---- 1. masks, face classes, slots
  uint8_t *m0, *m1;
  EB_TRY(tmp.get(&m0, N));
  EB_TRY(tmp.get(&m1, N));
  k_mark<<<nblk(N, 256), 256, 0, s>>>(dm, st->flag, m0); eb::count_launch();
  uint8_t* cur = m0;
  uint8_t* nxt = m1;
  for (int ax = 0; ax < D; ++ax) {
    k_dilate<<<nblk(N, 256), 256, 0, s>>>(dm, ax, R, cur, nxt); eb::count_launch();
    std::swap(cur, nxt);
  }
  uint8_t* dil = cur;
  const int M = R + 3;
  int64_t nkeys = 3;
  for (int d = 0; d < D; ++d) nkeys *= (int64_t)M * M;
  int64_t* class_rep;
  EB_TRY(tmp.get(&class_rep, nkeys));
  EB_CUDA(cudaMemsetAsync(class_rep, 0xFF, nkeys * 8, s));
  int32_t* state[3] = {nullptr, nullptr, nullptr};
  int32_t* isu[3] = {nullptr, nullptr, nullptr};
  int64_t* upos[3] = {nullptr, nullptr, nullptr};
  int64_t nu[3] = {0, 0, 0};
  for (int d = 0; d < D; ++d) {
    EB_TRY(tmp.get(&state[d], dm.nface[d]));
    EB_TRY(tmp.get(&isu[d], dm.nface[d]));
    EB_TRY(tmp.get(&upos[d], dm.nface[d]));
    k_classify_faces<<<nblk(dm.nface[d], 256), 256, 0, s>>>(dm, d, st->face_flag[d], dil, state[d], class_rep, isu[d]); eb::count_launch();
    EB_CUDA(cudaGetLastError());
    EB_TRY(scan<int32_t>(isu[d], dm.nface[d], upos[d], &nu[d], s, tmp));
  }
  std::vector<int64_t> h_rep(nkeys);
  EB_CUDA(cudaMemcpyAsync(h_rep.data(), class_rep, nkeys * 8, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  int64_t n_unique_grid = nu[0] + nu[1] + nu[2];
  int64_t n_unique = n_unique_grid + nc;
  std::vector<int32_t> h_class_slot(nkeys, -1);
  std::vector<int64_t> class_faces;
  int32_t* tmpl_slot_h = c.tmpl_slot_h;
  for (int64_t k = 0; k < nkeys; ++k) {
    if (h_rep[k] == -1) continue;
    h_class_slot[k] = (int32_t)(n_unique + class_faces.size());
    class_faces.push_back(h_rep[k]);
  }
  // template class of direction d: every clamped distance at its maximum
  for (int d = 0; d < D; ++d) {
    int64_t key = 0;
    for (int k = D - 1; k >= 0; --k) key = (key * M + (M - 1)) * M + (M - 1);
    key = key * 3 + d;
    tmpl_slot_h[d] = h_class_slot[key];
  }
  const int64_t n_slots = n_unique + (int64_t)class_faces.size();
  st->n_slots = n_slots;
  st->n_unique = n_unique;
  st->n_classes = (int32_t)class_faces.size();
  EB_TRY(dalloc(st, &st->slot_face, n_slots));
  int32_t* class_slot_d;
  EB_TRY(tmp.get(&class_slot_d, nkeys));
  EB_CUDA(cudaMemcpyAsync(class_slot_d, h_class_slot.data(), nkeys * 4, cudaMemcpyHostToDevice, s));
  if (!class_faces.empty())
    EB_CUDA(cudaMemcpyAsync(st->slot_face + n_unique, class_faces.data(), class_faces.size() * 8,
                            cudaMemcpyHostToDevice, s));
  int64_t ub = 0;
  for (int d = 0; d < D; ++d) {
    EB_TRY(dalloc(st, &st->face_slot[d], dm.nface[d]));
    k_face_slots<<<nblk(dm.nface[d], 256), 256, 0, s>>>(dm, d, state[d], upos[d], ub, class_slot_d,
                                                       st->face_slot[d], st->slot_face); eb::count_launch();
    ub += nu[d];
  }
  EB_TRY(dalloc(st, &st->eb_slot, nc));
  if (nc > 0) k_eb_slots<<<nblk(nc, 256), 256, 0, s>>>(nc, n_unique_grid, dm.n_grid_faces, st->slot_face, st->eb_slot); eb::count_launch();
  EB_CUDA(cudaGetLastError());
  EB_CUDA(cudaEventRecord(ev[1], s));

  // ---- 2. reach masks of cells whose neighbourhood sees a non-full cell
  int32_t *sel, *near_list, *reach_idx;
  int64_t* near_pos;
  int64_t n_near = 0;
  EB_TRY(tmp.get(&sel, N));
  EB_TRY(tmp.get(&near_pos, N));
  EB_TRY(tmp.get(&reach_idx, N));
  k_flag_list<<<nblk(N, 256), 256, 0, s>>>(dil, st->flag, N, sel); eb::count_launch();
  EB_TRY(scan<int32_t>(sel, N, near_pos, &n_near, s, tmp));
  EB_TRY(tmp.get(&near_list, n_near));
  k_compact<<<nblk(N, 256), 256, 0, s>>>(sel, near_pos, N, near_list, reach_idx); eb::count_launch();
  Mask* masks;
  EB_TRY(tmp.get(&masks, n_near));
  if (n_near > 0)
    k_reach<<<nblk(n_near, 128), 128, 0, s>>>(dm, near_list, n_near, st->flag, st->face_flag[0],
                                              D > 1 ? st->face_flag[1] : st->face_flag[0],
                                              D > 2 ? st->face_flag[2] : st->face_flag[0], masks); eb::count_launch();
  EB_CUDA(cudaGetLastError());

  // ---- 3. gather row lists
  GatherArgs ga;
  memset(&ga, 0, sizeof(ga));
  ga.dm = dm;
  ga.flag = st->flag;
  for (int d = 0; d < 3; ++d) ga.ff[d] = d < D ? st->face_flag[d] : st->face_flag[0];
  ga.reach_idx = reach_idx;
  ga.masks = masks;
  ga.cut_of_cell = st->cut_of_cell;
  ga.slot_face = st->slot_face;
  int64_t* counts;
  int32_t* too_many;
  EB_TRY(tmp.get(&counts, n_slots + 1));
  EB_TRY(tmp.get(&too_many, 1));
  EB_CUDA(cudaMemsetAsync(too_many, 0, 4, s));
  ga.count = counts;
  ga.too_many = too_many;
  ga.row_ptr = nullptr;
  k_gather<<<nblk(n_slots, 128), 128, 0, s>>>(ga, n_slots, st->cut_cell); eb::count_launch();
  EB_CUDA(cudaGetLastError());
  EB_TRY(dalloc(st, &st->row_ptr, n_slots + 1));
  int64_t nnz = 0;
  EB_CUDA(cudaMemsetAsync(counts + n_slots, 0, 8, s));
  EB_TRY(scan<int64_t>(counts, n_slots + 1, st->row_ptr, &nnz, s, tmp));
  int32_t h_too = 0;
  EB_CUDA(cudaMemcpyAsync(&h_too, too_many, 4, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  if (h_too) { set_error("a face has more LS rows than the kernel supports"); return EB_ERR_CAPACITY; }
  EB_TRY(dalloc(st, &st->row_desc, nnz));
  EB_TRY(dalloc(st, &st->row_val, nnz));
  ga.row_ptr = st->row_ptr;
  ga.row_desc = st->row_desc;
  k_gather<<<nblk(n_slots, 128), 128, 0, s>>>(ga, n_slots, st->cut_cell); eb::count_launch();
  EB_CUDA(cudaGetLastError());
  // ---- 4. weighted least squares (FP64): inputs here, the launch in build_ls
  int dev = 0, nsm = 0;
  EB_CUDA(cudaGetDevice(&dev));
  EB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  double *ftab, *wtab;
  EB_TRY(tmp.get(&ftab, (size_t)TAB_N * MAXK));
  EB_TRY(tmp.get(&wtab, TAB_N));
  k_full_rows<<<nblk(TAB_N, 128), 128, 0, s>>>(dm, dT, ftab, wtab); eb::count_launch();
  int32_t* status;
  EB_TRY(tmp.get(&status, std::max<int64_t>(n_slots, 1)));
  LsArgs& la = c.la;
  memset(&la, 0, sizeof(la));
  la.dm = dm;
  la.T = dT;
  la.flag = st->flag;
  la.cut_of_cell = st->cut_of_cell;
  la.cut_cell = st->cut_cell;
  la.vol_mom = st->vol_mom;
  la.eb_mom = st->eb_mom;
  la.eb_nmom = st->eb_nmom;
  la.eb_bc = st->eb_bc;
  for (int d = 0; d < 3; ++d) {
    la.cutface_of[d] = d < D ? st->cutface_of[d] : st->cutface_of[0];
    la.face_mom[d] = d < D ? st->face_mom[d] : st->face_mom[0];
  }
  la.slot_face = st->slot_face;
  la.row_ptr = st->row_ptr;
  la.row_desc = st->row_desc;
  la.row_val = st->row_val;
  la.n_slots = n_slots;
  la.status = status;
  la.ftab = ftab;
  la.wtab = wtab;
  c.P = P;
  c.R = R;
  c.D = D;
  c.N = N;
  c.nsm = nsm;
  c.n_slots = n_slots;
  c.n_unique = n_unique;
  c.status = status;
  return EB_OK;
}

// The least-squares launch for n builds (one launch; n > 1: the systems of all geometries share one
// work counter, each system finding its geometry from the prefix sums of the systems per build).
static eb_status build_ls(BuildCtx* const* cs, int n, cudaStream_t s) {
  BuildCtx& c0 = *cs[0];
  int64_t total = 0;
  std::vector<int64_t> base(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    if (cs[i]->T.K != c0.T.K || cs[i]->D != c0.D) { set_error("a batch mixes dimensions or orders"); return EB_ERR_INVALID; }
    base[i] = total;
    total += cs[i]->n_slots;
  }
  base[n] = total;
  Tmp tmp;
  tmp.s = s;
  EB_CUDA(lsq_prepare());
  const bool fp32 = c0.P.ls_precision == EB_LS_MIXED;
  for (int i = 1; i < n; ++i)
    if (cs[i]->P.ls_precision != c0.P.ls_precision) { set_error("a batch mixes LS precisions"); return EB_ERR_INVALID; }
  auto blocks_for = [&](int64_t systems, int per_cta) {
    return std::max<int64_t>(1, std::min<int64_t>(c0.nsm, (systems + per_cta - 1) / per_cta));
  };
  const int64_t nb_d = blocks_for(total, LS_SYS), nb_f = blocks_for(total, LS_SYS_F);
  double* scratch;
  EB_TRY(tmp.get(&scratch, (size_t)std::max(nb_d * LS_SYS, fp32 ? nb_f * LS_SYS_F : 0) * LS_SCRATCH));
  int32_t *next, *lerr, *nfb, *fblist = nullptr;
  double* flops;
  EB_TRY(tmp.get(&next, 1));
  EB_TRY(tmp.get(&lerr, 1));
  EB_TRY(tmp.get(&nfb, 1));
  EB_TRY(tmp.get(&flops, 2));
  EB_CUDA(cudaMemsetAsync(flops, 0, 16, s));
  EB_CUDA(cudaMemsetAsync(next, 0, 4, s));
  EB_CUDA(cudaMemsetAsync(lerr, 0, 4, s));
  EB_CUDA(cudaMemsetAsync(nfb, 0, 4, s));
  LsArgs a0 = c0.la;
  a0.n_slots = total;
  a0.slot_list = nullptr;
  a0.next = next;
  a0.err = lerr;
  a0.scratch = scratch;
  a0.flops = flops;
  LsArgs* dbatch = nullptr;
  int64_t* dbase = nullptr;
  if (n > 1) {
    std::vector<LsArgs> hb(n);
    for (int i = 0; i < n; ++i) {
      hb[i] = cs[i]->la;
      hb[i].slot_list = nullptr;
    }
    EB_TRY(tmp.get(&dbatch, n));
    EB_TRY(tmp.get(&dbase, n + 1));
    EB_CUDA(cudaMemcpyAsync(dbatch, hb.data(), n * sizeof(LsArgs), cudaMemcpyHostToDevice, s));
    EB_CUDA(cudaMemcpyAsync(dbase, base.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s));
  }
  for (int i = 0; i < n; ++i) EB_CUDA(cudaEventRecord(cs[i]->ev[2], s));
  if (total > 0) {
    if (fp32) {
      // FP32 factorisation for every system, then the FP64 one for those it left (status 3)
      EB_CUDA(lsq_launch(true, (unsigned)nb_f, s, a0, c0.T, n > 1 ? dbatch : nullptr, dbase, n));
      eb::count_launch();
      EB_TRY(tmp.get(&fblist, total));
      for (int i = 0; i < n; ++i) {
        EB_CUDA(lsq_fallback_list(cs[i]->status, cs[i]->n_slots, base[i], fblist, nfb, s));
        eb::count_launch();
      }
      int32_t hn = 0;
      EB_CUDA(cudaMemcpyAsync(&hn, nfb, 4, cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      if (hn > 0) {
        EB_CUDA(cudaMemsetAsync(next, 0, 4, s));
        a0.slot_list = fblist;
        a0.n_slots = hn;
        EB_CUDA(lsq_launch(false, (unsigned)blocks_for(hn, LS_SYS), s, a0, c0.T, n > 1 ? dbatch : nullptr, dbase, n));
        eb::count_launch();
      }
    } else {
      EB_CUDA(lsq_launch(false, (unsigned)nb_d, s, a0, c0.T, n > 1 ? dbatch : nullptr, dbase, n));
      eb::count_launch();
    }
  }
  for (int i = 0; i < n; ++i) EB_CUDA(cudaEventRecord(cs[i]->ev[3], s));
  int32_t h = 0;
  double hf[2] = {0.0, 0.0};
  EB_CUDA(cudaMemcpyAsync(&h, lerr, 4, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaMemcpyAsync(hf, flops, 16, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) {  // a batch's totals shared out by the systems' counts
    const double share = total > 0 ? (double)cs[i]->n_slots / (double)total : 0.0;
    cs[i]->ls_flops[0] = hf[0] * share;
    cs[i]->ls_flops[1] = hf[1] * share;
  }
  if (h) { set_error("a bounded device wait gave up in the least-squares kernel"); return EB_ERR_TIMEOUT; }
  return EB_OK;
}

static eb_status build_post(BuildCtx& c) {
  const eb_geom* g = c.g;
  eb_stencils* st = c.st;
  eb_build_info* info = c.info;
  cudaStream_t s = c.s;
  Tmp& tmp = c.tmp;
  cudaEvent_t* ev = c.ev;
  Tables& T = c.T;
  Dims& dm = st->dm;
  const int R = c.R, D = c.D, nsm = c.nsm;
  const int64_t N = c.N, n_slots = c.n_slots, n_unique = c.n_unique, nc = g->n_cut;
  const int32_t* tmpl_slot_h = c.tmpl_slot_h;
  int32_t* status = c.status;
  double* invk = c.invk;
  const int M = R + 3;
  {
    std::vector<int32_t> hs(n_slots);
    EB_CUDA(cudaMemcpyAsync(hs.data(), status, n_slots * 4, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    int unbuilt = 0, nbad = 0;
    int64_t nfp64 = 0;
    for (int64_t i = 0; i < n_slots; ++i) {
      if (hs[i] == 1) ++nbad;
      if (hs[i] == 2) unbuilt = 1;  // a row flagged by the row builder
      if (hs[i] == 4) ++nfp64;      // left by the FP32 factorisation, solved by the FP64 one
    }
    info->n_ls_fp64 = c.P.ls_precision == EB_LS_FP64 ? n_slots : nfp64;
    info->ls_fp64_flops = c.ls_flops[0];
    info->ls_fp32_flops = c.ls_flops[1];
    if (unbuilt) { set_error("an LS row could not be built"); return EB_ERR_INVALID; }
    if (nbad) {
      // every face whose system failed: a class slot stands for all the faces of its class, so the
      // faces are listed from the face -> slot maps (ascending global face id)
      for (int d = 0; d < D; ++d) {
        std::vector<int32_t> fs(dm.nface[d]);
        EB_CUDA(cudaMemcpyAsync(fs.data(), st->face_slot[d], dm.nface[d] * 4, cudaMemcpyDeviceToHost, s));
        EB_CUDA(cudaStreamSynchronize(s));
        for (int64_t f = 0; f < dm.nface[d]; ++f)
          if (fs[f] >= 0 && hs[fs[f]] == 1) g_bad_faces.push_back(dm.face_base[d] + f);
      }
      if (nc > 0) {
        std::vector<int32_t> es(nc);
        EB_CUDA(cudaMemcpyAsync(es.data(), st->eb_slot, nc * 4, cudaMemcpyDeviceToHost, s));
        EB_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < nc; ++i)
          if (es[i] >= 0 && hs[es[i]] == 1) g_bad_faces.push_back(dm.n_grid_faces + i);
      }
    }
    if (!g_bad_faces.empty()) {
      set_error("rank-deficient LS systems: " + std::to_string(g_bad_faces.size()) + " faces");
      return EB_ERR_RANK_DEFICIENT;
    }
  }

  // ---- 5. operator rows and boundary matrix
  // footprint
  {
    std::vector<int32_t> off;
    std::vector<int8_t> dd;
    int L = R + 1, S = 2 * L + 1;
    std::vector<int16_t> lut(S * S * S, -1);
    int zr = D == 3 ? L : 0;
    for (int z = -zr; z <= zr; ++z)
      for (int y = -L; y <= L; ++y)
        for (int x = -L; x <= L; ++x) {
          if (!in_footprint(x, y, z, R, dm.nbr_box)) continue;
          lut[(x + L) + S * ((y + L) + S * (z + L))] = (int16_t)off.size();
          off.push_back((int32_t)((int64_t)x + (int64_t)dm.n[0] * ((int64_t)y + (int64_t)dm.n[1] * z)));
          dd.push_back((int8_t)x);
          dd.push_back((int8_t)y);
          dd.push_back((int8_t)z);
        }
    st->nfoot = (int)off.size();
    EB_TRY(dalloc(st, &st->foot_off, off.size()));
    EB_TRY(dalloc(st, &st->foot_d, dd.size()));
    int16_t* dlut;
    EB_TRY(tmp.get(&dlut, lut.size()));
    EB_CUDA(cudaMemcpyAsync(st->foot_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice, s));
    EB_CUDA(cudaMemcpyAsync(st->foot_d, dd.data(), dd.size(), cudaMemcpyHostToDevice, s));
    EB_CUDA(cudaMemcpyAsync(dlut, lut.data(), lut.size() * 2, cudaMemcpyHostToDevice, s));
    int center = lut[L + S * (L + S * L)];
    st->foot_center = center;
    int64_t nrk = 1;
    for (int d = 0; d < D; ++d) nrk *= (int64_t)M * M;
    nrk += 1;  // key 0: template
    int64_t* row_rep;
    int32_t *rowkey, *isuc, *tslot;
    int64_t* upc;
    EB_TRY(tmp.get(&row_rep, nrk));
    EB_TRY(tmp.get(&rowkey, N));
    EB_TRY(tmp.get(&isuc, N));
    EB_TRY(tmp.get(&upc, N));
    EB_TRY(tmp.get(&tslot, 3));
    EB_CUDA(cudaMemsetAsync(row_rep, 0xFF, nrk * 8, s));
    EB_CUDA(cudaMemcpyAsync(tslot, tmpl_slot_h, 12, cudaMemcpyHostToDevice, s));
    EB_TRY(dalloc(st, &st->cell_kind, N));
    k_cell_kind<<<nblk(N, 256), 256, 0, s>>>(dm, st->flag, st->face_slot[0], D > 1 ? st->face_slot[1] : nullptr,
                                            D > 2 ? st->face_slot[2] : nullptr, n_unique, tslot, st->cell_kind,
                                            rowkey, row_rep, isuc); eb::count_launch();
    EB_CUDA(cudaGetLastError());
    int64_t n_ucell = 0;
    EB_TRY(scan<int32_t>(isuc, N, upc, &n_ucell, s, tmp));
    std::vector<int64_t> h_rrep(nrk);
    EB_CUDA(cudaMemcpyAsync(h_rrep.data(), row_rep, nrk * 8, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    // rows: [template (always row 0, even if unused)] [class rows] [unique rows]
    std::vector<int32_t> key_row(nrk, -1), rep_cells;
    rep_cells.push_back(h_rrep[0] >= 0 ? (int32_t)h_rrep[0] : -1);
    key_row[0] = 0;
    for (int64_t k = 1; k < nrk; ++k)
      if (h_rrep[k] >= 0) {
        key_row[k] = (int32_t)rep_cells.size();
        rep_cells.push_back((int32_t)h_rrep[k]);
      }
    int64_t n_class_rows = (int64_t)rep_cells.size();
    st->n_row_classes = (int32_t)n_class_rows;
    st->n_rows = n_class_rows + n_ucell;
    // irregular list
    int32_t* k2;
    int64_t* k2pos;
    EB_TRY(tmp.get(&k2, N));
    EB_TRY(tmp.get(&k2pos, N));
    k_is_kind2<<<nblk(N, 256), 256, 0, s>>>(N, st->cell_kind, k2); eb::count_launch();
    EB_TRY(scan<int32_t>(k2, N, k2pos, &st->n_irr, s, tmp));
    EB_TRY(dalloc(st, &st->irr_cell, st->n_irr));
    EB_TRY(dalloc(st, &st->irr_row, st->n_irr));
    int32_t *key_row_d, *rep_d;
    EB_TRY(tmp.get(&key_row_d, nrk));
    EB_TRY(tmp.get(&rep_d, st->n_rows));
    EB_CUDA(cudaMemcpyAsync(key_row_d, key_row.data(), nrk * 4, cudaMemcpyHostToDevice, s));
    EB_CUDA(cudaMemcpyAsync(rep_d, rep_cells.data(), n_class_rows * 4, cudaMemcpyHostToDevice, s));
    k_irr_list<<<nblk(N, 256), 256, 0, s>>>(N, st->cell_kind, k2pos, rowkey, key_row_d, upc, n_class_rows,
                                           st->irr_cell, st->irr_row, rep_d); eb::count_launch();
    EB_CUDA(cudaGetLastError());
    // operator rows
    EB_TRY(dalloc(st, &st->rows64, (size_t)st->nfoot * st->n_rows));
    EB_TRY(dalloc(st, &st->rows32, (size_t)st->nfoot * st->n_rows));
    AsmArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.dm = dm;
    aa.flag = st->flag;
    aa.cut_of_cell = st->cut_of_cell;
    for (int d = 0; d < 3; ++d) {
      aa.face_slot[d] = d < D ? st->face_slot[d] : nullptr;
      aa.ff[d] = d < D ? st->face_flag[d] : nullptr;
    }
    aa.eb_slot = st->eb_slot;
    aa.slot_face = st->slot_face;
    aa.row_ptr = st->row_ptr;
    aa.row_desc = st->row_desc;
    aa.row_val = st->row_val;
    aa.nfoot = st->nfoot;
    aa.foot_lut = dlut;
    aa.n_rows = st->n_rows;
    aa.rows64 = st->rows64;
    aa.rows32 = st->rows32;
    aa.inv_h2 = 1.0 / (dm.h * dm.h);
    aa.eb_bc = st->eb_bc;
    aa.eb_mom = st->eb_mom;
    int32_t* aerr;
    EB_TRY(tmp.get(&aerr, 1));
    EB_CUDA(cudaMemsetAsync(aerr, 0, 4, s));
    // the template row may have no representative on small grids: build the others, fill it below
    int first = rep_cells[0] >= 0 ? 0 : 1;
    int64_t nrep = st->n_rows - first;
    if (first) EB_CUDA(cudaMemsetAsync(st->rows64, 0, 8, s));  // row 0 of entry 0 only; the template row is unused
    if (nrep > 0) {
      size_t sm = (size_t)8 * st->nfoot * 8;
      k_assemble_rows<<<nblk(nrep, 8), 256, sm, s>>>(aa, rep_d + first, nrep, first, aerr); eb::count_launch();
    }
    EB_CUDA(cudaGetLastError());
    EB_TRY(dalloc(st, &st->tmpl64, st->nfoot));
    EB_TRY(dalloc(st, &st->tmpl32, st->nfoot));
    EB_CUDA(cudaMemsetAsync(st->tmpl64, 0, st->nfoot * 8, s));
    EB_CUDA(cudaMemsetAsync(st->tmpl32, 0, st->nfoot * 4, s));
    if (first == 0) {
      EB_CUDA(cudaMemcpy2DAsync(st->tmpl64, 8, st->rows64, st->n_rows * 8, 8, st->nfoot, cudaMemcpyDeviceToDevice, s));
      EB_CUDA(cudaMemcpy2DAsync(st->tmpl32, 4, st->rows32, st->n_rows * 4, 4, st->nfoot, cudaMemcpyDeviceToDevice, s));
    }
    // Jacobi diagonal of the kappa-weighted operator
    double* dinv64;
    float* dinv32;
    EB_TRY(dalloc(st, &dinv64, N));
    EB_TRY(dalloc(st, &dinv32, N));
    k_diag_inv<<<nblk(N, 256), 256, 0, s>>>(N, st->cell_kind, nullptr, st->tmpl64, center, dinv64, dinv32); eb::count_launch();
    if (st->n_irr > 0)
      k_diag_irr<<<nblk(st->n_irr, 256), 256, 0, s>>>(st->n_irr, st->irr_cell, st->irr_row, st->rows64, st->n_rows,
                                                       center, dinv64, dinv32); eb::count_launch();
    EB_CUDA(cudaGetLastError());
    // boundary matrix over irregular cells
    int64_t *bcnt, nbnz = 0;
    EB_TRY(tmp.get(&bcnt, st->n_irr + 1));
    EB_CUDA(cudaMemsetAsync(bcnt, 0, (st->n_irr + 1) * 8, s));
    if (st->n_irr > 0)
      k_assemble_b<<<nblk(st->n_irr, 128), 128, 0, s>>>(aa, st->irr_cell, st->n_irr, bcnt, nullptr, nullptr, nullptr,
                                                        nullptr); eb::count_launch();
    EB_TRY(dalloc(st, &st->b_ptr, st->n_irr + 1));
    EB_TRY(scan<int64_t>(bcnt, st->n_irr + 1, st->b_ptr, &nbnz, s, tmp));
    EB_TRY(dalloc(st, &st->b_col, nbnz));
    EB_TRY(dalloc(st, &st->b_val, nbnz));
    if (st->n_irr > 0)
      k_assemble_b<<<nblk(st->n_irr, 128), 128, 0, s>>>(aa, st->irr_cell, st->n_irr, nullptr, st->b_ptr, st->b_col,
                                                        st->b_val, nullptr); eb::count_launch();
    EB_CUDA(cudaGetLastError());
    int32_t h_aerr = 0;
    EB_CUDA(cudaMemcpyAsync(&h_aerr, aerr, 4, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    if (h_aerr) { set_error("stencil column outside the operator footprint"); return EB_ERR_INVALID; }
    // wall faces (ascending id) and the position of each B wall entry in that list
    {
      std::vector<int64_t> cand;
      for (int d = 0; d < D; ++d) {
        int64_t m0 = dm.n[0] + (d == 0), m1 = dm.n[1] + (d == 1);
        int nz = dm.n[2] + (d == 2), ny = dm.n[1] + (d == 1), nx = dm.n[0] + (d == 0);
        for (int z = 0; z < nz; ++z)
          for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
              int c[3] = {x, y, z};
              if (c[d] != 0 && c[d] != dm.n[d]) {
                if (d == 0) x = dm.n[0] - 1;  // jump to the high wall
                continue;
              }
              cand.push_back(dm.face_base[d] + x + m0 * ((int64_t)y + m1 * z));
            }
      }
      std::sort(cand.begin(), cand.end());
      int64_t nc2 = (int64_t)cand.size();
      int64_t* dcand;
      uint8_t* dfl;
      EB_TRY(tmp.get(&dcand, nc2));
      EB_TRY(tmp.get(&dfl, nc2));
      EB_CUDA(cudaMemcpyAsync(dcand, cand.data(), nc2 * 8, cudaMemcpyHostToDevice, s));
      std::vector<uint8_t> hfl(nc2);
      for (int d = 0; d < D; ++d) {
        // candidates of direction d are contiguous after sorting (global ids are direction-major)
        int64_t lo = std::lower_bound(cand.begin(), cand.end(), dm.face_base[d]) - cand.begin();
        int64_t hi = std::lower_bound(cand.begin(), cand.end(), dm.face_base[d] + dm.nface[d]) - cand.begin();
        if (hi > lo) {
          // shift ids to local indices on the fly
          std::vector<int64_t> loc(cand.begin() + lo, cand.begin() + hi);
          for (auto& v : loc) v -= dm.face_base[d];
          int64_t* dloc;
          EB_TRY(tmp.get(&dloc, hi - lo));
          EB_CUDA(cudaMemcpyAsync(dloc, loc.data(), (hi - lo) * 8, cudaMemcpyHostToDevice, s));
          k_gather_flags<<<nblk(hi - lo, 256), 256, 0, s>>>(st->face_flag[d], dloc, hi - lo, dfl + lo); eb::count_launch();
          EB_CUDA(cudaMemcpyAsync(hfl.data() + lo, dfl + lo, hi - lo, cudaMemcpyDeviceToHost, s));
          EB_CUDA(cudaStreamSynchronize(s));
        }
      }
      st->wall_ids_host.clear();
      for (int64_t i = 0; i < nc2; ++i)
        if (hfl[i]) st->wall_ids_host.push_back(cand[i]);
      st->n_wall = (int64_t)st->wall_ids_host.size();
      EB_TRY(dalloc(st, &st->wall_ids, st->n_wall));
      if (st->n_wall)
        EB_CUDA(cudaMemcpyAsync(st->wall_ids, st->wall_ids_host.data(), st->n_wall * 8, cudaMemcpyHostToDevice, s));
      int64_t* wpos;
      EB_TRY(dalloc(st, &wpos, nbnz));
      if (nbnz > 0)
        k_wall_pos<<<nblk(nbnz, 256), 256, 0, s>>>(nbnz, st->b_col, dm.n_grid_faces, st->wall_ids, st->n_wall, wpos); eb::count_launch();
      EB_CUDA(cudaGetLastError());
      st->b_wpos = wpos;
      st->dinv64 = dinv64;
      st->dinv32 = dinv32;
      st->inv_kappa = invk;
    }
    info->n_irregular_rows = st->n_rows - n_class_rows;
    info->n_row_classes = (int32_t)n_class_rows;
  }
  // ---- apply plan: TMA template pass when the row stride suits TMA, irregular rows overlapped
  {
    ApplyPlan* pl = new ApplyPlan();
    st->plan = pl;
    pl->nx = dm.n[0];
    pl->ny = dm.n[1];
    pl->nz = dm.n[2];
    pl->dim = D;
    pl->R = R;
    pl->nsm = nsm;
    pl->side = nullptr;
    pl->fork = pl->join = nullptr;
    EB_TRY(dalloc(st, &pl->err, 1));
    EB_CUDA(cudaMemsetAsync(pl->err, 0, 4, s));
    std::vector<double> tm(st->nfoot);
    std::vector<int8_t> fd(st->nfoot * 3);
    EB_CUDA(cudaMemcpyAsync(tm.data(), st->tmpl64, st->nfoot * 8, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaMemcpyAsync(fd.data(), st->foot_d, st->nfoot * 3, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    int L = R + 1, S = 2 * L + 1;
    pl->cube64.assign(S * S * S, 0.0);
    pl->cube32.assign(S * S * S, 0.0f);
    for (int i = 0; i < st->nfoot; ++i) {
      int idx = (fd[3 * i] + L) + S * ((fd[3 * i + 1] + L) + S * (fd[3 * i + 2] + L));
      pl->cube64[idx] = tm[i];
      pl->cube32[idx] = (float)tm[i];
    }
    if (D == 3) {
      // z symmetry of the interior template (exact in the mathematics, to rounding in the LS solves)
      double mx = 0.0, dmax = 0.0;
      for (double v : pl->cube64) mx = std::max(mx, fabs(v));
      pl->zcube64 = pl->cube64;
      for (int z = 1; z <= L; ++z)
        for (int y = 0; y < S; ++y)
          for (int x = 0; x < S; ++x) {
            double& p = pl->zcube64[x + S * (y + S * (L + z))];
            double m = pl->cube64[x + S * (y + S * (L - z))];
            dmax = std::max(dmax, fabs(p - m));
            p = 0.5 * (p + m);
          }
      pl->zsym = dmax <= 64.0 * 2.220446049250313e-16 * mx;
      pl->zcube32.assign(pl->zcube64.begin(), pl->zcube64.end());
      // reflection symmetry in x, y and z: T(a, b, c) = mean of c(+-a, +-b, +-c) over the sign images
      const int F = L + 1;
      pl->fold64.assign(F * F * F, 0.0);
      double fmax = 0.0;
      for (int c = 0; c <= L; ++c)
        for (int b = 0; b <= L; ++b)
          for (int a = 0; a <= L; ++a) {
            double sum = 0.0;
            int cnt = 0;
            for (int sz = -1; sz <= 1; sz += 2)
              for (int sy = -1; sy <= 1; sy += 2)
                for (int sx = -1; sx <= 1; sx += 2) {
                  sum += pl->cube64[(sx * a + L) + S * ((sy * b + L) + S * (sz * c + L))];
                  ++cnt;
                }
            const double t = sum / cnt;
            pl->fold64[a + F * (b + F * c)] = t;
            for (int sz = -1; sz <= 1; sz += 2)
              for (int sy = -1; sy <= 1; sy += 2)
                for (int sx = -1; sx <= 1; sx += 2)
                  fmax = std::max(fmax, fabs(pl->cube64[(sx * a + L) + S * ((sy * b + L) + S * (sz * c + L))] - t));
          }
      pl->fsym = fmax <= 64.0 * 2.220446049250313e-16 * mx;
      pl->fold32.assign(pl->fold64.begin(), pl->fold64.end());
    }
    bool ok = dm.nbr_box && st->n_row_classes > 0;
    pl->tma32 = ok && (dm.n[0] % 4 == 0);
    pl->tma64 = ok && (dm.n[0] % 2 == 0);
    pl->seg = dm.nbr_box;
    if (pl->seg && D == 3 && (R == 2 || R == 3) && st->n_irr > 0) EB_TRY(build_quad_plan(st, pl, R, s, tmp));
    EB_CUDA(cudaStreamCreateWithFlags(&pl->side, cudaStreamNonBlocking));
    EB_CUDA(cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming));
    EB_CUDA(cudaEventCreateWithFlags(&pl->join, cudaEventDisableTiming));
  }
  EB_CUDA(cudaEventRecord(ev[4], s));
  EB_CUDA(cudaStreamSynchronize(s));
  // ---- info
  info->n_unique_faces = n_unique;
  info->n_class_faces = 0;
  for (int d = 0; d < D; ++d) info->n_class_faces += dm.nface[d];  // refined below
  {
    int64_t n_open = 0, n_cls = 0;
    for (int d = 0; d < D; ++d) {
      std::vector<int32_t> hs(dm.nface[d]);
      EB_CUDA(cudaMemcpyAsync(hs.data(), st->face_slot[d], dm.nface[d] * 4, cudaMemcpyDeviceToHost, s));
      EB_CUDA(cudaStreamSynchronize(s));
      for (int32_t v : hs) {
        if (v >= 0) ++n_open;
        if (v >= n_unique) ++n_cls;
      }
    }
    info->n_flux_faces = n_open + nc;
    info->n_class_faces = n_cls;
  }
  info->n_classes = st->n_classes;
  {
    std::vector<int64_t> rp(n_slots + 1);
    EB_CUDA(cudaMemcpyAsync(rp.data(), st->row_ptr, (n_slots + 1) * 8, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    int32_t mx = 0;
    double fl = 0.0;
    int K = T.K;
    for (int64_t i = 0; i < n_slots; ++i) {
      int64_t n = rp[i + 1] - rp[i];
      mx = std::max<int32_t>(mx, (int32_t)n);
      // the method's count per system: Householder QR of the n x K matrix, the triangular solve and the
      // application of Q (2nK^2 - 2K^3/3 + 4nK + K^2)
      fl += 2.0 * n * K * K - 2.0 / 3.0 * K * K * K + 4.0 * n * K + 1.0 * K * K;
    }
    info->max_rows = mx;
    info->lsq_flops = (int64_t)fl;
  }
  float t01 = 0, t12 = 0, t23 = 0, t34 = 0;
  cudaEventElapsedTime(&t01, ev[0], ev[1]);
  cudaEventElapsedTime(&t12, ev[1], ev[2]);
  cudaEventElapsedTime(&t23, ev[2], ev[3]);
  cudaEventElapsedTime(&t34, ev[3], ev[4]);
  info->ms_classify = t01;
  info->ms_gather = t12;
  info->ms_lsq = t23;
  info->ms_assemble = t34;
  return EB_OK;
}

}  // extern "C"

// ====================================================================== apply / solve / query

namespace eb {

template <typename T>
static ApplyArgs<T> apply_args(const eb_stencils* st, int kw);

template <>
ApplyArgs<float> apply_args<float>(const eb_stencils* st, int kw) {
  ApplyArgs<float> a;
  a.ncell = st->dm.ncell;
  a.nfoot = st->nfoot;
  a.foot_off = st->foot_off;
  a.tmpl = st->tmpl32;
  a.kind = st->cell_kind;
  a.inv_kappa = st->inv_kappa;
  a.n_irr = st->n_irr;
  a.irr_cell = st->irr_cell;
  a.irr_row = st->irr_row;
  a.n_rows = st->n_rows;
  a.rows = st->rows32;
  a.phi = nullptr;
  a.y = nullptr;
  a.kappa_weighted = kw;
  a.plan = st->plan;
  return a;
}
template <>
ApplyArgs<double> apply_args<double>(const eb_stencils* st, int kw) {
  ApplyArgs<double> a;
  a.ncell = st->dm.ncell;
  a.nfoot = st->nfoot;
  a.foot_off = st->foot_off;
  a.tmpl = st->tmpl64;
  a.kind = st->cell_kind;
  a.inv_kappa = st->inv_kappa;
  a.n_irr = st->n_irr;
  a.irr_cell = st->irr_cell;
  a.irr_row = st->irr_row;
  a.n_rows = st->n_rows;
  a.rows = st->rows64;
  a.phi = nullptr;
  a.y = nullptr;
  a.kappa_weighted = kw;
  a.plan = st->plan;
  return a;
}

}  // namespace eb

extern "C" {

eb_status eb_apply(const eb_stencils* st, const void* phi, void* y, int32_t dtype, int32_t kappa_weighted,
                   eb_stream_t stream) {
  if (!st || !phi || !y) { set_error("null argument"); return EB_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == EB_F32) {
    ApplyArgs<float> a = apply_args<float>(st, kappa_weighted);
    a.phi = (const float*)phi;
    a.y = (float*)y;
    EB_CUDA(launch_apply<float>(a, s));
  } else if (dtype == EB_F64) {
    ApplyArgs<double> a = apply_args<double>(st, kappa_weighted);
    a.phi = (const double*)phi;
    a.y = (double*)y;
    EB_CUDA(launch_apply<double>(a, s));
  } else {
    set_error("dtype must be EB_F32 or EB_F64");
    return EB_ERR_INVALID;
  }
  return EB_OK;
}

eb_status eb_bc_rhs(const eb_stencils* st, const double* g_eb, const double* g_wall, double* Bg,
                    int32_t kappa_weighted, eb_stream_t stream) {
  if (!st || !Bg) { set_error("null argument"); return EB_ERR_INVALID; }
  if ((st->dm.n_cut > 0 && !g_eb) || (st->n_wall > 0 && !g_wall)) { set_error("missing boundary data"); return EB_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  EB_CUDA(vec_fill64(st->dm.ncell, Bg, 0.0, s));
  EB_CUDA(launch_bg(st->n_irr, st->irr_cell, st->b_ptr, st->b_col, st->b_val, st->dm.n_grid_faces, st->b_wpos, g_eb,
                    g_wall, st->inv_kappa, kappa_weighted, Bg, s));
  return EB_OK;
}

eb_status eb_norms(const eb_stencils* st, const double* err, double* out_host, eb_stream_t stream) {
  if (!st || !err || !out_host) { set_error("null argument"); return EB_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  double* d;
  EB_CUDA(cudaMallocAsync((void**)&d, 4 * sizeof(double), s));
  EB_CUDA(cudaMemsetAsync(d, 0, 4 * sizeof(double), s));
  EB_CUDA(launch_norms(st->dm.ncell, st->flag, st->kappa, err, d, s));
  double h[4];
  EB_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaFreeAsync(d, s));
  EB_CUDA(cudaStreamSynchronize(s));
  double sw = h[2] > 0 ? h[2] : 1.0;
  out_host[0] = h[3];
  out_host[1] = h[0] / sw;
  out_host[2] = sqrt(h[1] / sw);
  return EB_OK;
}

// the stencils' multigrid preconditioner, set up at its first use
static eb_status ensure_mg(const eb_stencils* st, cudaStream_t s) {
  if (!st->mg) {
    Multigrid* m = new Multigrid();
    MgFineInput in;
    in.dim = st->dm.dim;
    for (int d = 0; d < 3; ++d) in.n[d] = st->dm.n[d];
    in.h = st->dm.h;
    in.flag = st->flag;
    for (int d = 0; d < 3; ++d) {
      int dd = d < st->dm.dim ? d : 0;
      in.ff[d] = st->face_flag[dd];
      in.cf[d] = st->cutface_of[dd];
      in.fm[d] = st->face_mom[dd];
    }
    in.KFS = st->dm.KFS;
    in.dinv_high = st->dinv64;
    in.rows64 = st->rows64;
    in.rows32 = st->rows32;
    in.n_rows = st->n_rows;
    in.nfoot = st->nfoot;
    in.center = st->foot_center;
    in.irr_cell = st->irr_cell;
    in.irr_row = st->irr_row;
    in.n_irr = st->n_irr;
    in.kind = st->cell_kind;
    in.tmpl64 = st->tmpl64;
    in.tmpl32 = st->tmpl32;
    in.foot_off = st->foot_off;
    in.R = st->dm.R;
    in.box = st->dm.nbr_box;
    cudaError_t me = mg_setup(in, m, s);
    if (me != cudaSuccess) {
      mg_free(m);
      delete m;
      return cuda_status(me, "multigrid setup");
    }
    const_cast<eb_stencils*>(st)->mg = m;
  }
  return EB_OK;
}

eb_status eb_solve(const eb_stencils* st, const double* rho, const double* g_eb, const double* g_wall, double tol,
                   const eb_solve_opts* opts, double* phi, eb_solve_info* info, eb_stream_t stream) {
  if (!st || !rho || !phi) { set_error("null argument"); return EB_ERR_INVALID; }
  g_err.clear();
  eb_solve_opts o = {1, 1e-5, 20000, 30, 200000, 1, 1};
  if (opts) o = *opts;
  eb_solve_info loc;
  memset(&loc, 0, sizeof(loc));
  eb_solve_info* inf = info ? info : &loc;
  memset(inf, 0, sizeof(*inf));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = st->dm.ncell;
  Tmp tmp;
  tmp.s = s;
  double *bg, *rhs, *y64, *r64, *dscr;
  EB_TRY(tmp.get(&bg, n));
  EB_TRY(tmp.get(&rhs, n));
  EB_TRY(tmp.get(&y64, n));
  EB_TRY(tmp.get(&r64, n));
  EB_TRY(tmp.get(&dscr, 16));
  EB_TRY(eb_bc_rhs(st, g_eb, g_wall, bg, 1, stream));
  EB_CUDA(compute_rhs(n, st->flag, st->kappa, rho, bg, rhs, s));
  double bnorm = 0.0;
  EB_CUDA(norm2_64(n, rhs, dscr, &bnorm, s));
  if (bnorm == 0.0) bnorm = 1.0;
  ApplyArgs<double> A64 = apply_args<double>(st, 1);
  eb_status ret = EB_OK;
  const Multigrid* mg = nullptr;
  if (o.precond == 1) {
    EB_TRY(ensure_mg(st, s));
    mg = st->mg;
    inf->precond_blocks = mg->nblk;
  }
  void* timer = o.check_every < 0 ? new_apply_timer() : nullptr;  // check_every < 0: time every Krylov apply
  set_apply_timer(timer);
  struct TimerGuard {
    void*& t;
    eb_solve_info* inf;
    ~TimerGuard() {
      set_apply_timer(nullptr);
      double ms = 0;
      long long n = 0;
      if (t) free_apply_timer(t, &ms, &n);
      inf->apply_ms = ms;
      inf->n_applies = (int32_t)n;
    }
  } tg{timer, inf};
  if (o.mixed) {
    float *w32, *b32, *x32;
    EB_TRY(tmp.get(&w32, 8 * n));
    EB_TRY(tmp.get(&b32, n));
    EB_TRY(tmp.get(&x32, n));
    ApplyArgs<float> A32 = apply_args<float>(st, 1);
    int total = 0;
    bool phi_nonzero = true;  // a zero initial guess needs no FP64 apply for the first residual
    EB_CUDA(any_nonzero64(n, phi, reinterpret_cast<int32_t*>(dscr), &phi_nonzero, s));
    for (int sweep = 0;; ++sweep) {
      if (sweep > 0 || phi_nonzero) {
        A64.phi = phi;
        A64.y = y64;
        EB_CUDA(launch_apply<double>(A64, s));
      } else {
        EB_CUDA(vec_fill64(n, y64, 0.0, s));
      }
      EB_CUDA(resid64(n, rhs, y64, r64, s));
      double rn = 0.0;
      EB_CUDA(norm2_64(n, r64, dscr, &rn, s));
      inf->rel_residual = rn / bnorm;
      if (inf->n_history < 64) inf->history[inf->n_history++] = inf->rel_residual;
      if (inf->rel_residual <= tol) break;
      if (sweep >= o.max_outer || total >= o.max_iters) { ret = EB_ERR_NOT_CONVERGED; break; }
      EB_CUDA(to32(n, r64, 1.0 / rn, b32, s));
      EB_CUDA(fill32(n, x32, 0.0f, s));
      int it = 0;
      double rr = 0.0;
      int cap = std::min(o.max_inner, o.max_iters - total);
      EB_CUDA(bicgstab<float>(A32, b32, x32, st->dinv32, w32, n, o.inner_tol, cap, dscr, &it, &rr, s, mg));
      total += it;
      inf->sweeps = sweep + 1;
      if (!isfinite(rr)) {  // an FP32 breakdown produced no usable correction: stop, phi unchanged
        ret = EB_ERR_NOT_CONVERGED;
        set_error("FP32 inner solve broke down (non-finite residual)");
        break;
      }
      EB_CUDA(add32(n, phi, rn, x32, s));
    }
    inf->iterations = total;
  } else {
    double* w64;
    EB_TRY(tmp.get(&w64, 8 * n));
    int it = 0;
    double rr = 0.0;
    EB_CUDA(bicgstab<double>(A64, rhs, phi, st->dinv64, w64, n, tol, o.max_iters, dscr, &it, &rr, s, mg));
    inf->iterations = it;
    A64.phi = phi;
    A64.y = y64;
    EB_CUDA(launch_apply<double>(A64, s));
    EB_CUDA(resid64(n, rhs, y64, r64, s));
    double rn = 0.0;
    EB_CUDA(norm2_64(n, r64, dscr, &rn, s));
    inf->rel_residual = rn / bnorm;
    inf->history[0] = inf->rel_residual;
    inf->n_history = 1;
    if (inf->rel_residual > tol * 10) ret = EB_ERR_NOT_CONVERGED;
  }
  EB_CUDA(cudaStreamSynchronize(s));
  if (st->plan && st->plan->err) {
    int32_t h = 0;
    EB_CUDA(cudaMemcpy(&h, st->plan->err, 4, cudaMemcpyDeviceToHost));
    if (h) { set_error("a bounded device wait gave up in the operator apply"); return EB_ERR_TIMEOUT; }
  }
  if (ret != EB_OK && g_err.empty()) set_error("solve did not reach the requested tolerance");
  return ret;
}

}  // extern "C"

struct eb_batch_solver {
  std::vector<const eb_stencils*> st;
  eb_solve_opts o;
  std::vector<BatchSys> sys;
  BatchCtl* ctl = nullptr;  // device [n]
  std::vector<void*> mem;   // device arrays
  // copies of each system's apply plan for the two captured loop bodies, each with its own side
  // stream and events (a stream joins one capture at a time)
  std::deque<ApplyPlan> plans;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

void eb_batch_solver_destroy(eb_batch_solver* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (ApplyPlan& pl : b->plans) {
    if (pl.fork) cudaEventDestroy(pl.fork);
    if (pl.join) cudaEventDestroy(pl.join);
    if (pl.side) cudaStreamDestroy(pl.side);
  }
  for (void* p : b->mem) cudaFree(p);
  delete b;
}

eb_status eb_batch_solver_create(const eb_stencils* const* st, int32_t n, const eb_solve_opts* opts,
                                 eb_batch_solver** out, eb_stream_t stream) {
  if (!st || !out || n < 1) { set_error("eb_batch_solver_create: null argument or empty batch"); return EB_ERR_INVALID; }
  *out = nullptr;
  g_err.clear();
  eb_solve_opts o = {1, 1e-5, 20000, 30, 200000, 1, 1};
  if (opts) o = *opts;
  if (!o.mixed) { set_error("eb_batch_solver_create: the batched solve is the mixed-precision refinement"); return EB_ERR_INVALID; }
  if (o.max_inner < 1 || o.max_outer < 1 || o.max_iters < 1 || !(o.inner_tol > 0.0)) {
    set_error("eb_batch_solver_create: iteration caps must be positive and inner_tol > 0");
    return EB_ERR_INVALID;
  }
  for (int32_t k = 0; k < n; ++k)
    if (!st[k]) { set_error("eb_batch_solver_create: null stencils"); return EB_ERR_INVALID; }
  {
    // a stencil set's multigrid vectors and apply scratch serve one system of the graph at a time
    std::vector<const eb_stencils*> seen(st, st + n);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) {
      set_error("eb_batch_solver_create: a stencil set appears twice in the batch");
      return EB_ERR_INVALID;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  eb_batch_solver* b = new eb_batch_solver();
  b->o = o;
  b->st.assign(st, st + n);
  auto fail = [&](eb_status r) {
    eb_batch_solver_destroy(b);
    return r;
  };
  auto get = [&](void** p, size_t bytes) -> eb_status {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return cuda_status(e, "batched solve allocation");
    b->mem.push_back(*p);
    return EB_OK;
  };
  eb_status r;
  if ((r = get((void**)&b->ctl, sizeof(BatchCtl) * n)) != EB_OK) return fail(r);
  b->sys.resize(n);
  for (int32_t k = 0; k < n; ++k) {
    const eb_stencils* S = st[k];
    if (o.precond == 1 && (r = ensure_mg(S, s)) != EB_OK) return fail(r);
    BatchSys& y = b->sys[k];
    y = BatchSys();
    y.n = S->dm.ncell;
    y.A64 = apply_args<double>(S, 1);
    y.A32 = apply_args<float>(S, 1);
    if (S->plan) {
      for (int c = 0; c < 2; ++c) {
        b->plans.push_back(*S->plan);
        ApplyPlan& pl = b->plans.back();
        pl.side = nullptr;
        pl.fork = pl.join = nullptr;
        cudaError_t e = S->plan->side ? cudaStreamCreateWithFlags(&pl.side, cudaStreamNonBlocking) : cudaSuccess;
        if (e == cudaSuccess && S->plan->side) e = cudaEventCreateWithFlags(&pl.fork, cudaEventDisableTiming);
        if (e == cudaSuccess && S->plan->side) e = cudaEventCreateWithFlags(&pl.join, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(cuda_status(e, "batched solve streams"));
        (c == 0 ? y.A64.plan : y.A32.plan) = &pl;
      }
    }
    y.mg = o.precond == 1 ? S->mg : nullptr;
    y.dinv32 = S->dinv32;
    const size_t n8 = (size_t)y.n * 8, n4 = (size_t)y.n * 4;
    void* p;
    if ((r = get(&p, 4 * n8)) != EB_OK) return fail(r);
    y.rhs = (double*)p;
    y.phi = y.rhs + y.n;
    y.y64 = y.phi + y.n;
    y.r64 = y.y64 + y.n;
    if ((r = get(&p, 10 * n4)) != EB_OK) return fail(r);
    y.w32 = (float*)p;
    y.b32 = y.w32 + 8 * y.n;
    y.x32 = y.b32 + y.n;
    if ((r = get(&p, (SC_N + 2) * 8)) != EB_OK) return fail(r);
    y.sc = (double*)p;
    y.ctl = b->ctl + k;
  }
  EB_CUDA(cudaStreamSynchronize(s));
  cudaError_t e = batch_graph(b->sys, &b->graph, &b->exec, s);
  if (e != cudaSuccess) return fail(cuda_status(e, "batched solve graph"));
  *out = b;
  return EB_OK;
}

eb_status eb_batch_solve(eb_batch_solver* b, const double* const* rho, const double* const* g_eb,
                         const double* const* g_wall, double tol, double* const* phi, eb_solve_info* infos,
                         eb_stream_t stream) {
  if (!b || !rho || !phi) { set_error("eb_batch_solve: null argument"); return EB_ERR_INVALID; }
  g_err.clear();
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t n = (int32_t)b->sys.size();
  std::vector<BatchCtl> h(n);
  for (int32_t k = 0; k < n; ++k) {
    const eb_stencils* S = b->st[k];
    BatchSys& y = b->sys[k];
    if (!rho[k] || !phi[k]) { set_error("eb_batch_solve: null rho or phi"); return EB_ERR_INVALID; }
    EB_TRY(eb_bc_rhs(S, g_eb ? g_eb[k] : nullptr, g_wall ? g_wall[k] : nullptr, y.y64, 1, stream));
    EB_CUDA(compute_rhs(y.n, S->flag, S->kappa, rho[k], y.y64, y.rhs, s));
    EB_CUDA(cudaMemcpyAsync(y.phi, phi[k], (size_t)y.n * 8, cudaMemcpyDeviceToDevice, s));
    BatchCtl& c = h[k];
    memset(&c, 0, sizeof(c));
    c.tol = tol;
    c.inner_tol = b->o.inner_tol;
    c.max_outer = b->o.max_outer;
    c.max_inner = b->o.max_inner;
    c.max_iters = b->o.max_iters;
  }
  // the control blocks up to the loop handles, which the graph owns
  for (int32_t k = 0; k < n; ++k)
    EB_CUDA(cudaMemcpyAsync(b->ctl + k, &h[k], offsetof(BatchCtl, ho), cudaMemcpyHostToDevice, s));
  for (int32_t k = 0; k < n; ++k) EB_CUDA(batch_dots(b->sys[k].n, b->sys[k].rhs, &b->ctl[k].bnorm2, s));
  EB_CUDA(cudaGraphLaunch(b->exec, s));
  for (int32_t k = 0; k < n; ++k)
    EB_CUDA(cudaMemcpyAsync(phi[k], b->sys[k].phi, (size_t)b->sys[k].n * 8, cudaMemcpyDeviceToDevice, s));
  EB_CUDA(cudaMemcpyAsync(h.data(), b->ctl, sizeof(BatchCtl) * n, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  eb_status ret = EB_OK;
  for (int32_t k = 0; k < n; ++k) {
    const BatchCtl& c = h[k];
    eb::count_launches((long long)c.runs * b->sys[k].k_sweep + (long long)c.total * b->sys[k].k_iter);
    if (infos) {
      eb_solve_info& f = infos[k];
      memset(&f, 0, sizeof(f));
      f.iterations = c.total;
      f.sweeps = c.sweeps;
      f.rel_residual = c.rel_residual;
      f.n_history = std::min(c.n_hist, 64);
      for (int i = 0; i < f.n_history; ++i) f.history[i] = c.hist[i];
      f.precond_blocks = b->sys[k].mg ? b->sys[k].mg->nblk : 0;
    }
    if (c.status != 1 && ret == EB_OK) {
      ret = EB_ERR_NOT_CONVERGED;
      set_error("eb_batch_solve: system " + std::to_string(k) +
                (c.status == 3 ? " broke down (non-finite residual)" : " did not reach the tolerance within the caps"));
    }
    const eb_stencils* S = b->st[k];
    if (S->plan && S->plan->err) {
      int32_t fl = 0;
      EB_CUDA(cudaMemcpy(&fl, S->plan->err, 4, cudaMemcpyDeviceToHost));
      if (fl) { set_error("a bounded device wait gave up in the operator apply"); return EB_ERR_TIMEOUT; }
    }
  }
  return ret;
}

eb_status eb_wall_faces(const eb_stencils* st, int64_t* ids_host, int64_t cap, int64_t* n) {
  if (!st || !n) { set_error("null argument"); return EB_ERR_INVALID; }
  *n = st->n_wall;
  for (int64_t i = 0; i < cap && i < st->n_wall && ids_host; ++i) ids_host[i] = st->wall_ids_host[i];
  return EB_OK;
}

eb_status eb_stencil_query(const eb_stencils* st, int64_t face, int32_t* n, int64_t* cols_host, double* coef_host,
                           int32_t cap, eb_stream_t stream) {
  if (!st || !n) { set_error("null argument"); return EB_ERR_INVALID; }
  const Dims& dm = st->dm;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t slot = -1;
  int base[3] = {0, 0, 0};
  if (face < 0 || face >= dm.n_grid_faces + dm.n_cut) { set_error("face id out of range"); return EB_ERR_INVALID; }
  if (face >= dm.n_grid_faces) {
    int64_t cut = face - dm.n_grid_faces;
    EB_CUDA(cudaMemcpyAsync(&slot, st->eb_slot + cut, 4, cudaMemcpyDeviceToHost, s));
    int32_t c = 0;
    EB_CUDA(cudaMemcpyAsync(&c, st->cut_cell + cut, 4, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    base[0] = c % dm.n[0];
    base[1] = (c / dm.n[0]) % dm.n[1];
    base[2] = c / (dm.n[0] * dm.n[1]);
  } else {
    int d = 0;
    for (int k = 0; k < dm.dim; ++k)
      if (face >= dm.face_base[k]) d = k;
    int64_t f = face - dm.face_base[d];
    EB_CUDA(cudaMemcpyAsync(&slot, st->face_slot[d] + f, 4, cudaMemcpyDeviceToHost, s));
    EB_CUDA(cudaStreamSynchronize(s));
    int64_t m0 = dm.n[0] + (d == 0), m1 = dm.n[1] + (d == 1);
    base[0] = (int)(f % m0);
    base[1] = (int)((f / m0) % m1);
    base[2] = (int)(f / (m0 * m1));
  }
  if (slot < 0) { *n = 0; return EB_OK; }
  int64_t rp[2];
  EB_CUDA(cudaMemcpyAsync(rp, st->row_ptr + slot, 16, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  int32_t cnt = (int32_t)(rp[1] - rp[0]);
  *n = cnt;
  if (!cols_host) return EB_OK;
  if (cap < cnt) { set_error("capacity too small"); return EB_ERR_INVALID; }
  std::vector<uint32_t> desc(cnt);
  EB_CUDA(cudaMemcpyAsync(desc.data(), st->row_desc + rp[0], cnt * 4, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaMemcpyAsync(coef_host, st->row_val + rp[0], cnt * 8, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  for (int32_t i = 0; i < cnt; ++i) {
    uint32_t ds = desc[i];
    int c[3];
    for (int d = 0; d < 3; ++d) c[d] = base[d] + (d < dm.dim ? rd_off(ds, d) : 0);
    int64_t cid = (int64_t)c[0] + (int64_t)dm.n[0] * ((int64_t)c[1] + (int64_t)dm.n[1] * c[2]);
    int kind = rd_kind(ds);
    if (kind == 0) cols_host[i] = cid;
    else if (kind == 1) {
      int32_t cut = -1;
      EB_CUDA(cudaMemcpy(&cut, st->cut_of_cell + cid, 4, cudaMemcpyDeviceToHost));
      cols_host[i] = -(1 + dm.n_grid_faces + cut);
    } else {
      int wd = rd_wdir(ds);
      if (rd_wside(ds)) c[wd] += 1;
      int64_t m0 = dm.n[0] + (wd == 0), m1 = dm.n[1] + (wd == 1);
      cols_host[i] = -(1 + dm.face_base[wd] + c[0] + m0 * ((int64_t)c[1] + m1 * c[2]));
    }
  }
  return EB_OK;
}

}  // extern "C"

// ================================================================= FP64 FMA throughput probe

namespace eb {
// eight independent FMA chains per thread; the sum keeps them live
__global__ void k_dfma_probe(int64_t iters, double seed, double* sink) {
  double a[8];
  for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x + k;
  const double m = 0.9999999, c = 1e-9;
  for (int64_t i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  double t = 0.0;
  for (int k = 0; k < 8; ++k) t += a[k];
  if (t == 1234.5678) *sink = t;
}
}  // namespace eb

extern "C" eb_status eb_fp64_fma_rate(int32_t blocks_per_sm, int64_t iters, double* tflops_host, eb_stream_t stream) {
  if (!tflops_host || blocks_per_sm < 1 || iters < 1) { set_error("eb_fp64_fma_rate: bad argument"); return EB_ERR_INVALID; }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  EB_CUDA(cudaGetDevice(&dev));
  EB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  double* sink;
  EB_CUDA(cudaMallocAsync((void**)&sink, 8, s));
  cudaEvent_t e0, e1;
  EB_CUDA(cudaEventCreate(&e0));
  EB_CUDA(cudaEventCreate(&e1));
  const unsigned blocks = (unsigned)(nsm * blocks_per_sm);
  k_dfma_probe<<<blocks, 256, 0, s>>>(iters / 8 + 1, 1.0, sink);  // warm-up
  EB_CUDA(cudaEventRecord(e0, s));
  k_dfma_probe<<<blocks, 256, 0, s>>>(iters, 1.0, sink);
  EB_CUDA(cudaEventRecord(e1, s));
  eb::count_launches(2);
  EB_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  EB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  EB_CUDA(cudaFreeAsync(sink, s));
  *tflops_host = 2.0 * 8.0 * (double)iters * blocks * 256.0 / (ms * 1e-3) / 1e12;
  return EB_OK;
}

// ================================================================= adjoint with respect to the radii

namespace eb {

// rhs = kappa h^D phi (the gradient of J = 1/2 sum |V| phi^2) and v = (kappa h^D)^(1/2) phi (J = |v|^2 / 2)
__global__ void k_adj_rhs(int64_t n, const uint8_t* flag, const double* kappa, const double* phi, double hd,
                          double* rhs, double* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double w = flag[i] ? kappa[i] * hd : 0.0;
  rhs[i] = w * phi[i];
  v[i] = sqrt(w) * phi[i];
}

__global__ void k_adj_rowmap(int64_t n_irr, const int32_t* irr_cell, const int32_t* irr_row, int32_t* row_of) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_irr) row_of[irr_cell[t]] = irr_row[t];
}

// sum over the cut cells of (h^D phi^2 / 2 + lam) d kappa (kappa = the zeroth volume moment)
__global__ void k_adj_kappa(int64_t n_cut, const int32_t* cut_cell, const double* dvol, int KS, const double* phi,
                            const double* lam, double hd, double* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (t < n_cut) {
    const int32_t c = cut_cell[t];
    v = (0.5 * hd * phi[c] * phi[c] + lam[c]) * dvol[t * KS];
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

}  // namespace eb

namespace {

// timing events, destroyed with the scope
struct Events {
  cudaEvent_t e[4] = {};
  int n = 0;
  cudaError_t create(int k) {
    for (; n < k; ++n) {
      const cudaError_t r = cudaEventCreate(&e[n]);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  }
  ~Events() {
    for (int i = 0; i < n; ++i) cudaEventDestroy(e[i]);
  }
};

// J and, when dJ_host is given, dJ/dp for the boundary velocities vel (one parameter each)
eb_status adjoint_shape(const eb_geometry* g, const eb_stencils* st, const double* phi,
                        const std::vector<ShapeVel>& vel, double* J_host, double* dJ_host, eb_adjoint_info* info,
                        cudaStream_t s) {
  g_err.clear();
  const Dims& dm = st->dm;
  if (!geometry_matches(g, dm.dim, dm.n, dm.n_cut)) {
    set_error("eb_adjoint: the stencils were not built from this geometry");
    return EB_ERR_INVALID;
  }
  const int64_t n = dm.ncell;
  const double hd = pow(dm.h, dm.dim);
  Tmp tmp;
  tmp.s = s;
  double *rhs, *v, *dscr;
  EB_TRY(tmp.get(&rhs, n));
  EB_TRY(tmp.get(&v, n));
  EB_TRY(tmp.get(&dscr, 16));
  k_adj_rhs<<<nblk(n, 256), 256, 0, s>>>(n, st->flag, st->kappa, phi, hd, rhs, v);
  eb::count_launch();
  double nv = 0.0;
  EB_CUDA(norm2_64(n, v, dscr, &nv, s));
  *J_host = 0.5 * nv * nv;
  if (!dJ_host) return EB_OK;
  // ---- adjoint solve (kappa L)^T lam = kappa h^D phi: BiCGStab on the transposed operator (gather
  // form), Jacobi (the transpose has the same diagonal)
  double *lam, *work;
  int32_t* row_of;
  EB_TRY(tmp.get(&lam, n));
  EB_TRY(tmp.get(&work, 8 * n));
  EB_TRY(tmp.get(&row_of, n));
  EB_CUDA(cudaMemsetAsync(lam, 0, n * 8, s));
  EB_CUDA(cudaMemsetAsync(row_of, 0xFF, n * 4, s));
  if (st->n_irr > 0) {
    k_adj_rowmap<<<nblk(st->n_irr, 256), 256, 0, s>>>(st->n_irr, st->irr_cell, st->irr_row, row_of);
    eb::count_launch();
  }
  ApplyArgs<double> AT = apply_args<double>(st, 1);
  AT.transpose = 1;
  AT.row_of_cell = row_of;
  AT.foot_d = st->foot_d;
  AT.nx = dm.n[0];
  AT.ny = dm.n[1];
  AT.nz = dm.n[2];
  int it = 0;
  double rr = 0.0;
  Events ev;
  EB_CUDA(ev.create(4));
  EB_CUDA(cudaEventRecord(ev.e[0], s));
  if (st->mg) {
    // the forward solve's multigrid, its block solves transposed; Jacobi if that does not converge
    Multigrid* mg = st->mg;
    mg->transpose = 1;
    const cudaError_t e = bicgstab<double>(AT, rhs, lam, st->dinv64, work, n, 1e-12, 2000, dscr, &it, &rr, s, mg);
    mg->transpose = 0;
    EB_CUDA(e);
  }
  if (!st->mg || !(rr <= 1e-10)) {
    EB_CUDA(cudaMemsetAsync(lam, 0, n * 8, s));
    int it2 = 0;
    EB_CUDA(bicgstab<double>(AT, rhs, lam, st->dinv64, work, n, 1e-12, 20000, dscr, &it2, &rr, s, nullptr));
    it += it2;
  }
  EB_CUDA(cudaEventRecord(ev.e[1], s));
  if (info) {
    info->iterations = it;
    info->rel_residual = rr;
  }
  if (!(rr <= 1e-10)) { set_error("eb_adjoint: the adjoint solve did not converge"); return EB_ERR_NOT_CONVERGED; }
  // ---- per parameter: the moment tables' derivatives and the kappa terms; then one pass of the
  // stencil-solve adjoints over all parameters
  Tables T;
  if (!make_tables(dm.dim, dm.order, dm.mdeg, &T)) { set_error("table construction failed"); return EB_ERR_INVALID; }
  LsArgs la;
  memset(&la, 0, sizeof(la));
  la.dm = dm;
  la.flag = st->flag;
  la.cut_of_cell = st->cut_of_cell;
  la.cut_cell = st->cut_cell;
  la.vol_mom = st->vol_mom;
  la.eb_mom = st->eb_mom;
  la.eb_nmom = st->eb_nmom;
  la.eb_bc = st->eb_bc;
  for (int d = 0; d < 3; ++d) {
    la.cutface_of[d] = d < dm.dim ? st->cutface_of[d] : st->cutface_of[0];
    la.face_mom[d] = d < dm.dim ? st->face_mom[d] : st->face_mom[0];
  }
  la.slot_face = st->slot_face;
  la.row_ptr = st->row_ptr;
  la.row_desc = st->row_desc;
  int32_t *next, *lerr;
  EB_TRY(tmp.get(&next, 1));
  EB_TRY(tmp.get(&lerr, 1));
  EB_CUDA(cudaMemsetAsync(lerr, 0, 4, s));
  la.err = lerr;
  int dev = 0, nsm = 0;
  EB_CUDA(cudaGetDevice(&dev));
  EB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t nu = st->n_unique;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * 4, (nu + ADJ_WARPS - 1) / ADJ_WARPS));
  double* scratch;
  EB_TRY(tmp.get(&scratch, (size_t)blocks * ADJ_WARPS * MAXROWS * ADJ_SCRATCH));
  const int KS = dm.KS, KFS = dm.KFS, nc = dm.n_cut;
  const int np = (int)vel.size();
  AdjArgs ga;
  memset(&ga, 0, sizeof(ga));
  ga.s_vol = (int64_t)std::max(1, nc) * KS;
  ga.s_ebn = ga.s_vol * dm.dim;
  double *dvol, *deb, *debn, *acc;
  EB_TRY(tmp.get(&dvol, (size_t)np * ga.s_vol));
  EB_TRY(tmp.get(&deb, (size_t)np * ga.s_vol));
  EB_TRY(tmp.get(&debn, (size_t)np * ga.s_ebn));
  double* dface[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < dm.dim; ++d) {
    ga.s_face[d] = std::max<int64_t>(1, geometry_cutfaces(g, d)) * KFS;
    EB_TRY(tmp.get(&dface[d], (size_t)np * ga.s_face[d]));
  }
  EB_TRY(tmp.get(&acc, std::max(1, np)));
  EB_CUDA(cudaMemsetAsync(acc, 0, std::max(1, np) * 8, s));
  for (int p = 0; p < np; ++p) {
    double* dfp[3] = {nullptr, nullptr, nullptr};
    for (int d = 0; d < dm.dim; ++d) dfp[d] = dface[d] + p * ga.s_face[d];
    EB_CUDA(geometry_shape_derivative(g, vel[p], dvol + p * ga.s_vol, deb + p * ga.s_vol, debn + p * ga.s_ebn, dfp, s));
    if (nc > 0) {
      k_adj_kappa<<<nblk(nc, 256), 256, 0, s>>>(nc, st->cut_cell, dvol + p * ga.s_vol, KS, phi, lam, hd, acc + p);
      eb::count_launch();
    }
  }
  EB_CUDA(cudaEventRecord(ev.e[2], s));
  ga.lam = lam;
  ga.phi = phi;
  ga.dvol = dvol;
  ga.deb = deb;
  ga.debn = debn;
  for (int d = 0; d < 3; ++d) {
    ga.dface[d] = d < dm.dim ? dface[d] : dface[0];
    if (d >= dm.dim) ga.s_face[d] = ga.s_face[0];
  }
  ga.n_par = np;
  ga.n_slots = nu;
  ga.next = next;
  ga.scratch = scratch;
  ga.dJ = acc;
  EB_CUDA(cudaMemsetAsync(next, 0, 4, s));
  if (nu > 0 && np > 0) {
    EB_CUDA(stencil_adjoint_launch(blocks, s, la, T, ga));
    eb::count_launch();
  }
  EB_CUDA(cudaEventRecord(ev.e[3], s));
  std::vector<double> h(std::max(1, np));
  int32_t herr = 0;
  EB_CUDA(cudaMemcpyAsync(h.data(), acc, std::max(1, np) * 8, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaMemcpyAsync(&herr, lerr, 4, cudaMemcpyDeviceToHost, s));
  EB_CUDA(cudaStreamSynchronize(s));
  if (info) {
    float ms[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < 3; ++k) EB_CUDA(cudaEventElapsedTime(&ms[k], ev.e[k], ev.e[k + 1]));
    info->solve_ms = ms[0];
    info->tables_ms = ms[1];
    info->stencils_ms = ms[2];
  }
  if (herr) { set_error("eb_adjoint: a stencil system was singular in the adjoint"); return EB_ERR_RANK_DEFICIENT; }
  for (int p = 0; p < np; ++p) dJ_host[p] = h[p];
  return EB_OK;
}

}  // namespace

extern "C" eb_status eb_adjoint_radii(const eb_geometry* g, const eb_stencils* st, const double* phi, double* J_host,
                                      double* dJ_host, eb_stream_t stream) {
  if (!g || !st || !phi || !J_host) { set_error("eb_adjoint_radii: null argument"); return EB_ERR_INVALID; }
  std::vector<ShapeVel> vel(geometry_bodies(g));
  for (size_t b = 0; b < vel.size(); ++b) {
    memset(&vel[b], 0, sizeof(ShapeVel));
    vel[b].kind = 0;
    vel[b].body = (int)b;
  }
  return adjoint_shape(g, st, phi, vel, J_host, dJ_host, nullptr, (cudaStream_t)stream);
}

extern "C" eb_status eb_adjoint_shape(const eb_geometry* g, const eb_stencils* st, const double* phi,
                                      int32_t n_modes, const double* modes_host, double* J_host,
                                      double* dJ_radii_host, double* dJ_modes_host, eb_adjoint_info* info,
                                      eb_stream_t stream) {
  if (!g || !st || !phi || !J_host || n_modes < 0 || (n_modes > 0 && !modes_host)) {
    set_error("eb_adjoint_shape: null argument or negative mode count");
    return EB_ERR_INVALID;
  }
  const int nb = geometry_bodies(g);
  const bool want = dJ_radii_host || dJ_modes_host;
  if (want && ((!dJ_radii_host && nb > 0) || (!dJ_modes_host && n_modes > 0))) {
    set_error("eb_adjoint_shape: give the derivative arrays of both the radii and the modes, or neither");
    return EB_ERR_INVALID;
  }
  std::vector<ShapeVel> vel(nb + n_modes);
  for (int p = 0; p < nb + n_modes; ++p) {
    memset(&vel[p], 0, sizeof(ShapeVel));
    if (p < nb) {
      vel[p].kind = 0;
      vel[p].body = p;
    } else {
      const double* m = modes_host + 4 * (p - nb);
      vel[p].kind = 1;
      for (int d = 0; d < 3; ++d) vel[p].k[d] = m[d];
      vel[p].theta = m[3];
    }
  }
  if (!want) return adjoint_shape(g, st, phi, vel, J_host, nullptr, info, (cudaStream_t)stream);
  std::vector<double> dj(std::max<size_t>(1, vel.size()));
  const eb_status r = adjoint_shape(g, st, phi, vel, J_host, dj.data(), info, (cudaStream_t)stream);
  if (r != EB_OK) return r;
  for (int b = 0; b < nb; ++b) dJ_radii_host[b] = dj[b];
  for (int m = 0; m < n_modes; ++m) dJ_modes_host[m] = dj[nb + m];
  return EB_OK;
}
