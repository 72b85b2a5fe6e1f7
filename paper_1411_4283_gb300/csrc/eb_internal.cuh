// Internal definitions shared by the library's translation units.
// Paper: Devendran, Graves, Johansen, "A higher-order finite-volume
// discretization method for Poisson's equation in cut cell geometries"
// (arXiv:1411.4283).  Section references are to that paper.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/eb.h"
#include "eb_apply.cuh"
#include "eb_mg.cuh"

struct eb_geometry;

namespace eb {

// A normal velocity of the embedded boundary, along N = (x - c)/r (out of each body), for the moment
// tables' shape derivatives (eb_geom.cu): kind 0 the radius of body `body` (unit speed on its boundary);
// kind 1 the amplitude a of the level-set mode a sin(2 pi k . x + theta) added to the distance function
// of every body, at a = 0 (speed -sin(...) outside the bodies, +sin(...) inside one).
struct ShapeVel {
  int kind, body;
  double k[3], theta;
};
// the tables' derivatives for sv, laid out like the tables (eb_geom.cu)
cudaError_t geometry_shape_derivative(const eb_geometry* g, const ShapeVel& sv, double* dvol, double* deb,
                                      double* debn, double* const* dface, cudaStream_t s);
int geometry_bodies(const eb_geometry* g);
int64_t geometry_cutfaces(const eb_geometry* g, int d);
bool geometry_matches(const eb_geometry* g, int dim, const int* n, int n_cut);

constexpr int MAXK = 35;        // monomials of degree <= 4 in 3-D
constexpr int MAXK_STORE = 84;  // stored moment tables up to degree 6 in 3-D
constexpr int MAXROWS = 640;    // LS rows per face supported by the LS kernel
constexpr int MAX_FOOT = 637;   // operator footprint (3-D, R_n = 3, box neighbourhood)

// Row descriptor of one LS row, relative to the face's base cell (the high
// cell of a grid face; the cut cell of an EB face):
//   bits 0-1  kind: 0 volume, 1 EB face of the cut cell at the offset, 2 wall face
//   bits 2-3  wall direction, bit 4 wall side (0 low wall, 1 high wall)
//   bits 8-11, 12-15, 16-19: offsets dx, dy, dz (signed 4 bit)
__host__ __device__ inline uint32_t rd_pack(int kind, int wdir, int wside, int dx, int dy, int dz) {
  return (uint32_t)kind | ((uint32_t)wdir << 2) | ((uint32_t)wside << 4) | (((uint32_t)dx & 15u) << 8) |
         (((uint32_t)dy & 15u) << 12) | (((uint32_t)dz & 15u) << 16);
}
__host__ __device__ inline int rd_kind(uint32_t r) { return (int)(r & 3u); }
__host__ __device__ inline int rd_wdir(uint32_t r) { return (int)((r >> 2) & 3u); }
__host__ __device__ inline int rd_wside(uint32_t r) { return (int)((r >> 4) & 1u); }
__host__ __device__ inline int rd_off(uint32_t r, int d) {
  int v = (int)((r >> (8 + 4 * d)) & 15u);
  return v >= 8 ? v - 16 : v;
}

// Geometry and discretisation constants visible to the kernels.
struct Dims {
  int dim;
  int n[3];
  int64_t ncell;
  int64_t nface[3];       // faces normal to d
  int64_t face_base[3];   // global id of the first face normal to d
  int64_t n_grid_faces;
  int order, K, R;        // Q, monomial count, path radius
  int nbr_box;            // 1: box neighbourhoods
  int weighted;
  double w_threshold, w_power;
  int mdeg, KS, KFS;      // stored moment degree, its D-dim and (D-1)-dim monomial counts
  double h;
  int n_cut;
};

// Device-resident library state (owned by eb_stencils).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace eb

namespace eb {
// Bump allocation state over chunks of pooled device memory (see arena_alloc in eb_api.cu).
struct Arena {
  char* cur = nullptr;
  size_t left = 0;
  size_t next = (size_t)1 << 20;  // size of the next chunk
};
}  // namespace eb

struct eb_stencils {
  eb::Dims dm;
  // geometry copies
  uint8_t* flag = nullptr;        // [ncell]
  double* kappa = nullptr;        // [ncell] (0 covered)
  int32_t* cut_cell = nullptr;    // [n_cut]
  int32_t* cut_of_cell = nullptr; // [ncell] -> cut index or -1
  double* vol_mom = nullptr;      // [n_cut][KS]
  double* eb_mom = nullptr;       // [n_cut][KS]
  double* eb_nmom = nullptr;      // [n_cut][dim][KS]
  uint8_t* eb_bc = nullptr;       // [n_cut]
  uint8_t* face_flag[3] = {nullptr, nullptr, nullptr};
  int32_t* cutface_of[3] = {nullptr, nullptr, nullptr};  // [nface_d] -> cut-face index or -1
  double* face_mom[3] = {nullptr, nullptr, nullptr};
  // stencils: slots (unique faces first, then class representatives)
  int64_t n_slots = 0, n_unique = 0;
  int32_t n_classes = 0;
  int64_t* slot_face = nullptr;     // [n_slots] global face id solved for that slot
  int64_t* row_ptr = nullptr;       // [n_slots + 1]
  uint32_t* row_desc = nullptr;     // [nnz] row descriptors
  double* row_val = nullptr;        // [nnz] s_hat
  int32_t* face_slot[3] = {nullptr, nullptr, nullptr};  // [nface_d] slot per grid face (-1 closed)
  int32_t* eb_slot = nullptr;       // [n_cut]
  // operator rows (kappa-weighted, h^2 included): footprint-dense
  int nfoot = 0;
  int32_t* foot_off = nullptr;      // [nfoot] linear cell offset of each footprint entry
  int foot_center = 0;              // footprint index of the zero offset
  int8_t* foot_d = nullptr;         // [nfoot][3] offsets
  int64_t n_irr = 0;                // cells with a non-template row
  int32_t n_row_classes = 0;        // shared rows (class rows incl. template = row 0)
  int32_t* irr_cell = nullptr;      // [n_irr] ascending cell index
  int32_t* irr_row = nullptr;       // [n_irr] row index into rows_*
  int64_t n_rows = 0;               // n_row_classes + unique rows
  double* rows64 = nullptr;         // [nfoot][n_rows] (row-minor: coalesced across rows)
  float* rows32 = nullptr;          // [nfoot][n_rows]
  uint8_t* cell_kind = nullptr;     // [ncell]: 0 covered, 1 template, 2 irregular
  // template row for the fast pass
  double* tmpl64 = nullptr;         // [nfoot]
  float* tmpl32 = nullptr;
  // boundary matrix B (kappa-weighted), CSR over irregular cells
  int64_t* b_ptr = nullptr;         // [n_irr + 1]
  int64_t* b_col = nullptr;         // global boundary face id
  double* b_val = nullptr;
  // wall faces in ascending id
  int64_t n_wall = 0;
  int64_t* wall_ids = nullptr;      // device
  std::vector<int64_t> wall_ids_host;
  eb::ApplyPlan* plan = nullptr;
  eb::Multigrid* mg = nullptr;     // geometric multigrid preconditioner (built at the first solve)
  int64_t* b_wpos = nullptr;       // [nnz(B)] position of a wall column in the wall list (-1: EB)
  double* dinv64 = nullptr;         // [ncell] inverse diagonal of kappa L (0 on covered cells)
  float* dinv32 = nullptr;
  double* inv_kappa = nullptr;      // [ncell] 1/kappa (0 on covered cells)
  // scratch for solves
  void* work = nullptr;
  size_t work_bytes = 0;
  std::vector<void*> allocs;       // device memory owned by the stencils (chunks and large arrays from the pool)
  cudaStream_t build_stream = nullptr;  // stream the arrays are allocated in
  eb::Arena arena;                 // the stencils' small arrays share chunks
};

namespace eb {

// error handling shared by the host code
void set_error(const std::string& msg);
eb_status cuda_status(cudaError_t e, const char* what);

#define EB_CUDA(call)                                              \
  do {                                                             \
    cudaError_t _e = (call);                                       \
    if (_e != cudaSuccess) return ::eb::cuda_status(_e, #call);    \
  } while (0)

// host helpers
std::vector<std::vector<int>> monomials(int dim, int q);
// cumulative number of kernel launches issued by the library (all threads)
void count_launch();
void count_launches(long long n);
void uncount_launches(long long n);
long long launches_so_far();

}  // namespace eb
