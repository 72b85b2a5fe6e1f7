// Argument structures of the build kernels (eb_build.cu), shared with the host code.
#pragma once
#include <stdint.h>

#include "eb_internal.cuh"
#include "eb_tables.cuh"

namespace eb {

constexpr int RW = 6;  // 64-bit words of a (2R+1)^3 <= 343-bit mask

struct Mask {
  uint64_t w[RW];
};

struct GatherArgs {
  Dims dm;
  const uint8_t* flag;
  const uint8_t* ff[3];
  const int32_t* reach_idx;  // [ncell] index into masks or -1 (clean: whole box / ball)
  const Mask* masks;
  const int32_t* cut_of_cell;
  const int64_t* slot_face;
  const int64_t* row_ptr;    // null in the counting pass
  uint32_t* row_desc;
  int64_t* count;            // [n_slots] counting pass output
  int32_t* too_many;         // capacity flag
};

// LS kernel shape (compile-time; EB_LS_SYS / EB_LS_SYS_F / EB_LS_RPL override it for tuning builds)
#ifndef EB_LS_SYS
#define EB_LS_SYS 4
#endif
#ifndef EB_LS_SYS_F
#define EB_LS_SYS_F 6
#endif
#ifndef EB_LS_RPL
#define EB_LS_RPL 4
#endif
constexpr int LS_SYS = EB_LS_SYS;      // systems in flight per CTA, FP64 factorisation (shared memory bound)
constexpr int LS_SYS_F = EB_LS_SYS_F;  // systems in flight per CTA, FP32 factorisation
constexpr int LS_NW = 2;               // warps per system (each owns the columns j with j % LS_NW == its rank)
constexpr int RPL = EB_LS_RPL;  // rows per lane per chunk
constexpr int CH = 32 * RPL;  // rows per chunk
constexpr int KST = MAXK;     // row stride in shared memory (odd: conflict-free 32- and 64-bit access)
template <typename QT>
__host__ __device__ constexpr int ls_sys() {
  return sizeof(QT) == 8 ? LS_SYS : LS_SYS_F;
}

// Per-system shared memory; QT is the precision of the factorisation (the corrected semi-normal
// equations run in FP64 either way)
template <typename QT>
struct __align__(16) LsSysSmem {
  QT R[MAXK * MAXK + 1];     // triangular factor, row-major (one pad entry keeps C 8-byte aligned)
  QT C[CH * KST];            // current chunk of weighted rows
  QT P[32 * KST];            // partial dot products, column j in P[lane][j] (each column owned by one warp)
  double vec[5 * MAXK];      // F, y, z, tau, 1/R_kk
  double xch[LS_NW * MAXK];  // the warps' partial sums (corrected semi-normal equations)
  QT hs[2][4];               // Householder scalars (beta, v0, gamma, reflect) of step k in hs[k % 2]
  unsigned long long bar;    // barrier of the system's warps (mbarrier, 32 * LS_NW arrivals per phase)
  int32_t slot;              // system being solved
  int32_t bad[LS_NW];        // per-warp row flags
  int32_t hs_seq[2];         // step number whose scalars hs[k % 2] holds (posted after the values)
  int32_t done;              // corrections converged (FP32 factorisation)
};
static_assert(sizeof(LsSysSmem<double>) % 16 == 0 && sizeof(LsSysSmem<float>) % 16 == 0,
              "per-system blocks stay 16-byte aligned");
static_assert(LS_SYS * sizeof(LsSysSmem<double>) <= 232448 && LS_SYS_F * sizeof(LsSysSmem<float>) <= 232448,
              "the systems of a CTA fit in 227 KB of shared memory");
// per-system global scratch (doubles): the rows column-major (MAXROWS x MAXK), the weights and t
// (MAXROWS each), and the FP64 row staging of the FP32 factorisation (CH x KST)
constexpr int64_t LS_SCRATCH = (int64_t)MAXROWS * (MAXK + 2) + (int64_t)CH * KST;

// offsets in units of h/2 span [-11, 11] on each axis (volume, EB and wall rows)
constexpr int TAB_S = 23;
constexpr int TAB_N = TAB_S * TAB_S * TAB_S;

struct LsArgs {
  Dims dm;
  const Tables* T;
  const uint8_t* flag;
  const int32_t* cut_of_cell;
  const int32_t* cut_cell;
  const double* vol_mom;
  const double* eb_mom;
  const double* eb_nmom;
  const uint8_t* eb_bc;
  const int32_t* cutface_of[3];
  const double* face_mom[3];
  const int64_t* slot_face;
  const int64_t* row_ptr;
  const uint32_t* row_desc;
  double* row_val;
  int64_t n_slots;
  const int32_t* slot_list;  // [n_slots] systems to solve (null: 0 .. n_slots-1)
  int32_t* next;       // work counter
  int32_t* status;     // [n_slots]: 0 ok, 1 rank deficient, 2 unsupported row, 3 left to the FP64 path
  double* scratch;     // per system in flight: LS_SCRATCH doubles
  int32_t* err;        // set when a bounded wait between the two warps of a system gives up
  double* flops;       // [2] executed flops, accumulated: FP64 (factorisation, corrections), FP32 (factorisation)
  const double* ftab;  // [TAB_N][MAXK] weighted rows of full cells, by offset
  const double* wtab;  // [TAB_N] weights, by offset
};

struct AsmArgs {
  Dims dm;
  const uint8_t* flag;
  const int32_t* cut_of_cell;
  const int32_t* face_slot[3];
  const int32_t* eb_slot;
  const int64_t* slot_face;
  const int64_t* row_ptr;
  const uint32_t* row_desc;
  const double* row_val;
  const uint8_t* ff[3];
  int nfoot;
  const int16_t* foot_lut;  // [(2R+3)^3] footprint index of an offset, -1 outside
  int64_t n_rows;
  double* rows64;
  float* rows32;
  double inv_h2;
  const uint8_t* eb_bc;   // [n_cut] 0 Dirichlet, 1 Neumann
  const double* eb_mom;   // [n_cut][KS] (the EB area fraction is entry 0)
};

__global__ void k_mark(Dims dm, const uint8_t* flag, uint8_t* mark);
__global__ void k_dilate(Dims dm, int axis, int R, const uint8_t* in, uint8_t* out);
__global__ void k_classify_faces(Dims dm, int d, const uint8_t* fflag, const uint8_t* dil, int32_t* state,
                                 int64_t* class_rep, int32_t* is_unique);
__global__ void k_face_slots(Dims dm, int d, const int32_t* state, const int64_t* upos, int64_t ubase,
                             const int32_t* class_slot, int32_t* slot, int64_t* slot_face);
__global__ void k_reach(Dims dm, const int32_t* cells, int64_t ncells, const uint8_t* flag, const uint8_t* ff0,
                        const uint8_t* ff1, const uint8_t* ff2, Mask* out);
__global__ void k_gather(GatherArgs a, int64_t n_slots, const int32_t* cut_cell);
// Adjoint of the stencil solves with respect to the moment tables (k_stencil_adjoint, eb_build.cu)
struct AdjArgs {
  const double* lam;        // [ncell] adjoint solution
  const double* phi;        // [ncell] forward solution
  // derivatives of the moment tables for parameter 0; parameter p's at + p * the stride
  const double* dvol;       // [n_cut][KS] of the volume moments (stride s_vol)
  const double* deb;        // [n_cut][KS] of the EB moments (stride s_vol)
  const double* debn;       // [n_cut][dim][KS] of the normal-weighted EB moments (stride s_ebn)
  const double* dface[3];   // [n_cutface[d]][KFS] of the face moments (stride s_face[d])
  int n_par;                // parameters
  int64_t s_vol, s_ebn, s_face[3];
  int64_t n_slots;          // systems [0, n_slots) (the individually solved ones)
  int32_t* next;            // work counter
  double* scratch;          // per warp: MAXROWS * ADJ_SCRATCH doubles
  double* dJ;               // [n_par] accumulated derivatives
};
constexpr int ADJ_WARPS = 4;
constexpr int ADJ_SCRATCH = MAXK + 10;  // doubles per row of a warp's scratch
cudaError_t stencil_adjoint_launch(unsigned blocks, cudaStream_t s, const LsArgs& a, const Tables& T,
                                   const AdjArgs& g);
// k_lsq launchers (eb_build.cu): shared-memory attribute, then one launch over the systems of one
// geometry (batch == null) or of several (batch[g] per geometry, slot_base prefix sums of their systems)
// fp32: the FP32-factorisation kernel (systems it cannot finish get status 3), else the FP64 one
cudaError_t lsq_prepare();
size_t lsq_smem(bool fp32);
cudaError_t lsq_launch(bool fp32, unsigned blocks, cudaStream_t s, const LsArgs& a0, const Tables& T,
                       const LsArgs* batch, const int64_t* slot_base, int n_geom);
// the systems with status 3 (global numbers: + base) appended to list[*count]
cudaError_t lsq_fallback_list(const int32_t* status, int64_t n, int64_t base, int32_t* list, int32_t* count,
                              cudaStream_t s);
__global__ void k_full_rows(Dims dm, const Tables* T, double* ftab, double* wtab);
__global__ void k_assemble_rows(AsmArgs a, const int32_t* rep_cell, int64_t nrep, int64_t row0, int32_t* err);
__global__ void k_assemble_b(AsmArgs a, const int32_t* cells, int64_t ncells, int64_t* cnt, const int64_t* bptr,
                             int64_t* bcol, double* bval, const int32_t* unused);

}  // namespace eb
