/*
 * eb.h -- C ABI of the GB300 library for the higher-order cut-cell
 * finite-volume Poisson discretisation of Devendran, Graves and Johansen
 * (arXiv:1411.4283).
 *
 * The method (Sec. 2): on a Cartesian grid cut by an embedded boundary (EB),
 * every face f carries a flux stencil s_f = W (A^T W)^+ F (Eq. "stencil
 * equation solution"), the minimum-||W^-1 s|| solution of A^T s = F, where
 * the rows of A are volume averages of the monomials (x - x0)^p, |p| <= Q,
 * over the neighbouring volumes and face averages over the neighbouring
 * boundary faces (Sec. 2.2.1), F_p is the integral over f of
 * grad (x - x0)^p . n, and W is the distance weight of Sec. 2.4.  The
 * Laplacian of a volume is its flux divergence (1/|V_v|) sum_f s_f^T Phi
 * (Sec. 2.3); boundary values enter through a matrix B.
 *
 * Conventions for every entry point:
 *   - All array arguments are DEVICE pointers unless the name ends in _host;
 *     the caller owns them; the library never frees or retains them beyond
 *     the call (eb_build_stencils copies what it needs).
 *   - All calls are ordered on the given CUDA stream (NULL = legacy default
 *     stream).  eb_build_stencils and eb_solve synchronise that stream to
 *     read back small scalars (counts, status, residual norms); eb_apply and
 *     eb_bc_rhs do not synchronise.
 *   - Device memory of builds and solves comes from a library-owned,
 *     stream-ordered memory pool per device that keeps freed memory cached
 *     (small arrays share chunks of it); eb_stencils_destroy synchronises the
 *     device before returning the stencils' memory to the pool.
 *   - Errors are returned as eb_status; nothing is thrown across the ABI.
 *     eb_last_error_message() gives a human-readable reason for the last
 *     failure on the calling thread.
 *   - Cells are indexed c = x + nx*(y + ny*z); faces normal to d are indexed
 *     x + (nx+[d==0])*(y + (ny+[d==1])*z), where the face with coordinate i_d
 *     lies at x_d = i_d*h.  Global face ids: faces normal to 0, then 1, then
 *     2, each block in that order; EB faces follow, id = n_grid_faces + cut
 *     index.  Cut cells are listed in ascending cell index.
 *   - Moments are in h-scaled coordinates xi = (x - centre)/h about the cell
 *     centre (volumes, EB patches) or the face centre (grid faces), divided by
 *     h^D (volumes) or h^(D-1) (faces), for the graded monomials of degree
 *     <= moment_degree: degree 0, then for each degree q the exponents
 *     (p0, p1, ...) with p0 from q down to 0, p1 from q - p0 down to 0, ....
 *     Face moments use the face's tangential coordinates in ascending
 *     dimension order.  EB normals point out of the fluid.
 */
#ifndef EB_GB300_H
#define EB_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* eb_stream_t; /* = cudaStream_t */

typedef enum {
  EB_OK = 0,
  EB_ERR_INVALID = 1,        /* malformed descriptor or argument */
  EB_ERR_RANK_DEFICIENT = 2, /* some face's weighted LS system has rank < K (face ids recorded) */
  EB_ERR_MULTIVALUED = 3,    /* geometry needs more than one volume per cell (unsupported) */
  EB_ERR_NOT_CONVERGED = 4,  /* solve stopped at its iteration limit */
  EB_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
  EB_ERR_CUDA = 6,           /* a CUDA runtime call failed */
  EB_ERR_OOM = 7,            /* device allocation failed */
  EB_ERR_CAPACITY = 8        /* a face needs more LS rows than the kernels support */
} eb_status;

enum { EB_F32 = 0, EB_F64 = 1 };
enum { EB_DIRICHLET = 0, EB_NEUMANN = 1 };
enum { EB_NBR_BOX = 0, EB_NBR_PATH = 1 };

/* Geometry descriptor: the EB moment tables the paper takes from its
 * geometry generator (Sec. 2.1: volume moments m^p_v, face moments m^p_f,
 * normal-weighted EB moments m^p_{d,f}).  All pointers are device pointers. */
typedef struct eb_geom {
  int32_t dim;               /* 2 or 3 */
  int32_t n[3];              /* cells per dimension (n[2] = 1 in 2D) */
  double h;                  /* grid spacing */
  int32_t moment_degree;     /* degree of the stored moment tables (>= order) */
  const uint8_t* cell_flag;  /* [ncell]: 0 covered, 1 full, 2 cut */
  int32_t n_cut;
  const int32_t* cut_cell;   /* [n_cut] ascending cell indices */
  const double* vol_mom;     /* [n_cut][K_D] volume moments */
  const double* eb_mom;      /* [n_cut][K_D] EB-patch moments */
  const double* eb_nmom;     /* [n_cut][dim][K_D] EB moments weighted by the normal component */
  const uint8_t* eb_bc;      /* [n_cut] EB_DIRICHLET/EB_NEUMANN, or NULL = all Dirichlet.  Neumann
                              * rows are the Sec. 2.2.1 b_{f_b p}, weighed as in the physical
                              * minimum-norm problem; the flux through a Neumann EB face is its
                              * datum |A_f| <grad phi . n>_f (a column of B) */
  const uint8_t* face_flag[3];  /* per direction [nface_d]: 0 covered, 1 full, 2 cut */
  int32_t n_cutface[3];
  const int32_t* cutface[3];    /* [n_cutface[d]] ascending face indices */
  const double* face_mom[3];    /* [n_cutface[d]][K_{D-1}] tangential moments */
} eb_geom;

/* Discretisation parameters (Sec. 2.4).  Defaults: order 4, path radius 3
 * (2 for order 2), box neighbourhoods, weight threshold 1/2, power 5. */
typedef struct eb_params {
  int32_t order;         /* Q: interpolant degree, 2 or 4 (P = Q + 1) */
  int32_t path_radius;   /* R_n; <= 0 selects the paper's value for the order */
  int32_t nbr_metric;    /* EB_NBR_BOX (default) or EB_NBR_PATH */
  int32_t weighted;      /* 1: W_ii as in Sec. 2.4; 0: W = I (unstable control) */
  double w_threshold;    /* 0.5 */
  double w_power;        /* 5 */
  int32_t ls_precision;  /* EB_LS_MIXED (default): each least-squares system is factorised in FP32
                            and solved by FP64 corrected semi-normal iterations preconditioned by that
                            factor, a system the FP32 factor cannot carry going to the FP64 path;
                            EB_LS_FP64: FP64 Householder factorisation for every system.  Both give
                            the FP64 minimum-norm stencil to rounding (Sec. 2.2.1). */
} eb_params;
enum { EB_LS_MIXED = 0, EB_LS_FP64 = 1 };

typedef struct eb_stencils eb_stencils; /* opaque, library-owned */

typedef struct eb_build_info {
  int64_t n_flux_faces;     /* open grid faces + EB faces */
  int64_t n_unique_faces;   /* faces whose LS system was solved individually */
  int64_t n_class_faces;    /* faces sharing a translation-invariant class stencil */
  int32_t n_classes;        /* class stencils solved (includes the interior template) */
  int32_t max_rows;         /* largest LS system (rows) */
  int64_t n_irregular_rows; /* cells with their own operator row */
  int32_t n_row_classes;    /* shared operator rows (wall classes and template) */
  int64_t lsq_flops;        /* the method's flop count of the LS solves, 2nK^2 - 2K^3/3 + 4nK + K^2
                               per system (Householder QR, triangular solve, application of Q),
                               whichever path ran */
  double ms_classify, ms_gather, ms_lsq, ms_assemble; /* device time per phase */
  int64_t n_ls_fp64;        /* systems solved by the FP64 factorisation (all of them with
                               EB_LS_FP64; with EB_LS_MIXED those the FP32 factor could not carry) */
  double ls_fp64_flops;     /* FP64 flops the LS kernels executed (factorisations, semi-normal
                               solves and corrections; row construction not counted) */
  double ls_fp32_flops;     /* FP32 flops of the FP32 factorisations (EB_LS_MIXED).  For a batch
                               both are the launch's totals shared out by the systems' counts. */
} eb_build_info;

/* Build all flux stencils and the operator (Sec. 2.2-2.4).
 * Rank-deficient systems return EB_ERR_RANK_DEFICIENT (no fallback); query
 * the offending faces with eb_last_error_faces.  *out is NULL on failure. */
eb_status eb_build_stencils(const eb_geom* geom, const eb_params* params, eb_stencils** out, eb_build_info* info,
                            eb_stream_t stream);

/* Build the stencils of n_geom geometries (Sec. 2.2-2.4 for each) with one
 * least-squares launch: the LS systems of all geometries share one work
 * queue, each system carrying its geometry.  geoms: host array of n_geom
 * descriptors (device arrays as for eb_build_stencils), all of the same
 * dimension; params apply to all.  out: host array of n_geom handles, each
 * destroyed with eb_stencils_destroy; infos: optional host array of n_geom
 * (ms_lsq is the shared launch's time in every entry).  The results equal
 * those of n calls of eb_build_stencils.  The per-geometry phases before and
 * after the shared launch run on up to 8 library-owned host threads, each
 * with its own stream ordered after `stream`; the call returns when all of
 * them are done, with `stream` ordered after the work.  On any failure every
 * handle is NULL, nothing is left allocated, and the status, message and
 * faces are those of the lowest-numbered failing geometry (EB_ERR_INVALID
 * also for n_geom < 1 or mixed dimensions). */
eb_status eb_build_stencils_batch(const eb_geom* geoms, int32_t n_geom, const eb_params* params, eb_stencils** out,
                                  eb_build_info* infos, eb_stream_t stream);

/* y = L phi (kappa_weighted = 0) or kappa .* (L phi) (kappa_weighted = 1):
 * the homogeneous part of the discrete Laplacian (boundary values zero;
 * Sec. 2.3).  phi, y: [ncell] of dtype EB_F32 or EB_F64; covered cells of y
 * are set to 0 and covered entries of phi are ignored.  Never synchronises. */
eb_status eb_apply(const eb_stencils* st, const void* phi, void* y, int32_t dtype, int32_t kappa_weighted,
                   eb_stream_t stream);

/* Bg = B g, the boundary-data part of the Laplacian (FP64; kappa-weighted
 * when kappa_weighted = 1): the boundary-face columns of the flux stencils
 * (Sec. 2.2.1, boundary rows b_{f_b p}) summed into each volume's flux
 * divergence (Sec. 2.3).  Bg: [ncell], written on every cell (0 where no
 * boundary face reaches).  g_eb: [n_cut] face averages on the EB faces
 * (Dirichlet: <phi>_f; Neumann: <grad phi . n>_f); g_wall: values on the
 * open wall faces in ascending global face id (eb_wall_faces lists them). */
eb_status eb_bc_rhs(const eb_stencils* st, const double* g_eb, const double* g_wall, double* Bg,
                    int32_t kappa_weighted, eb_stream_t stream);

typedef struct eb_solve_opts {
  int32_t mixed;          /* 1: FP32 BiCGStab inner solves + FP64 iterative refinement; 0: FP64 BiCGStab */
  double inner_tol;       /* relative residual target of each inner solve (mixed), e.g. 1e-5 */
  int32_t max_inner;      /* iteration cap per inner solve */
  int32_t max_outer;      /* refinement sweeps (mixed) */
  int32_t max_iters;      /* total iteration cap */
  int32_t check_every;    /* < 0: time every Krylov operator apply with CUDA events (eb_solve_info.apply_ms) */
  int32_t precond;        /* 0: Jacobi (kappa-weighted diagonal); 1 (default): geometric multigrid
                             V-cycle followed by exact solves of the high-order operator on 3x3x3
                             blocks around the cut cells whose diagonal is weak or positive (3-D) */
} eb_solve_opts;

typedef struct eb_solve_info {
  int32_t iterations;     /* total Krylov iterations */
  int32_t sweeps;         /* refinement sweeps (mixed) */
  double rel_residual;    /* final ||rhs - kappa L phi||_2 / ||rhs||_2, FP64 */
  double history[64];     /* FP64 relative residual after each sweep (mixed) or check (FP64) */
  int32_t n_history;
  int32_t n_applies;      /* Krylov operator applies timed (check_every < 0) */
  double apply_ms;        /* their summed device time */
  int32_t precond_blocks; /* exact local block solves in the preconditioner (0 for Jacobi) */
} eb_solve_info;

/* Solve the discrete Poisson problem L phi = rho - B g of Sec. 2.3 (the
 * paper solves it with preconditioned GMRES, Sec. 3.2; here BiCGStab with
 * FP64 iterative refinement) to a relative residual tol of the
 * kappa-weighted system kappa L phi = kappa (rho - B g).  rho: [ncell] cell
 * averages of the source; phi: [ncell] initial guess on entry, solution on
 * exit (FP64); g_eb, g_wall as for eb_bc_rhs.  Returns
 * EB_ERR_NOT_CONVERGED (phi holds the last iterate) when the iteration caps
 * are reached first.  Synchronises the stream to read residual norms. */
eb_status eb_solve(const eb_stencils* st, const double* rho, const double* g_eb, const double* g_wall, double tol,
                   const eb_solve_opts* opts, double* phi, eb_solve_info* info, eb_stream_t stream);

/* Batched solve: the mixed-precision refinement of eb_solve (Sec. 2.3 system,
 * solved as eb_solve does) for n independent stencil sets at once, as one
 * CUDA graph launch per call.  Per system, a graph loop (conditional WHILE
 * node) runs the refinement sweeps -- FP64 residual with the FP64 operator,
 * an inner FP32 BiCGStab as a nested loop, the FP64 correction -- and
 * one-thread kernels set the loop conditions on the device from the
 * device-resident scalars: no host synchronisation inside the solve, the
 * systems' loops side by side.  Every loop stops at its iteration cap.
 *
 * eb_batch_solver_create: st[n] (host array of distinct handles, which must
 * outlive the solver and are not used concurrently by other solves; a handle
 * given twice is refused with EB_ERR_INVALID, since a stencil set's solver
 * state serves one system at a time); opts as for
 * eb_solve (mixed must be 1; check_every is ignored); sets up each system's
 * preconditioner, its vectors (about 72 bytes per cell) and the graph.
 * eb_batch_solve: host arrays of device pointers rho[n], g_eb[n], g_wall[n]
 * (the arrays may be NULL when no system has EB or wall faces), phi[n]
 * (in: initial guess, out: solution, FP64); tol as for eb_solve;
 * infos[n] (may be NULL) as for eb_solve without the apply timings.
 * Returns EB_ERR_NOT_CONVERGED naming the first system that did not
 * converge (its phi holds the last iterate; the others are solved).
 * Synchronises the stream once, at the end. */
typedef struct eb_batch_solver eb_batch_solver;
eb_status eb_batch_solver_create(const eb_stencils* const* st, int32_t n, const eb_solve_opts* opts,
                                 eb_batch_solver** out, eb_stream_t stream);
eb_status eb_batch_solve(eb_batch_solver* b, const double* const* rho, const double* const* g_eb,
                         const double* const* g_wall, double tol, double* const* phi, eb_solve_info* infos,
                         eb_stream_t stream);
void eb_batch_solver_destroy(eb_batch_solver* b);

/* Error norms of Sec. 3.3 over the volumes: L_inf, L1 = sum |e||V| / sum|V|,
 * L2 = (sum e^2 |V| / sum |V|)^(1/2).  err: [ncell] FP64 device; out_host[3]. */
eb_status eb_norms(const eb_stencils* st, const double* err, double* out_host, eb_stream_t stream);

/* Debug / parity: the flux stencil s_f of Sec. 2.2.1 (the minimum-||W^-1 s||
 * solution of A^T s = F) of a face (global face id).  Columns:
 * volume -> cell index; boundary face -> -(1 + global face id).  Values are
 * the h-scaled stencil s_hat (s = h^(D-2) s_hat), rows in canonical order
 * (volumes ascending, wall faces ascending, EB faces ascending).  With
 * cols_host == NULL only *n is written.  Synchronises the stream. */
eb_status eb_stencil_query(const eb_stencils* st, int64_t face, int32_t* n, int64_t* cols_host, double* coef_host,
                           int32_t cap, eb_stream_t stream);

/* Open wall faces in ascending global face id (the g_wall order). */
eb_status eb_wall_faces(const eb_stencils* st, int64_t* ids_host, int64_t cap, int64_t* n);

/* Faces whose LS system was rank deficient in the last failed build on the
 * calling thread (Sec. 2.4 uses one R_n everywhere, so no fallback is
 * applied): every such face in ascending global face id, including each face
 * of a translation class whose shared system failed.  With ids_host == NULL
 * only *n is written; at most cap ids are copied. */
eb_status eb_last_error_faces(int64_t* ids_host, int32_t cap, int32_t* n);

/* Batched weighted minimum-norm least squares that allocates nothing (the
 * paper has no counterpart; this is a service for callers that cannot
 * allocate device memory where they solve, e.g. code running inside a fixed
 * memory pool or arena, real-time hosts that allocate only at start-up, or
 * plugin hosts that forbid allocation in callbacks).
 * For each system q (rows row_ptr[q] .. row_ptr[q+1]-1, at most 256 rows and
 * K <= 35 unknowns): B holds the weighted rows W A ([nnz][K], row-major), w
 * the weights W_ii, F the right-hand side ([n_sys][K]); s receives the
 * stencil s = W t with t the least-||t|| solution of B^T t = F (the
 * weighted minimum-norm problem, for rows the caller formed); status[q] = 0 ok, 1 rank deficient or
 * fewer rows than K, 3 more than 256 rows.  All pointers are device pointers
 * owned by the caller.  max_rows is the caller's bound on the rows of any
 * system; above 256 the call returns EB_ERR_CAPACITY without launching.
 * Working storage is one fixed 9.4 MB array compiled into the library (held
 * by every GPU that loads it until the process exits); nothing is allocated.
 * The first call on each device looks up that array's device address (with
 * the device current) and should come before any stream capture.  Every call
 * shares the array, so calls that overlap on the GPU (other streams, other
 * host threads) race: serialise them.  The array's address is cached per
 * device for the life of the process; after a cudaDeviceReset the process
 * must not call this entry point on that device again.  Never synchronises. */
eb_status eb_lsq_batch_noalloc(const double* B, const double* w, const double* F, const int64_t* row_ptr,
                               int32_t n_sys, int32_t K, int32_t max_rows, double* s, int32_t* status,
                               eb_stream_t stream);

/* Moment tables computed on the device (Sec. 2.1: volume moments m^p_v,
 * face moments m^p_f and the EB-patch moments, plain and weighted by each
 * normal component; exact to rounding, which meets the O(h^{6+D}) of Sec.
 * 3.1), for the unit square [0,1]^2 on an N x N grid minus n_body circles
 * (inside = 0: fluid outside every circle) or inside one circle (inside = 1,
 * n_body = 1).  centers_host: [n_body][2], radii_host: [n_body] (host
 * arrays); moment_degree 0..6 (>= the order of the stencils built on it).
 * On success *out owns the device tables and *desc points into them, in the
 * layout eb_geom documents (cut cells and cut faces ascending; cells with
 * volume fraction <= 1e-14 count as covered, >= 1 - 1e-14 as full, faces
 * likewise, and a face next to a covered cell is closed); desc can be passed
 * to eb_build_stencils as it is.  A cell or face that two circles reach into
 * gives EB_ERR_MULTIVALUED.  Synchronises the stream.  Free with
 * eb_geometry_destroy (which synchronises the device) after the last use of
 * desc. */
typedef struct eb_geometry eb_geometry; /* opaque, library-owned */
/* The same for the unit cube [0,1]^3 on an N^3 grid minus n_body spheres
 * (centers_host [n_body][3]) or inside one sphere; moment_degree 0..4.  Face
 * moments by the disk each sphere cuts from the face plane (closed form in
 * one tangential coordinate, sin^2-mapped Gauss-Legendre in the other), EB
 * moments by the sphere's area element R^2 sin(th) dth dphi on polar-angle
 * panels split at the patch's tangencies, volume moments by the divergence
 * theorem. */
eb_status eb_geometry_spheres(int32_t N, int32_t n_body, const double* centers_host, const double* radii_host,
                              int32_t inside, int32_t moment_degree, eb_geometry** out, eb_geom* desc,
                              eb_stream_t stream);
eb_status eb_geometry_circles(int32_t N, int32_t n_body, const double* centers_host, const double* radii_host,
                              int32_t inside, int32_t moment_degree, eb_geometry** out, eb_geom* desc,
                              eb_stream_t stream);
void eb_geometry_destroy(eb_geometry* g);

/* Copy one table of a device geometry to host memory (dir: face direction
 * for the face tables).  *bytes receives the table's size; with dst_host ==
 * NULL nothing is copied.  Synchronous. */
enum { EB_TABLE_CELL_FLAG = 0, EB_TABLE_CUT_CELL = 1, EB_TABLE_VOL_MOM = 2, EB_TABLE_EB_MOM = 3,
       EB_TABLE_EB_NMOM = 4, EB_TABLE_FACE_FLAG = 5, EB_TABLE_CUTFACE = 6, EB_TABLE_FACE_MOM = 7 };
eb_status eb_geometry_table(const eb_geometry* g, int32_t which, int32_t dir, void* dst_host, int64_t cap_bytes,
                            int64_t* bytes);

/* One table of the shape derivatives of g's moment tables (d/dt of the table
 * when the boundary moves with a normal speed, the cut sets held fixed), as
 * the adjoint entry points below compute them: kind 0 the radius of body
 * `body`; kind 1 the amplitude of the level-set mode mode_host = (k_x, k_y,
 * k_z, theta) at zero amplitude (see eb_adjoint_shape).  which:
 * EB_TABLE_VOL_MOM, EB_TABLE_EB_MOM, EB_TABLE_EB_NMOM or EB_TABLE_FACE_MOM
 * (dir: face direction); laid out like the table.  *bytes receives the size;
 * with dst_host == NULL nothing is computed.  Synchronous; for tests and
 * inspection (it allocates and frees its work arrays). */
eb_status eb_geometry_shape_table(const eb_geometry* g, int32_t kind, int32_t body, const double* mode_host,
                                  int32_t which, int32_t dir, double* dst_host, int64_t cap_bytes, int64_t* bytes);

/* The objective J = 1/2 sum_v |V_v| phi_v^2 of a solution phi on the stencils
 * st built from the device geometry g, and (dJ_host != NULL) its derivatives
 * with respect to the radii of g's bodies (dJ_host[n_body]), by the adjoint
 * method, with phi the solution of kappa L phi = kappa rho for the Dirichlet
 * problem with homogeneous data (Sec. 2.3): the adjoint solve
 * (kappa L)^T lam = |V| phi (transposed operator, FP64), then
 *   dJ/dr = sum_v (h^D phi_v^2 / 2 + lam_v) d kappa_v / dr
 *           - lam^T (d (kappa L) / dr) phi,
 * where kappa L changes through every stencil s = W (A^T W)^+ F whose rows
 * or right-hand side hold moments of the moving boundary (Sec. 2.2.1): the
 * reverse-mode derivative of each stencil solve with respect to A and F,
 * contracted with the rows' and F's derivatives, which follow from the shape
 * derivatives of the moment tables (recomputed on the device, not stored).
 * The cut-cell and cut-face sets are held fixed.  Circles (2-D) and spheres
 * (3-D), Dirichlet EB.  phi: [ncell] device (FP64).  Synchronises the stream. */
eb_status eb_adjoint_radii(const eb_geometry* g, const eb_stencils* st, const double* phi, double* J_host,
                           double* dJ_host, eb_stream_t stream);

/* eb_adjoint_radii with level-set modes as further parameters: the boundary
 * is the zero set of psi + sum_m a_m sin(2 pi k_m . x + theta_m), psi the
 * signed distance of g's bodies (positive in the fluid), and the derivatives
 * are taken at a = 0 (g's geometry): mode m moves the boundary with the
 * normal speed -sin(2 pi k_m . x + theta_m) along the direction out of each
 * body (+ for the inside of one body).  modes_host: [n_modes][4] host
 * (k_x, k_y, k_z, theta; k_z ignored in 2-D).  dJ_radii_host[n_body] and
 * dJ_modes_host[n_modes] receive the derivatives (both NULL: J only).  One
 * adjoint solve serves all parameters; the stencil-solve adjoints run in one
 * pass over the systems for all parameters.  info (may be NULL) receives the
 * transposed solve's iterations and the phases' device times when the
 * derivatives are asked for.  Synchronises the stream. */
typedef struct eb_adjoint_info {
  int32_t iterations;     /* BiCGStab iterations of the transposed solve */
  double rel_residual;    /* its final relative residual */
  double solve_ms;        /* device time of the transposed solve */
  double tables_ms;       /* of the moment tables' derivatives and kappa terms, all parameters */
  double stencils_ms;     /* of the stencil-solve adjoints, all parameters */
} eb_adjoint_info;
eb_status eb_adjoint_shape(const eb_geometry* g, const eb_stencils* st, const double* phi, int32_t n_modes,
                           const double* modes_host, double* J_host, double* dJ_radii_host, double* dJ_modes_host,
                           eb_adjoint_info* info, eb_stream_t stream);

void eb_stencils_destroy(eb_stencils* st);
const char* eb_status_string(eb_status s);
const char* eb_last_error_message(void);
int32_t eb_abi_version(void);

/* Measured FP64 FMA throughput of the device (the FP64 roofline's
 * denominator): blocks_per_sm x SM-count blocks of 256 threads, each thread
 * eight independent FMA chains of iters steps, timed with CUDA events after a
 * warm-up launch; *tflops_host = 2 x FMAs / time in TFLOP/s.  Synchronous. */
eb_status eb_fp64_fma_rate(int32_t blocks_per_sm, int64_t iters, double* tflops_host, eb_stream_t stream);

/* Cumulative number of CUDA kernels this library has launched in the
 * process (all threads); differences around a region count its launches. */
int64_t eb_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif
