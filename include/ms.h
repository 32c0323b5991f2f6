/*
 * ms.h -- C ABI of the GB300 multiscale multibasis pressure solver.
 *
 * The library solves the linear pressure system A p = q (Eq. (9) of
 * Klemetsdal, Moyner & Lie, "Accelerating Multiscale Simulation of Complex
 * Geomodels by Use of Dynamically Adapted Basis Functions") obtained from a
 * two-point flux (TPFA) discretisation of div(K grad p) = q on a Cartesian
 * grid with optional inactive cells, face multipliers and non-neighbour
 * connections (Sec. 3).  It builds restriction-smoothed (MsRSB) prolongation
 * operators P on coarse partitions (Sec. 5, Sec. 5.1), Galerkin coarse
 * operators A_c = P^T A P (Eq. (10)), dynamically adapted extra bases from
 * pressure updates (Sec. 5.1), and runs the multiscale multibasis iteration
 * (Eq. (11)) inside a Richardson loop (Sec. 5.2) on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Cells.   Grid cell (i,j,k) has grid index i + nx*(j + ny*k).  The unknowns
 *          are the ACTIVE cells in increasing grid index ("active index").
 *          Vectors over unknowns (q, p, dp, mobility) use active indexing.
 * Memory.  Array arguments marked "host or device" may point to host memory
 *          (pageable or pinned) or to device memory of the context's device;
 *          the library detects which.  Arrays marked "host" must be host
 *          memory.  The caller keeps ownership of every array it passes; the
 *          library reads or writes it only during the call (in stream order
 *          for device arrays: results are complete when the context's stream
 *          reaches the end of the call; host results are complete on return).
 * Handles. ms_ctx, ms_system, ms_basis and ms_coarse are owned by the
 *          library and hold device memory until released.  A handle is used
 *          by one host thread and one stream at a time.
 * Errors.  Every call returns an ms_status.  On error no output handle is
 *          created and ms_last_error() describes the failure.  Device-side
 *          waits are bounded; a wait that runs out returns MS_ERR_TIMEOUT.
 *          Null handles or arrays, sizes out of range and non-finite inputs
 *          are MS_ERR_INVALID_ARG; calls that need matrix values (SpMV,
 *          matrix copies, ILU(0), bases, coarse operators, solves) on a
 *          system never assembled are MS_ERR_STATE; failed allocations are
 *          MS_ERR_OOM and failed CUDA runtime calls MS_ERR_CUDA.
 * Precision. MS_PREC_FP64 computes everything in double precision.
 *          MS_PREC_MIXED stores and applies the basis, the smoother and the
 *          coarse inverse in single precision (single-precision accumulation)
 *          and keeps the outer residual, the convergence check and the
 *          coarse-solve refinement in double precision.
 */
#ifndef MS_H
#define MS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MS_ABI_VERSION 10

typedef enum {
    MS_OK = 0,
    MS_ERR_INVALID_ARG = 1,     /* bad size, pointer, option or input value      */
    MS_ERR_OOM = 2,             /* device or host allocation failed              */
    MS_ERR_CUDA = 3,            /* a CUDA runtime call failed                    */
    MS_ERR_NOT_CONVERGED = 4,   /* iteration cap reached; outputs hold last iterate */
    MS_ERR_COARSE_SINGULAR = 5, /* coarse factorisation met a zero / non-positive pivot */
    MS_ERR_TIMEOUT = 6,         /* a bounded device-side wait ran out            */
    MS_ERR_STATE = 7            /* call made on a handle in the wrong state      */
} ms_status;

typedef enum { MS_PREC_FP64 = 0, MS_PREC_MIXED = 1 } ms_precision;
typedef enum { MS_SMOOTHER_ILU0 = 0, MS_SMOOTHER_JACOBI = 1 } ms_smoother;
/* Outer iteration (Sec. 5.2: "Richardson or GMRES"): Richardson cycles, or
 * restarted GMRES right-preconditioned with one multistage cycle. */
typedef enum { MS_OUTER_RICHARDSON = 0, MS_OUTER_GMRES = 1 } ms_outer;
/* Restriction of a coarse stage (Sec. 5, choice of R): the Galerkin R = P^T,
 * or the finite-volume R that sums the fine cells of each block (Sec. 6.4:
 * b = 1, one entry per cell). */
typedef enum { MS_RESTRICT_GALERKIN = 0, MS_RESTRICT_FV = 1 } ms_restriction;
typedef enum {
    MS_SUPPORT_BOX = 0,   /* Cartesian block box grown by floor(b/2) per side, cells reachable inside it */
    MS_SUPPORT_HOP = 1,   /* general partitions: block + neighbour-block cells nearer (in hops) to the
                             block than to the neighbour's centre cell                                */
    MS_SUPPORT_BLOCK = 2  /* support = the block (constant basis functions)                           */
} ms_support_rule;

typedef struct ms_ctx ms_ctx;
typedef struct ms_system ms_system;
typedef struct ms_basis ms_basis;
typedef struct ms_coarse ms_coarse;

/* Grid description (all arrays host memory, read during ms_system_create).
 * Face multiplier layouts: x-face (i,j,k)-(i+1,j,k) at i + (nx-1)*(j + ny*k);
 * y-face (i,j,k)-(i,j+1,k) at i + nx*(j + (ny-1)*k); z-face (i,j,k)-(i,j,k+1)
 * at i + nx*(j + ny*k).  A multiplier <= 0 removes the face.  A
 * non-neighbour connection e joins grid cells nnc[2e], nnc[2e+1]; its
 * transmissibility uses the permeability component, face area and cell
 * length of axis nnc_axis[e] (0,1,2) and multiplier nnc_mult[e]. */
typedef struct {
    int32_t nx, ny, nz;
    double dx, dy, dz;            /* cell sizes (m)                              */
    const uint8_t *active;        /* nx*ny*nz, nonzero = active; NULL = all       */
    const double *mult_x;         /* (nx-1)*ny*nz or NULL (all 1)                */
    const double *mult_y;         /* nx*(ny-1)*nz or NULL                        */
    const double *mult_z;         /* nx*ny*(nz-1) or NULL                        */
    int32_t n_nnc;
    const int32_t *nnc;           /* 2*n_nnc grid indices                        */
    const int8_t *nnc_axis;       /* n_nnc                                       */
    const double *nnc_mult;       /* n_nnc                                       */
} ms_grid;

typedef struct {
    int64_t n;          /* active cells (unknowns)                      */
    int64_t n_faces;    /* two-point connections                        */
    int32_t ell_width;  /* off-diagonal slots per row in device storage */
    int32_t n_levels;   /* wavefront levels of the natural-order ILU(0) */
    int32_t ref_cell;   /* pinned reference cell (active index)         */
} ms_system_info;

typedef struct {
    double omega;       /* Jacobi relaxation of the basis smoothing (reading: 2/3)   */
    double tol;         /* stop when max |P_new - P_old| < tol (reading: 1e-3)       */
    int32_t max_iter;   /* iteration cap (reading: 500)                               */
    int32_t precision;  /* ms_precision                                               */
    int32_t support;    /* ms_support_rule                                            */
    int32_t bx, by, bz; /* Cartesian block size, used by MS_SUPPORT_BOX               */
} ms_basis_opts;

typedef struct {
    int32_t M;          /* coarse blocks                                 */
    int64_t nnz;        /* sum of support sizes (entries of P)           */
    int32_t max_overlap;/* b: largest number of bases covering one cell  */
    int32_t iters;      /* smoothing iterations of the last build/update */
    double last_increment;
} ms_basis_info;

typedef struct {
    int32_t n_bins;     /* bins of log10|dp| (reading: 8)                        */
    double eps;         /* |dp| floored at eps * max|dp| (reading: 1e-8)          */
    int32_t smoothed;   /* 0: constant basis (the paper's); 1: MsRSB on hop supports */
    double omega, tol;  /* smoothing parameters when smoothed                     */
    int32_t max_iter;
    int32_t precision;  /* ms_precision of the basis made by ms_add_adaptive_basis   */
} ms_adapt_opts;

typedef struct {
    double tol;            /* relative residual ||q - A p||_2 / ||q||_2 target (1e-6) */
    int32_t max_iter;      /* Richardson cycle cap                                    */
    int32_t smoother;      /* ms_smoother                                             */
    int32_t precision;     /* ms_precision                                            */
    double jacobi_omega;   /* relaxation of the Jacobi smoother (reading: 2/3)       */
    int32_t adapt_schedule;/* 0 none; 1 rebuild the dynamic stage after every cycle; */
                           /* 2 after cycles 1 and 2 only (Sec. 5.1 schedule)          */
    ms_adapt_opts adapt;   /* dynamic-stage options (used when adapt_schedule != 0)  */
    int32_t use_x0;        /* 1: p holds the initial guess; 0: start from p = 0      */
    int32_t outer;         /* ms_outer                                                */
    int32_t restart;       /* GMRES: Arnoldi steps per restart (0: 30)                */
} ms_solve_opts;

typedef struct {
    int32_t iters;         /* Richardson cycles performed                 */
    int32_t converged;     /* 1 if rel_residual <= tol                    */
    double rel_residual;   /* final ||q - A p||_2 / ||q||_2 (pinned system) */
    double *history;       /* caller array of max_iter+1 entries or NULL:
                              relative residual before cycle 1 and after each cycle */
    int32_t *dyn_blocks;   /* caller array of max_iter entries or NULL:
                              blocks of the dynamic stage used in each cycle (0 = none) */
    double seconds;        /* wall time of the call                       */
} ms_solve_info;

/* ---------------------------------------------------------------- context */
/* Create a context on CUDA device `device` that launches on `stream`
 * (a cudaStream_t, or NULL for the default stream).  A device index outside
 * [0, device count) is MS_ERR_INVALID_ARG.  ms_destroy releases the context
 * (handles made with it must be released first); ms_set_stream changes the
 * stream later calls launch on. */
ms_status ms_create(ms_ctx **ctx, int32_t device, void *stream);
ms_status ms_destroy(ms_ctx *ctx);
ms_status ms_set_stream(ms_ctx *ctx, void *stream);
const char *ms_status_string(ms_status s);
/* Detail of the last failure on this context (empty string if none). */
const char *ms_last_error(const ms_ctx *ctx);
int32_t ms_abi_version(void);

/* ----------------------------------------------------------------- system */
/* Analyse the grid (host): active-cell numbering, two-point connection list
 * (Sec. 3), device ELL storage of A's pattern, and the wavefront levels of
 * the natural-order ILU(0).  `ref_cell` is the active index of the cell whose
 * pressure is fixed at 0 (the problem statement's reference cell; row and
 * column ref_cell lose their off-diagonal entries and q[ref_cell] is taken as
 * 0).  No values are computed until ms_assemble_tpfa.  Non-positive sizes,
 * a grid of more than 2^30 cells or without active cells, invalid
 * non-neighbour connections and a ref_cell outside the active cells are
 * MS_ERR_INVALID_ARG. */
ms_status ms_system_create(ms_ctx *ctx, const ms_grid *grid, int32_t ref_cell, ms_system **out);
ms_status ms_system_release(ms_system *sys);
ms_status ms_system_get_info(const ms_system *sys, ms_system_info *info);

/* Two-point flux assembly (Sec. 3; Eq. (9)) on the GPU.  perm: host or
 * device, 3*nx*ny*nz doubles, (Kx,Ky,Kz) of each grid cell in m^2, all
 * finite and >= 0.  For each connection, T = mult / (1/t_a + 1/t_b) with
 * half transmissibility t = K_axis * face_area / (cell_length / 2).
 * mobility: host or device, n doubles (total mobility per active cell) or
 * NULL; when given, T is multiplied by the face mobility, taken from the
 * upstream cell by the sign of p_prev[a] - p_prev[b] (single-point upstream
 * weighting) or the mean of the two cells when p_prev is NULL or on a tie.
 * Writes A (unpinned, for basis smoothing) and its pinned copy (for the
 * Galerkin operators and the solve).  Invalid permeability (negative, NaN or
 * infinite) returns MS_ERR_INVALID_ARG. */
ms_status ms_assemble_tpfa(ms_ctx *ctx, ms_system *sys, const double *perm, const double *mobility,
                           const double *p_prev);

/* Copy A out in ELL form (host arrays): col[w*n + i] and val[w*n + i] for the
 * w-th off-diagonal slot of row i (padding slots have col = i, val = 0),
 * diag[i].  pinned selects the pinned (1) or unpinned (0) values. */
ms_status ms_system_get_matrix(ms_ctx *ctx, const ms_system *sys, int32_t pinned, int32_t *col, double *val,
                               double *diag);

/* y = A x with the pinned matrix (x, y host or device, n doubles). */
ms_status ms_spmv(ms_ctx *ctx, const ms_system *sys, const double *x, double *y);

/* z = (L U)^{-1} r with the natural-order ILU(0) factors of the pinned A
 * (Sec. 5.1 smoother; Sec. 6.4): forward then backward triangular sweep.
 * Factors are computed on first use after each assembly.  precision selects
 * FP64 or FP32 factors. */
ms_status ms_ilu_apply(ms_ctx *ctx, ms_system *sys, int32_t precision, const double *r, double *z);

/* Allocation-free ILU(0) application.  The paper has no counterpart: this
 * is a deployment variant of ms_ilu_apply for callers that cannot allocate
 * at the point of the call -- for example an application that has handed
 * all free device memory to its own pool allocator, or a latency-critical
 * loop that cannot afford an allocation's implicit device synchronisation
 * or its failure under memory pressure.  It computes z = (L U)^{-1} r with
 * the system's FP64 factors by the level-ordered sweeps, keeping every
 * scratch buffer (sweep counters, per-row completion flags, the
 * forward-sweep vector) in one fixed device array inside the library: the
 * call performs no cudaMalloc, cudaFree or other allocating call.
 *  - Limit: n <= 1,048,576 unknowns.  The array takes 12 MiB + 256 bytes on
 *    every GPU that loads the library, until the process exits.  Larger
 *    systems return MS_ERR_INVALID_ARG.
 *  - r and z must be device memory of the context's device (host arrays
 *    would need staging buffers): otherwise MS_ERR_INVALID_ARG.
 *  - The FP64 ILU(0) factors of the current assembly must already exist
 *    (made by an earlier ms_ilu_apply or ms_solve with the ILU(0)
 *    smoother); otherwise MS_ERR_STATE.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and keeps it for the
 *    life of the process; make that first call before any stream capture,
 *    and do not reset the device (cudaDeviceReset) while the library is in
 *    use.
 *  - Every call shares the one array and it keeps the last call's contents;
 *    each call clears the counters that must start at zero.  Calls that
 *    overlap on the GPU race on the array: do not overlap them.
 *  - Results equal ms_ilu_apply's up to rounding (on structured grids
 *    ms_ilu_apply uses the tiled sweeps).  Waits for the context's stream
 *    before returning, to report a timed-out sweep as MS_ERR_TIMEOUT. */
ms_status ms_ilu_apply_noalloc(ms_ctx *ctx, const ms_system *sys, const double *r, double *z);

/* Bound of one device-side wait in this system's ILU(0) sweeps and its
 * structured ILU(0) factorisation (the paper runs on one CPU and has no
 * counterpart; the library bounds every wait so that a stalled dataflow
 * sweep returns an error instead of hanging the GPU).  A sweep whose wait
 * exceeds the bound stops waiting, the call returns MS_ERR_TIMEOUT, and the
 * system stays usable.  seconds in (0, 60]; 0 restores the default of 2 s;
 * anything else is MS_ERR_INVALID_ARG.  Ordered on the context's stream. */
ms_status ms_set_wait_limit(ms_ctx *ctx, ms_system *sys, double seconds);

/* Failure-path testing of the bounded waits (no counterpart in the paper):
 * the next forward ILU(0) segment sweep of this system (the sweeps of grids
 * with inactive cells or non-neighbour connections) starts handing out
 * segments at position `count` of its hand-out order, so the first `count`
 * segments are never solved and every segment that needs their results
 * waits until the bound of ms_set_wait_limit runs out; that call then
 * returns MS_ERR_TIMEOUT.  Nothing is written out of bounds and later sweeps
 * run normally.  Requires the ILU(0) factors of `precision` (MS_ERR_STATE
 * if missing, or if the system's sweeps are not the segment sweeps);
 * count in [1, number of segments), else MS_ERR_INVALID_ARG. */
ms_status ms_debug_withhold_segments(ms_ctx *ctx, ms_system *sys, int32_t precision, int32_t count);

/* Segments of the ILU(0) segment sweeps for a sparsity pattern (Sec. 5.1
 * smoother S, Sec. 6.4 "Smooth": the two triangular solves of natural-order
 * ILU(0)); the analysis ms_system_create runs on grids without the
 * structured line sweeps.  Host only, no device work; ctx may be NULL.
 * rowptr (n+1) and col (rowptr[n]) list row i's columns, host int32, in any
 * order (the diagonal and repeats are ignored).  A segment is a maximal run
 * of consecutive rows in which rows i-1 and i are coupled both ways, no row
 * has another coupling to a row of the run, and at most max_len (1..256)
 * rows.  Outputs, host and caller-allocated: seg_off (n+1 int32): first row
 * of each segment, then n; *n_seg; order (2n int32): the forward hand-out
 * order in [0, n_seg) and the backward one in [n_seg, 2 n_seg), segments by
 * wavefront level of the segment graph (forward over couplings to lower
 * rows, ties by ascending segment; backward over couplings to higher rows,
 * ties by descending segment); kg (2 int32): the most couplings of one row
 * that leave its segment towards lower / higher rows (the sweeps take at
 * most 8); *width: the most segments on one level, either direction.
 * Errors: MS_ERR_INVALID_ARG for a null array, n < 1, max_len outside
 * 1..256, a decreasing rowptr or a column outside [0, n). */
ms_status ms_plan_segments(ms_ctx *ctx, int32_t n, const int32_t *rowptr, const int32_t *col, int32_t max_len,
                           int32_t *seg_off, int32_t *n_seg, int32_t *order, int32_t *kg, int32_t *width);

/* ------------------------------------------------------------- partitions */
/* General structured partition (Sec. 5: non-overlapping coarse blocks;
 * Sec. 5.1 general partitions): cell (i,j,k) goes to Cartesian block
 * (i/bx, j/by, k/bz); blocks without active cells are dropped and the rest
 * numbered in increasing Cartesian block order (x fastest).  part: host, n
 * int32; *n_blocks receives the block count. */
ms_status ms_partition_cartesian(ms_ctx *ctx, const ms_system *sys, int32_t bx, int32_t by, int32_t bz,
                                 int32_t *part, int32_t *n_blocks);

/* Well partition (Sec. 6.2, well bases): the cells of well w (active
 * indices well_cells[well_ptr[w] .. well_ptr[w+1]), host arrays) form block
 * w and every other cell block n_wells, which keeps the partition of unity;
 * MsRSB on hop supports over it gives the well basis functions.  A cell
 * listed twice or out of range is MS_ERR_INVALID_ARG.  part: host, n int32;
 * *n_blocks = n_wells + 1. */
ms_status ms_partition_wells(ms_ctx *ctx, const ms_system *sys, int32_t n_wells, const int32_t *well_ptr,
                             const int32_t *well_cells, int32_t *part, int32_t *n_blocks);

/* Face-connected components of cells with equal class (host or device cls,
 * n int32), numbered by their lowest active index (Sec. 5.1 static
 * partitions: class = general block x facies).  part: host or device, n
 * int32 output; *n_blocks receives the number of components. */
ms_status ms_partition_components(ms_ctx *ctx, const ms_system *sys, const int32_t *cls, int32_t *part,
                                  int32_t *n_blocks);

/* Dynamic partition from a pressure update (Sec. 5.1): bin
 * log10(max(|dp|, eps*max|dp|)) into n_bins equal bins, then face-connected
 * components per bin numbered by lowest active index.  dp host or device
 * (n doubles); part host or device (n int32). */
ms_status ms_partition_dynamic(ms_ctx *ctx, const ms_system *sys, const double *dp, int32_t n_bins, double eps,
                               int32_t *part, int32_t *n_blocks);

/* ------------------------------------------------------------------ basis */
/* Build the prolongation P for a partition (host int32[n], block ids in
 * [0, n_blocks), every block non-empty) (Sec. 5 requirements 1-3):
 * supports by opts->support, then MsRSB smoothing from the block indicator
 * until the largest increment falls below opts->tol (MS_SUPPORT_BLOCK gives
 * the constant basis and no smoothing).  *iters receives the smoothing
 * iterations (may be NULL).  Requires an assembled system. */
ms_status ms_build_basis(ms_ctx *ctx, ms_system *sys, const int32_t *partition, int32_t n_blocks,
                         const ms_basis_opts *opts, ms_basis **out, int32_t *iters);
/* Recompute the basis values of an existing basis from the block indicator
 * with the system's current A (same pattern, no allocation). */
ms_status ms_basis_rebuild(ms_ctx *ctx, ms_system *sys, ms_basis *basis, int32_t *iters);
/* Local basis update (Sec. 5.1): continue smoothing from the current values
 * with the system's current A for at most max_iter iterations or until the
 * increment falls below tol. */
ms_status ms_basis_update(ms_ctx *ctx, ms_system *sys, ms_basis *basis, double tol, int32_t max_iter,
                          int32_t *iters);
ms_status ms_basis_release(ms_basis *basis);
ms_status ms_basis_get_info(const ms_basis *basis, ms_basis_info *info);
/* Copy P out column by column (host arrays): cptr[M+1], cells[nnz] (active
 * indices ascending within each column), val[nnz]. */
ms_status ms_basis_get(ms_ctx *ctx, const ms_basis *basis, int32_t *cptr, int32_t *cells, double *val);

/* Dynamically adapted extra basis (Sec. 5.1): dynamic partition of dp
 * (host or device, n doubles) and its constant basis (opts->smoothed = 0,
 * the paper's) or an MsRSB basis on hop supports (opts->smoothed = 1). */
ms_status ms_add_adaptive_basis(ms_ctx *ctx, ms_system *sys, const double *dp, const ms_adapt_opts *opts,
                                ms_basis **out);

/* --------------------------------------------------------- coarse operator */
/* Galerkin coarse operator A_c = P^T A P with the pinned A (Eq. (10),
 * R = P^T) and its dense Cholesky factorisation and inverse for the coarse
 * solve.  precision MS_PREC_MIXED factors in FP32 and refines in FP64 (an
 * FP32 factor that fails falls back to FP64).  A non-positive pivot in FP64
 * is MS_ERR_COARSE_SINGULAR. */
ms_status ms_galerkin(ms_ctx *ctx, ms_system *sys, const ms_basis *basis, int32_t precision, ms_coarse **out);
/* Coarse stage with the chosen restriction (ms_restriction): A_c = R A P with
 * the pinned A.  MS_RESTRICT_GALERKIN is ms_galerkin.  MS_RESTRICT_FV takes
 * R_ji = 1 for the cells i of block j of the basis's partition; A_c is then
 * not symmetric and is inverted by Gauss-Jordan elimination with partial
 * pivoting (MS_ERR_COARSE_SINGULAR on a zero pivot column).  A cycle whose
 * last stage is a finite-volume stage leaves a residual that sums to zero
 * over every block (local conservation).  Richardson iteration with a
 * finite-volume stage is not guaranteed to converge (the correction is not
 * an energy-norm projection); GMRES is the outer iteration to use with it.
 * MS_PREC_MIXED: FP32 inverse of the equilibrated A_c (positive diagonal
 * required, else FP64) with FP64 refinement, as for the Galerkin stage. */
ms_status ms_coarse_create(ms_ctx *ctx, ms_system *sys, const ms_basis *basis, int32_t precision,
                           int32_t restriction, ms_coarse **out);
/* Dense inverse X = A^{-1} by the Gauss-Jordan elimination with partial
 * pivoting that inverts finite-volume coarse operators (FP64; A and X host
 * arrays of M*M row-major doubles).  MS_ERR_COARSE_SINGULAR when a pivot
 * column is zero.  For checking that kernel on arbitrary matrices; stages
 * reach it through ms_coarse_create. */
ms_status ms_dense_inverse(ms_ctx *ctx, int32_t M, const double *A, double *X);
/* Inverse of a symmetric positive definite matrix by the blocked symmetric
 * sweep that inverts Galerkin coarse operators ((A_c)^{-1} of Eq. (11);
 * Sec. 6.4 "solve for p_c"): each step sweeps a 32-wide pivot block (its
 * Cholesky factor G, W = U G^{-T} for the column panel U) and applies the
 * rank-32 update A <- mask(A) - W W^T to the whole matrix, all steps in one
 * cooperative launch.  MS_PREC_FP64: FP64 on the CUDA cores.  MS_PREC_MIXED:
 * the symmetrically equilibrated matrix in FP32 with the rank-32 updates on
 * the tensor cores (tcgen05, TF32 operands split into high and low parts,
 * FP32 accumulation), scaled back, returned widened to FP64.  A and X: host
 * arrays of M*M row-major doubles; A must be symmetric (only the lower
 * triangle is read).  A pivot block that is not positive definite is
 * MS_ERR_COARSE_SINGULAR.  For checking the kernel on arbitrary matrices;
 * stages reach it through ms_galerkin / ms_coarse_create. */
ms_status ms_spd_inverse(ms_ctx *ctx, int32_t M, const double *A, double *X, int32_t precision);
/* The coarse inverse a stage applies (host, M*M row-major doubles, may be
 * NULL), whether it is FP64 (*fp64 = 1) or the FP32 inverse of a mixed
 * stage, widened (*fp64 = 0); for a mixed stage *inv_error receives
 * ||X A_c v - v|| / ||v|| on the stage's test vector and *refine_steps the
 * FP64 refinement steps of each coarse solve (0 when the FP64 inverse is
 * used).  Any output pointer may be NULL. */
ms_status ms_coarse_get_inverse(ms_ctx *ctx, const ms_coarse *coarse, double *X, int32_t *M, int32_t *fp64,
                                double *inv_error, int32_t *refine_steps);
/* Recompute A_c and its factors in place from the basis and the current A. */
ms_status ms_coarse_refresh(ms_ctx *ctx, ms_system *sys, ms_coarse *coarse);
ms_status ms_coarse_release(ms_coarse *coarse);
/* Copy A_c out (host, M*M doubles, row-major). */
ms_status ms_coarse_get(ms_ctx *ctx, const ms_coarse *coarse, double *Ac, int32_t *M);

/* ----------------------------------------------------- CPR pressure stage */
/* Compressible two-phase (water / oil) properties for the CPR pressure stage:
 * rho_a(p) = rho_a0 exp(c_a (p - p_ref)), phi(p) = phi0 exp(c_r (p - p_ref)),
 * Corey mobilities kr_a(s) / mu_a as in ms_fluid.  SI units. */
typedef struct {
    double mu_w, mu_o;        /* viscosities (Pa s)                    */
    double n_w, n_o;          /* Corey exponents (>= 1)                */
    double s_wc, s_or;        /* residual saturations                  */
    double phi0;              /* porosity at p_ref                     */
    double rho_w0, rho_o0;    /* densities at p_ref (kg/m^3)           */
    double c_w, c_o, c_r;     /* water, oil and rock compressibility (1/Pa) */
    double p_ref;             /* reference pressure (Pa)               */
} ms_cpr_fluid;

/* Pressure stage of CPR (Sec. 4, quasi-IMPES decoupling; the predictor of
 * the paper's Fig. 3) for one fully implicit step of the compressible
 * two-phase system with primary variables p and s = s_w per cell:
 *   R_a,i = V/dt [phi rho_a s_a - (phi rho_a s_a)^0] + sum_j T_ij (lambda_a
 *   rho_a)(up) (p_i - p_j) - q_a,i,   up = the higher-pressure cell (lower
 *   index on a tie), T_ij the geometric TPFA transmissibilities of perm.
 * Quasi-IMPES weights w_w + w_o = 1 cancel the diagonal saturation
 * derivatives, w_w dR_w/ds_i + w_o dR_o/ds_i = 0, and the system's matrix is
 * replaced by J* = W_w dR_w/dp + W_o dR_o/dp (not symmetric, no reference-cell
 * pinning: compressibility makes it nonsingular); rhs = -(W_w R_w + W_o R_o),
 * so ms_solve(q = rhs) returns the pressure update of the predictor.  Galerkin
 * stages formed afterwards are not symmetrised and are inverted by
 * Gauss-Jordan elimination.  The basis is not touched (smooth it on the TPFA
 * matrix first, or on J* with ms_basis_rebuild).  ms_assemble_tpfa restores
 * a symmetric pinned TPFA matrix.
 * perm: 3N; p, s, p0, s0 (state at the start of the step), q_w, q_o (fixed
 * mass rates, kg/s): n doubles each; rhs: n doubles out; weights: 2n out
 * (w_w then w_o) or NULL; host or device arrays; dt > 0. */
ms_status ms_cpr_pressure_system(ms_ctx *ctx, ms_system *sys, const double *perm, const ms_cpr_fluid *fluid,
                                 const double *p, const double *s, const double *p0, const double *s0,
                                 const double *q_w, const double *q_o, double dt, double *rhs, double *weights);

/* ------------------------------------------------------------------ solve */
/* Multiscale multibasis iteration (Eq. (11)) in a Richardson loop
 * (Sec. 5.2).  Per cycle, for each stage l = 0..n_stages-1 (then the
 * dynamic stage, if any):  p += S(q - A p);  p += P_l A_c,l^{-1} P_l^T (q - A p).
 * After each cycle the cycle stops when ||q - A p||_2 <= tol ||q||_2.
 * With opts->outer = MS_OUTER_GMRES the same cycle, from a zero guess, is
 * the right preconditioner of restarted flexible GMRES (Arnoldi by classical
 * Gram-Schmidt applied twice, Givens rotations); iters then counts Arnoldi
 * steps (one cycle each), history holds the GMRES residual estimate after
 * each step and the true residual at each restart, and max_iter bounds the
 * steps.  GMRES takes no adaptive schedule (MS_ERR_INVALID_ARG).
 * q: host or device, n doubles; p: host or device, n doubles (initial guess
 * if opts->use_x0, else overwritten from 0; holds the last iterate on
 * return, also on MS_ERR_NOT_CONVERGED).  stages: coarse operators built on
 * this system.  info may be NULL. */
ms_status ms_solve(ms_ctx *ctx, ms_system *sys, ms_coarse *const *stages, int32_t n_stages, const double *q,
                   double *p, const ms_solve_opts *opts, ms_solve_info *info);

/* One member of a batched solve: an independent system with its own stages,
 * sources and result.  `rebuild` (or NULL): a basis of this system to
 * re-smooth from its block indicator before the solve (Sec. 3 basis
 * construction), after which every stage built on it is re-formed (Galerkin
 * product and coarse factor); `basis_iters` receives its iteration count.
 * `status` receives the member's result (MS_ERR_NOT_CONVERGED keeps the last
 * iterate in p, as for ms_solve). */
typedef struct {
    ms_system *sys;
    ms_coarse *const *stages;
    int32_t n_stages;
    const double *q;       /* host or device, n doubles */
    double *p;             /* host or device, n doubles */
    ms_solve_info *info;   /* or NULL */
    ms_basis *rebuild;     /* or NULL */
    int32_t basis_iters;   /* out */
    ms_status status;      /* out */
} ms_batch_member;

/* Batched solve of independent members (no counterpart in the paper, which
 * solves one system at a time): members run concurrently on `n_workers`
 * worker streams of this context's device (0: min(16, n_members)), each
 * worker taking the largest remaining member next, so the small kernels of
 * many members overlap on the GPU; the bases of members with `rebuild` set
 * are first re-smoothed together, as by ms_basis_rebuild_batch.  Each member computes exactly what
 * ms_solve (after ms_basis_rebuild / ms_coarse_refresh when `rebuild` is set)
 * computes for it alone.  The batch is ordered after earlier work on the
 * context's stream and later work on that stream is ordered after it; the
 * call returns when every member is done.  Returns MS_OK when every member
 * converged, MS_ERR_NOT_CONVERGED when some did not (and none failed), else
 * the first failing member's status.  Handles of different members must be
 * distinct. */
ms_status ms_solve_batch(ms_ctx *ctx, ms_batch_member *members, int32_t n_members, const ms_solve_opts *opts,
                         int32_t n_workers);

/* Batched basis re-smoothing (no counterpart in the paper, which builds one
 * basis at a time; Sec. 5.1 gives the smoothing): re-smooths every basis
 * bases[m] of system sys[m] from its block indicator with the system's
 * current A, in one persistent launch per precision that takes
 * (member, tile) work items from a device queue, so many small systems fill
 * the GPU together.  Results (values, iteration counts, stopping) are
 * bitwise those of ms_basis_rebuild on each member.  Members the launch cannot
 * take (constant bases, rows with more than 8 connections) are re-smoothed
 * one by one.  iters (n entries, host, or NULL) receives the iteration
 * counts.  Systems and bases must be distinct and assembled; ordered on the
 * context's stream; returns after the smoothing. */
ms_status ms_basis_rebuild_batch(ms_ctx *ctx, ms_system *const *sys, ms_basis *const *bases, int32_t n,
                                 int32_t *iters);
/* Work-item shape of the batched smoothing (used by ms_basis_rebuild_batch
 * and ms_solve_batch): cells per item (a multiple of 256 in [256, 16384];
 * default 1024) and resident blocks per SM of the persistent launch (1..8;
 * default 4).  paper_2001_01624_gb300.autotune picks them per device. */
ms_status ms_set_batch_tuning(ms_ctx *ctx, int32_t tile_cells, int32_t ctas_per_sm);

/* ------------------------------------------------------------- two-phase */
/* Water / oil fluid for sequential-implicit time steps (Sec. 2): Corey
 * relative permeabilities krw = Se^n_w, kro = (1 - Se)^n_o with
 * Se = (S - s_wc) / (1 - s_wc - s_or) clipped to [0, 1], viscosities in
 * consistent units, porosity, and the CFL number of the transport substeps. */
typedef struct {
    double mu_w, mu_o;
    double n_w, n_o;
    double s_wc, s_or;
    double porosity;
    double cfl;
} ms_fluid;

/* Total mobility lambda_t = krw/mu_w + kro/mu_o per active cell (the
 * `mobility` argument of ms_assemble_tpfa).  S, lambda: host or device, n
 * doubles. */
ms_status ms_total_mobility(ms_ctx *ctx, const ms_system *sys, const ms_fluid *fluid, const double *S,
                            double *lambda);

/* Advance the water saturation S over dt with explicit single-point
 * upstream transport: total fluxes u = T (p_a - p_b) from the transmissibilities
 * of the last assembly (with its face mobilities) and the pressure p; water
 * flux u f_w(S_upstream), f_w = (krw/mu_w) / lambda_t; sources q (total
 * rate, + injection of water, - production at the cell's f_w); substeps of
 * equal length h <= cfl * min_i (phi V_i / outflow_i) / max f_w', where
 * outflow_i sums the fluxes leaving cell i and its production and max f_w'
 * is the largest slope of f_w from central differences on 2000 intervals.
 * p, q: host or device, n doubles; S: host or device, n doubles, updated in
 * place; substeps (or NULL) receives the substep count. */
ms_status ms_transport_step(ms_ctx *ctx, ms_system *sys, const ms_fluid *fluid, const double *p, const double *q,
                            double dt, double *S, int32_t *substeps);

/* Pressure update dp = p - p_prev over the n unknowns (device arrays of the
 * context's device); the dynamically adapted basis of the next step is
 * built from it (Sec. 5.1, the pressure change between successive steps).
 * Ordered on the context's stream. */
ms_status ms_pressure_update(ms_ctx *ctx, const ms_system *sys, const double *p, const double *p_prev, double *dp);

/* Device allocations of the library (all go through one allocator): bytes
 * allocated so far by library calls made on the calling host thread
 * (*thread_bytes), and the number of device allocations made so far in the
 * process (*allocations).  Either pointer may be NULL.  Serving measures a
 * model's footprint with the first; tests use the second to check that a
 * call allocates nothing. */
ms_status ms_allocation_stats(int64_t *thread_bytes, int64_t *allocations);

/* ---------------------------------------------------------------- tracing */
/* Process-wide kernel tracing.  Launch counts are always kept; when enabled,
 * each launch is also timed with a pair of CUDA events recorded on the
 * stream it runs on, and its algorithmic bytes (what the method must move
 * for that launch in this library's storage layout) are accumulated. */
typedef struct {
    char name[32];           /* kernel family                                   */
    int64_t launches;        /* launches since the last reset                   */
    int64_t timed_launches;  /* launches timed with events (tracing enabled)    */
    double total_ms;         /* summed device time of the timed launches        */
    double bytes;            /* summed algorithmic bytes of the timed launches  */
} ms_kernel_stat;

ms_status ms_profile_enable(int32_t on);
ms_status ms_profile_reset(void);
/* Fills up to `capacity` entries (out may be NULL to query the count);
 * *count receives the number of kernel families, *total_launches the launch
 * count over all families.  Waits for the timed launches to finish. */
ms_status ms_profile_read(ms_kernel_stat *out, int32_t capacity, int32_t *count, int64_t *total_launches);

#ifdef __cplusplus
}
#endif
#endif /* MS_H */
