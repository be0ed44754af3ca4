/*
 * gmg.h -- C ABI of the GB300 (sm_103a) cell-centred geometric multigrid library.
 *
 * The library solves the variable-coefficient equation of the paper's linear-solver
 * section (AMReX, arXiv 2009.12009, Sec. "Linear Solvers"):
 *
 *        a * alpha * phi - b * div(beta grad phi) = rhs,
 *
 * phi, rhs and alpha at cell centres, beta on cell faces, on a BoxArray (Sec. "Basic
 * data structures") with one ghost cell per box (Sec. "Containers for mesh data").  The
 * solver is a multigrid V-cycle: ghost-cell exchange (Sec. "Operations on a level",
 * fused into one gather kernel as in Sec. "Communication"), red-black Gauss-Seidel
 * smoothing, residual, average-down restriction and piecewise-constant interpolation
 * (Sec. "Operations between levels"), box aggregation on coarse levels and a BiCGStab
 * bottom solve (Sec. "Linear Solvers").
 *
 * Conventions
 *   - Every pointer to field data is a DEVICE pointer.  Pointers to index lists, scalars,
 *     parameter and info structs are HOST pointers.
 *   - The caller owns all device memory: the fields it passes and one workspace buffer
 *     (gmg_workspace_size / gmg_set_workspace).  The library never allocates device
 *     memory; it keeps the workspace pointer until it is replaced or the context is
 *     destroyed, and borrows field pointers for the duration of a call only.
 *   - All device work is ordered on the stream given to gmg_create.  Calls that return a
 *     host-visible result (norms, iteration counts) synchronise that stream.
 *   - Field layout ("boxed layout"): per MG level and element type, each box is a
 *     ghosted 3-D block, x fastest.  Valid cell (i,j,k), i in [0,nx), lives at element
 *         box_offset + (gx + i) + sx * ((j + 1) + (ny + 2) * (k + 1)),
 *     with gx = 8 for every element type (so the first valid cell of a row is 16-byte
 *     aligned for bfloat16, 32-byte for float, 64-byte for double) and sx = the row
 *     stride returned by gmg_mg_layout (a multiple of 32 elements).  Offsets count
 *     elements, so buffers of different element types on one level share offsets.  Ghost cells sit at
 *     i = -1, i = nx, j = -1, ... .  Face arrays use the same layout: slot i holds the
 *     face at i - 1/2, i in [0, nx].  gmg_pack / gmg_unpack convert to and from a dense
 *     array over the level's domain.
 *   - Errors: every call returns a gmg_status.  Negative values are errors; the message
 *     of the last failing call on a context is returned by gmg_last_error.  No call
 *     aborts the process or traps on the device.
 */
#ifndef GMG_H
#define GMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmg_ctx gmg_ctx;

typedef enum {
  GMG_OK = 0,
  GMG_ERR_BAD_INPUT = -1,      /* invalid arguments, geometry or unsolvable singular rhs */
  GMG_ERR_NOT_CONVERGED = -2,  /* max_iter reached; the last iterate is returned */
  GMG_ERR_DIVERGED = -3,       /* non-finite residual */
  GMG_ERR_CUDA = -4,           /* a CUDA runtime call failed */
  GMG_ERR_DEVICE_TIMEOUT = -5, /* a bounded device-side wait ran out */
  GMG_ERR_NO_WORKSPACE = -6,   /* workspace missing or too small for the request */
  GMG_ERR_STATE = -7           /* call out of order (e.g. solve before coefficients) */
} gmg_status;

/* Boundary condition of one domain side (Sec. "Basic data structures": BCRec; Sec.
   "Linear Solvers": the operator equation's boundary conditions).  Walls are homogeneous
   inside the solver: a Dirichlet ghost is minus the adjacent interior value (phi = 0 on the
   face), a Neumann ghost equals it (zero normal derivative); the face beta of a wall is the
   interior cell's.  Nonzero wall values (phi = g on a Dirichlet face, outward normal
   derivative g on a Neumann face) enter through gmg_wall_values_rhs.  A problem without a
   Dirichlet wall and with a = 0 is singular (constants in the null space).
   GMG_BC_DIRICHLET0 is the older name of GMG_BC_DIRICHLET.
   GMG_BC_DIRICHLET_QUAD: a Dirichlet side whose ghost is the parabola through the wall
   value and the two nearest interior cells, read half a cell outside the face: ghost =
   8g/3 - 2 phi_0 + phi_1 / 3 (exact for quadratics; the linear rule 2g - phi_0 is exact for
   linear functions only).  Boxes one cell thick along the wall normal keep the linear rule.
   The operator is then not symmetric: a wall cell's row holds the extra entry
   -b beta_f / (3 h^2) on phi_1.  Gauss-Seidel solves each wall cell's row exactly (the
   -2 phi_0 part is in the diagonal).  Taken on every multigrid level.  Not offered with:
   composite (AMR) contexts, conjugate gradients (krylov = 2, bottom_solver = 1),
   trilinear interpolation (prolongation = 1).  The transpose, adjoint solve and beta
   gradient of a one-level context take it into account. */
typedef enum {
  GMG_BC_PERIODIC = 0,
  GMG_BC_DIRICHLET = 1,
  GMG_BC_DIRICHLET0 = 1,
  GMG_BC_NEUMANN = 2,
  GMG_BC_DIRICHLET_QUAD = 3
} gmg_bc;

/* Arithmetic of the V-cycle.  FP64: everything in double.  MIXED_FP32: the V-cycle
   (smoothing, residual, restriction, interpolation) runs in float inside an FP64
   iterative-refinement loop (FP64 outer residual and solution update, FP64 bottom
   solve).  MIXED_BF16: as MIXED_FP32 with the V-cycle's correction and residual
   stored as bfloat16 (float arithmetic, float coefficients). */
typedef enum { GMG_FP64 = 0, GMG_MIXED_FP32 = 1, GMG_MIXED_BF16 = 2 } gmg_precision;

/* Element types of boxed-layout buffers. */
typedef enum { GMG_DT_F64 = 0, GMG_DT_F32 = 1, GMG_DT_BF16 = 2 } gmg_dtype;

typedef struct {
  int nu1;              /* pre-smoothing sweeps (red + black), default 2 */
  int nu2;              /* post-smoothing sweeps, default 2 */
  int max_iter;         /* outer iterations, default 100 */
  int bottom_max_iter;  /* BiCGStab iterations, default 200 */
  double bottom_tol;    /* BiCGStab relative L-inf tolerance, default 1e-4 */
  int precision;        /* gmg_precision, default GMG_FP64 */
  int project_mean;     /* singular (no Dirichlet wall, a = 0): project a nonzero-mean rhs
                           instead of returning GMG_ERR_BAD_INPUT; default 0 */
  int use_graph;        /* 1 (default): replay one outer iteration as a captured CUDA graph
                           (one level and batched: the V-cycle, update and residual; several
                           AMR levels: the composite iteration, and in the adjoint solve its
                           two preconditioner-and-transpose steps); 0: direct launches */
  int profile;          /* record CUDA events around every finest-level smoother and
                           outer-residual launch (inside the graph too; with fused sweeps
                           the region pass of each sweep); default 0 */
  int fused_coarse;     /* 1: each problem's V-cycle levels from the first one with at most
                           512 of its cells (never level 0) down to its bottom run as ONE
                           thread block per problem (same arithmetic as the per-level
                           launches; only the bottom solve's dot products add in another
                           order); 0: one grid launch per step on every level; 2 (default):
                           the gmg_autotune choice, 1 before tuning */
  int fused_sweep;      /* 1 or 2: on MG levels of at least 2^17 smoothed cells whose ghosts are
                           pushed, the colour passes of each smoothing step (up to 4, e.g.
                           black, red, black after the residual's red half-sweep) run as ONE
                           dataflow launch: items of ~128 cells (box, plane, rows) of every
                           pass are handed out to warps in an order where an item starts once
                           the previous pass has finished on the z-slabs it reads, so the
                           second colour's reads can come from L2.  Every value is computed
                           from the operands of the two-pass sweep: results are bitwise those
                           of fused_sweep = 0.  0 (default): one launch per colour -- measured
                           faster on GB300 (abec256 level 0: 165 us per colour pass in FP64,
                           115 in float, against ~270 for the dataflow launch, whose per-item
                           GPU-scope release/acquire dominates).  A dependency wait that gives up
                           (it cannot in a correct build) makes the call return
                           GMG_ERR_DEVICE_TIMEOUT. */
  int ghost_push;       /* 1: in the V-cycle the smoother and the interpolation write every
                           new value also into the ghost cells that copy it, so the ghost
                           exchanges before each colour and before the restriction are not
                           needed (levels whose every box face is copied whole into one
                           ghost rectangle and whose periodic lengths are all even, so a
                           ghost has its source's colour); same values as the exchange.
                           0: ghost exchange before every colour.  2 (default): per level,
                           the gmg_autotune choice; before tuning, push on levels of fewer
                           than 2^22 cells (where the exchange is launch-latency bound) */
  int vector_smooth;    /* 1: float and bfloat16 colour sweeps on levels whose box widths
                           are multiples of 4 run one thread per 4 consecutive cells with
                           128-bit (float) / 64-bit (bfloat16) loads, and double sweeps read
                           each cell pair of every array with one 128-bit load; bitwise the
                           same results as one thread per cell pair with scalar loads (0).
                           2 (default): per level, the gmg_autotune choice; before tuning,
                           bfloat16 only */
  int pdl;              /* 1: the V-cycle kernels are launched for programmatic dependent
                           launch -- each may be scheduled while its predecessor finishes
                           and waits for it on the device before touching memory; 0: plain
                           launches; 2 (default): dependent launch outside CUDA graph
                           capture only.  Same results. */
  int fuse_residual_sweep; /* 1 (default): the outer residual kernel also performs the
                           first red half-sweep of the next V-cycle on level 0 (from a zero
                           correction it is e = r / D on red cells, 0 on black), saving one
                           pass over the finest level per iteration; 0: separate.  Same
                           results (up to the sign of zero corrections). */
  int krylov;           /* top-level method of gmg_solve (Sec. "Linear Solvers": native
                           Krylov solvers next to multigrid).  0 (default): the multigrid
                           iteration phi += V(rhs - A phi).  1: BiCGStab preconditioned on the
                           right by one V-cycle per application.  2: conjugate gradients
                           preconditioned by the symmetric V-cycle (post-smoothing colours
                           reversed, whatever post_reverse says; A must be symmetric, which
                           it is for one level).  Krylov vectors are FP64 and need a
                           workspace sized with krylov != 0; the V-cycle runs in `precision`.
                           One-level, single-problem contexts.  The stopping test uses the
                           recursive residual of the Krylov recurrence.
                           With krylov = 0 the multigrid iteration can stall on coefficients
                           of very high contrast (measured: beta = exp(3 N(0,1)), 8 decades,
                           stops near 1e-5 and returns GMG_ERR_NOT_CONVERGED after max_iter);
                           krylov = 2 (or 1) reaches 1e-10 there -- use it when a solve reports
                           a residual history that levels off. */
  int bottom_solver;    /* 0 (default): BiCGStab bottom; 1: conjugate gradients (the bottom
                           operator is symmetric) */
  int post_reverse;     /* 1: post-smoothing sweeps take black before red, the reverse of
                           pre-smoothing (a symmetric V-cycle); 0 (default): red first */
  int fuse_correction;  /* 1 (default): in the multigrid iteration, the last colour pass of
                           the finest level's post-smoothing also adds the correction to phi
                           (one pass over phi and e fewer per iteration); 0: separate.  Same
                           results. */
  int settled_zero;     /* 1 (default): an FP64 residual taken right after a Gauss-Seidel
                           half-sweep (the restriction after pre-smoothing; the multigrid
                           iteration's residual after post-smoothing) stores 0 for the cells of
                           the colour updated last, except next to walls:
                           such a cell reads only the other colour, unchanged since the update
                           made its residual zero up to rounding.  0: every residual is
                           computed.  Results differ by rounding. */
  int flow_warps;       /* resident warps per SM of the dataflow sweep launches (each warp
                           takes one work item at a time); 0 (default): 32.  Same results. */
  int flow_lag_kcells;  /* dataflow sweeps: in the hand-out order, the items of colour pass
                           c trail those of pass c - 1 they depend on by this many x 1024
                           cells of the level (more lag: fewer waits, more data between the
                           passes that L2 must hold); 0 (default): 1024 (2^20 cells).  Same
                           results. */
  int serpentine;       /* 1 (default): the level-sweep kernels of a level (smoothers, residual,
                           residual-restriction, interpolation) alternate the direction in
                           which they walk the level's boxes, so each starts on the data the
                           previous one touched last (still in L2); 0: always first box first.
                           Same results. */
  int prolongation;     /* interpolation of the coarse correction in the V-cycle (Sec.
                           "Operations between levels" names interpolation without its order):
                           0 (default) piecewise constant; 1 trilinear -- weights 3/4 and 1/4
                           per axis from the parent and its neighbours towards the fine cell,
                           the coarse correction extended past walls by the homogeneous rule
                           (Dirichlet: negative mirror, Neumann: mirror), periodic images
                           wrapped.  Trilinear turns the one-block coarse end (fused_coarse) off
                           and, with this smoother, needs more V-cycles (abec64: 12 against 9).
                           The interpolation between AMR levels is not affected. */
  int wave_sweep;       /* 1: on MG levels whose ghosts are pushed, whose box widths are even and
                           whose boxes meet face to face (every face copied whole from one box,
                           or a wall; z-neighbours given opposite marching directions), each
                           red-first Gauss-Seidel sweep runs as ONE wavefront launch: thread
                           blocks take bands of rows of a box and march through its planes a
                           slab at a time, red cells of the slab, a report, then the black
                           cells whose reds on both sides are done; a block waits (bounded) for
                           the bands beside it to report before those black cells.  Bitwise the
                           results of 0; the first pre-smoothing sweep from a zero correction
                           computes its red cells as r / D itself (the outer residual then skips
                           that half-sweep).  Levels whose problems have more bands than the
                           device holds at once, and the black-first post-smoothing of the
                           symmetric V-cycle, keep one launch per colour.  A wait that gives up
                           (it cannot in a correct build) makes the call return
                           GMG_ERR_DEVICE_TIMEOUT.  0 (default): one launch per colour -- measured
                           faster on GB300 (abec256 level 0: 350 us per FP64 sweep, 228 in float,
                           against 508 and 329 for the wavefront launch, whose threads each own a
                           column of cells and so have one update's loads in flight at a time). */
  int tail_dense;       /* 1 (default): the coarse end of fused_coarse holds each problem's
                           levels in shared memory, every level as one padded array over the
                           problem's domain there (a problem's boxes tile it), loaded once
                           per V-cycle, so each of its steps reads on-chip memory instead of
                           global memory; problems whose levels do not fit keep the global-
                           memory coarse end.  Bitwise the results of 0; 0: the coarse end
                           reads and writes the levels' global arrays at every step. */
  int fuse_restriction_sweep; /* 1 (default): the residual restriction into each coarse level
                           that the grid launches smooth also performs that level's first red
                           half-sweep from the zero correction (a red cell becomes r / D, a
                           black one 0, every valid cell written, ghosts pushed), saving a
                           colour pass and a zero fill per level and V-cycle; the same values
                           as 0 (a -0.0 right-hand side aside). */
  int fuse_prolongation; /* 1 (default): where a level's post-smoothing starts with a red pass
                           of the grid launches and the coarser level's ghosts are pushed
                           (linear walls, piecewise-constant interpolation, red-first
                           post-smoothing), that red pass reads each neighbour as the
                           interpolation of the coarse correction would leave it (its value
                           plus its parent's) and the interpolation pass is not launched -- the
                           black cells it would have changed are rewritten by the black pass
                           that follows without being read.  Where that pass cannot (the fine
                           level exchanges its ghosts), the coarser level's last post-smoothing
                           pass adds its final values to the children instead (every coarse box
                           with one child box of twice its extent).  Bitwise the results of 0.
                           1 leaves out FP64 fine levels of at least 2^22 cells, whose passes
                           are bound by the FP64 pipe (the added additions cost more than the
                           pass they save); 2: every level where it applies. */
  int fork_bottoms;     /* 1 (default): in a batched context, the bottom solves of the problems
                           whose bottom is a level other problems go below run on a second
                           stream of the context, overlapping those problems' coarser levels,
                           and are joined before the interpolation from that level.  Same
                           results; 0: one stream. */
} gmg_params;

typedef struct {
  int iterations;        /* outer (V-cycle) iterations taken */
  int status;            /* gmg_status of the solve */
  double rhs_norm;       /* ||rhs||_inf (after mean projection for singular problems) */
  double initial_resid;  /* ||r_0||_inf */
  double final_resid;    /* ||r||_inf at exit, FP64 residual */
  int hist_len;          /* entries in resid_hist */
  double resid_hist[256];/* ||r||_inf after each iteration (index 0 = initial) */
  int bottom_iters;      /* BiCGStab iterations of the last bottom solve */
  double solve_ms;       /* wall time of the solve call (host clock) */
  long long kernel_launches; /* kernels launched by the call (graph nodes counted per replay) */
  double smooth0_ms;     /* with profile: summed device time of finest-level smoother launches */
  int smooth0_launches;  /* ... and their number */
  double resid0_ms;      /* with profile: summed device time of the outer FP64 residual launches */
  int resid0_launches;
  int smooth0_passes;    /* colour passes (red or black half-sweeps) covered by the timed
                            smoother launches (a dataflow launch covers several) */
} gmg_solve_info;

/* ---------------------------------------------------------------- context */

/* Default parameters of the solve (Sec. "Linear Solvers": the multigrid solver's settings --
   2 + 2 red-black Gauss-Seidel sweeps per V-cycle, BiCGStab bottom to 1e-4 in at most 200
   iterations -- and the launch options of this implementation, which change no result
   unless documented otherwise).  p: host pointer, written. */
gmg_status gmg_default_params(gmg_params* p);

/* Create a context bound to a CUDA stream (cudaStream_t passed as void*; NULL = the
   legacy default stream).  *out receives the context.  A context is one problem of the
   operator equation of Sec. "Linear Solvers" posed on the data model of Sec. "Basic data
   structures" (Geometry, BoxArray, BCRec) with one ghosted array per box (Sec.
   "Containers for mesh data"); it owns host metadata only (device memory is the caller's,
   see gmg_set_workspace).  GMG_ERR_BAD_INPUT if out is NULL. */
gmg_status gmg_create(gmg_ctx** out, void* cuda_stream);
/* Destroy a context (its cached tables and CUDA graphs; not the caller's device memory):
   the problem of Sec. "Linear Solvers" on the data model of Sec. "Basic data structures",
   as made by gmg_create.  NULL is accepted. */
gmg_status gmg_destroy(gmg_ctx* ctx);
/* Message of the last error on ctx ("" if none); no counterpart in the paper (the error
   model of this library: a status code and a message, never an abort).  ctx may be NULL
   (creation errors).  The returned string lives until the next call on ctx. */
const char* gmg_last_error(const gmg_ctx* ctx);

/* ---------------------------------------------------------------- geometry */

/* Problem domain (Sec. "Basic data structures": Geometry + BCRec): inclusive cell-index
   box [lo, hi], physical extent [prob_lo, prob_hi], one boundary condition per side.
   A periodic direction must be periodic on both sides. */
gmg_status gmg_define_domain(gmg_ctx* ctx, const int lo[3], const int hi[3], const double prob_lo[3],
                             const double prob_hi[3], const int bc_lo[3], const int bc_hi[3]);

/* BoxArray of AMR level `lev`: nboxes boxes given as box_lohi[6*b + 0..2] = lo,
   [6*b + 3..5] = hi (inclusive), disjoint.
   lev 0: the boxes cover the domain; builds the multigrid hierarchy (per-box coarsening,
     then aggregation into one box, Sec. "Linear Solvers").  Resets any AMR level above.
   lev >= 1 (composite form, Sec. "Basic data structures": refinement ratio; Sec.
     "Operations between levels"), defined in order, up to GMG_MAX_AMR_LEVELS levels in
     all; defining level lev drops the levels above it: ref_ratio must be 2; boxes in level
     lev's index space (the domain scaled by 2^lev), aligned to the ratio, each coarsened
     box inside one box of level lev - 1, faces either shared with another box of the level
     or wholly on its coarse/fine boundary, and at least one uncovered cell of level lev - 1
     between the level and any other of its boxes, a wall or the edge of level lev - 1 (the
     coarse/fine interpolation reads coarse neighbours).  Single-problem contexts.  Call
     before gmg_workspace_size; the workspace then holds every level.  The adjoint solve,
     apply_transpose and the beta gradient over three or more levels also need every level
     at least two of its cells inside the coarse/fine boundary of the level it refines (the
     two fine cells a coarse/fine ghost reads must not be covered): GMG_ERR_BAD_INPUT
     otherwise. */
#define GMG_MAX_AMR_LEVELS 4
gmg_status gmg_define_level(gmg_ctx* ctx, int lev, int nboxes, const int* box_lohi, int ref_ratio);

/* Convenience: BoxArray of level `lev` = the domain chopped into boxes of at most
   max_grid_size cells per axis (Sec. "Regridding": max_grid_size). */
gmg_status gmg_chop_domain(gmg_ctx* ctx, int lev, int max_grid_size);

/* Number of multigrid levels of the hierarchy (level 0 = the user's BoxArray; the coarser
   levels by per-box coarsening, then aggregation, Sec. "Linear Solvers"). */
gmg_status gmg_mg_nlevels(const gmg_ctx* ctx, int* nlevels);

/* MG level m: number of boxes and domain (dom[0..2] = lo, dom[3..5] = hi) (Sec. "Basic
   data structures": a level's BoxArray and Geometry). */
gmg_status gmg_mg_level_info(const gmg_ctx* ctx, int m, int* nboxes, int* dom);

/* MG level m: boxes (6 ints each) and, for each box, the box of level m+1 that holds its
   coarsened image (-1 on the bottom level) (Sec. "Linear Solvers": the coarsened
   BoxArrays of the multigrid hierarchy).  Either pointer may be NULL. */
gmg_status gmg_mg_level_boxes(const gmg_ctx* ctx, int m, int* box_lohi, int* parents);

/* The work tiles of the wavefront red-black sweep on MG level m (the smoother of Sec. "Linear
   Solvers"; the tiling itself has no counterpart in the paper): *ntiles receives their number
   and *ppt the cell pairs per thread (0: the level keeps one launch per colour).  out (may be
   NULL) receives, for at most cap tiles in hand-out order, 13 ints each: box, first row y0,
   end row y1, marching direction (0: planes upward), the tiles across the x-, x+, y-, y+ sides
   and the z-, z+ faces (-1: a wall), the red planes the two z tiles must have reported before
   the black cells of the first (z-) and last (z+) plane, and the tile's problem (batched
   form).  Host only (no device work). */
gmg_status gmg_wave_tiles(const gmg_ctx* ctx, int m, int* ntiles, int* ppt, int* out, int cap);

/* The coarse ends that start on MG level m (fused_coarse; the coarse levels of the V-cycle
   of Sec. "Linear Solvers" run by one thread block per problem): *nblocks receives how many
   (one per problem; 0: none starts there) and *dense_bytes the shared memory of their dense
   form in element type dt (gmg_dtype; 0: they keep the global-memory form, because a
   problem's boxes do not tile its domain on one of the levels or the arrays do not fit).
   Host only (no device work).  Either pointer may be NULL. */
gmg_status gmg_tail_plan(const gmg_ctx* ctx, int m, int dt, int* nblocks, long long* dense_bytes);

/* Boxed layout of MG level m for element type dt: total elements, per-box element
   offsets (nboxes entries, may be NULL) and row strides sx (nboxes entries, may be
   NULL) (Sec. "Containers for mesh data": one array per box, ghost cells included). */
gmg_status gmg_mg_layout(const gmg_ctx* ctx, int m, int dt, int64_t* nelems, int64_t* box_offsets, int* row_strides);

/* FP64 boxed layout of AMR level lev (0: MG level 0; 1: the fine level) (Sec.
   "Containers for mesh data"). */
gmg_status gmg_layout(const gmg_ctx* ctx, int lev, int64_t* nelems, int64_t* box_offsets);

/* Boxes of AMR level lev (count, 6 ints each, row strides); NULL pointers are skipped
   (Sec. "Basic data structures": the BoxArray of an AMR level). */
gmg_status gmg_amr_level_boxes(const gmg_ctx* ctx, int lev, int* nboxes, int* box_lohi, int* row_strides);

/* Dense (nz, ny, nx) FP64 array over the bounding box of AMR level lev's boxes (level 0:
   the domain) <-> FP64 boxed layout of that level (valid cells only) (Sec. "Containers for
   mesh data").  Device pointers; GMG_ERR_BAD_INPUT for an undefined level. */
gmg_status gmg_pack_amr(gmg_ctx* ctx, int lev, const double* dense, double* boxed);
gmg_status gmg_unpack_amr(gmg_ctx* ctx, int lev, const double* boxed, double* dense);

/* Dense (nz, ny, nx) FP64 device array over MG level m's domain <-> boxed layout of
   element type dt (Sec. "Containers for mesh data").  pack writes valid cells only
   (ghosts untouched); unpack reads valid cells only. */
gmg_status gmg_pack(gmg_ctx* ctx, int m, int dt, const double* dense, void* boxed);
gmg_status gmg_unpack(gmg_ctx* ctx, int m, int dt, const void* boxed, double* dense);

/* ------------------------------------------------------------- coefficients */

/* Scalars a and b of the operator equation a alpha phi - b div(beta grad phi) = rhs (Sec.
   "Linear Solvers").  Any finite values; a problem with a = 0 and no Dirichlet wall is
   singular.  Coefficients of every level are rebuilt at the next solve. */
gmg_status gmg_set_scalars(gmg_ctx* ctx, double a, double b);

/* Cell-centred alpha of AMR level lev (FP64, that level's boxed layout, device), the alpha
   of the operator equation (Sec. "Linear Solvers"; coarse levels take the mean of 8
   children, Sec. "Operations between levels").  Not calling it means alpha = 1.  The
   library copies it (the pointer is not kept). */
gmg_status gmg_set_acoef(gmg_ctx* ctx, int lev, const double* alpha_cc);

/* Cell-centred beta of AMR level lev (FP64, that level's boxed layout, device), from which
   the face beta of the operator equation (Sec. "Linear Solvers") is made: face
   beta = harmonic mean of the two cells, the interior cell's value on a wall face and
   (level 1) on a coarse/fine face.  Builds the coefficients of every MG level (coarse
   alpha = mean of 8 children, coarse face beta = mean of the 4 fine faces) once every
   defined AMR level has its beta.  Needs the workspace. */
gmg_status gmg_set_bcoef_cell(gmg_ctx* ctx, int lev, const double* beta_cc);

/* Face beta given directly (the face-centred beta of the operator equation, Sec. "Linear
   Solvers"): three FP64 face arrays in the boxed layout (slot i = face i - 1/2).  Builds
   every MG level's coefficients.  Needs the workspace. */
gmg_status gmg_set_bcoef_face(gmg_ctx* ctx, int lev, const double* bx, const double* by, const double* bz);

/* Scaled face weights w_d = b * beta_d / h_d^2 and diagonal D = a*alpha + sum of the six
   weights (plus 2 w_f per quadratic Dirichlet wall face f of the cell) of MG level m (the
   discrete operator of Sec. "Linear Solvers" on that level),
   copied into caller buffers of element type dt (NULL to skip). */
gmg_status gmg_get_coeffs(gmg_ctx* ctx, int m, int dt, void* wx, void* wy, void* wz, void* diag);

/* ---------------------------------------------------------------- workspace */

/* Bytes of device workspace needed for solves with parameters p (NULL = defaults; a
   mixed precision needs its float buffers in addition to the FP64 ones).  The workspace
   plays the part of the pre-allocated memory pool of Sec. "Memory management" (one large
   block handed out in pieces), except that the caller allocates it.  A context with a
   quadratic Dirichlet side (GMG_BC_DIRICHLET_QUAD) always includes the Krylov vectors
   (its adjoint solve is a BiCGStab on A^T). */
gmg_status gmg_workspace_size(const gmg_ctx* ctx, const gmg_params* p, size_t* bytes);

/* Hand the library a device buffer of at least gmg_workspace_size bytes, 256-byte
   aligned (Sec. "Memory management": the library carves every level array and table out
   of this one block).  Uploads the index tables.  The buffer stays in use until replaced;
   GMG_ERR_NO_WORKSPACE if it is too small. */
gmg_status gmg_set_workspace(gmg_ctx* ctx, void* dptr, size_t bytes);

/* ------------------------------------------------------------------- solve */

/* Sec. "Linear Solvers": solve the operator equation by geometric multigrid (V-cycles with a
   Krylov bottom solver; over several AMR levels, the multi-level solve with the coarse/fine
   operations of Sec. "Operations between levels").
   Solve A phi = rhs from phi = 0 (phi's input content is ignored) until
   ||rhs - A phi||_inf <= max(tol_rel * ||rhs||_inf, tol_abs) or p->max_iter outer
   iterations.  phi[l], rhs[l]: FP64 device arrays in AMR level l's layout.  One level:
   the multigrid V-cycle iteration.  Several AMR levels: A is the composite operator on the
   cells not covered by a finer level (fine ghosts on each coarse/fine boundary by quadratic
   interpolation from the level below, cells next to a finer level refluxed: the mean of
   the 4 fine fluxes replaces the coarse flux on a shared face), solved by the composite
   multigrid iteration (down the levels: smoothing of each refined level's correction,
   restriction of its correction residual and reflux into the level below; a V-cycle of
   level 0's hierarchy; up: interpolation and smoothing); with use_graph one captured
   iteration is replayed.  On return covered cells of phi[l] hold the average of the finer
   solution, and the rhs entries of covered cells are ignored; FP64 only.  info may be
   NULL.  Returns GMG_OK, GMG_ERR_NOT_CONVERGED (phi holds the last iterate),
   GMG_ERR_DIVERGED or GMG_ERR_BAD_INPUT (nonzero-mean rhs of a singular problem without
   project_mean; with several levels the mean is volume-weighted over the composite
   cells). */
gmg_status gmg_solve(gmg_ctx* ctx, void* const* phi, const void* const* rhs, double tol_rel, double tol_abs,
                     const gmg_params* p, gmg_solve_info* info);

/* out = A phi, the operator of Sec. "Linear Solvers" (FP64; phi's ghost cells are
   overwritten).  Several AMR levels: the composite operator (coarse/fine interpolation and
   refluxing, Sec. "Operations between levels"); covered entries of out are 0. */
gmg_status gmg_apply(gmg_ctx* ctx, void* const* out, void* const* phi);

/* out = A^T y, the transpose of the operator of Sec. "Linear Solvers" (the transpose
   itself has no counterpart in the paper; it serves the adjoint below).  One level: A is
   symmetric (same as gmg_apply) unless a side is GMG_BC_DIRICHLET_QUAD; then A^T moves each
   quadratic wall cell's entry -w/3 on phi_1 (w = b beta_f / h^2) into phi_1's row (single-
   problem contexts; y's ghosts are overwritten).  Several AMR levels: the
   transpose of the composite operator (the level stencils plus, for each pair of
   consecutive levels, the transposed interpolation and reflux couplings); covered entries
   of y are taken as 0 and those of out are 0; y's ghosts are overwritten. */
gmg_status gmg_apply_transpose(gmg_ctx* ctx, void* const* out, void* const* y);

/* Adjoint of the solve of Sec. "Linear Solvers" (no counterpart in the paper: the
   differentiation of its operator equation).
   Adjoint solve A^T lambda = g (FP64), so that lambda = dL/d(rhs) for a loss L(phi) with
   dL/dphi = g.  One level: a forward solve (A symmetric); with a GMG_BC_DIRICHLET_QUAD side,
   BiCGStab on A^T right-preconditioned by the V-cycle of A (the Krylov vectors of the
   workspace; precision of p for the V-cycle), to the same stopping test.  Several AMR levels: BiCGStab on A^T,
   right-preconditioned by the composite multigrid correction of A, to ||g - A^T lambda||_inf
   <= tol_rel ||g||_inf (max_iter Krylov iterations).  Singular problems (no Dirichlet wall,
   a = 0): g is projected onto the range of A^T (g - V sum(g)/sum(V), V the cell volumes;
   one level: g minus its mean) and lambda returned with zero sum.  lambda, g as in
   gmg_solve; covered entries of g are ignored and those of lambda are 0. */
gmg_status gmg_solve_adjoint(gmg_ctx* ctx, void* const* lambda, const void* const* g, double tol_rel,
                             const gmg_params* p, gmg_solve_info* info);

/* Derivative of the solve of Sec. "Linear Solvers" with respect to its beta (no counterpart
   in the paper: the differentiation of its operator equation).
   Gradient of a loss with respect to the cell-centred beta of each level, given the
   solution phi and the adjoint lambda:  per face, dL/dbeta_face = -lambda^T (dA/dbeta_face) phi
   (-(b/h^2)(phi_R - phi_L)(lambda_R - lambda_L) on an interior face; on a coarse/fine face
   also the reflux row's share), then through the rule that made the face value from cell
   beta (harmonic mean: d/dbeta_L = 2 beta_R^2 / (beta_L + beta_R)^2; wall and coarse/fine
   faces: 1 for the adjacent cell).  Uses the beta last passed to gmg_set_bcoef_cell.
   dbeta[l]: FP64 output in level l's layout for every AMR level (covered cells get 0: their
   beta shapes only the correction operator).  phi's and lambda's ghosts are overwritten. */
gmg_status gmg_beta_grad(gmg_ctx* ctx, void* const* dbeta, void* const* phi, void* const* lambda);

/* ------------------------------------------------------------- wall values */
/* Inhomogeneous boundary conditions of the operator equation (Sec. "Linear Solvers";
   Sec. "Basic data structures": BCRec).
   Nonzero values on the level-0 walls of a single-level, single-problem context.  A wall
   value g makes the wall's ghost rule affine -- Dirichlet: ghost = 2g - interior (the line
   through the interior value and g on the face); Neumann: ghost = interior + h g (h the cell
   size normal to the face) -- and its phi-independent part is a constant of the operator:
   A_g phi = A_0 phi + A_g(0).  Solving A_0 phi = rhs - A_g(0) (gmg_solve, homogeneous walls)
   gives the solution with the wall values; the stopping test is then relative to
   ||rhs - A_g(0)||_inf, the initial residual.

   values[f], f = 2*d + side (x-, x+, y-, y+, z-, z+): FP64 device array over face f's two
   tangential axes in increasing order, the lower one fastest (n_t1 * n_t2 values; for a
   face normal to y: x fastest, then z), or NULL for g = 0.  A periodic face must be NULL;
   a context with several problems or several AMR levels accepts only NULLs (GMG_ERR_BAD_INPUT).
   All work is enqueued on the context stream; nothing is synchronised. */

/* Wall values (Sec. "Linear Solvers": inhomogeneous boundary conditions of the operator
   equation).  out = rhs - A_g(0): rhs plus, in each cell next to a wall face with a value, 2 w g
   (Dirichlet; 8 w g / 3 under the quadratic rule) or w h g (Neumann), w = b beta_face / h^2
   the face's weight; faces are added
   in the order x-, x+, y-, y+, z-, z+.  rhs, out: FP64 level-0 boxed device arrays; out may
   equal rhs (in place); otherwise rhs is copied first. */
gmg_status gmg_wall_values_rhs(gmg_ctx* ctx, void* out, const void* rhs, const void* const* values);

/* Wall values, adjoint (no counterpart in the paper: the differentiation of the operator
   equation's boundary data).  The transpose of the map g -> rhs - A_g(0): dvalues[f][t] = c * lambda[q] for the wall
   cell q behind face position t, c = 2 w (Dirichlet; 8 w / 3 quadratic) or w h (Neumann); with lambda the
   adjoint (gmg_solve_adjoint of dL/dphi) this is dL/dg.  dvalues[f]: FP64 device arrays in
   the layout of values above, written whole; NULL entries are skipped. */
gmg_status gmg_wall_values_grad(gmg_ctx* ctx, const void* lambda, void* const* dvalues);

/* Wall values, beta gradient (no counterpart in the paper: the differentiation of the
   operator equation of Sec. "Linear Solvers").  gmg_beta_grad for a solution with wall
   values: phi's wall ghosts take the affine rule
   (values as above, NULL entries g = 0) before the face terms, so a wall face adds
   lambda_q w (ghost - phi_q) / beta_face to its cell.  values == NULL: gmg_beta_grad. */
gmg_status gmg_beta_grad_walls(gmg_ctx* ctx, void* const* dbeta, void* const* phi, void* const* lambda,
                               const void* const* values);

/* ------------------------------------------------ individual hot-path steps */
/* Each step acts on MG level m with caller buffers of element type dt in that level's
   boxed layout.  Coefficients come from the last gmg_set_bcoef_* call (float copies
   for GMG_DT_F32 / GMG_DT_BF16 fields need a mixed-precision workspace). */

/* Sec. "Operations on a level" (FillBoundary; fused into one gather kernel as in Sec.
   "Communication").
   FillBoundary: copy every face ghost cell from the box that owns it (periodic images
   included) or apply the homogeneous wall rule (Dirichlet: minus, Neumann: plus the
   adjacent interior value).  colour = 0 or 1 fills only
   the ghosts whose global (i+j+k) parity is that colour; -1 fills all. */
gmg_status gmg_fill_boundary(gmg_ctx* ctx, int m, int dt, void* field, int colour);

/* One red-black Gauss-Seidel half sweep of colour 0 (red, i+j+k even) or 1 (black),
   preceded by the ghost fill it needs (the smoother of the geometric multigrid of Sec.
   "Linear Solvers"). */
gmg_status gmg_smooth(gmg_ctx* ctx, int m, int dt, void* phi, const void* rhs, int colour);

/* r = rhs - A phi (ghosts of phi filled first), the residual of the operator equation of
   Sec. "Linear Solvers" (its max-norm is a reduction of Sec. "Parallel Reductions").  r has
   element type rdt.  If norm is non-NULL, *norm receives ||r||_inf (synchronises the
   stream). */
gmg_status gmg_residual(gmg_ctx* ctx, int m, int dt, void* phi, const void* rhs, int rdt, void* r, double* norm);

/* Average-down restriction of a cell field from MG level m to m+1 (mean of 8 children;
   Sec. "Operations between levels": restriction by averaging fine data). */
gmg_status gmg_restrict(gmg_ctx* ctx, int m, int dt, const void* fine, void* coarse);

/* fine += piecewise-constant interpolation of coarse (MG level m+1 -> m; Sec. "Operations
   between levels": interpolation). */
gmg_status gmg_prolong_add(gmg_ctx* ctx, int m, int dt, const void* coarse, void* fine);

/* fine += trilinear interpolation of coarse (MG level m+1 -> m; Sec. "Operations between
   levels": interpolation, here of second order -- the gmg_params.prolongation = 1 option).
   Fills coarse's ghost cells first (faces, edges and corners, by the homogeneous boundary
   rule), so coarse's ghosts are overwritten. */
gmg_status gmg_prolong_add_trilinear(gmg_ctx* ctx, int m, int dt, void* coarse, void* fine);

/* BiCGStab on the bottom level: x = A_bottom^-1 rhs to bottom_tol (FP64 arithmetic,
   buffers of type dt) (Sec. "Linear Solvers": the Krylov bottom solve of the multigrid
   hierarchy).  *iters (host, may be NULL) receives the iteration count. */
gmg_status gmg_bottom_solve(gmg_ctx* ctx, int dt, const void* rhs, void* x, const gmg_params* p, int* iters);

/* One V-cycle on the correction equation of MG level 0: e = V(r), element type dt (Sec.
   "Linear Solvers": the geometric multigrid cycle). */
gmg_status gmg_vcycle(gmg_ctx* ctx, int dt, void* e, const void* r, const gmg_params* p);

/* -------------------------------------------------------------- autotuning */

/* Launch-shape autotuner (no counterpart in the paper).  For the V-cycle of the given
   precision it times, on this context's own levels and buffers (CUDA events, a few
   repetitions each), (1) per MG level: a red-black sweep four ways -- ghost exchange before
   each colour or ghost push, one thread per cell pair or per 4 cells (float/bfloat16) --
   and (2) whole V-cycles with the fused coarse end against per-level launches, and keeps
   the fastest of each.  Solves and V-cycles whose params have ghost_push = 2,
   vector_smooth = 2, fused_coarse = 2 (the defaults) use the choices; the results do not
   depend on them.  rhs: FP64 level-0 boxed right-hand side (device), used
   to fill the correction equation.  Clobbers the V-cycle work buffers only; drops cached
   graphs. */
gmg_status gmg_autotune(gmg_ctx* ctx, int precision, const void* rhs, const gmg_params* p);

/* Autotuner results (no counterpart in the paper).  The tuned choice for MG level m and
   precision: *push = bit 0 ghost push, bit 1 4-cell
   threads, -1 not tuned (no smoothing there); the best measured ms per sweep with push and
   with the exchange (0 if push is not possible there); *fused_coarse = 1/0/-1 and the
   measured ms per V-cycle with (fused) and without (levels) the fused coarse end.  Any
   output pointer may be NULL. */
gmg_status gmg_tuned(const gmg_ctx* ctx, int precision, int m, int* push, double* ms_push, double* ms_pull,
                     int* fused_coarse, double* ms_vcycle_fused, double* ms_vcycle_levels);

/* ------------------------------------------------------------ batched form */

/* The batched form (no counterpart in the paper; each problem is a Geometry + BoxArray of
   Sec. "Basic data structures" solved as in Sec. "Linear Solvers").
   Several independent problems in one context (the batched form of the solve: many
   solves with boxes of uneven sizes run as one set of launches per V-cycle step).
   Problem s has domain dom_lohi[6s..6s+5] (lo, hi inclusive), physical extent
   prob_lo[3s..], prob_hi[3s..], boundary conditions bc_lo[3s..], bc_hi[3s..] and
   nboxes[s] boxes; box_lohi lists the boxes of problem 0, then of problem 1, ... (6 ints
   each).  Every problem's boxes must be disjoint and cover its domain.  Each problem
   gets its own multigrid hierarchy (Sec. "Linear Solvers": per-box coarsening, then
   aggregation) and its own bottom level; MG level m of the context is the union of level
   m of every problem that still has one.  Replaces any previous definition. */
gmg_status gmg_define_batch(gmg_ctx* ctx, int nsolves, const int* dom_lohi, const double* prob_lo,
                            const double* prob_hi, const int* bc_lo, const int* bc_hi, const int* nboxes,
                            const int* box_lohi);

/* Number of independent problems in the context (1 after gmg_define_domain) (batched form,
   no counterpart in the paper). */
gmg_status gmg_num_solves(const gmg_ctx* ctx, int* nsolves);

/* Boxes of problem `solve` on MG level m: index of its first box and count (-1, 0 if the
   problem has no boxes on that level) (batched form; Sec. "Basic data structures"). */
gmg_status gmg_solve_boxes(const gmg_ctx* ctx, int m, int solve, int* first, int* count);

/* Batched form, Sec. "Containers for mesh data":
   gmg_pack / gmg_unpack for one problem: dense (nz, ny, nx) FP64 array over that
   problem's domain on MG level m <-> its boxes in the level's boxed layout. */
gmg_status gmg_pack_solve(gmg_ctx* ctx, int m, int dt, int solve, const double* dense, void* boxed);
gmg_status gmg_unpack_solve(gmg_ctx* ctx, int m, int dt, int solve, const void* boxed, double* dense);

/* Batched solve (Sec. "Linear Solvers" for each problem; the batching has no counterpart in
   the paper).
   Solve every problem of the context from phi = 0: phi and rhs are FP64 level-0 boxed
   buffers holding all problems.  Each problem stops at its own tolerance
   max(tol_rel * ||rhs_s||_inf, tol_abs) (or max_iter); problems that have converged are
   masked out of the remaining V-cycles, so each one performs exactly the iterations a
   solve of it alone would.  infos: nsolves entries (may be NULL).  Returns GMG_OK when all
   converged, else the worst status (GMG_ERR_DIVERGED before GMG_ERR_NOT_CONVERGED). */
gmg_status gmg_batch_solve(gmg_ctx* ctx, void* phi, const void* rhs, double tol_rel, double tol_abs,
                           const gmg_params* p, gmg_solve_info* infos);

/* ------------------------------------------------- allocation-free box solve */

/* BiCGStab solve of one box that allocates nothing (the paper has no counterpart to this
   entry point).  It is for callers that cannot allocate device memory when they solve:
   an operator inside another framework that is handed only its input and output
   tensors, code running while its own stream is being captured into a CUDA graph
   (cudaMalloc is not allowed during capture), or a host that forbids allocation after
   start-up.  Such callers cannot provide a workspace, so no context is used: inputs and
   output are plain dense device arrays (x fastest) and the seven BiCGStab vectors live
   in one static device array of the library.

   Solves A x = rhs on an nx * ny * nz box with A = diag - (weighted neighbours):
     (A x)_c = diag_c x_c - sum over the six faces f of c of w_f x_nbr(f),
   the same operator and the same BiCGStab iteration as gmg_bottom_solve (x0 = 0, stop
   at ||r||_inf <= tol ||r0||_inf, after max_iter iterations, or on breakdown; FP64).
     wx: (nx+1)*ny*nz face weights, face i-1/2 of cell (i,j,k) at i + (nx+1)*(j + ny*k);
     wy: nx*(ny+1)*nz, face j-1/2 at i + nx*(j + (ny+1)*k);
     wz: nx*ny*(nz+1), face k-1/2 at i + nx*(j + ny*k);
     diag, rhs, x: nx*ny*nz.  All device pointers; x is written.
   bc_lo/bc_hi: GMG_BC_PERIODIC (both sides; wraps inside the box), GMG_BC_DIRICHLET
   (ghost = minus the adjacent cell) or GMG_BC_NEUMANN (ghost = the adjacent cell).  singular != 0 projects rhs and x onto zero mean.
   iters: device int receiving the iteration count, or NULL.

   Limit: (nx+2)(ny+2)(nz+2) <= 65536; larger boxes return GMG_ERR_BAD_INPUT.  The static
   scratch (65536 * 7 doubles = 3.5 MiB) is held by every GPU that loads the library until
   the process exits.  All calls share it and it keeps the previous call's contents (the
   kernel initialises what it reads); calls whose kernels overlap on the GPU race on it
   and must be serialised by the caller.  The first call on a device resolves the scratch
   address (cudaGetSymbolAddress) with that device current; make that first call before
   any stream capture.  Work is enqueued on cuda_stream; errors are reported through the
   return value and gmg_last_error(NULL). */
gmg_status gmg_box_bicgstab_noalloc(void* cuda_stream, int nx, int ny, int nz, const int bc_lo[3], const int bc_hi[3],
                                    int singular, const double* wx, const double* wy, const double* wz,
                                    const double* diag, const double* rhs, double* x, int max_iter, double tol,
                                    int* iters);

/* ------------------------------------------------- sharding plan (host only) */
/* Box ownership and ghost exchange for a solve split across ranks (Sec. "Basic data
   structures": the DistributionMapping that assigns boxes to processes, by a space-filling
   curve; Sec. "Communication": ghost-cell exchange between processes; Sec. "Linear
   Solvers": coarse multigrid levels consolidated onto fewer processes).  These calls build
   the tables only: every solve of this library runs on one GPU.  Host pointers throughout. */

/* Sec. "Basic data structures" (DistributionMapping by a space-filling curve) and Sec.
   "Linear Solvers" (coarse levels consolidated):
   Owner rank of every box of MG level m (owner: nboxes ints): boxes sorted along a Morton
   (Z-order) curve of their low corners (problem by problem), the curve cut into nranks
   pieces of about equal cell counts.  A level with fewer than nranks * min_cells_per_rank
   cells is consolidated: every box on rank 0. */
gmg_status gmg_partition(const gmg_ctx* ctx, int m, int nranks, long long min_cells_per_rank, int* owner);

/* Sec. "Communication" (the cached metadata of the ghost-cell exchange):
   The face-ghost rectangles of MG level m: *n receives the count; rects (may be NULL) gets
   14 ints per rectangle: dst_box, src_box, dst[3], src[3] (local coordinates of the first
   ghost cell and of its source cell), d1, d2 (tangential axes, d1 fastest), n1, n2
   (extents), sign (+1 copy or Neumann mirror, -1 Dirichlet reflection), kind (0 copy from a
   box of the level, periodic images included; 1 wall; 2 quadratic Dirichlet wall, whose
   source is the second cell inward and whose ghost holds a third of it, the rule's -2 phi_0
   being part of the diagonal). */
gmg_status gmg_ghost_rects(const gmg_ctx* ctx, int m, int* n, int* rects);

/* Sec. "Communication" (ghost-cell exchange between processes):
   Exchange plan of rank `rank` under owner[] (nboxes ints): the copy rectangles whose
   source box and destination box have different owners.  send (may be NULL): *nsend pairs
   (peer, rectangle) with the source on this rank; recv: *nrecv pairs with the destination
   on this rank; both sorted by (peer, rectangle), so a sender and its receiver list the
   rectangles between them in the same order.  A rectangle's values travel u (along d1)
   fastest, as gmg_ghost_rects describes them. */
gmg_status gmg_exchange_plan(const gmg_ctx* ctx, int m, const int* owner, int rank, int* nsend, int* send,
                             int* nrecv, int* recv);

/* ---------------------------------------------------------------- diagnostics */

/* FP64 throughput probe (no counterpart in the paper; a measurement helper for the roofline
   of the FP64-pipe-bound kernels): enqueues on cuda_stream one kernel of SMs x blocks_per_sm
   blocks of 256 threads, each thread running 16 independent chains of `iters` FP64 fused
   multiply-adds, and returns in *flops the floating-point operations it performs (2 per
   FMA).  The caller times it (events on the same stream).  Allocates nothing.
   GMG_ERR_BAD_INPUT for blocks_per_sm outside [1, 64], iters < 1 or flops NULL. */
gmg_status gmg_dfma_probe(void* cuda_stream, int blocks_per_sm, int iters, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* GMG_H */
