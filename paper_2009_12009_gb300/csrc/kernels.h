// kernels.h -- launch wrappers of the sm_103a kernels (kernels.cu, bottom.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace gmg {

// Per-solve geometry of one level, as the coefficient kernels see it.
struct DevGeom {
  int dlo[3], dhi[3];
  int wall_lo[3], wall_hi[3];  // wall on that side: 0 none (periodic), 1 Dirichlet, 2 Neumann,
                               // 3 Dirichlet with the quadratic ghost rule
  double ih2[3];               // 1 / h_d^2
};

// Device view of one level: its tables (uploaded once into the workspace).
struct LevelDev {
  const DevBox* boxes = nullptr;
  const DevGeom* geoms = nullptr;
  const GhostRect* ghosts = nullptr;
  const Chunk* ghost_chunks = nullptr;
  int n_ghost_chunks = 0;
  const Chunk* pair_chunks = nullptr;  // boxes that smooth on this level, 2 cells per item
  int n_pair_chunks = 0;
  const Chunk* quad_chunks = nullptr;  // the same, 4 cells per item (null: a width is not a multiple of 4)
  int n_quad_chunks = 0;
  const Chunk* pair_all_chunks = nullptr;  // every box, 2 cells per item
  int n_pair_all_chunks = 0;
  const Chunk* cell_chunks = nullptr;
  int n_cell_chunks = 0;
  const Chunk* coarse_chunks = nullptr;
  int n_coarse_chunks = 0;
  const int* parent = nullptr;
  const int* child = nullptr;       // per box: its one exact child box on the finer level, or -1
  const BotCell* bot_cells = nullptr;
  const BotGhost* bot_ghosts = nullptr;
  const BotDesc* bot_descs = nullptr;
  int n_bot = 0;
  int64_t nelem = 0;
  // per-solve data (batched form; one solve otherwise)
  int nsolves = 1;
  const int* active = nullptr;             // per solve: 0 = converged, its boxes are skipped; null = all
  const int* solve_chunk_range = nullptr;  // cell_chunks of solve s are [range[s], range[s+1])
  const double* inv_count = nullptr;       // per solve: 1 / number of cells on this level
  // the V-cycle's work lists when each problem's coarse end runs as one block (tail.cu)
  const Chunk* vc_ghost_chunks = nullptr;
  int n_vc_ghost_chunks = 0;
  const Chunk* vc_pair_chunks = nullptr;
  int n_vc_pair_chunks = 0;
  const Chunk* vc_quad_chunks = nullptr;
  int n_vc_quad_chunks = 0;
  const Chunk* vc_coarse_chunks = nullptr;
  int n_vc_coarse_chunks = 0;
  const BotDesc* vc_bot_descs = nullptr;
  int n_vc_bot = 0;
  // dataflow red-black sweep (flow.cu); n_flow_slabs == 0: one launch per colour here
  const FlowItem* flow_items = nullptr;
  const FlowSlab* flow_slabs = nullptr;
  int n_flow_slabs = 0;
  const FlowChunk* flow_order[FLOW_MAX_PHASES] = {};  // per number of phases n: [n - 1]
  int n_flow_order[FLOW_MAX_PHASES] = {};
  int* flow_cnt = nullptr;  // (FLOW_QUEUES + 1 + FLOW_MAX_PHASES * n_flow_slabs) * FLOW_CNT_STRIDE ints,
                            // zero between launches
  const int* flow_skip = nullptr;  // per solve: 1 = leave its items out (null: none)
  // wavefront red-black sweep (wave.cu): the level's tiles in hand-out order (problem by
  // problem); n_wave_tiles == 0: no wavefront sweep on this level
  const WaveTile* wave_tiles = nullptr;
  int n_wave_tiles = 0;
  int wave_ppt = 0;              // cell pairs per thread of the level's tiles (1, 2 or 4)
  int wave_max_solve_tiles = 0;  // tiles of the problem that has the most
  int64_t wave_layer_cells = 0;  // cells of one plane of every tiled box
  unsigned* wave_cnt = nullptr;  // 64 + n_wave_tiles words, zero between launches
  const PushFace* push_faces = nullptr;  // 6 per box (ghost push targets)
  int push_ok = 0;                       // push_faces usable for every box of the level
  const BotGhost* ec_ghosts = nullptr;  // edge and corner ghosts (levels >= 1), f[dst] = sign f[src]
  int n_ec_ghosts = 0;
  // SPLIT_RHS | SPLIT_INVD: the level's own right-hand side buffers (r, every element type)
  // and its 1/D are colour-split within rows; 0: the ordinary layout.  (A kernel given
  // another right-hand side -- a caller's -- reads it in the ordinary layout.)
  int split = 0;
  // 1: the level-sweep kernels (smoothers, residual, residual-restriction, interpolation)
  // take their work list last entry first.  Consecutive kernels on a level that alternate it
  // start on the boxes the previous one touched last, still in L2.  Same results.
  int rev = 0;
};

// Which arrays of a level are stored colour-split within rows (split_index, dev_util.cuh):
// the level's right-hand side of the smoother, its 1/D.  Ordinary layout otherwise.
enum { SPLIT_RHS = 1, SPLIT_INVD = 2 };

// Coefficients of one level in one element type (double for FP64 fields, float for
// float and bfloat16 fields): scaled face weights w = b*beta/h^2, diagonal
// D = a*alpha + sum of the six weights, and 1/D.
struct Coefs {
  const void* wx = nullptr;
  const void* wy = nullptr;
  const void* wz = nullptr;
  const void* D = nullptr;
  const void* invD = nullptr;
};

// ghost exchange; colour -1 = all ghosts; copy_mode 1: skip wall rectangles (coefficient
// fills, where the wall face is handled by the face kernel); 2: quadratic wall ghosts 0
// (the transposed operator: the rule's entry on phi_1 moves to phi_1's row)
void launch_fill(int dt, const LevelDev& L, void* f, int colour, int copy_mode, cudaStream_t s);
// one red-black colour (no ghost fill); push: also write each new value into the ghost
// cells that copy it (L.push_ok levels only)
// own_rhs: rhs is the level's own right-hand side buffer (colour-split where L.split says so;
// a caller's rhs is in the ordinary layout); 1/D is read as the level keeps it
void launch_smooth(int dt, const LevelDev& L, void* phi, const void* rhs, const Coefs& c, int colour,
                   cudaStream_t s, bool push = false, bool vec = false, bool own_rhs = false);
// One red-black colour fused with the piecewise-constant interpolation of the coarse
// correction ec of level Lc (Lc's ghosts current) that would precede it: the cells of the
// colour get the values of the interpolation followed by launch_smooth; the other colour's
// cells are left as they were (the next colour pass overwrites them without reading them).
void launch_smooth_pro(int dt, const LevelDev& L, const LevelDev& Lc, void* phi, const void* rhs, const Coefs& c,
                       int colour, const void* ec, cudaStream_t s, bool push, bool own_rhs = false);
// One red-black colour on coarse level L fused with the piecewise-constant interpolation of
// the level's correction onto the finer level Lf that follows it (fine += parent value; L's
// boxes each with one exact child, L.child): the values of launch_smooth followed by
// launch_prolong_add; push / fpush: write new values into the ghosts of L / Lf too.  The other
// colour's values must be final (this is the last pass of L's post-smoothing).
void launch_smooth_prolong(int dt, const LevelDev& L, const LevelDev& Lf, void* phi, const void* rhs, const Coefs& c,
                           int colour, void* fine, cudaStream_t s, bool push, bool fpush);
// r = (rhs - shift[solve]) - A phi on valid cells (ghosts of phi must be filled); rdt =
// type of r; maxbits (may be null): per-solve atomic max of |r| as IEEE bits; shift (may be
// null): per-solve device scalars
// own_r: r is the level's own right-hand side buffer, colour-split where L.split says so
// (and then invDe is the level's 1/D, split alike)
// e (may be null): also the first red half-sweep of a V-cycle on this r from e = 0 --
// e = r / D on red cells (invDe: 1/D in the coefficient type of rdt), 0 on black cells,
// pushed into e's ghosts when push is set
// settled (0 red, 1 black, -1 none; FP64 phi and r, a level whose ghosts have their
// source's colour): the colour a Gauss-Seidel half-sweep updated last.  A cell of that
// colour reads only cells of the other colour, unchanged since its update made its residual
// zero up to rounding -- except next to a wall, whose ghost is the cell's own image (those
// cells are computed).  Its r is stored as 0 without being computed.
void launch_residual(int dt, int rdt, const LevelDev& L, const void* phi, const void* rhs, const Coefs& c,
                     void* r, unsigned long long* maxbits, const double* shift, cudaStream_t s, void* e = nullptr,
                     const void* invDe = nullptr, bool push = false, int settled = -1, bool own_r = false);
// coarse r = restriction of (rhs - A phi) (ghosts of phi filled); settled_black: the last
// half-sweep on phi was black (as for launch_residual: black children count 0 unless they
// lie next to a wall).  ec non-null: also the coarse level's first red half-sweep from a zero
// correction, ec = r / D (invDc: the coarse 1/D) on red cells and 0 on black ones, every
// valid coarse cell written (cpush: and pushed into the coarse ghosts that copy it).
void launch_resid_restrict(int dt, const LevelDev& f, const LevelDev& c, const void* phi, const void* rhs,
                           const Coefs& cf, void* rc, cudaStream_t s, bool settled_black = false, bool own_rhs = false,
                           void* ec = nullptr, const void* invDc = nullptr, bool cpush = false);
void launch_restrict(int dt, const LevelDev& f, const LevelDev& c, const void* fine, void* coarse, cudaStream_t s);
void launch_prolong_add(int dt, const LevelDev& f, const LevelDev& c, const void* coarse, void* fine,
                        cudaStream_t s, bool push = false);
// fine += trilinear interpolation of coarse (weights 3/4, 1/4 per axis; summed z, y, x
// outermost first, unfused products -- the oracle's order); coarse's face, edge and corner
// ghosts must hold the homogeneous boundary rule's values (launch_fill + launch_fill_ec)
void launch_prolong_tri(int dt, const LevelDev& f, const LevelDev& c, const void* coarse, void* fine,
                        cudaStream_t s, bool push = false);
// edge and corner ghosts of a level from their owning valid cells (L.ec_ghosts)
void launch_fill_ec(int dt, const LevelDev& L, void* f, cudaStream_t s);
// phi (double) += e (type dt) on valid cells
// (push: also write the new phi into the ghost cells that copy it, L.push_ok levels only)
void launch_add_correction(int dt, const LevelDev& L, double* phi, const void* e, cudaStream_t s,
                           bool push = false);
// the last colour pass of the finest level's post-smoothing fused with phi += e on every
// smoothed cell (pair work list); push_phi: also write phi's new values into its ghosts
void launch_smooth_update(int dt, const LevelDev& L, void* e, const void* rhs, const Coefs& c, int colour,
                          double* phi, bool push_phi, cudaStream_t s, bool own_rhs = false);
// dense (nz,ny,nx) double over the level's (single-solve) domain <-> boxed type dt
void launch_pack(int dt, const LevelDev& L, const int dlo[3], const int dn[3], const double* dense, void* boxed,
                 cudaStream_t s);
void launch_unpack(int dt, const LevelDev& L, const int dlo[3], const int dn[3], const void* boxed, double* dense,
                   cudaStream_t s);
// |x|_inf of a double field per solve (atomic max into maxbits[solve])
void launch_norm_max(const LevelDev& L, const double* x, unsigned long long* maxbits, cudaStream_t s);
// deterministic per-solve mean of the valid cells of a double field: partial sums per
// block, then one block per solve adds its partials in order; out[s] = mean of solve s
void launch_sum(const LevelDev& L, const double* x, double* partials, double* out, cudaStream_t s);
// x += scale * c[solve] on valid cells
void launch_add_scalar(const LevelDev& L, double* x, const double* c, double scale, cudaStream_t s);
// x *= scale on valid cells
void launch_scale_valid(const LevelDev& L, double* x, double scale, cudaStream_t s);
void launch_copy_valid(const LevelDev& L, double* dst, const double* src, cudaStream_t s);

// ---- coefficients (FP64) ----
// acoef = a * alpha (alpha null: a)
void launch_acoef(const LevelDev& L, double a, const double* alpha, double* acoef, cudaStream_t s);
// face beta = harmonic mean of the two cells (wall faces: interior cell) from cell beta
// whose ghosts hold the neighbouring boxes' values
void launch_faces_from_cell(const LevelDev& L, const double* beta, double* bx, double* by, double* bz, cudaStream_t s);
// w_d = b * beta_d / h_d^2 from face arrays
void launch_faces_scale(const LevelDev& L, double b, const double* bx, const double* by, const double* bz, double* wx,
                        double* wy, double* wz, cudaStream_t s);
// coarse acoef = mean of 8; coarse w = (sum of 4 fine w) / 16
void launch_coarsen_coefs(const LevelDev& f, const LevelDev& c, const double* acf, const double* wxf,
                          const double* wyf, const double* wzf, double* acc, double* wxc, double* wyc, double* wzc,
                          cudaStream_t s);
void launch_diag(const LevelDev& L, const double* acoef, const double* wx, const double* wy, const double* wz,
                 double* D, double* invD, cudaStream_t s);
void launch_to_float(const double* src, float* dst, int64_t n, cudaStream_t s);
// copy a field of type dt into type dt2 (same layout, every element)
void launch_convert(int dt, int dt2, const void* src, void* dst, int64_t n, cudaStream_t s);
// the level's own right-hand side buffer (type dt; colour-split where L.split says so) = src
// (double, the ordinary layout) on the valid cells
void launch_to_rhs(int dt, const LevelDev& L, const double* src, void* dst, cudaStream_t s);
// the same from a type-dt source (a copy where the level is not split)
void launch_copy_to_rhs(int dt, const LevelDev& L, const void* src, void* dst, cudaStream_t s);

// programmatic dependent launch for the V-cycle kernels (fill, smooth, residuals,
// restriction, interpolation, correction, coarse end, bottom): each may start while its
// stream predecessor finishes and waits for it on the device (process-wide switch, set
// per solve from gmg_params.pdl)
void set_pdl(bool on);
bool pdl_enabled();

// number of kernel launches issued through these wrappers (host counter)
int64_t kernel_launch_count();
void count_launches(int n);

// ---- bottom solve (bottom.cu) ----
struct BottomArgs {
  int maxit;
  double tol;
  double* work;        // 7 double vectors of the bottom level's layout
  int* iters;          // device: iterations per bottom problem
  int cg = 0;          // 1: conjugate gradients instead of BiCGStab
};
void launch_bottom(int dt, const LevelDev& L, const void* rhs, void* x, const Coefs& c64, const BottomArgs& a,
                   cudaStream_t s);

// ---- wavefront red-black sweep (wave.cu) ----
// whether level L has wavefront-sweep tables (and pushed ghosts)
bool wave_ok(const LevelDev& L);
// One whole red-black sweep (red, then black) of level L in one launch, in place on e, with
// the values of two launch_smooth passes with push (bitwise).  zero_start: e is zero
// (valid cells and ghosts) before the sweep, so the red cells are rhs / D.  phi (double,
// level 0 only, not with zero_start): also phi += e on every smoothed cell afterwards, as
// launch_smooth_update does (push_phi: phi's new values into its ghosts).  A dependency wait
// that gives up sets *err.  Returns false (nothing launched) when the level has no tables or
// the problem with the most tiles cannot have them all resident at once.
bool launch_wave(int dt, const LevelDev& L, void* e, const void* rhs, const Coefs& c, bool zero_start, double* phi,
                 bool push_phi, int* err, cudaStream_t s);

// ---- dataflow red-black sweeps (flow.cu) ----
// whether level L has flow tables and pushes its ghosts (the flow kernel keeps every ghost
// current by push; it cannot run a ghost exchange between phases)
bool flow_ok(const LevelDev& L);
// nphase alternating colour phases starting with colour0 (0 red, 1 black), in one launch,
// in place on e; the same values as nphase launches of launch_smooth with push.  phi
// non-null: the last phase also adds both cells' e to phi on every pair (launch_smooth_update),
// pushing phi's new values into its ghosts if push_phi.  err: device flag raised if a
// dependency wait gave up.  Returns false (nothing launched) if the level has no flow tables.
// warps: resident warps per SM (0: the default).
bool launch_flow(int dt, const LevelDev& L, void* e, const void* rhs, const Coefs& c, int colour0, int nphase,
                 double* phi, bool push_phi, int* err, cudaStream_t s, int warps = 0);

// ---- coarse end of the V-cycle, one block per problem (tail.cu) ----
struct TailArgs {
  const TailDesc* descs = nullptr;  // block b runs descs[b]
  const TailLevel* levels = nullptr;
  const BotCell* cells = nullptr;
  const BotGhost* ghosts = nullptr;
  const TailXfer* xfer = nullptr;
  const BotGhost* dghosts = nullptr;     // dense-form ghosts (TailLevel.dghost0)
  const double* wx64[TAIL_MAXLEV] = {};  // FP64 coefficients (bottom solve)
  const double* wy64[TAIL_MAXLEV] = {};
  const double* wz64[TAIL_MAXLEV] = {};
  const double* D64[TAIL_MAXLEV] = {};
  double* work[TAIL_MAXLEV] = {};  // 7 double vectors of the level's layout (bottom levels)
  int64_t nelem[TAIL_MAXLEV] = {};
  int nu1 = 2, nu2 = 2, maxit = 200;
  double tol = 1e-4;
  int cg = 0;        // bottom by conjugate gradients instead of BiCGStab
  int post_rev = 0;  // post-smoothing black before red
  int* iters = nullptr;         // per solve: bottom iterations
  const int* active = nullptr;  // per solve: 0 = skip (null: all)
};
// one level's V-cycle buffers in the element type of the launch (coefficients double for
// FP64, float otherwise)
struct TailLevelBufs {
  void* e = nullptr;
  void* r = nullptr;
  const void *wx = nullptr, *wy = nullptr, *wz = nullptr, *D = nullptr, *invD = nullptr;
};
// dense_bytes > 0: the dense coarse end (k_vtail_dense) with that much dynamic shared memory
void launch_vtail(int dt, int nblocks, const TailArgs& a, const TailLevelBufs* lv, int nlev, int dense_bytes,
                  cudaStream_t s);

// Wall values on level 0 (walls.cu), one launch per face: mode 0 f[q] += c g, mode 1
// f[ghost] += (2 or h) g, mode 2 dg = c lam[q]; c = 2 w (kind 1, Dirichlet) or w h (kind 2,
// Neumann), w the FP64 face weight array of the face's direction.
void launch_wall_values(const LevelDev& L, int nboxes, int max_face_cells, int face, int kind, double h,
                        const double* w, const double* g, int mode, double* f, const double* lam, double* dg,
                        cudaStream_t s);

// Top-level Krylov vector kernels (krylov.cu): out = A in (ghosts of in filled first,
// FP64 coefficients); p = r + beta (p - omega v); x += a y + b z (flat, n elements).
void launch_apply(const LevelDev& L, const double* in, const Coefs& c64, double* out, cudaStream_t s);
void launch_bicg_direction(int64_t n, const double* r, double* p, const double* v, double beta, double omega,
                           cudaStream_t s);
void launch_add2(int64_t n, double* x, double a, const double* y, double b, const double* z, cudaStream_t s);

// ---- the same vector operations over every level of a composite vector in one launch
// (krylov.cu): nl levels of n[l] elements (ghosts included); per level the values of the
// one-level kernels above, bitwise.  Segments (level and vectors) of the reductions: up to
// ML_MAX_SEG.
constexpr int ML_MAX_SEG = 8;
// out_l = a[l] x_l + b[l] y_l
void launch_axpby_ml(int nl, const int64_t* n, const double* a, const double* const* x, const double* b,
                     const double* const* y, double* const* out, cudaStream_t s);
// o1_l = a[l] x_l, o2_l = o1_l (the values of launch_axpby(a, x, 0, x, o1) then
// launch_axpby(1, o1, 0, o1, o2))
void launch_scale2_ml(int nl, const int64_t* n, const double* a, const double* const* x, double* const* o1,
                      double* const* o2, cudaStream_t s);
void launch_bicg_direction_ml(int nl, const int64_t* n, const double* const* r, double* const* p,
                              const double* const* v, double beta, double omega, cudaStream_t s);
void launch_add2_ml(int nl, const int64_t* n, double* const* x, double a, const double* const* y, double b,
                    const double* const* z, cudaStream_t s);
// out[s] = sum over the valid cells of segment s (level L[s]) of x_s y_s: deterministic
// partial sums over groups of cell chunks, then one block per segment adds them in order
// (partials: one per cell chunk of all segments is enough)
void launch_dot_ml(int ns, const LevelDev* const* L, const double* const* x, const double* const* y,
                   double* partials, double* out, cudaStream_t s);
// maxbits[s] = max(maxbits[s], |x_s|_inf as IEEE bits) over the valid cells of segment s
void launch_norm_max_ml(int ns, const LevelDev* const* L, const double* const* x, unsigned long long* maxbits,
                        cudaStream_t s);

}  // namespace gmg
