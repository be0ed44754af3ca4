// meta.h -- host-side index-space metadata: boxes, BoxArrays, the multigrid hierarchy
// and the cached ghost-exchange / work tables (Sec. "Basic data structures",
// Sec. "Communication": box intersections are computed once and cached).
#pragma once

#include <string>
#include <vector>

#include "internal.h"

namespace gmg {

struct Box {
  int lo[3] = {0, 0, 0};
  int hi[3] = {-1, -1, -1};
  int n(int d) const { return hi[d] - lo[d] + 1; }
  bool empty() const { return n(0) <= 0 || n(1) <= 0 || n(2) <= 0; }
  int64_t volume() const { return empty() ? 0 : (int64_t)n(0) * n(1) * n(2); }
};

Box intersect(const Box& a, const Box& b);
Box shifted(const Box& a, int d, int s);

// Geometry of one independent problem on one level (Sec. "Basic data structures":
// Geometry, BCRec).
struct SolveGeom {
  Box domain;
  double h[3] = {1, 1, 1};
  int bclo[3] = {0, 0, 0};
  int bchi[3] = {0, 0, 0};
  int qlo[3] = {0, 0, 0};  // 1: that Dirichlet side takes the quadratic ghost rule
  int qhi[3] = {0, 0, 0};
  bool periodic(int d) const { return bclo[d] == 0; }
  bool has_quad() const {
    for (int d = 0; d < 3; ++d)
      if (qlo[d] || qhi[d]) return true;
    return false;
  }
  bool all_periodic() const { return bclo[0] == 0 && bclo[1] == 0 && bclo[2] == 0; }
  bool has_dirichlet() const {
    for (int d = 0; d < 3; ++d)
      if (bclo[d] == 1 || bchi[d] == 1) return true;
    return false;
  }
};

// One multigrid level of one or several independent problems.
struct CfSlab {
  int box, d, side;  // a face of a box whose ghosts lie on the coarse/fine boundary
};

struct LevelMeta {
  bool allow_cf = false;            // fine AMR level: uncovered face ghosts are coarse/fine
  std::vector<CfSlab> cf_slabs;
  std::vector<Box> boxes;
  std::vector<int> box_solve;       // per box: index into geoms
  std::vector<SolveGeom> geoms;     // per solve (indexed by solve id)
  std::vector<char> solve_present;  // per solve: has boxes on this level
  std::vector<char> solve_bottom;   // per solve: this level is its bottom
  std::vector<int> parent;          // per box: box on the next coarser level (-1: none)
  std::vector<int> child;           // per box: its one child box on the next finer level, whose
                                    // cells are exactly its own halved (-1: none or several)

  // layout (shared by every element type)
  std::vector<DevBox> dbox;
  int64_t nelem = 0;
  int64_t ncells = 0;

  // cached tables
  std::vector<GhostRect> ghosts;
  std::vector<PushFace> push_faces;  // 6 per box: where each face's cells are copied
  bool push_ok = false;  // every face copied whole into one ghost rectangle, every periodic
                         // length even (a ghost has its source's colour)
  std::vector<Chunk> ghost_chunks;
  std::vector<Chunk> pair_chunks;    // boxes of solves that smooth on this level, 2 cells per item
  std::vector<Chunk> quad_chunks;    // the same boxes, 4 cells per item (all widths multiples of 4)
  bool quad_ok = false;              // every smoothing box has a width that is a multiple of 4
  std::vector<Chunk> pair_all_chunks;  // every box, 2 cells per item
  std::vector<Chunk> cell_chunks;    // every box, 1 cell per item
  std::vector<Chunk> coarse_chunks;  // boxes with a parent, 1 coarse cell per item
  std::vector<BotCell> bot_cells;    // bottom problems on this level
  std::vector<BotGhost> bot_ghosts;
  std::vector<BotDesc> bot_descs;
  std::vector<int> solve_chunk_range;  // cell_chunks of solve s: [range[s], range[s+1])
  std::vector<double> inv_count;       // per solve: 1 / cells of the solve on this level (0 if absent)

  // work lists of the V-cycle's grid launches when the coarse ends of the problems run as
  // one thread block each: entries of problems whose tail covers this level are left out
  std::vector<Chunk> vc_ghost_chunks, vc_pair_chunks, vc_coarse_chunks, vc_quad_chunks;
  std::vector<BotDesc> vc_bot_descs;

  // dataflow red-black sweep (empty when the level has fewer than FLOW_MIN_CELLS smoothed
  // cells or its ghosts cannot be pushed): items grouped by slab, the slab table, and per
  // number of phases n the dispense order (flow_order[n - 1]: chunks of one slab's items)
  std::vector<FlowItem> flow_items;
  std::vector<FlowSlab> flow_slabs;
  std::vector<FlowChunk> flow_order[FLOW_MAX_PHASES];
  int64_t flow_lag = 0;  // the dispense lag (cells) flow_order was built with
  // per solve: 1 if the problem's coarse end (tail.cu) covers this level, so the V-cycle's
  // flow launches skip its items
  std::vector<int> vc_flow_skip;

  // wavefront sweep (wave.cu, tables by build_wave; empty when the level cannot run it): the
  // tiles in hand-out order (problem by problem), cell pairs per thread, and the number of
  // tiles of the problem that has the most
  std::vector<WaveTile> wave_tiles;
  int wave_ppt = 0;
  int wave_max_solve_tiles = 0;
  int64_t wave_layer_cells = 0;  // cells of one plane of every tiled box (one step of every tile)

  // edge and corner ghosts (built on demand by build_ec_ghosts): f[dst] = sign * f[src]
  std::vector<BotGhost> ec_ghosts;
  bool ec_built = false;
};

// Tail tables: for every problem whose bottom level is small, the levels from the first
// one with at most TAIL_MAX_CELLS of its cells (never level 0) down to its bottom.
struct TailHost {
  std::vector<TailDesc> descs;  // ordered by m0
  std::vector<TailLevel> levels;
  std::vector<BotCell> cells;
  std::vector<BotGhost> ghosts;
  std::vector<TailXfer> xfer;
  std::vector<BotGhost> dghosts;        // dense-form ghosts (slots of the levels' dense arrays)
  std::vector<int> first_at, count_at;  // per MG level: descs whose m0 is that level
  std::vector<int> tail_from;           // per solve: m0, or -1 (no tail)
};

// Build the tail tables and the vc_* work lists of every level (after finalize_level of
// all levels).  Returns "" or an error message.
std::string build_tail(std::vector<LevelMeta>& L, TailHost& T);

// Checks that boxes are non-empty, inside the domain and pairwise disjoint; with
// must_cover, that they cover it.  Returns "" or an error message.
std::string validate_boxes(const std::vector<Box>& boxes, const Box& domain, bool must_cover);

// Chop a box into pieces of at most max_grid_size cells per axis (low end first).
std::vector<Box> chop(const Box& dom, int max_grid_size);

// Layout, ghost rectangles and work tables of a level whose boxes, box_solve, geoms and
// solve_present/solve_bottom are set.  Returns "" or an error message.
std::string finalize_level(LevelMeta& L);

// Edge and corner ghost cells of every box of a level (face ghosts are the exchange's): the
// source of ghost cell g is the valid cell that owns g under the homogeneous boundary rule
// applied per axis -- a periodic axis wraps, a wall mirrors the index into the domain (ghost
// -1 <-> cell 0) with the factor -1 for a Dirichlet wall and +1 for a Neumann wall.  Used by
// the trilinear interpolation, which reads the coarse correction diagonally.
void build_ec_ghosts(LevelMeta& L);

// Tables of the wavefront sweep (wave.cu) for a level whose layout, ghost rectangles and push
// faces are built.  The rows of every smoothed box are cut into bands of one height per level,
// each a tile; tile sizes are chosen so that every problem has at most `max_resident` tiles
// (the blocks of the sweep kernel the device holds at once).  Left empty (the level keeps one
// launch per colour) unless the ghosts are pushed, every box width is even, every box face
// is copied whole from one box (or is a wall) with rows and planes aligned, and the boxes of
// each problem can be given marching directions with z-neighbours opposite and x- and
// y-neighbours alike.
void build_wave(LevelMeta& L, int max_resident);
// Blocks of the wavefront sweep the device is assumed to hold at once when tables are built
// (default 8 per SM on 152 SMs); the launch checks the real figure.
void set_wave_capacity(int blocks);
int wave_capacity();

// Rebuild a level's flow dispense orders for a dispense lag of `lag` cells (same sizes).
void build_flow_order(LevelMeta& L, int64_t lag);

// Multigrid coarsening with aggregation (Sec. "Linear Solvers"), per solve:
//  - every box of the solve has even lo, even size and size >= 4: coarsen each box;
//  - else every box has even lo and even size, the boxes cover the solve's domain and
//    every domain edge is even and >= 4: the coarse level holds the coarsened domain as
//    one box (aggregation);
//  - else the solve's bottom is this level.
// Fills f.parent and f.solve_bottom, and c's boxes/geoms.  Returns false if no solve
// continues to a coarser level.
bool make_coarse(LevelMeta& f, LevelMeta& c);

}  // namespace gmg
