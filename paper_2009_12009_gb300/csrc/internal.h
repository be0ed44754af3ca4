// internal.h -- shared host/device definitions of the GB300 multigrid library.
//
// Data model (Sec. "Basic data structures", Sec. "Containers for mesh data"): a level is
// a list of disjoint boxes; every field on a level is one flat device buffer holding one
// ghosted block per box.  All element types share one layout per level (offsets are
// counted in elements), so a float field, a bfloat16 field and a double coefficient
// array of the same level are indexed with the same numbers.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace gmg {

enum { DT_F64 = 0, DT_F32 = 1, DT_BF16 = 2, NDT = 3 };

// Valid cell i of a row sits at element GX + i; GX elements = 16 B for bfloat16, 32 B for
// float, 64 B for double, so the first valid cell of every row is 16-byte aligned.
constexpr int GX = 8;
// Row strides are multiples of this many elements: 128 B (one DRAM line) for float, 256 B
// for double, so every row of a float or double array starts on a line boundary.
constexpr int ROW_ALIGN = 32;
// Box offsets are multiples of this many elements.
constexpr int BOX_ALIGN = 64;

// Threads per block of the cell/pair kernels and items per block.
constexpr int BLOCK = 256;
// Ghost elements handled by one block of the ghost-exchange kernel.
constexpr int GHOST_CHUNK = 1024;

struct DevBox {
  int64_t off;   // element offset of the box's ghosted block
  int64_t sy;    // plane stride (elements) = sx * (ny + 2)
  int nx, ny, nz;
  int sx;        // row stride (elements)
  int lo[3];     // global index of the box's first valid cell on its level
  int solve;     // index of the independent solve this box belongs to (batched form)
};

// Ghost push target of one box face (2 * axis + side): the cells of the face are copied,
// times sign, into box `box` at the same cell shifted by (dx, dy, dz); box < 0: none.
struct PushFace {
  int box;
  int sign;
  int dx, dy, dz;
  int direct;     // 1: same row and plane strides, the ghost of element q is q + delta
  int64_t delta;
  int wall;       // 1: a physical wall (the ghost is the cell's own image); 0: a copy
  int pad_;
};

// One rectangle of face ghost cells of box dst_box and where its values come from.
struct GhostRect {
  int dst_box, src_box;
  int dst[3];    // local coordinates of the rectangle's first ghost cell
  int src[3];    // local coordinates (in src_box) of its source cell
  int d1, d2;    // tangential axes iterated by u (fastest) and v
  int n1, n2;    // extents along d1, d2
  int sign;      // +1: copy (or homogeneous Neumann mirror); -1: homogeneous Dirichlet reflection
  int par0;      // global (i+j+k) parity of the first ghost cell
  int kind;      // 0: copy from a box of the same level (periodic images included); 1: wall;
                 // 2: quadratic Dirichlet wall -- the source is the second cell inward and the
                 //    ghost holds a third of it (the rule's -2 phi_0 sits in the diagonal D)
};

// the factor from a ghost rectangle's source value to its ghost value
inline double ghost_factor(const GhostRect& g) { return g.kind == 2 ? 1.0 / 3.0 : (double)g.sign; }

// Generic work-list entry: block b handles items [start, start + per-block) of `item`.
struct Chunk {
  int item;
  int start;
};

// A valid cell of the bottom level (for the single-block BiCGStab kernel).
struct BotCell {
  int64_t q;     // element offset
  int64_t sy;    // plane stride of its box
  int sx;        // row stride of its box
  int pad;
};

// Ghost assignment of the bottom level, flattened: f[dst] = sign * f[src].
struct BotGhost {
  int64_t dst, src;
  double sign;
};

// One bottom problem (one per independent solve in the batched form).
struct BotDesc {
  int cell0, ncell;     // range in the BotCell list
  int ghost0, nghost;   // range in the BotGhost list
  int singular;         // project onto zero mean
  int solve;
};

// Dataflow red-black sweep (flow.cu).  A smoothed level is cut, per independent problem,
// into z-slabs of whole planes of the problem's domain (about FLOW_SLAB_CELLS cells each);
// every box is cut into work items of its full x extent and about FLOW_ITEM_CELLS cells
// inside one slab (one warp's work).  One launch runs
// several colour phases (red, black, red, ...): an item of phase c may start once every item
// of phase c - 1 in its own slab and the two slabs next to it (periodic images included) has
// finished, which is exactly when the values it reads are those of the two-pass sweep and no
// value it overwrites is still to be read.
struct FlowItem {
  int box;
  int slab;      // index into the level's FlowSlab table
  int z0, z1;    // planes [z0, z1) of the box
  int y0, y1;    // rows [y0, y1) of the box
};

struct FlowSlab {
  int first, count;  // the slab's items: [first, first + count) of the item list
  int dep[3];        // slabs whose previous-phase items must be complete (-1: none)
  int solve;
};

// One entry of a dispense order: one item (box, planes, rows) of one slab in one phase.
struct FlowChunk {
  int phase_slab;  // phase << 24 | slab
  int box;
  int z0, z1, y0, y1;
};

constexpr int FLOW_MAX_PHASES = 4;          // colour phases one launch can run
constexpr int FLOW_SLAB_CELLS = 1 << 18;    // target cells per slab (whole planes, at most 16)
constexpr int FLOW_ITEM_CELLS = 128;        // target cells per work item (one warp: two updates per lane)
constexpr int FLOW_LAG_CELLS = 1 << 20;     // default dispense lag of phase c behind phase c - 1
constexpr int FLOW_MIN_CELLS = 1 << 17;     // levels with fewer smoothed cells keep one launch per colour
constexpr int FLOW_BLOCK = 128;             // threads per block of the flow kernel (4 warps)
constexpr int FLOW_WARPS_PER_SM = 32;       // default resident warps per SM
constexpr int FLOW_QUEUES = 16;             // hand-out counters (chunk k is handed out by queue k % FLOW_QUEUES)
constexpr int FLOW_CNT_STRIDE = 32;         // ints between completion counters (one 128-byte line each)

// Wavefront red-black sweep (wave.cu): one launch performs one whole Gauss-Seidel sweep
// (red then black) of a level, in place.  The level is cut into tiles -- a band of rows
// [y0, y1) of one box, all its x and all its planes -- and one thread block per tile marches
// through the tile's planes: at step m it updates the red cells of plane m (in the tile's
// marching order), then the black cells of plane m - 1.  A black cell on the tile's border
// reads red cells of the tile next to it, so before the black cells of a plane the block
// waits until each neighbouring tile has reported its red cells of that plane done; a red
// cell reads black cells of the neighbours, which they update only after this tile's report.
// Boxes next to each other along z march in opposite directions (their shared face is the
// first plane of both, or the last of both), and boxes next to each other along x or y march
// alike, so every wait is for a step the other tile reaches earlier: no wait can deadlock.
struct WaveTile {
  int box;
  int y0, y1;     // rows [y0, y1) of the box
  int dir;        // 0: planes 0, 1, ..., nz - 1; 1: nz - 1, ..., 0
  int nb[4];      // tiles across the x-, x+, y-, y+ sides whose reds of a plane this tile's blacks
                  // of that plane wait for (same planes, same marching order); -1: a wall
  int zb[2];      // tiles across the z- and z+ faces (-1: a wall)
  int zneed[2];   // red planes those tiles must have reported before the blacks of plane 0
                  // (z-) and of plane nz - 1 (z+)
  int solve;
};

constexpr int WAVE_BLOCK = 128;       // threads per block of the wavefront sweep
constexpr int WAVE_MAX_PPT = 4;       // cell pairs per thread (a tile holds up to WAVE_BLOCK * WAVE_MAX_PPT)
constexpr int WAVE_MAX_PLANES = 4095; // planes of a box the sweep handles (a 12-bit count)

// The coarse end of one problem's V-cycle run by one thread block (tail.cu): levels
// m0..mb of that problem, mb its bottom.  Cell and ghost lists reuse BotCell / BotGhost.
constexpr int TAIL_MAXLEV = 20;       // MG levels addressable by the tail kernel
constexpr int TAIL_MAX_CELLS = 512;   // a problem's level joins its tail at or below this size
constexpr int TAIL_WARP_CELLS = 128;  // bottoms up to this size run in one warp ...
constexpr int TAIL_WARP_SPAN = 2048;  // ... if their boxes span at most this many elements

struct TailLevel {
  int cell0, ncell[2];   // colour-0 cells at [cell0, cell0 + ncell[0]), colour 1 after them
  int ghost0, nghost[2]; // ghosts of parity 0, then parity 1 (walls included)
  int xfer0, nxfer;      // coarse cells of level m + 1 over this level's boxes (m < mb)
  // Dense form (the shared-memory coarse end): the problem's cells of this level tile one
  // box, the level's domain, held as one padded array of dne = (n0+2)(n1+2)(n2+2) elements
  // with strides 1, dsx, dsy.  A cell's slot is BotCell.pad (TAIL_SLOT_MASK bits, plus
  // TAIL_HI_* / TAIL_LO_* flags where its high / low face lies on the domain's boundary);
  // the ghosts outside the domain (walls, periodic images) are dense BotGhost entries of
  // parity 0, then 1.  face[2 a + side]: the rule of the domain's face on axis a, low (0) or
  // high (1) side -- +1 / -1 a wall whose ghost is +/- the cell inward, 2 periodic (the
  // ghost is the cell at the other end), 0 none -- with which a boundary cell writes its
  // new value into the ghosts that copy it.
  int dsx, dsy, dne;
  int dghost0, ndghost[2];
  int face[6];
};
constexpr int TAIL_SLOT_MASK = (1 << 24) - 1;
constexpr int TAIL_HI_X = 1 << 24, TAIL_HI_Y = 1 << 25, TAIL_HI_Z = 1 << 26;
constexpr int TAIL_LO_X = 1 << 27, TAIL_LO_Y = 1 << 28, TAIL_LO_Z = 1 << 29;
// shared-memory budget of the dense coarse end's arrays (dynamic shared memory per block)
constexpr int TAIL_SMEM_MAX = 160 * 1024;

// Bytes of one level's arrays in the dense coarse end: e and r (element size es) and, on a
// smoothed level, wx, wy, wz, 1/D and D (coefficient size cs), each 16-byte aligned.
__host__ __device__ inline int64_t tail_level_bytes(int dne, int es, int cs, bool smoothed) {
  const int64_t a = ((int64_t)dne * es + 15) & ~(int64_t)15;
  const int64_t b = ((int64_t)dne * cs + 15) & ~(int64_t)15;
  return 2 * a + (smoothed ? 5 * b : 0);
}

// one coarse cell of the next level and its 8 children on this level:
// qf + {0,1} + sx*{0,1} + sy*{0,1}
struct TailXfer {
  int64_t qc, qf;
  int sx, sy;
  int dqc, dqf;  // the same two cells' slots in the dense form
  int dfl;       // TAIL_LO_* flags of child (0,0,0) and TAIL_HI_* flags of child (1,1,1)
};

struct TailDesc {
  int solve;
  int m0, mb;       // first tail level and bottom level (absolute MG levels)
  int lev0;         // TailLevel of m0; level m is lev0 + m - m0
  int singular;     // bottom projects onto zero mean
  int bot_span;     // elements from bot_base to the end of the problem's last bottom box
  int64_t bot_base; // first element of the problem's first bottom box
  int dense;        // 1: every level of the tail has its dense form
  int pad_;
};

__host__ __device__ inline int64_t elem_index(const DevBox& B, int i, int j, int k) {
  return B.off + GX + i + (int64_t)B.sx * (j + 1) + B.sy * (k + 1);
}

}  // namespace gmg
