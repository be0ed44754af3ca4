// capi.cpp -- C ABI (include/gmg.h) and the host driver of the V-cycle / outer loop.
//
// The host side owns only metadata: the hierarchy, the cached exchange tables and the
// carve-up of the caller's workspace.  Every step of the solve runs in the kernels of
// kernels.cu / bottom.cu; the host decides the launch order and reads back one norm per
// problem per outer iteration.
//
// A context holds one problem (gmg_define_domain + gmg_define_level / gmg_chop_domain) or
// several independent problems (gmg_define_batch).  Either way each MG level is ONE list
// of boxes over all problems, so one launch per step covers every problem; a device mask
// of still-active problems makes converged ones skip their work.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/gmg.h"
#include "amr_meta.h"
#include "kernels.h"
#include "meta.h"

using namespace gmg;

namespace {

thread_local std::string g_create_error;

size_t dt_size(int dt) { return dt == DT_F64 ? 8 : (dt == DT_F32 ? 4 : 2); }

struct LevelBufs {
  // FP64 coefficients
  double *acoef = nullptr, *wx = nullptr, *wy = nullptr, *wz = nullptr, *D = nullptr, *invD = nullptr;
  // float coefficients (mixed precision)
  float *fwx = nullptr, *fwy = nullptr, *fwz = nullptr, *fD = nullptr, *finvD = nullptr;
  // V-cycle correction and right-hand side per element type
  void* e[NDT] = {nullptr, nullptr, nullptr};
  void* r[NDT] = {nullptr, nullptr, nullptr};
  // bottom work vectors (7 doubles per element) if a bottom problem lives here
  double* bot_work = nullptr;
};

// bump allocator over the caller's workspace; run once with base = nullptr to size
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  void* take(size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
  // A level array of elem-byte elements that kernels read without its x ghosts
  // (coefficients, right-hand sides): 128 - 8 elem bytes past a 256-byte boundary.  Rows of
  // the boxed layout start on 128-byte lines (float, double) and their first valid cell sits
  // at element 8, so here the valid cells of a row begin on a line: 64 doubles are 4 lines
  // instead of 5, 64 floats 2 instead of 3.  DRAM traffic follows whole lines (abec256
  // level-0 FP64 sweep: 1.02 -> 0.87 GB per colour); fields read with their x ghosts (phi,
  // e) keep the plain placement, where the ghosts share the end lines.
  void* take_rows(size_t bytes, size_t elem) {
    off = ((off + 255) & ~(size_t)255) + ((128 - 8 * elem) & 127);
    void* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  }
};

}  // namespace

namespace gmg {
// errors of calls that have no context; read back through gmg_last_error(NULL)
void set_thread_error(const std::string& msg) { g_create_error = msg; }
}  // namespace gmg

// One AMR level above level 0: its boxes (one MG level whose coarse correction is the level
// below), the tables of the pair (level below, this level), device views, coefficients and
// work fields.
struct AmrLevel {
  LevelMeta M;
  AmrHost H;  // covered cells of the level below, this level's coarse/fine ghosts, reflux, averaging
  AmrDev A;
  LevelDev D;
  LevelBufs B;
  double *alpha = nullptr, *bx = nullptr, *by = nullptr, *bz = nullptr, *beta_cell = nullptr;
  double *rhs = nullptr, *res = nullptr, *tmp = nullptr, *zero = nullptr;  // projected rhs, residual
  double* kf[9] = {};  // adjoint BiCGStab vectors
  double* phi = nullptr;  // the composite solve's iterate on this level
  bool have_beta = false, have_alpha = false;
};

struct gmg_ctx {
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
  // batched contexts: a second stream for bottom solves that overlap the other problems'
  // coarser levels, with a fork and a join event per MG level
  cudaStream_t side_stream = nullptr;
  std::vector<cudaEvent_t> ev_fork, ev_join;
  std::string err;

  bool have_domain = false;
  std::vector<SolveGeom> geoms;  // level-0 geometry per independent problem
  std::vector<LevelMeta> L;      // multigrid levels, 0 = the user's BoxArray(s)
  double a = 0.0, b = 1.0;

  // workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool mixed = false;  // float buffers present
  std::vector<LevelDev> dev;
  std::vector<LevelBufs> buf;
  double *alpha0 = nullptr, *bx0 = nullptr, *by0 = nullptr, *bz0 = nullptr, *tmp0 = nullptr;
  // top-level Krylov vectors (level-0 FP64, after everything else in the workspace when it
  // was sized for them): b, r, rhat, p, v, y, s, t, z
  static constexpr int NKV = 9;
  double* kv[NKV] = {};
  // per-problem device scalars
  unsigned long long* normbits = nullptr;  // [0, ns): outer residual norms; [ns, 2ns): rhs / step norms
  double* partials = nullptr;
  double* scal = nullptr;  // [0, ns): rhs means; [ns, 2ns): phi means
  int* bot_iters = nullptr;
  int* dev_err = nullptr;  // raised by a kernel whose bounded wait gave up
  int* active = nullptr;  // per problem: 1 while it iterates
  int max_cell_chunks = 0;

  bool have_beta = false, have_alpha = false;
  bool coefs_dirty = true;

  // pinned host mirrors
  unsigned long long* h_bits = nullptr;
  double* h_scal = nullptr;
  int* h_iters = nullptr;
  int* h_active = nullptr;
  size_t h_cap = 0;

  // graphs of one outer iteration, keyed by (phi, rhs, precision, nu1, nu2, bottom, profile)
  struct GraphEntry {
    cudaGraphExec_t exec;
    int64_t launches;
    int n_ev_smooth, n_ev_resid;  // profiling event pairs recorded per replay
    std::vector<int> passes;      // colour passes of each smoother event pair
  };
  std::map<
      std::tuple<void*, const void*, int, int, int, int, double, int, int, int, int, int, int, int, int, int, int, int>,
      GraphEntry>
      graphs;
  // preconditioner V-cycles of the top-level Krylov solvers, per (input, output, params)
  std::map<std::tuple<const void*, void*, int, int, int, int, double, int, int, int, int, int, int, int, int>, GraphEntry>
      kgraphs;

  // profiling events (pairs around finest-level smoother / outer residual launches)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_smooth, ev_resid;
  int n_ev_smooth = 0, n_ev_resid = 0;
  std::vector<int> ev_smooth_passes;  // colour passes covered by each smoother event pair

  // cell beta of level 0 as last set (ghosts filled), for beta gradients
  double* betac_cell = nullptr;

  // autotuned choices (gmg_autotune), per element type: ghost push per MG level (-1: not
  // tuned), fused coarse end (-1: not tuned); graphs are rebuilt after tuning
  std::vector<signed char> push_choice[NDT];
  int tail_choice[NDT] = {-1, -1, -1};
  std::vector<double> tune_ms_push[NDT], tune_ms_pull[NDT];
  double tune_ms_tail[NDT][2] = {{0, 0}, {0, 0}, {0, 0}};

  // serpentine order (gmg_params.serpentine, set per call): per MG level, the direction the
  // last level-sweep launch took its work list in
  bool serp = true;
  std::vector<int> dir;

  // per MG level: the vc_flow_skip table on the device (the V-cycle's view of the flow sweep)
  std::vector<const int*> vc_flow_skip;

  // coarse ends of the problems' V-cycles, one thread block each (tail.cu)
  TailHost tail;
  bool tail_ok = false;  // tables built and addressable (hierarchy within TAIL_MAXLEV levels)
  TailDesc* tdescs = nullptr;
  TailLevel* tlevels = nullptr;
  BotCell* tcells = nullptr;
  BotGhost* tghosts = nullptr;
  TailXfer* txfer = nullptr;
  BotGhost* tdghosts = nullptr;

  // composite form: AMR levels 1, 2, ... (ratio 2 each) over part of the level below;
  // amrl[l - 1] is AMR level l
  bool amr = false;
  std::vector<AmrLevel> amrl;
  double *crhs = nullptr, *cres = nullptr;  // level 0: projected rhs, composite residual
  double *ctmp = nullptr, *czero = nullptr;
  double* kc[9] = {};  // level 0's adjoint BiCGStab vectors
  double* cphi = nullptr;  // level 0's iterate of the composite solve

  int ns() const { return (int)geoms.size(); }
};

#define SETERR(ctx, code, msg) \
  do {                          \
    (ctx)->err = (msg);         \
    return (code);              \
  } while (0)

#define CK(ctx, call)                                                  \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return GMG_ERR_CUDA;                                             \
    }                                                                  \
  } while (0)

namespace {

void drop_graphs(gmg_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
  c->graphs.clear();
  for (auto& kv : c->kgraphs) cudaGraphExecDestroy(kv.second.exec);
  c->kgraphs.clear();
}

// event pair k of a list (created on first use, outside any capture)
cudaEvent_t* ev_pair(std::vector<cudaEvent_t>& v, int k) {
  while ((int)v.size() < 2 * (k + 1)) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    v.push_back(e);
  }
  return &v[2 * k];
}

// no Dirichlet wall and a = 0: the constants span the null space of A
bool singular(const gmg_ctx* c, int s) { return !c->geoms[s].has_dirichlet() && c->a == 0.0; }
bool any_singular(const gmg_ctx* c) {
  for (int s = 0; s < c->ns(); ++s)
    if (singular(c, s)) return true;
  return false;
}

int nlev(const gmg_ctx* c) { return (int)c->L.size(); }
// AMR levels of the context (level 0 included)
int namr(const gmg_ctx* c) { return 1 + (int)c->amrl.size(); }

Coefs coefs_of(const gmg_ctx* c, int m, int dt) {
  const LevelBufs& B = c->buf[m];
  Coefs k;
  if (dt == DT_F64) {
    k.wx = B.wx; k.wy = B.wy; k.wz = B.wz; k.D = B.D; k.invD = B.invD;
  } else {
    k.wx = B.fwx; k.wy = B.fwy; k.wz = B.fwz; k.D = B.fD; k.invD = B.finvD;
  }
  return k;
}

Coefs coefs64(const gmg_ctx* c, int m) { return coefs_of(c, m, DT_F64); }

gmg_status check_level(gmg_ctx* c, int m, int dt) {
  if (c->L.empty()) SETERR(c, GMG_ERR_STATE, "no BoxArray defined");
  if (m < 0 || m >= nlev(c)) SETERR(c, GMG_ERR_BAD_INPUT, "MG level out of range");
  if (dt < 0 || dt >= NDT) SETERR(c, GMG_ERR_BAD_INPUT, "bad element type");
  if (!c->ws) SETERR(c, GMG_ERR_NO_WORKSPACE, "no workspace set");
  if (dt != DT_F64 && !c->mixed) SETERR(c, GMG_ERR_NO_WORKSPACE, "workspace has no float buffers (size it for a mixed precision)");
  return GMG_OK;
}

// Carve the workspace (base = nullptr: size only).  Returns bytes.

// Whether the finest level of a context keeps its right-hand side and 1/D colour-split within
// rows (split_index): every box smooths there (none has its bottom on it), every width is
// even, and no AMR level sits above it (the composite solve writes its own right-hand sides).
// A colour pass then reads half of each of those two arrays' sectors instead of all of them.
bool split_level_ok(const gmg_ctx* c, const LevelMeta& M) {
  if (c->amr || c->L.size() < 2 || !M.bot_descs.empty() || M.pair_chunks.empty()) return false;
  for (const Box& b : M.boxes)
    if (b.n(0) % 2 != 0) return false;
  return true;
}

size_t carve(gmg_ctx* c, void* base, bool mixed, bool fill) {
  Carver cv(base);
  const int n = nlev(c);
  const size_t ns = (size_t)std::max(1, c->ns());
  if (fill) {
    c->dev.assign(n, LevelDev());
    c->buf.assign(n, LevelBufs());
  }
  int* active = (int*)cv.take(4 * ns);
  int maxchunks = 1;
  std::vector<const int*> vc_skip(n, nullptr);
  for (int m = 0; m < n; ++m) {
    const LevelMeta& M = c->L[m];
    const size_t ne = (size_t)M.nelem;
    LevelDev D;
    LevelBufs B;
    D.nelem = M.nelem;
    D.nsolves = (int)ns;
    D.active = active;
    D.boxes = (const DevBox*)cv.take(sizeof(DevBox) * M.dbox.size());
    D.geoms = (const DevGeom*)cv.take(sizeof(DevGeom) * M.geoms.size());
    D.ghosts = (const GhostRect*)cv.take(sizeof(GhostRect) * M.ghosts.size());
    D.ghost_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.ghost_chunks.size());
    D.n_ghost_chunks = (int)M.ghost_chunks.size();
    D.pair_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.pair_chunks.size());
    D.n_pair_chunks = (int)M.pair_chunks.size();
    D.quad_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.quad_chunks.size());
    D.n_quad_chunks = (int)M.quad_chunks.size();
    D.pair_all_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.pair_all_chunks.size());
    D.n_pair_all_chunks = (int)M.pair_all_chunks.size();
    D.cell_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.cell_chunks.size());
    D.n_cell_chunks = (int)M.cell_chunks.size();
    D.coarse_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.coarse_chunks.size());
    D.n_coarse_chunks = (int)M.coarse_chunks.size();
    D.parent = (const int*)cv.take(sizeof(int) * M.parent.size());
    D.child = (const int*)cv.take(sizeof(int) * M.child.size());
    D.bot_cells = (const BotCell*)cv.take(sizeof(BotCell) * M.bot_cells.size());
    D.bot_ghosts = (const BotGhost*)cv.take(sizeof(BotGhost) * M.bot_ghosts.size());
    D.bot_descs = (const BotDesc*)cv.take(sizeof(BotDesc) * M.bot_descs.size());
    D.n_bot = (int)M.bot_descs.size();
    D.solve_chunk_range = (const int*)cv.take(sizeof(int) * M.solve_chunk_range.size());
    D.inv_count = (const double*)cv.take(sizeof(double) * M.inv_count.size());
    D.vc_ghost_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.vc_ghost_chunks.size());
    D.n_vc_ghost_chunks = (int)M.vc_ghost_chunks.size();
    D.vc_pair_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.vc_pair_chunks.size());
    D.n_vc_pair_chunks = (int)M.vc_pair_chunks.size();
    D.vc_quad_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.vc_quad_chunks.size());
    D.n_vc_quad_chunks = (int)M.vc_quad_chunks.size();
    D.vc_coarse_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.vc_coarse_chunks.size());
    D.n_vc_coarse_chunks = (int)M.vc_coarse_chunks.size();
    D.vc_bot_descs = (const BotDesc*)cv.take(sizeof(BotDesc) * M.vc_bot_descs.size());
    D.n_vc_bot = (int)M.vc_bot_descs.size();
    D.flow_items = (const FlowItem*)cv.take(sizeof(FlowItem) * M.flow_items.size());
    D.flow_slabs = (const FlowSlab*)cv.take(sizeof(FlowSlab) * M.flow_slabs.size());
    D.n_flow_slabs = (int)M.flow_slabs.size();
    for (int q = 0; q < FLOW_MAX_PHASES; ++q) {
      D.flow_order[q] = (const FlowChunk*)cv.take(sizeof(FlowChunk) * M.flow_order[q].size());
      D.n_flow_order[q] = (int)M.flow_order[q].size();
    }
    D.flow_cnt = M.flow_slabs.empty()
                     ? nullptr
                     : (int*)cv.take(sizeof(int) * FLOW_CNT_STRIDE *
                                     (FLOW_QUEUES + 1 + FLOW_MAX_PHASES * M.flow_slabs.size()));
    vc_skip[m] = (const int*)cv.take(sizeof(int) * M.vc_flow_skip.size());
    D.ec_ghosts = (const BotGhost*)cv.take(sizeof(BotGhost) * M.ec_ghosts.size());
    D.n_ec_ghosts = (int)M.ec_ghosts.size();
    D.push_faces = (const PushFace*)cv.take(sizeof(PushFace) * M.push_faces.size());
    D.push_ok = M.push_ok ? 1 : 0;
    D.split = (m == 0 && split_level_ok(c, M)) ? (SPLIT_RHS | SPLIT_INVD) : 0;
    D.wave_tiles = (const WaveTile*)cv.take(sizeof(WaveTile) * M.wave_tiles.size());
    D.n_wave_tiles = (int)M.wave_tiles.size();
    D.wave_ppt = M.wave_ppt;
    D.wave_max_solve_tiles = M.wave_max_solve_tiles;
    D.wave_layer_cells = M.wave_layer_cells;
    D.wave_cnt = M.wave_tiles.empty() ? nullptr : (unsigned*)cv.take(sizeof(unsigned) * (64 + M.wave_tiles.size()));
    maxchunks = std::max(maxchunks, D.n_cell_chunks);
    B.acoef = (double*)cv.take_rows(8 * ne, 8);
    B.wx = (double*)cv.take_rows(8 * ne, 8);
    B.wy = (double*)cv.take_rows(8 * ne, 8);
    B.wz = (double*)cv.take_rows(8 * ne, 8);
    B.D = (double*)cv.take_rows(8 * ne, 8);
    B.invD = (double*)cv.take_rows(8 * ne, 8);
    B.e[DT_F64] = cv.take(8 * ne);
    B.r[DT_F64] = cv.take_rows(8 * ne, 8);
    if (mixed) {
      B.fwx = (float*)cv.take_rows(4 * ne, 4);
      B.fwy = (float*)cv.take_rows(4 * ne, 4);
      B.fwz = (float*)cv.take_rows(4 * ne, 4);
      B.fD = (float*)cv.take_rows(4 * ne, 4);
      B.finvD = (float*)cv.take_rows(4 * ne, 4);
      B.e[DT_F32] = cv.take(4 * ne);
      B.r[DT_F32] = cv.take_rows(4 * ne, 4);
      B.e[DT_BF16] = cv.take(2 * ne);
      B.r[DT_BF16] = cv.take_rows(2 * ne, 2);
    }
    if (!M.bot_descs.empty()) B.bot_work = (double*)cv.take(8 * 7 * ne);
    if (fill) {
      c->dev[m] = D;
      c->buf[m] = B;
    }
  }
  if (fill) c->vc_flow_skip = vc_skip;
  const size_t ne0 = c->L.empty() ? 0 : (size_t)c->L[0].nelem;
  double* alpha0 = (double*)cv.take(8 * ne0);
  double* bx0 = (double*)cv.take(8 * ne0);
  double* by0 = (double*)cv.take(8 * ne0);
  double* bz0 = (double*)cv.take(8 * ne0);
  double* tmp0 = (double*)cv.take(8 * ne0);
  double* betac = (double*)cv.take(8 * ne0);
  if (fill) c->betac_cell = betac;
  {
    const TailHost& T = c->tail;
    TailDesc* td = (TailDesc*)cv.take(sizeof(TailDesc) * T.descs.size());
    TailLevel* tl = (TailLevel*)cv.take(sizeof(TailLevel) * T.levels.size());
    BotCell* tc = (BotCell*)cv.take(sizeof(BotCell) * T.cells.size());
    BotGhost* tg = (BotGhost*)cv.take(sizeof(BotGhost) * T.ghosts.size());
    TailXfer* tx = (TailXfer*)cv.take(sizeof(TailXfer) * T.xfer.size());
    BotGhost* tdg = (BotGhost*)cv.take(sizeof(BotGhost) * T.dghosts.size());
    if (fill) {
      c->tdescs = td; c->tlevels = tl; c->tcells = tc; c->tghosts = tg; c->txfer = tx; c->tdghosts = tdg;
    }
  }
  for (size_t al = 0; al < c->amrl.size(); ++al) {  // AMR level al + 1
    const LevelMeta& M = c->amrl[al].M;
    const AmrHost& H = c->amrl[al].H;
    const size_t nf = (size_t)M.nelem;
    LevelDev D;
    LevelBufs B;
    D.nelem = M.nelem;
    D.nsolves = 1;
    D.active = active;
    D.boxes = (const DevBox*)cv.take(sizeof(DevBox) * M.dbox.size());
    D.geoms = (const DevGeom*)cv.take(sizeof(DevGeom) * M.geoms.size());
    D.ghosts = (const GhostRect*)cv.take(sizeof(GhostRect) * M.ghosts.size());
    D.ghost_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.ghost_chunks.size());
    D.n_ghost_chunks = (int)M.ghost_chunks.size();
    D.pair_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.pair_chunks.size());
    D.n_pair_chunks = (int)M.pair_chunks.size();
    D.pair_all_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.pair_all_chunks.size());
    D.n_pair_all_chunks = (int)M.pair_all_chunks.size();
    D.cell_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.cell_chunks.size());
    D.n_cell_chunks = (int)M.cell_chunks.size();
    D.coarse_chunks = (const Chunk*)cv.take(sizeof(Chunk) * M.coarse_chunks.size());
    D.n_coarse_chunks = (int)M.coarse_chunks.size();
    D.parent = (const int*)cv.take(sizeof(int) * M.parent.size());
    D.solve_chunk_range = (const int*)cv.take(sizeof(int) * M.solve_chunk_range.size());
    D.inv_count = (const double*)cv.take(sizeof(double) * M.inv_count.size());
    D.push_faces = (const PushFace*)cv.take(sizeof(PushFace) * M.push_faces.size());
    D.push_ok = M.push_ok ? 1 : 0;
    D.wave_tiles = (const WaveTile*)cv.take(sizeof(WaveTile) * M.wave_tiles.size());
    D.n_wave_tiles = (int)M.wave_tiles.size();
    D.wave_ppt = M.wave_ppt;
    D.wave_max_solve_tiles = M.wave_max_solve_tiles;
    D.wave_layer_cells = M.wave_layer_cells;
    D.wave_cnt = M.wave_tiles.empty() ? nullptr : (unsigned*)cv.take(sizeof(unsigned) * (64 + M.wave_tiles.size()));
    maxchunks = std::max(maxchunks, D.n_cell_chunks);
    B.acoef = (double*)cv.take_rows(8 * nf, 8);
    B.wx = (double*)cv.take_rows(8 * nf, 8);
    B.wy = (double*)cv.take_rows(8 * nf, 8);
    B.wz = (double*)cv.take_rows(8 * nf, 8);
    B.D = (double*)cv.take_rows(8 * nf, 8);
    B.invD = (double*)cv.take_rows(8 * nf, 8);
    B.e[DT_F64] = cv.take(8 * nf);
    B.r[DT_F64] = cv.take_rows(8 * nf, 8);
    AmrDev A;
    A.cf = (const CfGhost*)cv.take(sizeof(CfGhost) * H.cf.size());
    A.ncf = (int)H.cf.size();
    A.rcells = (const RefluxCell*)cv.take(sizeof(RefluxCell) * H.rcells.size());
    A.nrcell = (int)H.rcells.size();
    A.rfaces = (const RefluxFace*)cv.take(sizeof(RefluxFace) * H.rfaces.size());
    A.covered_list = (const int64_t*)cv.take(sizeof(int64_t) * H.covered_list.size());
    A.ncov = (int)H.covered_list.size();
    A.covered = (const unsigned char*)cv.take(H.covered.size());
    A.cfidx = (const int*)cv.take(sizeof(int) * H.cfidx.size());
    A.hf_over_hc = 0.5;
    A.avg_faces = (const AvgFace*)cv.take(sizeof(AvgFace) * H.avg_faces.size());
    A.navg_face = (int)H.avg_faces.size();
    A.avg_cells = (const AvgCell*)cv.take(sizeof(AvgCell) * H.avg_cells.size());
    A.navg_cell = (int)H.avg_cells.size();
    double* f5[5];
    for (int q = 0; q < 5; ++q) f5[q] = (double*)cv.take(8 * nf);
    double* cc[5] = {};
    if (al == 0)
      for (int q = 0; q < 5; ++q) cc[q] = (double*)cv.take(8 * ne0);
    double* ff[5];
    for (int q = 0; q < 5; ++q) ff[q] = (double*)cv.take(8 * nf);
    double *kc[9] = {}, *kf[9] = {};  // the adjoint solve's vectors
    for (int q = 0; q < 9; ++q) {
      if (al == 0) kc[q] = (double*)cv.take(8 * ne0);
      kf[q] = (double*)cv.take(8 * nf);
    }
    if (fill) {
      AmrLevel& V = c->amrl[al];
      V.D = D;
      V.B = B;
      V.A = A;
      V.alpha = f5[0]; V.bx = f5[1]; V.by = f5[2]; V.bz = f5[3]; V.beta_cell = f5[4];
      if (al == 0) {
        c->crhs = cc[0]; c->cres = cc[1]; c->ctmp = cc[2]; c->czero = cc[3]; c->cphi = cc[4];
        for (int q = 0; q < 9; ++q) c->kc[q] = kc[q];
      }
      V.rhs = ff[0]; V.res = ff[1]; V.tmp = ff[2]; V.zero = ff[3]; V.phi = ff[4];
      for (int q = 0; q < 9; ++q) V.kf[q] = kf[q];
    }
  }
  unsigned long long* nb = (unsigned long long*)cv.take(8 * (2 * ns + 8));
  // (multi-level dot products keep the partials of every composite level twice)
  int mlchunks = c->L.empty() ? 0 : (int)c->L[0].cell_chunks.size();
  for (const AmrLevel& V : c->amrl) mlchunks += (int)V.M.cell_chunks.size();
  double* partials = (double*)cv.take(8 * (size_t)std::max(maxchunks, 2 * mlchunks));
  double* scal = (double*)cv.take(8 * (2 * ns + 8));
  int* iters = (int*)cv.take(4 * (ns + 1));  // bottom iterations per problem, then the device error flag
  if (fill) {
    c->alpha0 = alpha0; c->bx0 = bx0; c->by0 = by0; c->bz0 = bz0; c->tmp0 = tmp0;
    c->normbits = nb; c->partials = partials; c->scal = scal; c->bot_iters = iters;
    c->dev_err = iters + ns;
    c->active = active;
    c->max_cell_chunks = maxchunks;
  }
  return cv.off + 256;
}

template <class V>
gmg_status upload(gmg_ctx* c, const void* dst, const std::vector<V>& v) {
  if (v.empty()) return GMG_OK;
  CK(c, cudaMemcpyAsync((void*)dst, v.data(), sizeof(V) * v.size(), cudaMemcpyHostToDevice, c->stream));
  return GMG_OK;
}

std::vector<DevGeom> dev_geoms(const LevelMeta& M) {
  std::vector<DevGeom> g(M.geoms.size());
  for (size_t s = 0; s < g.size(); ++s) {
    const SolveGeom& G = M.geoms[s];
    for (int d = 0; d < 3; ++d) {
      g[s].dlo[d] = G.domain.lo[d];
      g[s].dhi[d] = G.domain.hi[d];
      // the boundary codes: 0 periodic, 1 Dirichlet, 2 Neumann, 3 quadratic Dirichlet
      g[s].wall_lo[d] = G.qlo[d] ? 3 : G.bclo[d];
      g[s].wall_hi[d] = G.qhi[d] ? 3 : G.bchi[d];
      g[s].ih2[d] = 1.0 / (G.h[d] * G.h[d]);
    }
  }
  return g;
}

gmg_status upload_tables(gmg_ctx* c) {
  for (int m = 0; m < nlev(c); ++m) {
    const LevelMeta& M = c->L[m];
    const LevelDev& D = c->dev[m];
    gmg_status st;
    if ((st = upload(c, D.boxes, M.dbox))) return st;
    if ((st = upload(c, D.geoms, dev_geoms(M)))) return st;
    if ((st = upload(c, D.ghosts, M.ghosts))) return st;
    if ((st = upload(c, D.ghost_chunks, M.ghost_chunks))) return st;
    if ((st = upload(c, D.pair_chunks, M.pair_chunks))) return st;
    if ((st = upload(c, D.quad_chunks, M.quad_chunks))) return st;
    if ((st = upload(c, D.pair_all_chunks, M.pair_all_chunks))) return st;
    if ((st = upload(c, D.cell_chunks, M.cell_chunks))) return st;
    if ((st = upload(c, D.coarse_chunks, M.coarse_chunks))) return st;
    if ((st = upload(c, D.parent, M.parent))) return st;
    if ((st = upload(c, D.child, M.child))) return st;
    if ((st = upload(c, D.bot_cells, M.bot_cells))) return st;
    if ((st = upload(c, D.bot_ghosts, M.bot_ghosts))) return st;
    if ((st = upload(c, D.bot_descs, M.bot_descs))) return st;
    if ((st = upload(c, D.solve_chunk_range, M.solve_chunk_range))) return st;
    if ((st = upload(c, D.inv_count, M.inv_count))) return st;
    if ((st = upload(c, D.vc_ghost_chunks, M.vc_ghost_chunks))) return st;
    if ((st = upload(c, D.vc_pair_chunks, M.vc_pair_chunks))) return st;
    if ((st = upload(c, D.vc_quad_chunks, M.vc_quad_chunks))) return st;
    if ((st = upload(c, D.vc_coarse_chunks, M.vc_coarse_chunks))) return st;
    if ((st = upload(c, D.vc_bot_descs, M.vc_bot_descs))) return st;
    if ((st = upload(c, D.flow_items, M.flow_items))) return st;
    if ((st = upload(c, D.flow_slabs, M.flow_slabs))) return st;
    for (int q = 0; q < FLOW_MAX_PHASES; ++q)
      if ((st = upload(c, D.flow_order[q], M.flow_order[q]))) return st;
    if (D.flow_cnt)
      CK(c, cudaMemsetAsync(D.flow_cnt, 0,
                            sizeof(int) * FLOW_CNT_STRIDE * (FLOW_QUEUES + 1 + FLOW_MAX_PHASES * M.flow_slabs.size()),
                            c->stream));
    if ((st = upload(c, c->vc_flow_skip[m], M.vc_flow_skip))) return st;
    if ((st = upload(c, D.ec_ghosts, M.ec_ghosts))) return st;
    if ((st = upload(c, D.push_faces, M.push_faces))) return st;
    if ((st = upload(c, D.wave_tiles, M.wave_tiles))) return st;
    if (D.wave_cnt) CK(c, cudaMemsetAsync(D.wave_cnt, 0, sizeof(unsigned) * (64 + M.wave_tiles.size()), c->stream));
  }
  {
    const TailHost& T = c->tail;
    gmg_status st;
    if ((st = upload(c, c->tdescs, T.descs))) return st;
    if ((st = upload(c, c->tlevels, T.levels))) return st;
    if ((st = upload(c, c->tcells, T.cells))) return st;
    if ((st = upload(c, c->tghosts, T.ghosts))) return st;
    if ((st = upload(c, c->txfer, T.xfer))) return st;
    if ((st = upload(c, c->tdghosts, T.dghosts))) return st;
  }
  for (const AmrLevel& V : c->amrl) {
    const LevelMeta& M = V.M;
    const LevelDev& D = V.D;
    const AmrHost& H = V.H;
    const AmrDev& A = V.A;
    gmg_status st;
    if ((st = upload(c, D.boxes, M.dbox))) return st;
    if ((st = upload(c, D.geoms, dev_geoms(M)))) return st;
    if ((st = upload(c, D.ghosts, M.ghosts))) return st;
    if ((st = upload(c, D.ghost_chunks, M.ghost_chunks))) return st;
    if ((st = upload(c, D.pair_chunks, M.pair_chunks))) return st;
    if ((st = upload(c, D.pair_all_chunks, M.pair_all_chunks))) return st;
    if ((st = upload(c, D.cell_chunks, M.cell_chunks))) return st;
    if ((st = upload(c, D.coarse_chunks, M.coarse_chunks))) return st;
    if ((st = upload(c, D.parent, M.parent))) return st;
    if ((st = upload(c, D.solve_chunk_range, M.solve_chunk_range))) return st;
    if ((st = upload(c, D.inv_count, M.inv_count))) return st;
    if ((st = upload(c, D.push_faces, M.push_faces))) return st;
    if ((st = upload(c, A.cf, H.cf))) return st;
    if ((st = upload(c, A.rcells, H.rcells))) return st;
    if ((st = upload(c, A.rfaces, H.rfaces))) return st;
    if ((st = upload(c, A.covered_list, H.covered_list))) return st;
    if ((st = upload(c, A.covered, H.covered))) return st;
    if ((st = upload(c, A.cfidx, H.cfidx))) return st;
    if ((st = upload(c, A.avg_faces, H.avg_faces))) return st;
    if ((st = upload(c, A.avg_cells, H.avg_cells))) return st;
  }
  std::vector<int> ones(c->ns(), 1);
  gmg_status st = upload(c, c->active, ones);
  if (st) return st;
  CK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return GMG_OK;
}

void reset_problem(gmg_ctx* c) {
  drop_graphs(c);
  c->L.clear();
  c->ws = nullptr;
  c->ws_bytes = 0;
  c->have_beta = c->have_alpha = false;
  c->coefs_dirty = true;
  c->amr = false;
  c->amrl.clear();
  c->tail = TailHost();
  c->tail_ok = false;
  for (int d = 0; d < NDT; ++d) {
    c->push_choice[d].clear();
    c->tail_choice[d] = -1;
    c->tune_ms_push[d].clear();
    c->tune_ms_pull[d].clear();
  }
}

// Build the multigrid hierarchy from level-0 boxes (stored problem by problem).
gmg_status build_hierarchy(gmg_ctx* c, const std::vector<Box>& boxes, const std::vector<int>& box_solve) {
  const int ns = c->ns();
  for (int s = 0; s < ns; ++s) {
    std::vector<Box> mine;
    for (size_t b = 0; b < boxes.size(); ++b)
      if (box_solve[b] == s) mine.push_back(boxes[b]);
    if (mine.empty()) SETERR(c, GMG_ERR_BAD_INPUT, "problem " + std::to_string(s) + " has no boxes");
    std::string e = validate_boxes(mine, c->geoms[s].domain, true);
    if (!e.empty()) SETERR(c, GMG_ERR_BAD_INPUT, (ns > 1 ? "problem " + std::to_string(s) + ": " : std::string()) + e);
  }
  reset_problem(c);
  {  // wavefront tiles: at most 8 blocks of the sweep per SM are assumed resident
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ==
                                                  cudaSuccess && nsm > 0)
      set_wave_capacity(8 * nsm);
    else
      cudaGetLastError();
  }
  LevelMeta L0;
  L0.boxes = boxes;
  L0.box_solve = box_solve;
  L0.geoms = c->geoms;
  L0.solve_present.assign(ns, 1);
  L0.solve_bottom.assign(ns, 0);
  c->L.push_back(L0);
  for (int m = 0; m < 64; ++m) {
    LevelMeta C;
    bool more = make_coarse(c->L[m], C);
    std::string e = finalize_level(c->L[m]);
    if (!e.empty()) SETERR(c, GMG_ERR_BAD_INPUT, e);
    if (m > 0) build_ec_ghosts(c->L[m]);  // the coarse side of an interpolation (trilinear option)
    if (!more) break;
    c->L.push_back(C);
  }
  // child boxes: level m's box b has exactly one child on level m - 1, of twice its extent
  for (int m = 0; m < nlev(c); ++m) {
    LevelMeta& M = c->L[m];
    M.child.assign(M.boxes.size(), -1);
    if (m == 0) continue;
    const LevelMeta& F = c->L[m - 1];
    std::vector<int> nchild(M.boxes.size(), 0);
    for (int f = 0; f < (int)F.boxes.size(); ++f)
      if (F.parent[f] >= 0) {
        ++nchild[F.parent[f]];
        M.child[F.parent[f]] = f;
      }
    for (int b = 0; b < (int)M.boxes.size(); ++b) {
      const int f = M.child[b];
      if (f < 0) continue;
      bool exact = nchild[b] == 1;
      for (int d = 0; d < 3; ++d)
        exact = exact && F.boxes[f].lo[d] == 2 * M.boxes[b].lo[d] && F.boxes[f].n(d) == 2 * M.boxes[b].n(d);
      if (!exact) M.child[b] = -1;
    }
  }
  c->tail_ok = false;
  if (nlev(c) <= TAIL_MAXLEV) {
    std::string e = build_tail(c->L, c->tail);
    if (!e.empty()) SETERR(c, GMG_ERR_BAD_INPUT, e);
    c->tail_ok = true;
  }
  return GMG_OK;
}

// Coefficients of every level from the stored level-0 alpha and face beta.
gmg_status build_coefs(gmg_ctx* c) {
  if (!c->coefs_dirty) return GMG_OK;
  if (!c->have_beta) SETERR(c, GMG_ERR_STATE, "beta not set (gmg_set_bcoef_cell / gmg_set_bcoef_face)");
  cudaStream_t s = c->stream;
  launch_acoef(c->dev[0], c->a, c->have_alpha ? c->alpha0 : nullptr, c->buf[0].acoef, s);
  launch_faces_scale(c->dev[0], c->b, c->bx0, c->by0, c->bz0, c->buf[0].wx, c->buf[0].wy, c->buf[0].wz, s);
  if (c->amr) {
    // every AMR level's own coefficients; then, finest pair first, a level under the next
    // finer one takes the restriction of that level's coefficients; the diagonals last
    for (size_t al = 0; al < c->amrl.size(); ++al) {
      const AmrLevel& V = c->amrl[al];
      if (!V.have_beta) SETERR(c, GMG_ERR_STATE, "beta of AMR level " + std::to_string(al + 1) + " not set");
      launch_acoef(V.D, c->a, V.have_alpha ? V.alpha : nullptr, V.B.acoef, s);
      launch_faces_scale(V.D, c->b, V.bx, V.by, V.bz, V.B.wx, V.B.wy, V.B.wz, s);
    }
    for (int l = namr(c) - 1; l >= 1; --l) {
      const LevelBufs& B = c->amrl[l - 1].B;
      const LevelBufs& Bc = l == 1 ? c->buf[0] : c->amrl[l - 2].B;
      launch_avgdown_coefs(c->amrl[l - 1].A, B.acoef, B.wx, B.wy, B.wz, Bc.acoef, Bc.wx, Bc.wy, Bc.wz, s);
    }
    for (const AmrLevel& V : c->amrl) launch_diag(V.D, V.B.acoef, V.B.wx, V.B.wy, V.B.wz, V.B.D, V.B.invD, s);
  }
  for (int m = 0; m + 1 < nlev(c); ++m) {
    const LevelBufs& F = c->buf[m];
    const LevelBufs& C = c->buf[m + 1];
    launch_coarsen_coefs(c->dev[m], c->dev[m + 1], F.acoef, F.wx, F.wy, F.wz, C.acoef, C.wx, C.wy, C.wz, s);
  }
  for (int m = 0; m < nlev(c); ++m) {
    const LevelBufs& B = c->buf[m];
    launch_diag(c->dev[m], B.acoef, B.wx, B.wy, B.wz, B.D, B.invD, s);
    if (c->mixed) {
      const int64_t n = c->L[m].nelem;
      launch_convert(DT_F64, DT_F32, B.wx, B.fwx, n, s);
      launch_convert(DT_F64, DT_F32, B.wy, B.fwy, n, s);
      launch_convert(DT_F64, DT_F32, B.wz, B.fwz, n, s);
      launch_convert(DT_F64, DT_F32, B.D, B.fD, n, s);
      launch_convert(DT_F64, DT_F32, B.invD, B.finvD, n, s);
    }
  }
  // singular flag of the bottom problems
  for (int m = 0; m < nlev(c); ++m) {
    LevelMeta& M = c->L[m];
    for (auto& d : M.bot_descs) d.singular = singular(c, d.solve) ? 1 : 0;
    for (auto& d : M.vc_bot_descs) d.singular = singular(c, d.solve) ? 1 : 0;
    gmg_status st = upload(c, c->dev[m].bot_descs, M.bot_descs);
    if (st) return st;
    if ((st = upload(c, c->dev[m].vc_bot_descs, M.vc_bot_descs))) return st;
  }
  for (auto& d : c->tail.descs) d.singular = singular(c, d.solve) ? 1 : 0;
  if (gmg_status st = upload(c, c->tdescs, c->tail.descs)) return st;
  CK(c, cudaGetLastError());
  c->coefs_dirty = false;
  return GMG_OK;
}

// A timing event: inside a capture it must be an external event-record node (a plain
// record becomes a dependency edge without a timestamp); outside, a plain record.
void record_timing_event(gmg_ctx* c, cudaEvent_t e, cudaStream_t s) {
  if (s == c->cap_stream) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

// ghost push on level m: 1 always (where the level allows it), 2 on levels that run the
// dataflow sweep, elsewhere the tuned choice (before tuning: levels below 2^22 cells, whose
// ghost exchanges are launch-latency bound)
bool push_on(const gmg_ctx* c, const gmg_params& p, int dt, int m) {
  if (p.ghost_push == 0) return false;
  if (p.ghost_push == 1) return true;
  if (p.fused_sweep != 0 && flow_ok(c->dev[m])) return true;  // the dataflow sweep needs pushed ghosts
  if (p.wave_sweep != 0 && wave_ok(c->dev[m])) return true;    // and so does the wavefront sweep
  const auto& ch = c->push_choice[dt];
  if (m < (int)ch.size() && ch[m] >= 0) return (ch[m] & 1) != 0;
  return c->L[m].ncells < (1 << 22);
}

// 4-cell sweep threads on level m: 1 always (where possible), 2 the tuned choice (before
// tuning: bfloat16 only)
bool vec_on(const gmg_ctx* c, const gmg_params& p, int dt, int m) {
  if (p.vector_smooth != 2) return p.vector_smooth == 1;
  const auto& ch = c->push_choice[dt];
  if (m < (int)ch.size() && ch[m] >= 0) return (ch[m] & 2) != 0;
  return dt == DT_BF16;
}

// a problem of the context has a quadratic Dirichlet side
bool any_quad(const gmg_ctx* c) {
  for (const SolveGeom& G : c->geoms)
    if (G.has_quad()) return true;
  return false;
}

bool tail_on(const gmg_ctx* c, const gmg_params& p, int dt) {
  if (p.prolongation == 1) return false;  // the one-block coarse end interpolates piecewise constant
  if (any_quad(c)) return false;          // its ghost lists copy or negate only
  if (p.fused_coarse == 2) return c->tail_choice[dt] != 0;  // untuned: on
  return p.fused_coarse == 1;
}

// Serpentine order: a copy of D whose level-sweep kernels take their work list in the
// direction opposite to the previous such launch on level m (the first boxes they touch are
// the last ones the previous kernel touched, still in L2).  Forward if serpentine is off.
LevelDev dir_view(gmg_ctx* c, const LevelDev& D, int m) {
  LevelDev V = D;
  V.rev = 0;
  if (!c->serp) return V;
  if ((int)c->dir.size() <= m) c->dir.resize(m + 1, 0);
  c->dir[m] ^= 1;
  V.rev = c->dir[m];
  return V;
}

// whether the sweeps of level m run as dataflow launches (flow.cu): fused_sweep 1 or 2 on
// levels with flow tables whose ghosts are pushed (default 0: one launch per colour)
bool flow_on(const gmg_ctx* c, const gmg_params& p, const LevelDev& D, bool push) {
  (void)c;
  return p.fused_sweep != 0 && push && flow_ok(D);
}

// a profiling event pair around a finest-level smoother launch covering `passes` colour passes
cudaEvent_t* smooth_event(gmg_ctx* c, int passes) {
  const int k = c->n_ev_smooth++;
  if ((int)c->ev_smooth_passes.size() <= k) c->ev_smooth_passes.resize(k + 1, 0);
  c->ev_smooth_passes[k] = passes;
  return ev_pair(c->ev_smooth, k);
}

// push: the smoother writes its new values into the ghost cells that copy them, so no
// ghost exchange precedes a colour (the ghosts are kept current since e was cleared)
void smooth_colour(gmg_ctx* c, const LevelDev& D, int dt, int m, int colour, cudaStream_t s, bool fill = true,
                   bool push = false, bool vec = true) {
  const LevelBufs& B = c->buf[m];
  if (fill && !push) launch_fill(dt, D, B.e[dt], 1 - colour, 0, s);
  const bool prof = c->profiling && m == 0;
  cudaEvent_t* ev = prof ? smooth_event(c, 1) : nullptr;
  if (prof) record_timing_event(c, ev[0], s);
  launch_smooth(dt, dir_view(c, D, m), B.e[dt], B.r[dt], coefs_of(c, m, dt), colour, s, push, vec, true);
  if (prof) record_timing_event(c, ev[1], s);
}

// the red pass of smooth_colour fused with the interpolation of the coarse correction ec
// (level m + 1) that precedes it (launch_smooth_pro)
void smooth_colour_pro(gmg_ctx* c, const LevelDev& D, const LevelDev& Dc, int dt, int m, const void* ec,
                       cudaStream_t s, bool push) {
  const LevelBufs& B = c->buf[m];
  if (!push) launch_fill(dt, D, B.e[dt], 1, 0, s);
  const bool prof = c->profiling && m == 0;
  cudaEvent_t* ev = prof ? smooth_event(c, 1) : nullptr;
  if (prof) record_timing_event(c, ev[0], s);
  launch_smooth_pro(dt, dir_view(c, D, m), Dc, B.e[dt], B.r[dt], coefs_of(c, m, dt), 0, ec, s, push, true);
  if (prof) record_timing_event(c, ev[1], s);
}

// whether the sweeps of level m run as wavefront launches (wave.cu): wave_sweep on, the level
// has wavefront tables and pushes its ghosts (red-first sweeps only)
bool wave_on(const gmg_params& p, const LevelDev& D, bool push) { return p.wave_sweep != 0 && push && wave_ok(D); }

// One red-black sweep (red, then black) of level m as two launches; phi_last: the black pass
// also adds e to phi (k_smooth_update).
void black_pass(gmg_ctx* c, const LevelDev& D, int dt, int m, cudaStream_t s, bool push, bool vec, double* phi_last,
                bool push_phi) {
  if (!phi_last) {
    smooth_colour(c, D, dt, m, 1, s, true, push, vec);
    return;
  }
  const LevelBufs& B = c->buf[m];
  if (!push) launch_fill(dt, D, B.e[dt], 0, 0, s);
  const bool prof = c->profiling && m == 0;
  cudaEvent_t* ev = prof ? smooth_event(c, 1) : nullptr;
  if (prof) record_timing_event(c, ev[0], s);
  launch_smooth_update(dt, dir_view(c, D, m), B.e[dt], B.r[dt], coefs_of(c, m, dt), 1, phi_last, push_phi, s,
                       true);
  if (prof) record_timing_event(c, ev[1], s);
}
void two_pass_sweep(gmg_ctx* c, const LevelDev& D, int dt, int m, cudaStream_t s, bool fill_red, bool push, bool vec,
                    double* phi_last, bool push_phi) {
  smooth_colour(c, D, dt, m, 0, s, fill_red, push, vec);
  black_pass(c, D, dt, m, s, push, vec, phi_last, push_phi);
}

// nsweep red-black sweeps on level m.
// e_zero: e is zero including its ghosts (just cleared), so the first ghost fill would
// copy zeros and is skipped.
// red_done: the first red half-sweep was done by the residual kernel (level 0)
// reverse: black before red in every sweep (post-smoothing of the symmetric V-cycle)
// phi_last (finest level, red-first order): the last (black) pass also adds e to phi
// (k_smooth_update), pushing phi's new values into its ghosts if push_phi
// On levels with flow tables and pushed ghosts (fused_sweep != 0) the colour passes run
// as dataflow launches of up to FLOW_MAX_PHASES passes each, with the same values.
void smooth_sweeps(gmg_ctx* c, const LevelDev& D, int dt, int m, int nsweep, const gmg_params& p, cudaStream_t s,
                   bool e_zero = false, bool push = false, bool red_done = false, bool reverse = false,
                   double* phi_last = nullptr, bool push_phi = false, const void* pro_ec = nullptr,
                   const LevelDev* pro_c = nullptr, void* out_fine = nullptr, const LevelDev* out_f = nullptr,
                   bool out_push = false) {
  if (nsweep <= 0) return;
  if (!reverse && wave_on(p, D, push)) {
    const LevelBufs& B = c->buf[m];
    const Coefs k = coefs_of(c, m, dt);
    for (int it = 0; it < nsweep; ++it) {
      double* ph = (phi_last && it == nsweep - 1) ? phi_last : nullptr;
      if (red_done && it == 0) {  // the residual kernel did this sweep's red cells
        black_pass(c, D, dt, m, s, push, vec_on(c, p, dt, m), ph, push_phi);
        continue;
      }
      const bool zero = e_zero && it == 0 && !ph;
      const bool prof = c->profiling && m == 0;
      cudaEvent_t* ev = prof ? smooth_event(c, 2) : nullptr;
      if (prof) record_timing_event(c, ev[0], s);
      const bool ran = launch_wave(dt, D, B.e[dt], B.r[dt], k, zero, ph, push_phi, c->dev_err, s);
      if (prof) record_timing_event(c, ev[1], s);
      if (!ran) {  // (a problem's tiles do not fit on the device at once)
        if (prof) --c->n_ev_smooth;
        two_pass_sweep(c, D, dt, m, s, !(e_zero && it == 0), push, vec_on(c, p, dt, m), ph, push_phi);
      }
    }
    return;
  }
  if (flow_on(c, p, D, push)) {
    int first = reverse ? 1 : 0;
    int n = 2 * nsweep;
    if (red_done && !reverse) {
      first = 1;
      --n;
    }
    const LevelBufs& B = c->buf[m];
    const Coefs k = coefs_of(c, m, dt);
    for (int done = 0; done < n;) {
      const int np = std::min(FLOW_MAX_PHASES, n - done);
      const bool last = done + np == n;
      const bool prof = c->profiling && m == 0;
      cudaEvent_t* ev = prof ? smooth_event(c, np) : nullptr;
      if (prof) record_timing_event(c, ev[0], s);
      launch_flow(dt, D, B.e[dt], B.r[dt], k, (first + done) & 1, np, last && !reverse ? phi_last : nullptr,
                  push_phi, c->dev_err, s, p.flow_warps);
      if (prof) record_timing_event(c, ev[1], s);
      done += np;
    }
    return;
  }
  if (reverse) {
    for (int it = 0; it < nsweep; ++it) {
      smooth_colour(c, D, dt, m, 1, s, !(e_zero && it == 0), push, vec_on(c, p, dt, m));
      smooth_colour(c, D, dt, m, 0, s, true, push, vec_on(c, p, dt, m));
    }
    return;
  }
  for (int it = 0; it < nsweep; ++it) {
    if (pro_ec && it == 0)  // (the interpolation of the coarse correction, fused into the red pass)
      smooth_colour_pro(c, D, *pro_c, dt, m, pro_ec, s, push);
    else if (!(red_done && it == 0))
      smooth_colour(c, D, dt, m, 0, s, !(e_zero && it == 0), push, vec_on(c, p, dt, m));
    if (out_fine && it == nsweep - 1) {  // (the interpolation onto the finer level, fused)
      const LevelBufs& B = c->buf[m];
      if (!push) launch_fill(dt, D, B.e[dt], 0, 0, s);
      launch_smooth_prolong(dt, dir_view(c, D, m), *out_f, B.e[dt], B.r[dt], coefs_of(c, m, dt), 1, out_fine, s, push,
                            out_push);
    } else if (phi_last && it == nsweep - 1) {
      const LevelBufs& B = c->buf[m];
      if (!push) launch_fill(dt, D, B.e[dt], 0, 0, s);
      const bool prof = c->profiling && m == 0;
      cudaEvent_t* ev = prof ? smooth_event(c, 1) : nullptr;
      if (prof) record_timing_event(c, ev[0], s);
      launch_smooth_update(dt, dir_view(c, D, m), B.e[dt], B.r[dt], coefs_of(c, m, dt), 1, phi_last, push_phi, s,
                       true);
      if (prof) record_timing_event(c, ev[1], s);
    } else {
      smooth_colour(c, D, dt, m, 1, s, true, push, vec_on(c, p, dt, m));
    }
  }
}

// the graph-cache value of the sweep choices: fused_sweep, the flow launch width, serpentine,
// the interpolation, the wavefront sweep, the coarse end's form, the fused red passes
int sweep_key(const gmg_params& p) {
  return p.fused_sweep + 4 * p.flow_warps + 1024 * p.serpentine + 2048 * p.prolongation + 4096 * p.wave_sweep +
         8192 * p.tail_dense + 16384 * p.fuse_restriction_sweep + 32768 * p.fuse_prolongation +
         131072 * p.fork_bottoms;
}

// the symmetric V-cycle: post-smoothing black before red (asked for, or implied by the
// conjugate-gradient top level)
bool post_reversed(const gmg_params& p) { return p.post_reverse != 0 || p.krylov == 2; }

// Level m's tables with the V-cycle's work lists of the fused coarse ends: the grid
// launches leave out the problems whose tail covers level m.
LevelDev vc_view(const gmg_ctx* c, int m) {
  LevelDev D = c->dev[m];
  D.ghost_chunks = D.vc_ghost_chunks;
  D.n_ghost_chunks = D.n_vc_ghost_chunks;
  D.pair_chunks = D.vc_pair_chunks;
  D.n_pair_chunks = D.n_vc_pair_chunks;
  if (D.quad_chunks) {  // (null when the level's widths are not all multiples of 4)
    D.quad_chunks = D.vc_quad_chunks;
    D.n_quad_chunks = D.n_vc_quad_chunks;
  }
  D.coarse_chunks = D.vc_coarse_chunks;
  D.n_coarse_chunks = D.n_vc_coarse_chunks;
  D.bot_descs = D.vc_bot_descs;
  D.n_bot = D.n_vc_bot;
  if (m < (int)c->vc_flow_skip.size()) D.flow_skip = c->vc_flow_skip[m];
  return D;
}

// Shared memory (bytes) of the dense coarse end for the tails that start at level m in
// element type dt, or 0 if one of them has no dense form or needs more than TAIL_SMEM_MAX.
int64_t tail_dense_bytes(const gmg_ctx* c, int dt, int m) {
  const TailHost& T = c->tail;
  const int es = (int)dt_size(dt), cs = dt == DT_F64 ? 8 : 4;
  int64_t most = 0;
  for (int k = 0; k < T.count_at[m]; ++k) {
    const TailDesc& D = T.descs[T.first_at[m] + k];
    if (!D.dense) return 0;
    int64_t b = 0;
    for (int q = D.m0; q <= D.mb; ++q) b += tail_level_bytes(T.levels[D.lev0 + q - D.m0].dne, es, cs, q < D.mb);
    most = std::max(most, b);
  }
  return most <= TAIL_SMEM_MAX ? most : 0;
}

// the tails that start at level m: one block per problem runs its levels m..bottom
void launch_tails(gmg_ctx* c, int dt, int m, const gmg_params& p, cudaStream_t s) {
  const TailHost& T = c->tail;
  if (m >= (int)T.count_at.size() || T.count_at[m] == 0) return;
  TailArgs a;
  a.descs = c->tdescs + T.first_at[m];
  a.levels = c->tlevels;
  a.cells = c->tcells;
  a.ghosts = c->tghosts;
  a.xfer = c->txfer;
  a.dghosts = c->tdghosts;
  TailLevelBufs lv[TAIL_MAXLEV];
  for (int q = 0; q < nlev(c) && q < TAIL_MAXLEV; ++q) {
    const LevelBufs& B = c->buf[q];
    const Coefs k = coefs_of(c, q, dt);
    lv[q].e = B.e[dt];
    lv[q].r = B.r[dt];
    lv[q].wx = k.wx; lv[q].wy = k.wy; lv[q].wz = k.wz; lv[q].D = k.D; lv[q].invD = k.invD;
    a.wx64[q] = B.wx; a.wy64[q] = B.wy; a.wz64[q] = B.wz; a.D64[q] = B.D;
    a.work[q] = B.bot_work;
    a.nelem[q] = c->L[q].nelem;
  }
  a.nu1 = p.nu1;
  a.nu2 = p.nu2;
  a.maxit = p.bottom_max_iter;
  a.tol = p.bottom_tol;
  a.cg = p.bottom_solver;
  a.post_rev = post_reversed(p) ? 1 : 0;
  a.iters = c->bot_iters;
  a.active = c->active;
  const int64_t dense = p.tail_dense ? tail_dense_bytes(c, dt, m) : 0;
  launch_vtail(dt, T.count_at[m], a, lv, std::min(nlev(c), TAIL_MAXLEV), (int)dense, s);
}

// V-cycle on the correction equation of level m: e_m = V(r_m), e_m zeroed first.  Problems
// whose bottom is this level are solved here by BiCGStab; the others smooth, restrict,
// recurse, interpolate and smooth again.  With fused_coarse, each problem's levels from
// its first level of at most TAIL_MAX_CELLS cells down to its bottom run in one thread
// block (launched when the descent reaches that level) and the grid launches skip them.
// dependent launch on or off for the launches that follow: pdl = 2 (default) uses it
// outside CUDA graph capture only (measured: it shortens eager launch chains, e.g. the
// two-level solve 12.8 -> 11.5 ms, and costs ~0.3% inside replayed graphs)
void choose_pdl(const gmg_params& p, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  set_pdl(p.pdl == 1 || (p.pdl == 2 && cs == cudaStreamCaptureStatusNone));
}

// Whether the residual restriction into level m (>= 1) also performs that level's first red
// half-sweep of pre-smoothing: level m is smoothed by the grid launches (pair or 4-cell
// threads, red first) and pre-smooths at least once.
bool coarse_red(const gmg_ctx* c, const gmg_params& p, int dt, int m) {
  if (p.fuse_restriction_sweep == 0 || p.nu1 <= 0 || m < 1 || m + 1 >= nlev(c)) return false;
  const bool fused = tail_on(c, p, dt) && c->tail_ok;
  const LevelDev D = fused ? vc_view(c, m) : c->dev[m];
  return D.n_pair_chunks > 0;
}

// Whether level m's first post-smoothing (red) pass also performs the interpolation of level
// m + 1's correction before it (launch_smooth_pro): piecewise-constant interpolation, red-first
// post-smoothing by the grid's two-pass sweeps on level m, which pushes its ghosts (push),
// linear walls (a quadratic wall ghost is not the parent's image), and level m + 1's ghosts
// current when its post-smoothing ends: every problem on it is smoothed by grid launches that
// push them, or by a coarse end starting there (which fills them before it returns), none
// is solved by a bottom launch there.
bool prolong_fused(gmg_ctx* c, const gmg_params& p, int dt, int m, bool push, const LevelDev& D) {
  if (p.fuse_prolongation == 0 || p.prolongation != 0 || post_reversed(p) || p.nu2 <= 0 || any_quad(c) || !push)
    return false;
  // (FP64 on a large level: the colour pass is bound by the FP64 pipe, and the six additions
  // per update cost more than the interpolation pass they save -- measured on abec256)
  if (p.fuse_prolongation == 1 && dt == DT_F64 && c->L[m].ncells >= (1 << 22)) return false;
  if (m + 1 >= nlev(c)) return false;
  if (wave_on(p, D, push) || flow_on(c, p, D, push)) return false;
  const bool fused = tail_on(c, p, dt) && c->tail_ok;
  const LevelDev Dc = fused ? vc_view(c, m + 1) : c->dev[m + 1];
  if (Dc.n_bot > 0) return false;  // (a bottom solve leaves its ghosts as they were)
  if (Dc.n_pair_chunks > 0 && !(push_on(c, p, dt, m + 1) && Dc.push_ok)) return false;
  // (the problems not smoothed by the grid there are in coarse ends, which leave the ghosts
  // of their first level current)
  return Dc.n_pair_chunks > 0 || fused;
}

// Whether level m + 1's last post-smoothing pass also performs the interpolation of its
// correction onto level m (launch_smooth_prolong; used where the first red pass of level m
// does not): piecewise-constant interpolation, red-first post-smoothing with at least one
// sweep, level m + 1 smoothed for every problem by the grid's two-pass sweeps (no bottom
// solve, no coarse end, no wavefront or dataflow sweep there), and every box of level m + 1
// with one exact child box on level m.
bool smooth_prolong_ok(gmg_ctx* c, const gmg_params& p, int dt, int m) {
  if (p.fuse_prolongation == 0 || p.prolongation != 0 || post_reversed(p) || p.nu2 <= 0) return false;
  if (m + 2 >= nlev(c)) return false;
  // (FP64 onto a large level: the additions for the 8 children per coarse cell make the
  // coarse pass FP64-bound, slower than the interpolation pass -- measured on abec256)
  if (p.fuse_prolongation == 1 && dt == DT_F64 && c->L[m].ncells >= (1 << 22)) return false;
  const bool fused = tail_on(c, p, dt) && c->tail_ok;
  const LevelDev Dc = fused ? vc_view(c, m + 1) : c->dev[m + 1];
  if (Dc.n_bot > 0 || Dc.n_pair_chunks == 0 || Dc.n_pair_chunks != c->dev[m + 1].n_pair_chunks) return false;
  const bool cpush = push_on(c, p, dt, m + 1) && Dc.push_ok;
  if (wave_on(p, Dc, cpush) || flow_on(c, p, Dc, cpush)) return false;
  for (int b : c->L[m + 1].child)
    if (b < 0) return false;
  return true;
}

// phi_update (finest level only, see fuse_correction_on): the last post-smoothing pass also
// adds e to phi
void vcycle(gmg_ctx* c, int dt, int m, const gmg_params& p, cudaStream_t s, bool red_done = false,
            double* phi_update = nullptr, bool push_phi = false, void* out_fine = nullptr,
            const LevelDev* out_f = nullptr, bool out_push = false) {
  choose_pdl(p, s);
  c->serp = p.serpentine != 0;
  const bool fused = tail_on(c, p, dt) && c->tail_ok;
  const LevelDev D = fused ? vc_view(c, m) : c->dev[m];
  const LevelBufs& B = c->buf[m];
  // (red_done: the residual kernel wrote e on every valid cell -- r / D on red, 0 on black
  // -- and, with the push, its ghosts; no grid smoothing here: every problem on the level is
  // solved by a bottom launch or a coarse end, which write all its cells themselves)
  if (!red_done && D.n_pair_chunks > 0) cudaMemsetAsync(B.e[dt], 0, dt_size(dt) * (size_t)c->L[m].nelem, s);
  if (fused) launch_tails(c, dt, m, p, s);
  // Bottom solves of the problems whose bottom is this level: on the side stream when other
  // problems go on to coarser levels (the bottom touches only its problems' cells and the
  // level's bottom scratch), joined before this call returns -- the interpolation from this
  // level is the first step that reads their result.
  struct Join {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    ~Join() {
      if (ev) cudaStreamWaitEvent(s, ev, 0);
    }
  } join;
  if (D.n_bot) {
    BottomArgs a{p.bottom_max_iter, p.bottom_tol, B.bot_work, c->bot_iters, p.bottom_solver};
    const bool fork = p.fork_bottoms != 0 && c->side_stream && m < (int)c->ev_fork.size() && D.n_pair_chunks > 0 &&
                      m + 1 < nlev(c);
    if (fork) {
      cudaEventRecord(c->ev_fork[m], s);
      cudaStreamWaitEvent(c->side_stream, c->ev_fork[m], 0);
      launch_bottom(dt, D, B.r[dt], B.e[dt], coefs64(c, m), a, c->side_stream);
      cudaEventRecord(c->ev_join[m], c->side_stream);
      join.s = s;
      join.ev = c->ev_join[m];
    } else {
      launch_bottom(dt, D, B.r[dt], B.e[dt], coefs64(c, m), a, s);
    }
  }
  if (m + 1 >= nlev(c) || D.n_pair_chunks == 0) return;
  // ghost push (every value written also lands in the ghosts that copy it) on levels whose
  // ghosts share their source's colour, when the sweep is the two-pass one
  const bool push = push_on(c, p, dt, m) && D.push_ok;
  smooth_sweeps(c, D, dt, m, p.nu1, p, s, !red_done, push, red_done);
  if (p.nu1 > 0 && !push) launch_fill(dt, D, B.e[dt], -1, 0, s);  // (nu1 = 0: e and its ghosts are still zero)
  const LevelDev Dc = fused ? vc_view(c, m + 1) : c->dev[m + 1];
  // (pre-smoothing ends with a black half-sweep: black residuals vanish away from walls)
  const bool settled = dt == DT_F64 && p.nu1 > 0 && p.settled_zero != 0 && D.push_ok;
  // (fuse_restriction_sweep: the coarse level's first red half-sweep from e = 0 is done by
  // the restriction, which writes every valid coarse cell of e, so no zero fill either)
  const bool cred = coarse_red(c, p, dt, m + 1);
  const bool cpush = push_on(c, p, dt, m + 1) && Dc.push_ok;
  launch_resid_restrict(dt, dir_view(c, D, m), Dc, B.e[dt], B.r[dt], coefs_of(c, m, dt), c->buf[m + 1].r[dt], s,
                        settled, true, cred ? c->buf[m + 1].e[dt] : nullptr,
                        cred ? coefs_of(c, m + 1, dt).invD : nullptr, cpush);
  const bool pro = prolong_fused(c, p, dt, m, push, D);
  // (otherwise the coarse level's last post-smoothing pass may do the interpolation)
  const bool sprol = !pro && smooth_prolong_ok(c, p, dt, m);
  vcycle(c, dt, m + 1, p, s, cred, nullptr, false, sprol ? B.e[dt] : nullptr, &D, push);
  if (p.prolongation == 1) {  // trilinear: the coarse correction's ghosts, edges and corners too
    launch_fill(dt, c->dev[m + 1], c->buf[m + 1].e[dt], -1, 0, s);
    launch_fill_ec(dt, c->dev[m + 1], c->buf[m + 1].e[dt], s);
    launch_prolong_tri(dt, dir_view(c, D, m), Dc, c->buf[m + 1].e[dt], B.e[dt], s, push);
  } else if (pro) {
    // (the interpolation is done by the first post-smoothing red pass)
    smooth_sweeps(c, D, dt, m, p.nu2, p, s, false, push, false, false, phi_update, push_phi, c->buf[m + 1].e[dt], &Dc,
                  out_fine, out_f, out_push);
    return;
  } else if (!sprol) {
    launch_prolong_add(dt, dir_view(c, D, m), Dc, c->buf[m + 1].e[dt], B.e[dt], s, push);
  }
  smooth_sweeps(c, D, dt, m, p.nu2, p, s, false, push, false, post_reversed(p), phi_update, push_phi, nullptr, nullptr,
                out_fine, out_f, out_push);
}

// Whether the outer residual also performs the first red half-sweep of the next V-cycle
// (level 0 smooths with the pair/4-cell kernels and pre-smooths at least once), and
// whether level 0's V-cycle pushes ghosts (then that red half-sweep pushes too).
bool resid_red(const gmg_ctx* c, const gmg_params& p, int dt) {
  const LevelDev& D = c->dev[0];
  // (with the wavefront sweep on level 0, its first pre-smoothing sweep starts from e = 0
  // itself: r / D on red cells, then the black cells, in one launch)
  if (p.wave_sweep != 0 && push_on(c, p, dt, 0) && D.push_ok && wave_ok(D)) return false;
  return p.fuse_residual_sweep != 0 && p.nu1 > 0 && nlev(c) > 1 && D.n_pair_chunks > 0;
}
bool level0_push(const gmg_ctx* c, const gmg_params& p, int dt) {
  return push_on(c, p, dt, 0) && c->dev[0].push_ok;
}
// Whether the last post-smoothing pass on level 0 (black, red-first order) can also add the
// correction to phi: every level-0 box smooths there (no problem has level 0 as its
// bottom) with the two-pass sweep.
bool fuse_correction_on(const gmg_ctx* c, const gmg_params& p, int dt) {
  const LevelDev& D = c->dev[0];
  return p.fuse_correction != 0 && p.nu2 > 0 && !post_reversed(p) && nlev(c) > 1 && D.n_pair_chunks > 0 &&
         D.n_pair_chunks == D.n_pair_all_chunks;
}

// The colour whose residual vanishes away from walls after an outer iteration (-1: none):
// the level-0 colour smoothed last, when the correction was computed in FP64 (r - A e = 0
// there up to rounding, and rhs - A (phi + e) = r - A e), every level-0 box is smoothed and
// ghosts have their source's colour.  (In the batched form the residual of a problem that
// has stopped is not used again.)
int outer_settled(const gmg_ctx* c, const gmg_params& p, int dt) {
  const LevelDev& D = c->dev[0];
  if (!p.settled_zero || dt != DT_F64 || p.nu2 <= 0 || nlev(c) <= 1 || D.n_pair_chunks == 0 ||
      D.n_pair_chunks != D.n_pair_all_chunks || !D.push_ok)
    return -1;
  return post_reversed(p) ? 0 : 1;
}

// One outer iteration: e = V(r); phi += e; r = rhs - A phi with per-problem ||r||_inf into
// normbits[0, ns), copied to the pinned host mirror.
void outer_iteration(gmg_ctx* c, int dt, double* phi, const double* rhs, const gmg_params& p, cudaStream_t s) {
  const int ns = c->ns();
  c->serp = p.serpentine != 0;
  const bool rr = resid_red(c, p, dt);
  // phi's ghosts stay current by push (they were filled, or zero, before the first update)
  const bool push = p.ghost_push != 0 && c->dev[0].push_ok;
  const bool fc = fuse_correction_on(c, p, dt);
  // (sets the dependent-launch switch for the launches below too)
  vcycle(c, dt, 0, p, s, rr, fc ? phi : nullptr, push);
  if (!fc) launch_add_correction(dt, c->dev[0], phi, c->buf[0].e[dt], s, push);
  if (!push) launch_fill(DT_F64, c->dev[0], phi, -1, 0, s);
  cudaMemsetAsync(c->normbits, 0, 8 * (size_t)ns, s);
  cudaEvent_t* ev = c->profiling ? ev_pair(c->ev_resid, c->n_ev_resid++) : nullptr;
  if (ev) record_timing_event(c, ev[0], s);
  launch_residual(DT_F64, dt, dir_view(c, c->dev[0], 0), phi, rhs, coefs64(c, 0), c->buf[0].r[dt], c->normbits,
                  any_singular(c) ? c->scal : nullptr, s, rr ? c->buf[0].e[dt] : nullptr,
                  rr ? coefs_of(c, 0, dt).invD : nullptr, rr && level0_push(c, p, dt), outer_settled(c, p, dt), true);
  if (ev) record_timing_event(c, ev[1], s);
  cudaMemcpyAsync(c->h_bits, c->normbits, 8 * (size_t)ns, cudaMemcpyDeviceToHost, s);
}

// summed elapsed time (ms) of the first n event pairs of a list
double pair_ms(const std::vector<cudaEvent_t>& v, int n) {
  double t = 0.0;
  for (int k = 0; k < n; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, v[2 * k], v[2 * k + 1]) == cudaSuccess) t += ms;
    else cudaGetLastError();  // a missing timestamp is not an error of the solve
  }
  return t;
}

double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, 8);
  return d;
}

// Read and clear the device error flag (raised by a flow-sweep dependency wait that gave up);
// synchronises s.  GMG_ERR_DEVICE_TIMEOUT if it was raised.
gmg_status take_dev_err(gmg_ctx* c, cudaStream_t s) {
  int flag = 0;
  CK(c, cudaMemcpyAsync(&flag, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  if (!flag) return GMG_OK;
  CK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), s));
  SETERR(c, GMG_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up (flow sweep dependency)");
}

int dt_of_precision(int prec) { return prec == GMG_MIXED_FP32 ? DT_F32 : (prec == GMG_MIXED_BF16 ? DT_BF16 : DT_F64); }

gmg_status params_ok(gmg_ctx* c, const gmg_params& p) {
  if (p.nu1 < 0 || p.nu2 < 0 || p.nu1 + p.nu2 == 0 || p.max_iter < 0 || p.bottom_max_iter < 1 || !(p.bottom_tol > 0))
    SETERR(c, GMG_ERR_BAD_INPUT, "invalid parameters");
  if (p.precision < GMG_FP64 || p.precision > GMG_MIXED_BF16) SETERR(c, GMG_ERR_BAD_INPUT, "invalid precision");
  if (p.fused_coarse < 0 || p.fused_coarse > 2) SETERR(c, GMG_ERR_BAD_INPUT, "fused_coarse must be 0, 1 or 2");
  if (p.fused_sweep < 0 || p.fused_sweep > 2) SETERR(c, GMG_ERR_BAD_INPUT, "fused_sweep must be 0, 1 or 2");
  if (p.flow_warps < 0 || p.flow_warps > 64) SETERR(c, GMG_ERR_BAD_INPUT, "flow_warps must be in [0, 64]");
  if (p.flow_lag_kcells < 0) SETERR(c, GMG_ERR_BAD_INPUT, "flow_lag_kcells must be >= 0");
  if (p.serpentine != 0 && p.serpentine != 1) SETERR(c, GMG_ERR_BAD_INPUT, "serpentine must be 0 or 1");
  if (p.prolongation != 0 && p.prolongation != 1) SETERR(c, GMG_ERR_BAD_INPUT, "prolongation must be 0 or 1");
  if (p.wave_sweep != 0 && p.wave_sweep != 1) SETERR(c, GMG_ERR_BAD_INPUT, "wave_sweep must be 0 or 1");
  if (p.tail_dense != 0 && p.tail_dense != 1) SETERR(c, GMG_ERR_BAD_INPUT, "tail_dense must be 0 or 1");
  if (p.fuse_restriction_sweep != 0 && p.fuse_restriction_sweep != 1)
    SETERR(c, GMG_ERR_BAD_INPUT, "fuse_restriction_sweep must be 0 or 1");
  if (p.fuse_prolongation < 0 || p.fuse_prolongation > 2)
    SETERR(c, GMG_ERR_BAD_INPUT, "fuse_prolongation must be 0, 1 or 2");
  if (p.fork_bottoms != 0 && p.fork_bottoms != 1) SETERR(c, GMG_ERR_BAD_INPUT, "fork_bottoms must be 0 or 1");
  if (p.ghost_push < 0 || p.ghost_push > 2) SETERR(c, GMG_ERR_BAD_INPUT, "ghost_push must be 0, 1 or 2");
  if (p.vector_smooth < 0 || p.vector_smooth > 2) SETERR(c, GMG_ERR_BAD_INPUT, "vector_smooth must be 0, 1 or 2");
  if (p.pdl < 0 || p.pdl > 2) SETERR(c, GMG_ERR_BAD_INPUT, "pdl must be 0, 1 or 2");
  if (p.fuse_residual_sweep != 0 && p.fuse_residual_sweep != 1)
    SETERR(c, GMG_ERR_BAD_INPUT, "fuse_residual_sweep must be 0 or 1");
  if (p.krylov < 0 || p.krylov > 2) SETERR(c, GMG_ERR_BAD_INPUT, "krylov must be 0, 1 or 2");
  if (p.bottom_solver != 0 && p.bottom_solver != 1) SETERR(c, GMG_ERR_BAD_INPUT, "bottom_solver must be 0 or 1");
  if (p.post_reverse != 0 && p.post_reverse != 1) SETERR(c, GMG_ERR_BAD_INPUT, "post_reverse must be 0 or 1");
  if (p.fuse_correction != 0 && p.fuse_correction != 1)
    SETERR(c, GMG_ERR_BAD_INPUT, "fuse_correction must be 0 or 1");
  if (p.settled_zero != 0 && p.settled_zero != 1) SETERR(c, GMG_ERR_BAD_INPUT, "settled_zero must be 0 or 1");
  if (p.precision != GMG_FP64 && !c->mixed) SETERR(c, GMG_ERR_NO_WORKSPACE, "workspace was not sized for mixed precision");
  if (any_quad(c)) {
    if (p.krylov == 2 || p.bottom_solver == 1)
      SETERR(c, GMG_ERR_BAD_INPUT,
             "quadratic Dirichlet walls make the operator non-symmetric: conjugate gradients (krylov = 2, "
             "bottom_solver = 1) are not offered");
    if (p.prolongation == 1)
      SETERR(c, GMG_ERR_BAD_INPUT, "quadratic Dirichlet walls: trilinear interpolation is not offered");
  }
  return GMG_OK;
}

// Dispense orders of the flow sweeps for the lag the parameters ask for (flow_lag_kcells x
// 1024 cells; 0: FLOW_LAG_CELLS): rebuilt and uploaded (same sizes) when it changes.  Not
// during stream capture: called by the entry points before they launch anything.
gmg_status ensure_flow_lag(gmg_ctx* c, const gmg_params& p) {
  const int64_t lag = p.flow_lag_kcells > 0 ? 1024 * (int64_t)p.flow_lag_kcells : (int64_t)FLOW_LAG_CELLS;
  bool any = false;
  for (int m = 0; m < nlev(c); ++m) {
    LevelMeta& M = c->L[m];
    if (M.flow_slabs.empty() || M.flow_lag == lag) continue;
    build_flow_order(M, lag);
    const LevelDev& D = c->dev[m];
    for (int q = 0; q < FLOW_MAX_PHASES; ++q) {
      gmg_status st = upload(c, D.flow_order[q], M.flow_order[q]);
      if (st) return st;
    }
    any = true;
  }
  if (any) CK(c, cudaStreamSynchronize(c->stream));
  return GMG_OK;
}

// the level's cell work list restricted to one problem's boxes
LevelDev solve_view(const gmg_ctx* c, int m, int s) {
  LevelDev D = c->dev[m];
  const LevelMeta& M = c->L[m];
  D.cell_chunks += M.solve_chunk_range[s];
  D.n_cell_chunks = M.solve_chunk_range[s + 1] - M.solve_chunk_range[s];
  return D;
}

// Solve every problem of the context from phi = 0; infos[s] per problem (may be null).
gmg_status solve_impl(gmg_ctx* c, double* phi, const double* rhs, double tol_rel, double tol_abs, const gmg_params& p,
                      gmg_solve_info* infos) {
  const auto t0 = std::chrono::steady_clock::now();
  const int ns = c->ns();
  const int dt = dt_of_precision(p.precision);
  cudaStream_t s = c->stream;
  const LevelDev& D0 = c->dev[0];
  const int64_t ne0 = c->L[0].nelem;
  const bool sing = any_singular(c);
  if (infos) memset(infos, 0, sizeof(gmg_solve_info) * (size_t)ns);
  const int64_t l_pro = kernel_launch_count();
  // ||rhs||_inf per problem and, for singular problems, mean(rhs)
  CK(c, cudaMemsetAsync(c->normbits, 0, 8 * (size_t)(2 * ns), s));
  launch_norm_max(D0, rhs, c->normbits + ns, s);
  if (sing) launch_sum(D0, rhs, c->partials, c->scal, s);
  CK(c, cudaMemcpyAsync(c->h_bits + ns, c->normbits + ns, 8 * (size_t)ns, cudaMemcpyDeviceToHost, s));
  CK(c, cudaMemcpyAsync(c->h_scal, c->scal, 8 * (size_t)ns, cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  CK(c, cudaGetLastError());
  std::vector<double> rhsnorm(ns), target(ns);
  for (int q = 0; q < ns; ++q) {
    rhsnorm[q] = bits_to_double(c->h_bits[ns + q]);
    if (!std::isfinite(rhsnorm[q])) SETERR(c, GMG_ERR_BAD_INPUT, "rhs of problem " + std::to_string(q) + " is not finite");
    if (sing && singular(c, q)) {
      const double mean = c->h_scal[q];
      if (std::fabs(mean) > 1e-12 * rhsnorm[q] && !p.project_mean) {
        if (infos) infos[q].status = GMG_ERR_BAD_INPUT;
        SETERR(c, GMG_ERR_BAD_INPUT, "singular problem with a nonzero-mean rhs (set project_mean)");
      }
    } else {
      c->h_scal[q] = 0.0;  // no shift for nonsingular problems
    }
    target[q] = std::max(tol_rel * rhsnorm[q], tol_abs);
  }
  if (sing) CK(c, cudaMemcpyAsync(c->scal, c->h_scal, 8 * (size_t)ns, cudaMemcpyHostToDevice, s));
  // phi = 0; r = (rhs - mean) - A 0
  CK(c, cudaMemsetAsync(phi, 0, 8 * (size_t)ne0, s));
  CK(c, cudaMemsetAsync(c->normbits, 0, 8 * (size_t)ns, s));
  {
    const bool rr = resid_red(c, p, dt);
    launch_residual(DT_F64, dt, D0, phi, rhs, coefs64(c, 0), c->buf[0].r[dt], c->normbits, sing ? c->scal : nullptr,
                    s, rr ? c->buf[0].e[dt] : nullptr, rr ? coefs_of(c, 0, dt).invD : nullptr,
                    rr && level0_push(c, p, dt), -1, true);
  }
  CK(c, cudaMemcpyAsync(c->h_bits, c->normbits, 8 * (size_t)ns, cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  CK(c, cudaGetLastError());
  std::vector<std::vector<double>> hist(ns);
  std::vector<int> its(ns, 0), status(ns, GMG_OK);
  std::vector<char> live(ns, 0);
  int nlive = 0;
  for (int q = 0; q < ns; ++q) {
    const double rn = bits_to_double(c->h_bits[q]);
    hist[q].push_back(rn);
    live[q] = !(rn <= target[q]);
    if (live[q] && p.max_iter == 0) {
      status[q] = GMG_ERR_NOT_CONVERGED;
      live[q] = 0;
    }
    nlive += live[q];
    c->h_active[q] = live[q];
  }
  if (ns > 1) CK(c, cudaMemcpyAsync(c->active, c->h_active, 4 * (size_t)ns, cudaMemcpyHostToDevice, s));
  const int64_t prologue_launches = kernel_launch_count() - l_pro;

  cudaGraphExec_t gexec = nullptr;
  int64_t per_iter = 0;
  c->profiling = p.profile != 0;
  if (c->profiling) {  // events are created outside any capture
    ev_pair(c->ev_smooth, 2 * (p.nu1 + p.nu2) - 1);
    ev_pair(c->ev_resid, 0);
  }
  double sm_ms = 0.0, rs_ms = 0.0;
  int sm_n = 0, rs_n = 0, sm_passes = 0;
  if (p.use_graph && nlive) {
    auto key = std::make_tuple((void*)phi, (const void*)rhs, p.precision, p.nu1, p.nu2, p.bottom_max_iter,
                               p.bottom_tol, p.profile, p.fused_coarse, sweep_key(p), p.ghost_push,
                               p.vector_smooth, p.pdl, p.fuse_residual_sweep, p.bottom_solver,
                               p.post_reverse, p.fuse_correction, p.settled_zero);
    auto itg = c->graphs.find(key);
    if (itg != c->graphs.end()) {
      gexec = itg->second.exec;
      per_iter = itg->second.launches;
      c->n_ev_smooth = itg->second.n_ev_smooth;
      c->n_ev_resid = itg->second.n_ev_resid;
      c->ev_smooth_passes = itg->second.passes;
    } else {
      cudaGraph_t g;
      const int64_t l0 = kernel_launch_count();
      c->n_ev_smooth = c->n_ev_resid = 0;
      CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      outer_iteration(c, dt, phi, rhs, p, c->cap_stream);
      cudaError_t e1 = cudaStreamEndCapture(c->cap_stream, &g);
      if (e1 != cudaSuccess) SETERR(c, GMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
      cudaError_t e2 = cudaGraphInstantiate(&gexec, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) SETERR(c, GMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
      per_iter = kernel_launch_count() - l0;
      count_launches((int)-per_iter);  // captured, not launched
      c->graphs[key] = {gexec, per_iter, c->n_ev_smooth, c->n_ev_resid, c->ev_smooth_passes};
    }
  }
  int64_t launched = 0;
  while (nlive) {
    if (gexec) {
      CK(c, cudaGraphLaunch(gexec, s));
      launched += per_iter;
    } else {
      const int64_t l0 = kernel_launch_count();
      c->n_ev_smooth = c->n_ev_resid = 0;
      outer_iteration(c, dt, phi, rhs, p, s);
      launched += kernel_launch_count() - l0;
    }
    CK(c, cudaStreamSynchronize(s));
    CK(c, cudaGetLastError());
    if (c->profiling) {
      sm_ms += pair_ms(c->ev_smooth, c->n_ev_smooth);
      sm_n += c->n_ev_smooth;
      for (int k = 0; k < c->n_ev_smooth && k < (int)c->ev_smooth_passes.size(); ++k) sm_passes += c->ev_smooth_passes[k];
      rs_ms += pair_ms(c->ev_resid, c->n_ev_resid);
      rs_n += c->n_ev_resid;
    }
    bool changed = false;
    for (int q = 0; q < ns; ++q) {
      if (!live[q]) continue;
      const double rn = bits_to_double(c->h_bits[q]);
      ++its[q];
      hist[q].push_back(rn);
      if (!std::isfinite(rn)) status[q] = GMG_ERR_DIVERGED;
      else if (rn <= target[q]) status[q] = GMG_OK;
      else if (its[q] >= p.max_iter) status[q] = GMG_ERR_NOT_CONVERGED;
      else continue;
      live[q] = 0;
      c->h_active[q] = 0;
      --nlive;
      changed = true;
    }
    if (changed && nlive && ns > 1)
      CK(c, cudaMemcpyAsync(c->active, c->h_active, 4 * (size_t)ns, cudaMemcpyHostToDevice, s));
  }
  c->profiling = false;
  const int64_t l_epi = kernel_launch_count();
  // every problem active again for later calls
  if (ns > 1) {
    for (int q = 0; q < ns; ++q) c->h_active[q] = 1;
    CK(c, cudaMemcpyAsync(c->active, c->h_active, 4 * (size_t)ns, cudaMemcpyHostToDevice, s));
  }
  if (sing) {  // singular problems: phi -= mean(phi); the others keep a zero shift
    launch_sum(D0, phi, c->partials, c->scal + ns, s);
    for (int q = 0; q < ns; ++q)
      if (!singular(c, q)) CK(c, cudaMemsetAsync(c->scal + ns + q, 0, 8, s));
    launch_add_scalar(D0, phi, c->scal + ns, -1.0, s);
    CK(c, cudaGetLastError());
  }
  CK(c, cudaMemcpyAsync(c->h_iters, c->bot_iters, 4 * (size_t)(ns + 1), cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  gmg_status worst = GMG_OK;
  for (int q = 0; q < ns; ++q)
    if (status[q] != GMG_OK && (worst == GMG_OK || status[q] == GMG_ERR_DIVERGED)) worst = (gmg_status)status[q];
  if (c->h_iters[ns]) {  // a dependency wait of a flow sweep gave up: results are not trustworthy
    CK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), s));
    for (int q = 0; q < ns; ++q) status[q] = GMG_ERR_DEVICE_TIMEOUT;
    worst = GMG_ERR_DEVICE_TIMEOUT;
  }
  if (infos) {
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const int64_t tot = launched + prologue_launches + (kernel_launch_count() - l_epi);
    for (int q = 0; q < ns; ++q) {
      gmg_solve_info& I = infos[q];
      I.iterations = its[q];
      I.status = status[q];
      I.rhs_norm = rhsnorm[q];
      I.initial_resid = hist[q][0];
      I.final_resid = hist[q].back();
      I.hist_len = (int)std::min<size_t>(hist[q].size(), 256);
      for (int i = 0; i < I.hist_len; ++i) I.resid_hist[i] = hist[q][i];
      I.bottom_iters = c->h_iters[q];
      I.solve_ms = ms;
      I.kernel_launches = tot;
      I.smooth0_ms = sm_ms;
      I.smooth0_launches = sm_n;
      I.smooth0_passes = sm_passes;
      I.resid0_ms = rs_ms;
      I.resid0_launches = rs_n;
    }
  }
  if (worst == GMG_ERR_NOT_CONVERGED) c->err = "not converged within max_iter";
  if (worst == GMG_ERR_DIVERGED) c->err = "residual is not finite";
  if (worst == GMG_ERR_DEVICE_TIMEOUT) c->err = "a bounded device wait gave up (flow sweep dependency)";
  return worst;
}

// ------------------------------------------------------------ composite form

// per-level views of the AMR levels: level 0 is MG level 0, level l >= 1 is amrl[l - 1]
const LevelDev& adev(const gmg_ctx* c, int l) { return l == 0 ? c->dev[0] : c->amrl[l - 1].D; }
int64_t anelem(const gmg_ctx* c, int l) { return l == 0 ? c->L[0].nelem : c->amrl[l - 1].M.nelem; }
Coefs acoefs(const gmg_ctx* c, int l) {
  if (l == 0) return coefs64(c, 0);
  const LevelBufs& B = c->amrl[l - 1].B;
  Coefs k;
  k.wx = B.wx; k.wy = B.wy; k.wz = B.wz; k.D = B.D; k.invD = B.invD;
  return k;
}

// ghosts of level l >= 1: copies between its boxes, then its coarse/fine ghosts (interpolated
// from level l - 1's field cx, or zero coarse data when cx is null)
void level_fill(gmg_ctx* c, int l, double* f, const double* cx, int mode, cudaStream_t s) {
  launch_fill(DT_F64, adev(c, l), f, -1, 0, s);
  launch_cf_fill(c->amrl[l - 1].A, f, cx, mode, s);
}

// composite residual r_l = rhs_l - (A x)_l on every level (covered cells 0), ||r_l||_inf into
// nb[l] (nb may be null).  x's ghosts are overwritten.
void comp_residual_n(gmg_ctx* c, double* const* x, const double* const* rhs, double* const* r, unsigned long long* nb,
                     cudaStream_t s) {
  const int L = namr(c);
  for (int l = L - 1; l >= 1; --l) level_fill(c, l, x[l], x[l - 1], CF_INTERP, s);
  launch_fill(DT_F64, c->dev[0], x[0], -1, 0, s);
  if (nb) cudaMemsetAsync(nb, 0, 8 * (size_t)L, s);
  for (int l = 0; l < L; ++l) {
    const bool finest = l + 1 == L;
    launch_residual(DT_F64, DT_F64, adev(c, l), x[l], rhs[l], acoefs(c, l), r[l], finest && nb ? nb + l : nullptr,
                    nullptr, s);
    if (!finest) {
      launch_reflux(c->amrl[l].A, acoefs(c, l), acoefs(c, l + 1), x[l], x[l + 1], r[l], r[l], 1, s);
      launch_zero_covered(c->amrl[l].A, r[l], s);
      if (nb) launch_norm_max(adev(c, l), r[l], nb + l, s);
    }
  }
}
// One composite multigrid correction from the composite residuals r (per level): e_l in
// level l's e buffer.  Down, for l = L-1 .. 1: pre-smoothing of level l's correction
// equation (right-hand side rr_l; coarse/fine ghosts with a zero coarse correction); the
// right-hand side of level l-1: its composite residual with, on cells covered by level l,
// the average of level l's correction residual, and next to level l minus the correction's
// reflux.  Level 0: one V-cycle of its hierarchy.  Up, for l = 1 .. L-1: interpolation of
// e_(l-1), post-smoothing with coarse/fine ghosts from e_(l-1).  Then covered corrections
// := averages of their children, finest pair first.
void comp_correction_n(gmg_ctx* c, const gmg_params& p, const double* const* r, cudaStream_t s) {
  const int L = namr(c);
  double* e[GMG_MAX_AMR_LEVELS];
  const double* rr[GMG_MAX_AMR_LEVELS];
  for (int l = 0; l < L; ++l) e[l] = (double*)(l == 0 ? c->buf[0].e[DT_F64] : c->amrl[l - 1].B.e[DT_F64]);
  // right-hand sides: level 0 in its V-cycle buffer, middle levels in their own r buffers,
  // the finest level's is its composite residual
  double* rbuf[GMG_MAX_AMR_LEVELS];
  for (int l = 0; l < L; ++l) rbuf[l] = (double*)(l == 0 ? c->buf[0].r[DT_F64] : c->amrl[l - 1].B.r[DT_F64]);
  rr[L - 1] = r[L - 1];
  choose_pdl(p, s);
  // level l's box ghosts kept current by push (e_l starts at zero; every later write pushes);
  // the coarse/fine ghosts depend on the cells inward and are refilled every colour
  auto push_of = [&](int l) { return p.ghost_push != 0 && adev(c, l).push_ok; };
  auto fill = [&](int l, const double* cx) {
    if (push_of(l)) launch_cf_fill(c->amrl[l - 1].A, e[l], cx, CF_INTERP, s);
    else level_fill(c, l, e[l], cx, CF_INTERP, s);
  };
  for (int l = 1; l < L; ++l) cudaMemsetAsync(e[l], 0, 8 * (size_t)anelem(c, l), s);
  for (int l = L - 1; l >= 1; --l) {
    for (int it = 0; it < p.nu1; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        fill(l, nullptr);  // coarse correction 0
        launch_smooth(DT_F64, adev(c, l), e[l], rr[l], acoefs(c, l), colour, s, push_of(l));
      }
    fill(l, nullptr);
    cudaMemcpyAsync(rbuf[l - 1], r[l - 1], 8 * (size_t)anelem(c, l - 1), cudaMemcpyDeviceToDevice, s);
    // covered cells: average of level l's correction residual rr_l - A_l e_l
    launch_resid_restrict(DT_F64, adev(c, l), adev(c, l - 1), e[l], rr[l], acoefs(c, l), rbuf[l - 1], s);
    // cells next to level l: minus the correction's reflux
    launch_reflux(c->amrl[l - 1].A, acoefs(c, l - 1), acoefs(c, l), rbuf[l - 1], e[l], rbuf[l - 1], rbuf[l - 1], 0,
                  s);
    rr[l - 1] = rbuf[l - 1];
  }
  vcycle(c, DT_F64, 0, p, s);
  for (int l = 1; l < L; ++l) {
    launch_prolong_add(DT_F64, adev(c, l), adev(c, l - 1), e[l - 1], e[l], s, push_of(l));
    for (int it = 0; it < p.nu2; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        fill(l, e[l - 1]);
        launch_smooth(DT_F64, adev(c, l), e[l], rr[l], acoefs(c, l), colour, s, push_of(l));
      }
  }
  for (int l = L - 1; l >= 1; --l) launch_restrict(DT_F64, adev(c, l), adev(c, l - 1), e[l], e[l - 1], s);
}
// volume of a cell of each AMR level and the number of its composite cells (not covered)
struct CompLevels {
  double v[GMG_MAX_AMR_LEVELS], n[GMG_MAX_AMR_LEVELS];
};

CompLevels comp_levels(const gmg_ctx* c) {
  CompLevels z;
  const int L = namr(c);
  const SolveGeom& G = c->geoms[0];
  double v = G.h[0] * G.h[1] * G.h[2];
  for (int l = 0; l < L; ++l, v /= 8.0) {
    z.v[l] = v;
    const double ncell = (double)(l == 0 ? c->L[0].ncells : c->amrl[l - 1].M.ncells);
    const double ncov = l + 1 < L ? (double)c->amrl[l].H.covered_list.size() : 0.0;
    z.n[l] = ncell - ncov;
  }
  return z;
}

// per-level plain sums of the valid cells of x (covered entries must be zero)
gmg_status comp_sums_n(gmg_ctx* c, double* const* x, double* sums) {
  cudaStream_t s = c->stream;
  const int L = namr(c);
  for (int l = 0; l < L; ++l) launch_sum(adev(c, l), x[l], c->partials, c->scal + l, s);  // in stream order
  CK(c, cudaMemcpyAsync(c->h_scal, c->scal, 8 * (size_t)L, cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  for (int l = 0; l < L; ++l)  // launch_sum returns the mean over every cell of the level
    sums[l] = c->h_scal[l] * (double)(l == 0 ? c->L[0].ncells : c->amrl[l - 1].M.ncells);
  return GMG_OK;
}

// x_l += k[l] on every level (covered entries cleared afterwards)
gmg_status comp_add_const_n(gmg_ctx* c, double* const* x, const double* k) {
  cudaStream_t s = c->stream;
  const int L = namr(c);
  for (int l = 0; l < L; ++l) c->h_scal[4 + l] = k[l];
  CK(c, cudaMemcpyAsync(c->scal + 4, c->h_scal + 4, 8 * (size_t)L, cudaMemcpyHostToDevice, s));
  for (int l = 0; l < L; ++l) {
    launch_add_scalar(adev(c, l), x[l], c->scal + 4 + l, 1.0, s);
    if (l + 1 < L) launch_zero_covered(c->amrl[l].A, x[l], s);
  }
  CK(c, cudaGetLastError());
  return GMG_OK;
}

// max over n per-level norms in normbits[0, n) (NaN if any is NaN)
gmg_status read_norms_n(gmg_ctx* c, int n, double* rn) {
  CK(c, cudaMemcpyAsync(c->h_bits, c->normbits, 8 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaGetLastError());
  *rn = 0.0;
  for (int l = 0; l < n; ++l) {
    const double v = bits_to_double(c->h_bits[l]);
    if (std::isnan(v)) {
      *rn = NAN;
      break;
    }
    *rn = std::max(*rn, v);
  }
  return GMG_OK;
}

// volume-weighted mean of x over the composite cells (covered entries must be zero)
gmg_status comp_mean_n(gmg_ctx* c, double* const* x, double* mean) {
  cudaStream_t s = c->stream;
  const int L = namr(c);
  for (int l = 0; l < L; ++l) launch_sum(adev(c, l), x[l], c->partials, c->scal + l, s);
  CK(c, cudaMemcpyAsync(c->h_scal, c->scal, 8 * (size_t)L, cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  const SolveGeom& G = c->geoms[0];
  double v = G.h[0] * G.h[1] * G.h[2], num = 0.0, vol = 0.0;
  for (int l = 0; l < L; ++l, v /= 8.0) {
    const double ncell = (double)(l == 0 ? c->L[0].ncells : c->amrl[l - 1].M.ncells);
    const double ncov = l + 1 < L ? (double)c->amrl[l].H.covered_list.size() : 0.0;
    num += v * c->h_scal[l] * ncell;  // launch_sum gives the mean over every cell of the level
    vol += v * (ncell - ncov);
  }
  *mean = num / vol;
  return GMG_OK;
}

// x_l -= k on every level, covered entries cleared afterwards
gmg_status comp_shift_n(gmg_ctx* c, double* const* x, double k) {
  cudaStream_t s = c->stream;
  const int L = namr(c);
  c->h_scal[0] = -k;
  CK(c, cudaMemcpyAsync(c->scal, c->h_scal, 8, cudaMemcpyHostToDevice, s));
  for (int l = 0; l < L; ++l) {
    launch_add_scalar(adev(c, l), x[l], c->scal, 1.0, s);
    if (l + 1 < L) launch_zero_covered(c->amrl[l].A, x[l], s);
  }
  CK(c, cudaGetLastError());
  return GMG_OK;
}

// Composite multigrid solve over every AMR level (the oracle's multi-level iteration; with
// two levels its two-level one): residual, composite correction, update, average-down.
// (the iterate lives in the context's own buffers, so one captured iteration serves every
// call with the same parameters; it is copied to the caller's arrays at the end)
gmg_status solve_amr_n(gmg_ctx* c, double* const* phi_user, const double* const* rhs_user, double tol_rel,
                       double tol_abs, const gmg_params& p, gmg_solve_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = c->stream;
  const int L = namr(c);
  const int64_t l0 = kernel_launch_count();
  if (info) memset(info, 0, sizeof(*info));
  double *rhs[GMG_MAX_AMR_LEVELS], *res[GMG_MAX_AMR_LEVELS], *phi[GMG_MAX_AMR_LEVELS];
  for (int l = 0; l < L; ++l) {
    rhs[l] = l == 0 ? c->crhs : c->amrl[l - 1].rhs;
    res[l] = l == 0 ? c->cres : c->amrl[l - 1].res;
    phi[l] = l == 0 ? c->cphi : c->amrl[l - 1].phi;
    CK(c, cudaMemcpyAsync(rhs[l], rhs_user[l], 8 * (size_t)anelem(c, l), cudaMemcpyDeviceToDevice, s));
  }
  CK(c, cudaMemsetAsync(c->normbits, 0, 8 * (size_t)L, s));
  for (int l = 0; l < L; ++l) {
    if (l + 1 < L) launch_zero_covered(c->amrl[l].A, rhs[l], s);
    launch_norm_max(adev(c, l), rhs[l], c->normbits + l, s);
  }
  double rhsnorm;
  gmg_status st = read_norms_n(c, L, &rhsnorm);
  if (st) return st;
  if (!std::isfinite(rhsnorm)) SETERR(c, GMG_ERR_BAD_INPUT, "rhs is not finite");
  const bool sing = singular(c, 0);
  if (sing) {  // project onto zero volume-weighted mean (the range of the composite operator)
    double mean;
    if ((st = comp_mean_n(c, rhs, &mean))) return st;
    if (std::fabs(mean) > 1e-12 * rhsnorm && !p.project_mean)
      SETERR(c, GMG_ERR_BAD_INPUT, "singular problem with a nonzero-mean rhs (set project_mean)");
    if ((st = comp_shift_n(c, rhs, mean))) return st;
  }
  const double target = std::max(tol_rel * rhsnorm, tol_abs);
  for (int l = 0; l < L; ++l) CK(c, cudaMemsetAsync(phi[l], 0, 8 * (size_t)anelem(c, l), s));
  comp_residual_n(c, phi, rhs, res, c->normbits, s);
  double rn;
  if ((st = read_norms_n(c, L, &rn))) return st;
  std::vector<double> hist{rn};
  int it = 0;
  gmg_status result = GMG_OK;
  // one iteration: correction, update, covered := average, composite residual and its norms
  auto iteration = [&](cudaStream_t st_) {
    comp_correction_n(c, p, res, st_);
    for (int l = 0; l < L; ++l)
      launch_add_correction(DT_F64, adev(c, l), phi[l], l == 0 ? c->buf[0].e[DT_F64] : c->amrl[l - 1].B.e[DT_F64],
                            st_);
    for (int l = L - 1; l >= 1; --l) launch_restrict(DT_F64, adev(c, l), adev(c, l - 1), phi[l], phi[l - 1], st_);
    comp_residual_n(c, phi, rhs, res, c->normbits, st_);
  };
  cudaGraphExec_t gexec = nullptr;
  int64_t per_iter = 0;
  if (p.use_graph && !(rn <= target) && p.max_iter > 0) {
    // keyed by the context's own buffers (no caller pointer is captured) and the parameters
    // the iteration reads
    auto key = std::make_tuple((void*)phi[0], (const void*)rhs[0], L, p.nu1, p.nu2, p.bottom_max_iter, p.bottom_tol,
                               0, p.fused_coarse, sweep_key(p), p.ghost_push, p.vector_smooth, p.pdl, 0, p.bottom_solver,
                               p.post_reverse, 0, p.settled_zero);
    auto itg = c->graphs.find(key);
    if (itg != c->graphs.end()) {
      gexec = itg->second.exec;
      per_iter = itg->second.launches;
    } else {
      cudaGraph_t g;
      const int64_t lc0 = kernel_launch_count();
      CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      iteration(c->cap_stream);
      cudaError_t e1 = cudaStreamEndCapture(c->cap_stream, &g);
      if (e1 != cudaSuccess) SETERR(c, GMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
      cudaError_t e2 = cudaGraphInstantiate(&gexec, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) SETERR(c, GMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
      per_iter = kernel_launch_count() - lc0;
      count_launches((int)-per_iter);  // captured, not launched
      c->graphs[key] = {gexec, per_iter, 0, 0};
    }
  }
  while (!(rn <= target) && it < p.max_iter) {
    if (gexec) {
      CK(c, cudaGraphLaunch(gexec, s));
      count_launches((int)per_iter);
    } else {
      iteration(s);
    }
    if ((st = read_norms_n(c, L, &rn))) return st;
    ++it;
    hist.push_back(rn);
    if (!std::isfinite(rn)) {
      result = GMG_ERR_DIVERGED;
      break;
    }
  }
  if (result == GMG_OK && !(rn <= target)) result = GMG_ERR_NOT_CONVERGED;
  if (sing) {  // zero volume-weighted mean over the composite unknowns
    for (int l = 0; l + 1 < L; ++l) launch_zero_covered(c->amrl[l].A, phi[l], s);
    double mean;
    if ((st = comp_mean_n(c, phi, &mean))) return st;
    if ((st = comp_shift_n(c, phi, mean))) return st;
  }
  for (int l = L - 1; l >= 1; --l) launch_restrict(DT_F64, adev(c, l), adev(c, l - 1), phi[l], phi[l - 1], s);
  for (int l = 0; l < L; ++l)
    CK(c, cudaMemcpyAsync(phi_user[l], phi[l], 8 * (size_t)anelem(c, l), cudaMemcpyDeviceToDevice, s));
  CK(c, cudaStreamSynchronize(s));
  CK(c, cudaGetLastError());
  if (info) {
    info->iterations = it;
    info->status = result;
    info->rhs_norm = rhsnorm;
    info->initial_resid = hist[0];
    info->final_resid = rn;
    info->hist_len = (int)std::min<size_t>(hist.size(), 256);
    for (int i = 0; i < info->hist_len; ++i) info->resid_hist[i] = hist[i];
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->kernel_launches = kernel_launch_count() - l0;
  }
  if (result == GMG_ERR_NOT_CONVERGED) c->err = "not converged within max_iter";
  if (gmg_status e = take_dev_err(c, s)) {
    if (info) info->status = e;
    return e;
  }
  return result;
}

// out = A x (composite) over every level; x's ghosts are overwritten; covered entries 0
void comp_apply_n(gmg_ctx* c, double* const* x, double* const* out, cudaStream_t s) {
  const int L = namr(c);
  const double* zero[GMG_MAX_AMR_LEVELS];
  for (int l = 0; l < L; ++l) {
    double* z = l == 0 ? c->czero : c->amrl[l - 1].zero;
    cudaMemsetAsync(z, 0, 8 * (size_t)anelem(c, l), s);
    zero[l] = z;
  }
  comp_residual_n(c, x, zero, out, nullptr, s);
  for (int l = 0; l < L; ++l) launch_scale_valid(adev(c, l), out[l], -1.0, s);
}
// out = A^T y (composite) over every level: the level stencils (symmetric; coarse/fine
// ghosts zero, covered entries of y zero) plus, for each pair of consecutive levels, the
// transposed interpolation and reflux couplings.  y's ghosts are overwritten; its covered
// entries are cleared.
void comp_apply_transpose_n(gmg_ctx* c, double* const* y, double* const* out, cudaStream_t s) {
  const int L = namr(c);
  double* zero[GMG_MAX_AMR_LEVELS];
  for (int l = 0; l < L; ++l) {
    zero[l] = l == 0 ? c->czero : c->amrl[l - 1].zero;
    cudaMemsetAsync(zero[l], 0, 8 * (size_t)anelem(c, l), s);
    if (l + 1 < L) launch_zero_covered(c->amrl[l].A, y[l], s);
  }
  for (int l = 1; l < L; ++l) level_fill(c, l, y[l], nullptr, CF_ZERO, s);
  launch_fill(DT_F64, c->dev[0], y[0], -1, 0, s);
  for (int l = L - 1; l >= 0; --l) {
    launch_residual(DT_F64, DT_F64, adev(c, l), y[l], zero[l], acoefs(c, l), out[l], nullptr, nullptr, s);
    launch_scale_valid(adev(c, l), out[l], -1.0, s);
  }
  for (int l = 0; l + 1 < L; ++l)
    launch_composite_transpose_couplings(c->amrl[l].A, acoefs(c, l), acoefs(c, l + 1), y[l], y[l + 1], out[l],
                                         out[l + 1], s);
  for (int l = 0; l + 1 < L; ++l) launch_zero_covered(c->amrl[l].A, out[l], s);
}

// sum over the levels of <x_l, y_l> (covered entries zero in one of the two): one launch of
// partial sums over every level, one of per-level sums, one read-back
gmg_status comp_dot_n(gmg_ctx* c, double* const* x, double* const* y, double* out) {
  cudaStream_t s = c->stream;
  const int L = namr(c);
  const LevelDev* Ls[ML_MAX_SEG];
  for (int l = 0; l < L; ++l) Ls[l] = &adev(c, l);
  launch_dot_ml(L, Ls, (const double* const*)x, (const double* const*)y, c->partials, c->scal, s);
  CK(c, cudaMemcpyAsync(c->h_scal, c->scal, 8 * (size_t)L, cudaMemcpyDeviceToHost, s));
  CK(c, cudaStreamSynchronize(s));
  CK(c, cudaGetLastError());
  double sum = 0.0;
  for (int l = 0; l < L; ++l) sum += c->h_scal[l];
  *out = sum;
  return GMG_OK;
}

// sums over the levels of <x1_l, y1_l> (and, with x2, of <x2_l, y2_l>) and the max over the
// levels of ||z_l||_inf, with one read-back
gmg_status comp_dots_norm_n(gmg_ctx* c, double* const* x1, double* const* y1, double* const* x2,
                            double* const* y2, double* const* z, double* d1, double* d2, double* zn) {
  cudaStream_t s = c->stream;
  const int L = namr(c);
  const int nseg = x2 ? 2 * L : L;
  const LevelDev* Ls[ML_MAX_SEG];
  const double *xs[ML_MAX_SEG], *ys[ML_MAX_SEG];
  for (int l = 0; l < L; ++l) {
    Ls[l] = &adev(c, l);
    xs[l] = x1[l];
    ys[l] = y1[l];
    if (x2) {
      Ls[L + l] = &adev(c, l);
      xs[L + l] = x2[l];
      ys[L + l] = y2[l];
    }
  }
  launch_dot_ml(nseg, Ls, xs, ys, c->partials, c->scal, s);
  CK(c, cudaMemsetAsync(c->normbits, 0, 8 * (size_t)L, s));
  launch_norm_max_ml(L, Ls, (const double* const*)z, c->normbits, s);
  CK(c, cudaMemcpyAsync(c->h_scal, c->scal, 8 * (size_t)nseg, cudaMemcpyDeviceToHost, s));
  gmg_status st = read_norms_n(c, L, zn);  // (synchronises the stream)
  if (st) return st;
  double a = 0.0, b = 0.0;
  for (int l = 0; l < L; ++l) {
    a += c->h_scal[l];
    if (x2) b += c->h_scal[L + l];
  }
  *d1 = a;
  if (d2) *d2 = b;
  return GMG_OK;
}

// max over the levels of ||x_l||_inf
gmg_status comp_norm_n(gmg_ctx* c, double* const* x, double* out) {
  const int L = namr(c);
  CK(c, cudaMemsetAsync(c->normbits, 0, 8 * (size_t)L, c->stream));
  const LevelDev* Ls[ML_MAX_SEG];
  for (int l = 0; l < L; ++l) Ls[l] = &adev(c, l);
  launch_norm_max_ml(L, Ls, (const double* const*)x, c->normbits, c->stream);
  return read_norms_n(c, L, out);
}

// The transpose, the adjoint solve and the beta gradient treat the composite operator as a
// matrix over the unknowns.  That holds while no coarse/fine ghost of a level reads, through
// its two inward cells, a cell covered by the next finer level (whose value is then an
// average of finer data): every level must lie at least two cells inside the coarse/fine
// boundary of the level it refines.
gmg_status adjoint_layout_ok(gmg_ctx* c) {
  const int L = namr(c);
  for (int l = 0; l + 2 < L; ++l) {
    const std::vector<unsigned char>& cov = c->amrl[l + 1].H.covered;  // level l+1 under level l+2
    for (const CfGhost& G : c->amrl[l].H.cf)                          // level l+1's coarse/fine ghosts
      if (cov[G.f1] || cov[G.f2])
        SETERR(c, GMG_ERR_BAD_INPUT,
               "transpose/adjoint/gradient: a level lies closer than two cells to the coarse/fine boundary of the "
               "level it refines");
  }
  return GMG_OK;
}

// Adjoint solve A^T lambda = g of the composite operator over every AMR level: BiCGStab
// preconditioned on the right by the composite multigrid correction of A.  Singular
// problems: g is projected onto the range of A^T (g - V sum(g) / sum(V), V = cell volumes)
// and lambda onto zero plain sum.
gmg_status solve_adjoint_amr_n(gmg_ctx* c, double* const* lam, const double* const* g_user, double tol_rel,
                               const gmg_params& p, gmg_solve_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = c->stream;
  const int L = namr(c);
  const int64_t l0 = kernel_launch_count();
  if (info) memset(info, 0, sizeof(*info));
  // vectors per level: 0 r, 1 rhat, 2 p, 3 v, 4 s, 5 t, 6 phat, 7 shat, 8 g
  double* k[9][GMG_MAX_AMR_LEVELS];
  double *tmp[GMG_MAX_AMR_LEVELS], *e[GMG_MAX_AMR_LEVELS];
  int64_t ne[GMG_MAX_AMR_LEVELS];
  for (int l = 0; l < L; ++l) {
    for (int q = 0; q < 9; ++q) k[q][l] = l == 0 ? c->kc[q] : c->amrl[l - 1].kf[q];
    tmp[l] = l == 0 ? c->ctmp : c->amrl[l - 1].tmp;
    e[l] = (double*)(l == 0 ? c->buf[0].e[DT_F64] : c->amrl[l - 1].B.e[DT_F64]);
    ne[l] = anelem(c, l);
  }
  // out = a x + b y on every level (one launch)
  auto axpby = [&](double a, double* const* x, double b, double* const* y, double* const* out) {
    double av[ML_MAX_SEG], bv[ML_MAX_SEG];
    for (int l = 0; l < L; ++l) {
      av[l] = a;
      bv[l] = b;
    }
    launch_axpby_ml(L, ne, av, (const double* const*)x, bv, (const double* const*)y, out, s);
  };
  for (int l = 0; l < L; ++l) {
    CK(c, cudaMemcpyAsync(k[8][l], g_user[l], 8 * (size_t)ne[l], cudaMemcpyDeviceToDevice, s));
    if (l + 1 < L) launch_zero_covered(c->amrl[l].A, k[8][l], s);
  }
  const CompLevels z = comp_levels(c);
  double vol = 0.0;
  for (int l = 0; l < L; ++l) vol += z.v[l] * z.n[l];
  gmg_status st;
  const bool sing = singular(c, 0);
  double sums[GMG_MAX_AMR_LEVELS], shift[GMG_MAX_AMR_LEVELS];
  if (sing) {
    if ((st = comp_sums_n(c, k[8], sums))) return st;
    double tot = 0.0;
    for (int l = 0; l < L; ++l) tot += sums[l];
    for (int l = 0; l < L; ++l) shift[l] = -(tot / vol) * z.v[l];
    if ((st = comp_add_const_n(c, k[8], shift))) return st;
  }
  double gnorm;
  if ((st = comp_norm_n(c, k[8], &gnorm))) return st;
  for (int l = 0; l < L; ++l) {
    CK(c, cudaMemsetAsync(lam[l], 0, 8 * (size_t)ne[l], s));
    for (int q = 0; q < 8; ++q) CK(c, cudaMemsetAsync(k[q][l], 0, 8 * (size_t)ne[l], s));
  }
  axpby(1.0, k[8], 0.0, k[8], k[0]);
  axpby(1.0, k[8], 0.0, k[8], k[1]);
  const double target = tol_rel * gnorm;
  double rho_old = 1.0, alpha = 1.0, omega = 1.0, rn = gnorm;
  std::vector<double> hist{rn};
  int it = 0;
  gmg_status result = GMG_OK;
  // Preconditioner for A^T.  The composite operator is a flux divergence per cell volume,
  // A = V^-1 K with K nearly symmetric, so A^T = K V^-1 = V A V^-1 (exactly so away from the
  // coarse/fine couplings).  With M the composite multigrid correction (M ~ A^-1), the
  // preconditioner is V M V^-1: scale level l of the input by V_0 / V_l = 8^l, apply M,
  // scale level l of the output by 8^-l.  V^-1 also maps the range of A^T (zero sum) onto
  // the range of A (zero volume-weighted sum) for the singular problem.
  // mid = V M V^-1 in, then out = A^T mid (mid copied first: the transpose overwrites its
  // input's ghosts).  With use_graph each of the two (in, mid, out) triples of the iteration
  // is captured once and replayed.
  // (the scalings are one launch over every level each; mid and its copy come from one pass)
  double sc_in[ML_MAX_SEG], sc_out[ML_MAX_SEG], zeros[ML_MAX_SEG];
  for (int l = 0; l < L; ++l) {
    sc_in[l] = z.v[0] / z.v[l];
    sc_out[l] = z.v[l] / z.v[0];
    zeros[l] = 0.0;
  }
  auto prec_apply = [&](double* const* in, double* const* mid, double* const* out, cudaStream_t st_) {
    launch_axpby_ml(L, ne, sc_in, (const double* const*)in, zeros, (const double* const*)in, tmp, st_);
    comp_correction_n(c, p, tmp, st_);
    launch_scale2_ml(L, ne, sc_out, (const double* const*)e, mid, tmp, st_);
    comp_apply_transpose_n(c, tmp, out, st_);
  };
  auto run_pa = [&](double* const* in, double* const* mid, double* const* out) -> gmg_status {
    if (!p.use_graph) {
      prec_apply(in, mid, out, s);
      return GMG_OK;
    }
    auto key = std::make_tuple((void*)mid[0], (const void*)in[0], L, p.nu1, p.nu2, p.bottom_max_iter, p.bottom_tol, 1,
                               p.fused_coarse, 1 + 256 * sweep_key(p), p.ghost_push, p.vector_smooth, p.pdl, 1,
                               p.bottom_solver,
                               p.post_reverse, 1, p.settled_zero);
    auto itg = c->graphs.find(key);
    if (itg == c->graphs.end()) {
      cudaGraph_t g;
      cudaGraphExec_t ge;
      const int64_t lc0 = kernel_launch_count();
      CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      prec_apply(in, mid, out, c->cap_stream);
      cudaError_t e1 = cudaStreamEndCapture(c->cap_stream, &g);
      if (e1 != cudaSuccess) SETERR(c, GMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
      cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) SETERR(c, GMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
      const int64_t n = kernel_launch_count() - lc0;
      count_launches((int)-n);  // captured, not launched
      itg = c->graphs.emplace(key, gmg_ctx::GraphEntry{ge, n, 0, 0}).first;
    }
    CK(c, cudaGraphLaunch(itg->second.exec, s));
    count_launches((int)itg->second.launches);
    return GMG_OK;
  };
  // (read-backs per iteration: <rhat, v>; ||s|| with <t, t> and <t, s> -- t computed before
  // ||s|| is known, so the last iteration may apply the preconditioner once for nothing;
  // ||r|| with the next iteration's <rhat, r>)
  double rho_next = 0.0;
  while (!(rn <= target) && it < p.max_iter) {
    ++it;
    double rho = rho_next;
    if (it == 1 && (st = comp_dot_n(c, k[1], k[0], &rho))) return st;
    if (std::fabs(rho) < 1e-300) break;
    const double beta = (rho / rho_old) * (alpha / omega);
    // p = r + beta (p - omega v), one pass over every level
    launch_bicg_direction_ml(L, ne, (const double* const*)k[0], k[2], (const double* const*)k[3], beta, omega, s);
    if ((st = run_pa(k[2], k[6], k[3]))) return st;
    double rv;
    if ((st = comp_dot_n(c, k[1], k[3], &rv))) return st;
    if (std::fabs(rv) < 1e-300) break;
    alpha = rho / rv;
    axpby(1.0, k[0], -alpha, k[3], k[4]);
    if ((st = run_pa(k[4], k[7], k[5]))) return st;
    double sn, tt, ts;
    if ((st = comp_dots_norm_n(c, k[5], k[5], k[5], k[4], k[4], &tt, &ts, &sn))) return st;
    if (sn <= target) {
      axpby(1.0, lam, alpha, k[6], lam);
      rn = sn;
      hist.push_back(rn);
      break;
    }
    if (tt == 0.0) break;
    omega = ts / tt;
    launch_add2_ml(L, ne, lam, alpha, (const double* const*)k[6], omega, (const double* const*)k[7], s);  // one pass
    axpby(1.0, k[4], -omega, k[5], k[0]);
    if ((st = comp_dots_norm_n(c, k[1], k[0], nullptr, nullptr, k[0], &rho_next, nullptr, &rn))) return st;
    hist.push_back(rn);
    if (!std::isfinite(rn)) {
      result = GMG_ERR_DIVERGED;
      break;
    }
    rho_old = rho;
  }
  if (result == GMG_OK && !(rn <= target)) result = GMG_ERR_NOT_CONVERGED;
  for (int l = 0; l + 1 < L; ++l) launch_zero_covered(c->amrl[l].A, lam[l], s);
  if (sing) {  // remove the null-space component of A^T (span of V): zero plain sum
    if ((st = comp_sums_n(c, lam, sums))) return st;
    double tot = 0.0;
    for (int l = 0; l < L; ++l) tot += sums[l];
    for (int l = 0; l < L; ++l) shift[l] = -(tot / vol) * z.v[l];
    if ((st = comp_add_const_n(c, lam, shift))) return st;
  }
  CK(c, cudaStreamSynchronize(s));
  CK(c, cudaGetLastError());
  if (info) {
    info->iterations = it;
    info->status = result;
    info->rhs_norm = gnorm;
    info->initial_resid = hist[0];
    info->final_resid = rn;
    info->hist_len = (int)std::min<size_t>(hist.size(), 256);
    for (int i = 0; i < info->hist_len; ++i) info->resid_hist[i] = hist[i];
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->kernel_launches = kernel_launch_count() - l0;
  }
  if (result == GMG_ERR_NOT_CONVERGED) c->err = "adjoint solve not converged within max_iter";
  if (gmg_status e = take_dev_err(c, s)) {
    if (info) info->status = e;
    return e;
  }
  return result;
}

gmg_status ensure_pinned(gmg_ctx* c) {
  const size_t need = (size_t)std::max(1, c->ns()) * 3 + 16;
  if (c->h_cap >= need) return GMG_OK;
  if (c->h_bits) cudaFreeHost(c->h_bits);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_iters) cudaFreeHost(c->h_iters);
  if (c->h_active) cudaFreeHost(c->h_active);
  c->h_bits = nullptr;
  c->h_scal = nullptr;
  c->h_iters = nullptr;
  c->h_active = nullptr;
  c->h_cap = 0;
  CK(c, cudaHostAlloc((void**)&c->h_bits, need * sizeof(unsigned long long), cudaHostAllocDefault));
  CK(c, cudaHostAlloc((void**)&c->h_scal, need * sizeof(double), cudaHostAllocDefault));
  CK(c, cudaHostAlloc((void**)&c->h_iters, need * sizeof(int), cudaHostAllocDefault));
  CK(c, cudaHostAlloc((void**)&c->h_active, need * sizeof(int), cudaHostAllocDefault));
  c->h_cap = need;
  return GMG_OK;
}

gmg_status set_domain_geom(gmg_ctx* c, SolveGeom& G, const int lo[3], const int hi[3], const double plo[3],
                           const double phi[3], const int bclo[3], const int bchi[3]) {
  for (int d = 0; d < 3; ++d) {
    if (hi[d] < lo[d]) SETERR(c, GMG_ERR_BAD_INPUT, "empty domain");
    if (!(phi[d] > plo[d])) SETERR(c, GMG_ERR_BAD_INPUT, "prob_hi must exceed prob_lo");
    if (bclo[d] < GMG_BC_PERIODIC || bclo[d] > GMG_BC_DIRICHLET_QUAD || bchi[d] < GMG_BC_PERIODIC ||
        bchi[d] > GMG_BC_DIRICHLET_QUAD)
      SETERR(c, GMG_ERR_BAD_INPUT, "unknown boundary condition");
    if ((bclo[d] == GMG_BC_PERIODIC) != (bchi[d] == GMG_BC_PERIODIC))
      SETERR(c, GMG_ERR_BAD_INPUT, "a periodic direction must be periodic on both sides");
    G.domain.lo[d] = lo[d];
    G.domain.hi[d] = hi[d];
    // a quadratic Dirichlet side is a Dirichlet side with the quadratic flag
    G.qlo[d] = bclo[d] == GMG_BC_DIRICHLET_QUAD;
    G.qhi[d] = bchi[d] == GMG_BC_DIRICHLET_QUAD;
    G.bclo[d] = G.qlo[d] ? GMG_BC_DIRICHLET : bclo[d];
    G.bchi[d] = G.qhi[d] ? GMG_BC_DIRICHLET : bchi[d];
    G.h[d] = (phi[d] - plo[d]) / (double)(hi[d] - lo[d] + 1);
  }
  return GMG_OK;
}

}  // namespace

// ====================================================================== C ABI

namespace {

// workspace bytes of the top-level Krylov vectors
size_t krylov_bytes(const gmg_ctx* c) {
  const size_t ne0 = c->L.empty() ? 0 : (size_t)c->L[0].nelem;
  return 256 + gmg_ctx::NKV * ((((8 * ne0) + 255) & ~(size_t)255) + 256);
}

// Krylov solve of A phi = rhs from phi = 0, preconditioned by one V-cycle per application
// (Sec. "Linear Solvers": native Krylov solvers next to multigrid): krylov = 1 BiCGStab
// (van der Vorst 1992) preconditioned on the right, 2 conjugate gradients with the symmetric
// V-cycle.  Vectors FP64; the V-cycle in the precision of p.  Stops on the recursive
// residual, ||r||_inf <= max(tol_rel ||rhs||_inf, tol_abs), after max_iter iterations, or on
// breakdown.  Singular problems: rhs, every preconditioned vector and phi projected onto
// zero mean.  One-level, single-problem contexts.  transpose: solve A^T x = rhs instead (the
// adjoint of a context with quadratic walls; BiCGStab, still preconditioned by the V-cycle
// of A, which differs from A^T only in the wall couplings).
void apply_transpose_one(gmg_ctx* c, double* y, double* out, cudaStream_t s);
gmg_status krylov_solve(gmg_ctx* c, double* x, const double* rhs, double tol_rel, double tol_abs, const gmg_params& p,
                        gmg_solve_info* info, bool transpose = false) {
  const auto t0 = std::chrono::steady_clock::now();
  if (c->amr || c->ns() != 1) SETERR(c, GMG_ERR_BAD_INPUT, "krylov: one-level, single-problem contexts only");
  if (!c->kv[0]) SETERR(c, GMG_ERR_NO_WORKSPACE, "workspace was not sized for the Krylov vectors (krylov != 0)");
  if (info) memset(info, 0, sizeof(*info));
  cudaStream_t s = c->stream;
  const int dt = dt_of_precision(p.precision);
  const LevelDev& D0 = c->dev[0];
  const int64_t ne = c->L[0].nelem;
  const int64_t l0 = kernel_launch_count();
  double *b = c->kv[0], *r = c->kv[1], *rh = c->kv[2], *pp = c->kv[3], *v = c->kv[4], *y = c->kv[5],
         *sv = c->kv[6], *t = c->kv[7], *z = c->kv[8];
  const bool sing = singular(c, 0);
  gmg_status st;
  auto host_sync = [&]() -> gmg_status {
    CK(c, cudaStreamSynchronize(s));
    CK(c, cudaGetLastError());
    return GMG_OK;
  };
  auto norm = [&](const double* a, double* out) -> gmg_status {
    CK(c, cudaMemsetAsync(c->normbits, 0, 8, s));
    launch_norm_max(D0, a, c->normbits, s);
    CK(c, cudaMemcpyAsync(c->h_bits, c->normbits, 8, cudaMemcpyDeviceToHost, s));
    gmg_status e = host_sync();
    *out = bits_to_double(c->h_bits[0]);
    return e;
  };
  auto dot = [&](const double* a, const double* bb, double* out) -> gmg_status {
    launch_dot(D0, a, bb, c->partials, c->scal, s);
    CK(c, cudaMemcpyAsync(c->h_scal, c->scal, 8, cudaMemcpyDeviceToHost, s));
    gmg_status e = host_sync();
    *out = c->h_scal[0];
    return e;
  };
  auto project = [&](double* a) {  // a -= mean(a) on the valid cells (device only)
    launch_sum(D0, a, c->partials, c->scal + 1, s);
    launch_add_scalar(D0, a, c->scal + 1, -1.0, s);
  };
  auto axpby = [&](double al, const double* a, double be, const double* bb, double* out) {
    launch_axpby(ne, al, a, be, bb, out, s);
  };
  // out = V(in) on stream st: the V-cycle runs on in and out themselves in FP64 (the
  // level-0 buffers are swapped for the call), on float or bfloat16 copies otherwise
  auto precond_body = [&](const double* in, double* out, cudaStream_t st) {
    LevelBufs& B0 = c->buf[0];
    if (dt == DT_F64) {
      // (a colour-split finest level takes a split copy of in as its right-hand side)
      void* const sr = B0.r[DT_F64];
      void* const se = B0.e[DT_F64];
      if (D0.split & SPLIT_RHS) launch_to_rhs(DT_F64, D0, in, sr, st);
      else B0.r[DT_F64] = (void*)in;
      B0.e[DT_F64] = out;
      vcycle(c, dt, 0, p, st);
      B0.r[DT_F64] = sr;
      B0.e[DT_F64] = se;
    } else {
      launch_to_rhs(dt, D0, in, B0.r[dt], st);
      vcycle(c, dt, 0, p, st);
      launch_convert(dt, DT_F64, B0.e[dt], out, ne, st);
    }
    if (sing) {
      launch_sum(D0, out, c->partials, c->scal + 1, st);
      launch_add_scalar(D0, out, c->scal + 1, -1.0, st);
    }
  };
  int64_t graph_launches = 0;
  auto precond = [&](const double* in, double* out) -> gmg_status {
    if (!p.use_graph) {
      precond_body(in, out, s);
      return GMG_OK;
    }
    auto key = std::make_tuple((const void*)in, (void*)out, p.precision, p.nu1, p.nu2, p.bottom_max_iter, p.bottom_tol,
                               p.fused_coarse, p.ghost_push, p.vector_smooth, p.bottom_solver, post_reversed(p) ? 1 : 0,
                               p.pdl, p.settled_zero, sweep_key(p));
    auto itg = c->kgraphs.find(key);
    if (itg == c->kgraphs.end()) {
      cudaGraph_t g;
      cudaGraphExec_t ge;
      const int64_t lc = kernel_launch_count();
      CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
      precond_body(in, out, c->cap_stream);
      cudaError_t e1 = cudaStreamEndCapture(c->cap_stream, &g);
      if (e1 != cudaSuccess) SETERR(c, GMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
      cudaError_t e2 = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (e2 != cudaSuccess) SETERR(c, GMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
      const int64_t nl = kernel_launch_count() - lc;
      count_launches((int)-nl);  // captured, not launched
      itg = c->kgraphs.emplace(key, gmg_ctx::GraphEntry{ge, nl, 0, 0}).first;
    }
    CK(c, cudaGraphLaunch(itg->second.exec, s));
    graph_launches += itg->second.launches;
    return GMG_OK;
  };
  auto apply = [&](double* in, double* out) {  // out = A in (A^T in), homogeneous walls
    if (transpose) {
      apply_transpose_one(c, in, out, s);
      return;
    }
    launch_fill(DT_F64, D0, in, -1, 0, s);
    launch_apply(D0, in, coefs64(c, 0), out, s);
  };
  CK(c, cudaMemcpyAsync(b, rhs, 8 * (size_t)ne, cudaMemcpyDeviceToDevice, s));
  double bnorm;
  if ((st = norm(b, &bnorm))) return st;
  if (!std::isfinite(bnorm)) SETERR(c, GMG_ERR_BAD_INPUT, "rhs is not finite");
  if (sing) {
    launch_sum(D0, b, c->partials, c->scal, s);
    CK(c, cudaMemcpyAsync(c->h_scal, c->scal, 8, cudaMemcpyDeviceToHost, s));
    if ((st = host_sync())) return st;
    if (std::fabs(c->h_scal[0]) > 1e-12 * bnorm && !p.project_mean) {
      if (info) info->status = GMG_ERR_BAD_INPUT;
      SETERR(c, GMG_ERR_BAD_INPUT, "singular problem with a nonzero-mean rhs (set project_mean)");
    }
    launch_add_scalar(D0, b, c->scal, -1.0, s);
  }
  const double target = std::max(tol_rel * bnorm, tol_abs);
  CK(c, cudaMemsetAsync(x, 0, 8 * (size_t)ne, s));
  for (double* w : {pp, v, y, sv, t, z}) CK(c, cudaMemsetAsync(w, 0, 8 * (size_t)ne, s));
  CK(c, cudaMemcpyAsync(r, b, 8 * (size_t)ne, cudaMemcpyDeviceToDevice, s));
  double rn;
  if ((st = norm(r, &rn))) return st;
  std::vector<double> hist{rn};
  int it = 0;
  gmg_status result = GMG_OK;
  if (p.krylov == 1) {
    CK(c, cudaMemcpyAsync(rh, r, 8 * (size_t)ne, cudaMemcpyDeviceToDevice, s));
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    while (!(rn <= target) && it < p.max_iter) {
      ++it;
      double rho;
      if ((st = dot(rh, r, &rho))) return st;
      if (std::fabs(rho) < 1e-300) { --it; break; }
      const double beta = (rho / rho_old) * (alpha / omega);
      launch_bicg_direction(ne, r, pp, v, beta, omega, s);  // p = r + beta (p - omega v)
      if ((st = precond(pp, y))) return st;
      apply(y, v);
      double rv;
      if ((st = dot(rh, v, &rv))) return st;
      if (std::fabs(rv) < 1e-300) { --it; break; }
      alpha = rho / rv;
      axpby(1.0, r, -alpha, v, sv);
      double sn;
      if ((st = norm(sv, &sn))) return st;
      if (sn <= target) {
        axpby(1.0, x, alpha, y, x);
        rn = sn;
        hist.push_back(rn);
        break;
      }
      if ((st = precond(sv, z))) return st;
      apply(z, t);
      double tt, ts;
      if ((st = dot(t, t, &tt))) return st;
      if (tt == 0.0) { --it; break; }
      if ((st = dot(t, sv, &ts))) return st;
      omega = ts / tt;
      launch_add2(ne, x, alpha, y, omega, z, s);
      axpby(1.0, sv, -omega, t, r);
      if ((st = norm(r, &rn))) return st;
      hist.push_back(rn);
      if (!std::isfinite(rn)) {
        result = GMG_ERR_DIVERGED;
        break;
      }
      rho_old = rho;
    }
  } else {
    if ((st = precond(r, z))) return st;
    CK(c, cudaMemcpyAsync(pp, z, 8 * (size_t)ne, cudaMemcpyDeviceToDevice, s));
    double rho;
    if ((st = dot(r, z, &rho))) return st;
    while (!(rn <= target) && it < p.max_iter) {
      ++it;
      apply(pp, v);
      double pv;
      if ((st = dot(pp, v, &pv))) return st;
      if (!(pv > 0.0)) { --it; break; }
      const double alpha = rho / pv;
      axpby(1.0, x, alpha, pp, x);
      axpby(1.0, r, -alpha, v, r);
      if ((st = norm(r, &rn))) return st;
      hist.push_back(rn);
      if (!std::isfinite(rn)) {
        result = GMG_ERR_DIVERGED;
        break;
      }
      if (rn <= target) break;
      if ((st = precond(r, z))) return st;
      double rho_new;
      if ((st = dot(r, z, &rho_new))) return st;
      const double beta = rho_new / rho;
      rho = rho_new;
      axpby(1.0, z, beta, pp, pp);
    }
  }
  if (result == GMG_OK && !(rn <= target)) result = GMG_ERR_NOT_CONVERGED;
  if (sing) project(x);
  CK(c, cudaMemcpyAsync(c->h_iters, c->bot_iters, 4 * 2, cudaMemcpyDeviceToHost, s));
  if ((st = host_sync())) return st;
  if (c->h_iters[1]) {  // a dependency wait of a flow sweep gave up
    CK(c, cudaMemsetAsync(c->dev_err, 0, sizeof(int), s));
    result = GMG_ERR_DEVICE_TIMEOUT;
  }
  if (info) {
    info->iterations = it;
    info->status = result;
    info->rhs_norm = bnorm;
    info->initial_resid = hist[0];
    info->final_resid = rn;
    info->bottom_iters = c->h_iters[0];
    info->hist_len = (int)std::min<size_t>(hist.size(), 256);
    for (int i = 0; i < info->hist_len; ++i) info->resid_hist[i] = hist[i];
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->kernel_launches = kernel_launch_count() - l0 + graph_launches;
  }
  if (result == GMG_ERR_NOT_CONVERGED) c->err = "not converged within max_iter";
  return result;
}

}  // namespace

namespace {

// Time `body` (stream-ordered launches) reps times with CUDA events on the context stream;
// returns ms per rep.
template <class F>
double time_reps(gmg_ctx* c, int reps, F body) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  body();  // warm-up
  cudaEventRecord(a, c->stream);
  for (int i = 0; i < reps; ++i) body();
  cudaEventRecord(b, c->stream);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)ms / reps;
}

// Wall values are for single-level contexts holding one problem; a periodic face takes none.
gmg_status wall_values_check(gmg_ctx* c, const void* const* values) {
  bool any = false;
  for (int f = 0; f < 6; ++f) any |= values[f] != nullptr;
  if (!any) return GMG_OK;
  if (c->amr || c->ns() != 1) SETERR(c, GMG_ERR_BAD_INPUT, "wall values: single-level, single-problem contexts only");
  const SolveGeom& G = c->geoms[0];
  for (int f = 0; f < 6; ++f) {
    const int d = f / 2, bc = f % 2 ? G.bchi[d] : G.bclo[d];
    if (values[f] && bc == GMG_BC_PERIODIC)
      SETERR(c, GMG_ERR_BAD_INPUT, "wall values given for periodic face " + std::to_string(f));
  }
  if (c->L[0].boxes.size() > 65535u) SETERR(c, GMG_ERR_BAD_INPUT, "wall values: more than 65535 level-0 boxes");
  return GMG_OK;
}

// One k_wall_values launch per face with values, in face order (walls.cu).
gmg_status wall_values_pass(gmg_ctx* c, const void* const* values, int mode, double* f, const double* lam,
                            void* const* dg) {
  const LevelMeta& M = c->L[0];
  const SolveGeom& G = c->geoms[0];
  const Coefs k = coefs64(c, 0);
  const double* w[3] = {(const double*)k.wx, (const double*)k.wy, (const double*)k.wz};
  for (int face = 0; face < 6; ++face) {
    if (!values[face]) continue;
    const int d = face / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int kind = (face % 2 ? G.qhi[d] : G.qlo[d]) ? 3 : (face % 2 ? G.bchi[d] : G.bclo[d]);
    int maxf = 0;
    for (const Box& B : M.boxes) maxf = std::max(maxf, B.n(t1) * B.n(t2));
    launch_wall_values(c->dev[0], (int)M.boxes.size(), maxf, face, kind, G.h[d], w[d], (const double*)values[face],
                       mode, f, lam, mode == 2 ? (double*)dg[face] : nullptr, c->stream);
  }
  CK(c, cudaGetLastError());
  return GMG_OK;
}

// out = A^T y on level 0 of a one-level context with homogeneous walls (y's ghosts are
// overwritten).  Without quadratic walls A is symmetric and this is A y.  A quadratic wall
// cell's row holds, besides its symmetric entries, -w/3 on phi_1 (the cell next to it
// inward): A y with the quadratic ghosts 0 gives every other entry of A^T, then one
// k_wall_values pass per quadratic face adds -w/3 y_0 to the row of phi_1.
void apply_transpose_one(gmg_ctx* c, double* y, double* out, cudaStream_t s) {
  const LevelDev& D0 = c->dev[0];
  const bool quad = any_quad(c);
  launch_fill(DT_F64, D0, y, -1, quad ? 2 : 0, s);
  launch_apply(D0, y, coefs64(c, 0), out, s);
  if (!quad) return;
  const LevelMeta& M = c->L[0];
  const SolveGeom& G = c->geoms[0];
  const Coefs k = coefs64(c, 0);
  const double* w[3] = {(const double*)k.wx, (const double*)k.wy, (const double*)k.wz};
  for (int face = 0; face < 6; ++face) {
    const int d = face / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    if (!(face % 2 ? G.qhi[d] : G.qlo[d])) continue;
    int maxf = 0;
    for (const Box& B : M.boxes) maxf = std::max(maxf, B.n(t1) * B.n(t2));
    launch_wall_values(D0, (int)M.boxes.size(), maxf, face, 3, G.h[d], w[d], nullptr, 3, out, y, nullptr, s);
  }
}

}  // namespace

extern "C" {

gmg_status gmg_default_params(gmg_params* p) {
  if (!p) return GMG_ERR_BAD_INPUT;
  p->nu1 = 2;
  p->nu2 = 2;
  p->max_iter = 100;
  p->bottom_max_iter = 200;
  p->bottom_tol = 1e-4;
  p->precision = GMG_FP64;
  p->project_mean = 0;
  p->use_graph = 1;
  p->profile = 0;
  p->fused_coarse = 2;
  p->fused_sweep = 0;
  p->flow_warps = 0;
  p->flow_lag_kcells = 0;
  p->serpentine = 1;
  p->prolongation = 0;
  p->wave_sweep = 0;
  p->tail_dense = 1;
  p->fuse_restriction_sweep = 1;
  p->fuse_prolongation = 1;
  p->fork_bottoms = 1;
  p->ghost_push = 2;
  p->vector_smooth = 2;
  p->pdl = 2;
  p->fuse_residual_sweep = 1;
  p->krylov = 0;
  p->bottom_solver = 0;
  p->post_reverse = 0;
  p->fuse_correction = 1;
  p->settled_zero = 1;
  return GMG_OK;
}

gmg_status gmg_create(gmg_ctx** out, void* stream) {
  if (!out) return GMG_ERR_BAD_INPUT;
  *out = nullptr;
  gmg_ctx* c = new gmg_ctx();
  c->stream = (cudaStream_t)stream;
  *out = c;
  return GMG_OK;
}

gmg_status gmg_destroy(gmg_ctx* c) {
  if (!c) return GMG_OK;
  drop_graphs(c);
  for (cudaEvent_t e : c->ev_smooth) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_resid) cudaEventDestroy(e);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (cudaEvent_t e : c->ev_fork) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_join) if (e) cudaEventDestroy(e);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  if (c->h_bits) cudaFreeHost(c->h_bits);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_iters) cudaFreeHost(c->h_iters);
  if (c->h_active) cudaFreeHost(c->h_active);
  delete c;
  return GMG_OK;
}

const char* gmg_last_error(const gmg_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

gmg_status gmg_define_domain(gmg_ctx* c, const int lo[3], const int hi[3], const double plo[3], const double phi[3],
                             const int bclo[3], const int bchi[3]) {
  if (!c || !lo || !hi || !plo || !phi || !bclo || !bchi) return GMG_ERR_BAD_INPUT;
  SolveGeom G;
  gmg_status st = set_domain_geom(c, G, lo, hi, plo, phi, bclo, bchi);
  if (st) return st;
  reset_problem(c);
  c->geoms = {G};
  c->have_domain = true;
  c->err.clear();
  return GMG_OK;
}

gmg_status gmg_define_level(gmg_ctx* c, int lev, int nboxes, const int* lohi, int ref_ratio) {
  if (!c) return GMG_ERR_BAD_INPUT;
  if (!c->have_domain || c->ns() != 1) SETERR(c, GMG_ERR_STATE, "define one domain first (gmg_define_domain)");
  if (lev < 0 || lev >= GMG_MAX_AMR_LEVELS)
    SETERR(c, GMG_ERR_BAD_INPUT, "AMR level out of range (0 .. " + std::to_string(GMG_MAX_AMR_LEVELS - 1) + ")");
  if (nboxes <= 0 || !lohi) SETERR(c, GMG_ERR_BAD_INPUT, "no boxes");
  std::vector<Box> boxes(nboxes);
  for (int b = 0; b < nboxes; ++b)
    for (int d = 0; d < 3; ++d) {
      boxes[b].lo[d] = lohi[6 * b + d];
      boxes[b].hi[d] = lohi[6 * b + 3 + d];
    }
  if (lev == 0) return build_hierarchy(c, boxes, std::vector<int>(boxes.size(), 0));
  // AMR level lev >= 1: ratio 2 over part of level lev - 1 (Sec. "Basic data structures":
  // refinement ratio between levels; proper nesting inside the level below)
  if (c->L.empty()) SETERR(c, GMG_ERR_STATE, "define AMR level 0 first");
  if (c->geoms[0].has_quad())
    SETERR(c, GMG_ERR_BAD_INPUT, "quadratic Dirichlet walls: composite (AMR) contexts take the linear rule only");
  if (c->ns() != 1) SETERR(c, GMG_ERR_BAD_INPUT, "AMR levels: single-problem contexts only");
  if (lev > (int)c->amrl.size() + 1 || lev > GMG_MAX_AMR_LEVELS - 1)
    SETERR(c, GMG_ERR_BAD_INPUT, "define AMR levels in order (at most " + std::to_string(GMG_MAX_AMR_LEVELS) + ")");
  if (ref_ratio != 2) SETERR(c, GMG_ERR_BAD_INPUT, "only refinement ratio 2 is supported");
  SolveGeom G = c->geoms[0];
  for (int d = 0; d < 3; ++d) {
    G.domain.lo[d] = G.domain.lo[d] << lev;
    G.domain.hi[d] = ((G.domain.hi[d] + 1) << lev) - 1;
    G.h[d] /= (double)(1 << lev);
  }
  const std::string tag = "level " + std::to_string(lev) + ": ";
  std::string e = validate_boxes(boxes, G.domain, false);
  if (!e.empty()) SETERR(c, GMG_ERR_BAD_INPUT, tag + e);
  drop_graphs(c);
  c->ws = nullptr;
  c->ws_bytes = 0;
  c->have_beta = c->have_alpha = false;
  c->amrl.resize(lev - 1);  // a new level lev drops the levels above it
  for (AmrLevel& A : c->amrl) A.have_beta = A.have_alpha = false;
  c->coefs_dirty = true;
  AmrLevel N;
  N.M.allow_cf = true;
  N.M.boxes = boxes;
  N.M.box_solve.assign(boxes.size(), 0);
  N.M.geoms = {G};
  N.M.solve_present = {1};
  N.M.solve_bottom = {0};
  e = finalize_level(N.M);
  if (!e.empty()) SETERR(c, GMG_ERR_BAD_INPUT, tag + e);
  e = build_amr(lev == 1 ? c->L[0] : c->amrl[lev - 2].M, N.M, N.H);
  if (!e.empty()) SETERR(c, GMG_ERR_BAD_INPUT, tag + e);
  c->amrl.push_back(std::move(N));
  c->amr = true;
  return GMG_OK;
}

gmg_status gmg_chop_domain(gmg_ctx* c, int lev, int mgs) {
  if (!c) return GMG_ERR_BAD_INPUT;
  if (!c->have_domain || c->ns() != 1) SETERR(c, GMG_ERR_STATE, "define one domain first (gmg_define_domain)");
  if (lev != 0) SETERR(c, GMG_ERR_BAD_INPUT, "only AMR level 0 is supported by gmg_chop_domain");
  if (mgs < 1) SETERR(c, GMG_ERR_BAD_INPUT, "max_grid_size must be positive");
  std::vector<Box> boxes = chop(c->geoms[0].domain, mgs);
  return build_hierarchy(c, boxes, std::vector<int>(boxes.size(), 0));
}

gmg_status gmg_define_batch(gmg_ctx* c, int n, const int* dom_lohi, const double* prob_lo, const double* prob_hi,
                            const int* bc_lo, const int* bc_hi, const int* nboxes, const int* box_lohi) {
  if (!c || n < 1 || !dom_lohi || !prob_lo || !prob_hi || !bc_lo || !bc_hi || !nboxes || !box_lohi)
    return GMG_ERR_BAD_INPUT;
  std::vector<SolveGeom> geoms(n);
  std::vector<Box> boxes;
  std::vector<int> owner;
  int64_t k = 0;
  for (int s = 0; s < n; ++s) {
    gmg_status st = set_domain_geom(c, geoms[s], dom_lohi + 6 * s, dom_lohi + 6 * s + 3, prob_lo + 3 * s,
                                    prob_hi + 3 * s, bc_lo + 3 * s, bc_hi + 3 * s);
    if (st) return st;
    if (nboxes[s] < 1) SETERR(c, GMG_ERR_BAD_INPUT, "every problem needs at least one box");
    for (int b = 0; b < nboxes[s]; ++b, ++k) {
      Box B;
      for (int d = 0; d < 3; ++d) {
        B.lo[d] = box_lohi[6 * k + d];
        B.hi[d] = box_lohi[6 * k + 3 + d];
      }
      boxes.push_back(B);
      owner.push_back(s);
    }
  }
  reset_problem(c);
  c->geoms = geoms;
  c->have_domain = true;
  c->err.clear();
  return build_hierarchy(c, boxes, owner);
}

gmg_status gmg_num_solves(const gmg_ctx* c, int* n) {
  if (!c || !n) return GMG_ERR_BAD_INPUT;
  *n = c->ns();
  return GMG_OK;
}

gmg_status gmg_solve_boxes(const gmg_ctx* c, int m, int solve, int* first, int* count) {
  if (!c || m < 0 || m >= (int)c->L.size() || solve < 0 || solve >= c->ns()) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->L[m];
  int f = -1, n = 0;
  for (int b = 0; b < (int)M.boxes.size(); ++b)
    if (M.box_solve[b] == solve) {
      if (f < 0) f = b;
      ++n;
    }
  if (first) *first = f;
  if (count) *count = n;
  return GMG_OK;
}

gmg_status gmg_mg_nlevels(const gmg_ctx* c, int* n) {
  if (!c || !n) return GMG_ERR_BAD_INPUT;
  *n = (int)c->L.size();
  return GMG_OK;
}

gmg_status gmg_mg_level_info(const gmg_ctx* c, int m, int* nboxes, int* dom) {
  if (!c || m < 0 || m >= (int)c->L.size()) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->L[m];
  if (nboxes) *nboxes = (int)M.boxes.size();
  if (dom)
    for (int d = 0; d < 3; ++d) {
      dom[d] = M.geoms[0].domain.lo[d];
      dom[3 + d] = M.geoms[0].domain.hi[d];
    }
  return GMG_OK;
}

gmg_status gmg_mg_level_boxes(const gmg_ctx* c, int m, int* lohi, int* parents) {
  if (!c || m < 0 || m >= (int)c->L.size()) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->L[m];
  for (size_t b = 0; b < M.boxes.size(); ++b) {
    if (lohi)
      for (int d = 0; d < 3; ++d) {
        lohi[6 * b + d] = M.boxes[b].lo[d];
        lohi[6 * b + 3 + d] = M.boxes[b].hi[d];
      }
    if (parents) parents[b] = M.parent[b];
  }
  return GMG_OK;
}

gmg_status gmg_wave_tiles(const gmg_ctx* c, int m, int* ntiles, int* ppt, int* out, int cap) {
  if (!c || m < 0 || m >= (int)c->L.size() || cap < 0) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->L[m];
  if (ntiles) *ntiles = (int)M.wave_tiles.size();
  if (ppt) *ppt = M.wave_ppt;
  if (out)
    for (int t = 0; t < (int)M.wave_tiles.size() && t < cap; ++t) {
      const WaveTile& W = M.wave_tiles[t];
      const int row[13] = {W.box,   W.y0,    W.y1,    W.dir,      W.nb[0],    W.nb[1],   W.nb[2],
                           W.nb[3], W.zb[0], W.zb[1], W.zneed[0], W.zneed[1], W.solve};
      for (int u = 0; u < 13; ++u) out[13 * t + u] = row[u];
    }
  return GMG_OK;
}

gmg_status gmg_tail_plan(const gmg_ctx* c, int m, int dt, int* nblocks, long long* dense_bytes) {
  if (!c || m < 0 || m >= (int)c->L.size() || dt < 0 || dt >= NDT) return GMG_ERR_BAD_INPUT;
  const TailHost& T = c->tail;
  const bool any = c->tail_ok && m < (int)T.count_at.size() && T.count_at[m] > 0;
  if (nblocks) *nblocks = any ? T.count_at[m] : 0;
  if (dense_bytes) *dense_bytes = any ? (long long)tail_dense_bytes(c, dt, m) : 0;
  return GMG_OK;
}

// ------------------------------------------------------------- sharding plan (host only)

namespace {
// Morton (Z-order) key of a box's low corner: the bits of x, y, z interleaved
uint64_t morton_key(const Box& b, const Box& dom) {
  uint64_t k = 0;
  const uint32_t x = (uint32_t)(b.lo[0] - dom.lo[0]), y = (uint32_t)(b.lo[1] - dom.lo[1]),
                 z = (uint32_t)(b.lo[2] - dom.lo[2]);
  for (int bit = 20; bit >= 0; --bit)
    k = (k << 3) | (((z >> bit) & 1u) << 2) | (((y >> bit) & 1u) << 1) | ((x >> bit) & 1u);
  return k;
}
}  // namespace

gmg_status gmg_partition(const gmg_ctx* c, int m, int nranks, long long min_cells_per_rank, int* owner) {
  if (!c || m < 0 || m >= (int)c->L.size() || nranks < 1 || !owner || min_cells_per_rank < 0)
    return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->L[m];
  const int nb = (int)M.boxes.size();
  if (M.ncells < (int64_t)nranks * min_cells_per_rank || nranks == 1) {
    for (int b = 0; b < nb; ++b) owner[b] = 0;  // consolidated onto rank 0
    return GMG_OK;
  }
  std::vector<std::pair<std::pair<int, uint64_t>, int>> order(nb);  // ((solve, key), box)
  for (int b = 0; b < nb; ++b)
    order[b] = {{M.box_solve[b], morton_key(M.boxes[b], M.geoms[M.box_solve[b]].domain)}, b};
  std::sort(order.begin(), order.end());
  // cut the curve into nranks pieces of about equal cell counts: box i goes to the rank in
  // whose share the middle of its cells falls
  int64_t before = 0;
  for (const auto& o : order) {
    const int64_t v = M.boxes[o.second].volume();
    const double mid = (double)before + 0.5 * (double)v;
    owner[o.second] = std::min(nranks - 1, (int)(mid * nranks / (double)M.ncells));
    before += v;
  }
  return GMG_OK;
}

gmg_status gmg_ghost_rects(const gmg_ctx* c, int m, int* n, int* rects) {
  if (!c || m < 0 || m >= (int)c->L.size() || !n) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->L[m];
  *n = (int)M.ghosts.size();
  if (rects)
    for (size_t r = 0; r < M.ghosts.size(); ++r) {
      const GhostRect& g = M.ghosts[r];
      const int v[14] = {g.dst_box, g.src_box, g.dst[0], g.dst[1], g.dst[2], g.src[0], g.src[1], g.src[2],
                         g.d1,      g.d2,      g.n1,     g.n2,     g.sign,   g.kind};
      for (int q = 0; q < 14; ++q) rects[14 * r + q] = v[q];
    }
  return GMG_OK;
}

gmg_status gmg_exchange_plan(const gmg_ctx* c, int m, const int* owner, int rank, int* nsend, int* send, int* nrecv,
                             int* recv) {
  if (!c || m < 0 || m >= (int)c->L.size() || !owner || !nsend || !nrecv) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->L[m];
  std::vector<std::pair<int, int>> s, r;  // (peer, rectangle)
  for (int q = 0; q < (int)M.ghosts.size(); ++q) {
    const GhostRect& g = M.ghosts[q];
    if (g.kind != 0) continue;  // walls are filled where their box lives
    const int od = owner[g.dst_box], os = owner[g.src_box];
    if (od == os) continue;
    if (os == rank) s.push_back({od, q});
    if (od == rank) r.push_back({os, q});
  }
  std::sort(s.begin(), s.end());
  std::sort(r.begin(), r.end());
  *nsend = (int)s.size();
  *nrecv = (int)r.size();
  if (send)
    for (size_t i = 0; i < s.size(); ++i) { send[2 * i] = s[i].first; send[2 * i + 1] = s[i].second; }
  if (recv)
    for (size_t i = 0; i < r.size(); ++i) { recv[2 * i] = r[i].first; recv[2 * i + 1] = r[i].second; }
  return GMG_OK;
}

gmg_status gmg_mg_layout(const gmg_ctx* c, int m, int dt, int64_t* nelems, int64_t* offs, int* sx) {
  if (!c || m < 0 || m >= (int)c->L.size() || dt < 0 || dt >= NDT) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->L[m];
  if (nelems) *nelems = M.nelem;
  for (size_t b = 0; b < M.dbox.size(); ++b) {
    if (offs) offs[b] = M.dbox[b].off;
    if (sx) sx[b] = M.dbox[b].sx;
  }
  return GMG_OK;
}

gmg_status gmg_layout(const gmg_ctx* c, int lev, int64_t* nelems, int64_t* offs) {
  if (!c) return GMG_ERR_BAD_INPUT;
  if (lev == 0) return gmg_mg_layout(c, 0, DT_F64, nelems, offs, nullptr);
  if (lev < 1 || lev > (int)c->amrl.size()) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = c->amrl[lev - 1].M;
  if (nelems) *nelems = M.nelem;
  if (offs)
    for (size_t b = 0; b < M.dbox.size(); ++b) offs[b] = M.dbox[b].off;
  return GMG_OK;
}

gmg_status gmg_amr_level_boxes(const gmg_ctx* c, int lev, int* nboxes, int* lohi, int* row_strides) {
  if (!c || lev < 0 || lev > (int)c->amrl.size() || c->L.empty()) return GMG_ERR_BAD_INPUT;
  const LevelMeta& M = lev ? c->amrl[lev - 1].M : c->L[0];
  if (nboxes) *nboxes = (int)M.boxes.size();
  for (size_t b = 0; b < M.boxes.size(); ++b) {
    if (lohi)
      for (int d = 0; d < 3; ++d) {
        lohi[6 * b + d] = M.boxes[b].lo[d];
        lohi[6 * b + 3 + d] = M.boxes[b].hi[d];
      }
    if (row_strides) row_strides[b] = M.dbox[b].sx;
  }
  return GMG_OK;
}

// dense (nz, ny, nx) array over the bounding box of AMR level lev's boxes <-> boxed layout
gmg_status gmg_pack_amr(gmg_ctx* c, int lev, const double* dense, double* boxed) {
  if (!c || lev < 0) return GMG_ERR_BAD_INPUT;
  if (lev == 0) return gmg_pack_solve(c, 0, DT_F64, 0, dense, boxed);
  if (lev > (int)c->amrl.size()) SETERR(c, GMG_ERR_STATE, "no such AMR level");
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  const AmrLevel& V = c->amrl[lev - 1];
  Box bb = V.M.boxes[0];
  for (const Box& B : V.M.boxes)
    for (int d = 0; d < 3; ++d) {
      bb.lo[d] = std::min(bb.lo[d], B.lo[d]);
      bb.hi[d] = std::max(bb.hi[d], B.hi[d]);
    }
  int dn[3] = {bb.n(0), bb.n(1), bb.n(2)};
  launch_pack(DT_F64, V.D, bb.lo, dn, dense, boxed, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_unpack_amr(gmg_ctx* c, int lev, const double* boxed, double* dense) {
  if (!c || lev < 0) return GMG_ERR_BAD_INPUT;
  if (lev == 0) return gmg_unpack_solve(c, 0, DT_F64, 0, boxed, dense);
  if (lev > (int)c->amrl.size()) SETERR(c, GMG_ERR_STATE, "no such AMR level");
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  const AmrLevel& V = c->amrl[lev - 1];
  Box bb = V.M.boxes[0];
  for (const Box& B : V.M.boxes)
    for (int d = 0; d < 3; ++d) {
      bb.lo[d] = std::min(bb.lo[d], B.lo[d]);
      bb.hi[d] = std::max(bb.hi[d], B.hi[d]);
    }
  int dn[3] = {bb.n(0), bb.n(1), bb.n(2)};
  launch_unpack(DT_F64, V.D, bb.lo, dn, boxed, dense, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_pack_solve(gmg_ctx* c, int m, int dt, int solve, const double* dense, void* boxed) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if (solve < 0 || solve >= c->ns()) SETERR(c, GMG_ERR_BAD_INPUT, "problem index out of range");
  if (!c->L[m].solve_present[solve]) SETERR(c, GMG_ERR_BAD_INPUT, "problem has no boxes on this MG level");
  const SolveGeom& G = c->L[m].geoms[solve];
  int dn[3] = {G.domain.n(0), G.domain.n(1), G.domain.n(2)};
  launch_pack(dt, solve_view(c, m, solve), G.domain.lo, dn, dense, boxed, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_unpack_solve(gmg_ctx* c, int m, int dt, int solve, const void* boxed, double* dense) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if (solve < 0 || solve >= c->ns()) SETERR(c, GMG_ERR_BAD_INPUT, "problem index out of range");
  if (!c->L[m].solve_present[solve]) SETERR(c, GMG_ERR_BAD_INPUT, "problem has no boxes on this MG level");
  const SolveGeom& G = c->L[m].geoms[solve];
  int dn[3] = {G.domain.n(0), G.domain.n(1), G.domain.n(2)};
  launch_unpack(dt, solve_view(c, m, solve), G.domain.lo, dn, boxed, dense, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_pack(gmg_ctx* c, int m, int dt, const double* dense, void* boxed) {
  return gmg_pack_solve(c, m, dt, 0, dense, boxed);
}

gmg_status gmg_unpack(gmg_ctx* c, int m, int dt, const void* boxed, double* dense) {
  return gmg_unpack_solve(c, m, dt, 0, boxed, dense);
}

gmg_status gmg_set_scalars(gmg_ctx* c, double a, double b) {
  if (!c) return GMG_ERR_BAD_INPUT;
  if (!std::isfinite(a) || !std::isfinite(b) || b == 0.0) SETERR(c, GMG_ERR_BAD_INPUT, "a must be finite and b finite and nonzero");
  c->a = a;
  c->b = b;
  c->coefs_dirty = true;
  drop_graphs(c);
  return GMG_OK;
}

gmg_status gmg_set_acoef(gmg_ctx* c, int lev, const double* alpha) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if (!alpha || lev < 0 || lev > (int)c->amrl.size()) SETERR(c, GMG_ERR_BAD_INPUT, "alpha: bad level or null");
  if (lev >= 1) {
    AmrLevel& V = c->amrl[lev - 1];
    CK(c, cudaMemcpyAsync(V.alpha, alpha, 8 * (size_t)V.M.nelem, cudaMemcpyDeviceToDevice, c->stream));
    V.have_alpha = true;
    c->coefs_dirty = true;
    return GMG_OK;
  }
  CK(c, cudaMemcpyAsync(c->alpha0, alpha, 8 * (size_t)c->L[0].nelem, cudaMemcpyDeviceToDevice, c->stream));
  c->have_alpha = true;
  c->coefs_dirty = true;
  return GMG_OK;
}

gmg_status gmg_set_bcoef_cell(gmg_ctx* c, int lev, const double* beta) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if (!beta || lev < 0 || lev > (int)c->amrl.size()) SETERR(c, GMG_ERR_BAD_INPUT, "beta: bad level or null");
  cudaStream_t s = c->stream;
  auto all_set = [&]() {
    if (!c->have_beta) return false;
    for (const AmrLevel& V : c->amrl)
      if (!V.have_beta) return false;
    return true;
  };
  if (lev >= 1) {  // coarse/fine faces take the fine cell's beta: ghost := adjacent cell
    AmrLevel& V = c->amrl[lev - 1];
    CK(c, cudaMemcpyAsync(V.beta_cell, beta, 8 * (size_t)V.M.nelem, cudaMemcpyDeviceToDevice, s));
    launch_fill(DT_F64, V.D, V.beta_cell, -1, 1, s);
    launch_cf_fill(V.A, V.beta_cell, nullptr, CF_COPY, s);
    launch_faces_from_cell(V.D, V.beta_cell, V.bx, V.by, V.bz, s);
    CK(c, cudaGetLastError());
    V.have_beta = true;
    c->coefs_dirty = true;
    return all_set() ? build_coefs(c) : GMG_OK;
  }
  CK(c, cudaMemcpyAsync(c->betac_cell, beta, 8 * (size_t)c->L[0].nelem, cudaMemcpyDeviceToDevice, s));
  launch_fill(DT_F64, c->dev[0], c->betac_cell, -1, 1, s);
  launch_faces_from_cell(c->dev[0], c->betac_cell, c->bx0, c->by0, c->bz0, s);
  CK(c, cudaGetLastError());
  c->have_beta = true;
  c->coefs_dirty = true;
  if (!all_set()) return GMG_OK;  // built once every AMR level's beta is set
  return build_coefs(c);
}

gmg_status gmg_set_bcoef_face(gmg_ctx* c, int lev, const double* bx, const double* by, const double* bz) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if (lev != 0 || !bx || !by || !bz) SETERR(c, GMG_ERR_BAD_INPUT, "beta faces: only level 0, non-null");
  const size_t n = 8 * (size_t)c->L[0].nelem;
  CK(c, cudaMemcpyAsync(c->bx0, bx, n, cudaMemcpyDeviceToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->by0, by, n, cudaMemcpyDeviceToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->bz0, bz, n, cudaMemcpyDeviceToDevice, c->stream));
  c->have_beta = true;
  c->coefs_dirty = true;
  return build_coefs(c);
}

gmg_status gmg_get_coeffs(gmg_ctx* c, int m, int dt, void* wx, void* wy, void* wz, void* diag) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if ((st = build_coefs(c))) return st;
  const int64_t n = c->L[m].nelem;
  const int src = (dt == DT_F64) ? DT_F64 : DT_F32;
  const Coefs k = coefs_of(c, m, src);
  if (wx) launch_convert(src, dt, k.wx, wx, n, c->stream);
  if (wy) launch_convert(src, dt, k.wy, wy, n, c->stream);
  if (wz) launch_convert(src, dt, k.wz, wz, n, c->stream);
  if (diag) launch_convert(src, dt, k.D, diag, n, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_workspace_size(const gmg_ctx* cc, const gmg_params* p, size_t* bytes) {
  gmg_ctx* c = (gmg_ctx*)cc;
  if (!c || !bytes) return GMG_ERR_BAD_INPUT;
  if (c->L.empty()) SETERR(c, GMG_ERR_STATE, "no BoxArray defined");
  const bool mixed = p && p->precision != GMG_FP64;
  // Krylov vectors: asked for, or needed by the adjoint solve of quadratic walls
  *bytes = carve(c, nullptr, mixed, false) + ((p && p->krylov) || any_quad(c) ? krylov_bytes(c) : 0);
  return GMG_OK;
}

gmg_status gmg_set_workspace(gmg_ctx* c, void* dptr, size_t bytes) {
  if (!c) return GMG_ERR_BAD_INPUT;
  if (c->L.empty()) SETERR(c, GMG_ERR_STATE, "no BoxArray defined");
  if (!dptr || ((uintptr_t)dptr & 255)) SETERR(c, GMG_ERR_BAD_INPUT, "workspace must be non-null and 256-byte aligned");
  const size_t need64 = carve(c, nullptr, false, false);
  const size_t needmx = carve(c, nullptr, true, false);
  const size_t kb = krylov_bytes(c);
  // the sizes gmg_workspace_size gives, largest first: mixed with the Krylov vectors, FP64
  // with them (when that is more than mixed alone), mixed, FP64
  bool mixed;
  if (bytes >= needmx + kb) mixed = true;
  else if (needmx < need64 + kb && bytes >= need64 + kb) mixed = false;
  else if (bytes >= needmx) mixed = true;
  else if (bytes >= need64) mixed = false;
  else SETERR(c, GMG_ERR_NO_WORKSPACE, "workspace too small");
  drop_graphs(c);
  if (!c->cap_stream) CK(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  if (!c->side_stream && c->ns() > 1) {
    CK(c, cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
    c->ev_fork.assign(nlev(c), nullptr);
    c->ev_join.assign(nlev(c), nullptr);
    for (int m = 0; m < nlev(c); ++m) {
      CK(c, cudaEventCreateWithFlags(&c->ev_fork[m], cudaEventDisableTiming));
      CK(c, cudaEventCreateWithFlags(&c->ev_join[m], cudaEventDisableTiming));
    }
  }
  gmg_status st = ensure_pinned(c);
  if (st) return st;
  c->ws = dptr;
  c->ws_bytes = bytes;
  c->mixed = mixed;
  const size_t used = carve(c, dptr, mixed, true);
  // the Krylov vectors, if the workspace holds them after the rest
  const size_t ne0 = (size_t)c->L[0].nelem;
  const bool kr = bytes >= used + kb;
  // the V-cycle outputs y (5) and z (8) are read with their ghosts (plain placement); the
  // others start their rows' valid cells on a 128-byte line (see Carver::take_rows)
  const size_t stride = (((8 * ne0) + 255) & ~(size_t)255) + 256;
  for (int q = 0; q < gmg_ctx::NKV; ++q)
    c->kv[q] = kr ? (double*)((char*)dptr + ((used + 255) & ~(size_t)255) + (size_t)q * stride +
                              ((q == 5 || q == 8) ? 0 : 64))
                  : nullptr;
  CK(c, cudaMemsetAsync(c->ws, 0, c->ws_bytes, c->stream));
  st = upload_tables(c);
  if (st) return st;
  c->have_beta = c->have_alpha = false;
  c->coefs_dirty = true;
  return GMG_OK;
}

gmg_status gmg_fill_boundary(gmg_ctx* c, int m, int dt, void* f, int colour) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if (colour < -1 || colour > 1) SETERR(c, GMG_ERR_BAD_INPUT, "colour must be -1, 0 or 1");
  launch_fill(dt, c->dev[m], f, colour, 0, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_smooth(gmg_ctx* c, int m, int dt, void* phi, const void* rhs, int colour) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if (colour < 0 || colour > 1) SETERR(c, GMG_ERR_BAD_INPUT, "colour must be 0 or 1");
  if ((st = build_coefs(c))) return st;
  // the smoother's work list skips bottom boxes; a single step smooths every box
  LevelDev D = c->dev[m];
  D.pair_chunks = D.pair_all_chunks;
  D.n_pair_chunks = D.n_pair_all_chunks;
  launch_fill(dt, D, phi, 1 - colour, 0, c->stream);
  launch_smooth(dt, D, phi, rhs, coefs_of(c, m, dt), colour, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_residual(gmg_ctx* c, int m, int dt, void* phi, const void* rhs, int rdt, void* r, double* norm) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if (rdt < 0 || rdt >= NDT) SETERR(c, GMG_ERR_BAD_INPUT, "bad residual type");
  if (dt != DT_F64 && rdt == DT_F64) SETERR(c, GMG_ERR_BAD_INPUT, "a float residual pass cannot write double");
  if ((st = build_coefs(c))) return st;
  cudaStream_t s = c->stream;
  const int ns = c->ns();
  launch_fill(dt, c->dev[m], phi, -1, 0, s);
  unsigned long long* nb = c->normbits + ns;  // per-problem slots; the maximum is taken here
  CK(c, cudaMemsetAsync(nb, 0, 8 * (size_t)ns, s));
  launch_residual(dt, rdt, c->dev[m], phi, rhs, coefs_of(c, m, dt), r, norm ? nb : nullptr, nullptr, s);
  CK(c, cudaGetLastError());
  if (norm) {
    CK(c, cudaMemcpyAsync(c->h_bits + ns, nb, 8 * (size_t)ns, cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    double v = 0.0;
    for (int q = 0; q < ns; ++q) v = std::max(v, bits_to_double(c->h_bits[ns + q]));
    *norm = v;
  }
  return GMG_OK;
}

gmg_status gmg_restrict(gmg_ctx* c, int m, int dt, const void* fine, void* coarse) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if (m + 1 >= nlev(c)) SETERR(c, GMG_ERR_BAD_INPUT, "no coarser level");
  launch_restrict(dt, c->dev[m], c->dev[m + 1], fine, coarse, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_prolong_add(gmg_ctx* c, int m, int dt, const void* coarse, void* fine) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if (m + 1 >= nlev(c)) SETERR(c, GMG_ERR_BAD_INPUT, "no coarser level");
  launch_prolong_add(dt, c->dev[m], c->dev[m + 1], coarse, fine, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_prolong_add_trilinear(gmg_ctx* c, int m, int dt, void* coarse, void* fine) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, m, dt);
  if (st) return st;
  if (m + 1 >= nlev(c)) SETERR(c, GMG_ERR_BAD_INPUT, "no coarser level");
  launch_fill(dt, c->dev[m + 1], coarse, -1, 0, c->stream);
  launch_fill_ec(dt, c->dev[m + 1], coarse, c->stream);
  launch_prolong_tri(dt, c->dev[m], c->dev[m + 1], coarse, fine, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_bottom_solve(gmg_ctx* c, int dt, const void* rhs, void* x, const gmg_params* pp, int* iters) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_params p;
  gmg_default_params(&p);
  if (pp) p = *pp;
  gmg_status st = check_level(c, 0, dt);
  if (st) return st;
  if ((st = build_coefs(c))) return st;
  if (c->ns() != 1) SETERR(c, GMG_ERR_BAD_INPUT, "gmg_bottom_solve needs a single-problem context");
  const int m = nlev(c) - 1;
  BottomArgs a{p.bottom_max_iter, p.bottom_tol, c->buf[m].bot_work, c->bot_iters, p.bottom_solver};
  launch_bottom(dt, c->dev[m], rhs, x, coefs64(c, m), a, c->stream);
  CK(c, cudaGetLastError());
  if (iters) {
    CK(c, cudaMemcpyAsync(c->h_iters, c->bot_iters, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *iters = c->h_iters[0];
  }
  return GMG_OK;
}

gmg_status gmg_autotune(gmg_ctx* c, int precision, const void* rhs, const gmg_params* pp) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_params p;
  gmg_default_params(&p);
  if (pp) p = *pp;
  gmg_status st;
  if ((st = params_ok(c, p))) return st;
  if ((st = ensure_flow_lag(c, p))) return st;
  const int dt = dt_of_precision(precision);
  if ((st = check_level(c, 0, dt))) return st;
  if (!rhs) SETERR(c, GMG_ERR_BAD_INPUT, "autotune needs a level-0 right-hand side");
  if ((st = build_coefs(c))) return st;
  drop_graphs(c);
  cudaStream_t s = c->stream;
  const int n = nlev(c);
  const int reps = 5;
  // a realistic level-0 correction equation: r = rhs (its mean removed for singular problems
  // does not matter for timing), and one V-cycle to populate every level's r
  launch_to_rhs(dt, c->dev[0], (const double*)rhs, c->buf[0].r[dt], s);
  gmg_params q = p;
  q.fused_coarse = 1;
  q.ghost_push = 0;
  q.fused_sweep = 0;
  vcycle(c, dt, 0, q, s);
  // per level, a red-black sweep (two colour passes) four ways on the level's own buffers:
  // ghost exchange or push, one thread per cell pair or per 4 cells (float / bfloat16)
  c->push_choice[dt].assign(n, -1);
  c->tune_ms_push[dt].assign(n, 0.0);
  c->tune_ms_pull[dt].assign(n, 0.0);
  for (int m = 0; m < n; ++m) {
    const LevelDev& D = c->dev[m];
    if (D.n_pair_chunks == 0) continue;
    const LevelBufs& B = c->buf[m];
    const Coefs k = coefs_of(c, m, dt);
    // (4-cell threads for float / bfloat16; 128-bit pair loads for double)
    const bool can_vec = dt == DT_F64 || (D.quad_chunks && D.n_quad_chunks > 0);
    double best = 1e30;
    int best_v = 0;
    double best_push = 1e30, best_pull = 1e30;
    for (int v = 0; v < 4; ++v) {
      const bool push = v & 1, vec = (v & 2) != 0;
      if ((push && !D.push_ok) || (vec && !can_vec)) continue;
      const double ms = time_reps(c, reps, [&] {
        for (int colour = 0; colour < 2; ++colour) {
          if (!push) launch_fill(dt, D, B.e[dt], 1 - colour, 0, s);
          launch_smooth(dt, D, B.e[dt], B.r[dt], k, colour, s, push, vec, true);
        }
      });
      if (push) best_push = std::min(best_push, ms);
      else best_pull = std::min(best_pull, ms);
      // (the vector-load variants must win by 2%: on launch-bound levels the order is noise)
      if (vec ? ms < 0.98 * best : ms < best) {
        best = ms;
        best_v = v;
      }
    }
    c->tune_ms_pull[dt][m] = best_pull;
    c->tune_ms_push[dt][m] = best_push < 1e30 ? best_push : 0.0;
    c->push_choice[dt][m] = (signed char)best_v;
  }
  // fused coarse end vs per-level launches, whole V-cycles with the choices above
  q.ghost_push = 2;
  for (int f = 0; f < 2; ++f) {
    q.fused_coarse = f;
    c->tune_ms_tail[dt][f] = time_reps(c, reps, [&] { vcycle(c, dt, 0, q, s); });
  }
  c->tail_choice[dt] = c->tune_ms_tail[dt][1] <= c->tune_ms_tail[dt][0] ? 1 : 0;
  CK(c, cudaStreamSynchronize(s));
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_tuned(const gmg_ctx* c, int precision, int m, int* push, double* ms_push, double* ms_pull,
                     int* fused_coarse, double* ms_vcycle_fused, double* ms_vcycle_levels) {
  if (!c) return GMG_ERR_BAD_INPUT;
  const int dt = dt_of_precision(precision);
  if (dt < 0 || dt >= NDT || m < 0 || m >= (int)c->L.size()) return GMG_ERR_BAD_INPUT;
  const auto& ch = c->push_choice[dt];
  if (push) *push = m < (int)ch.size() ? ch[m] : -1;  // bit 0: push, bit 1: 4-cell threads
  if (ms_push) *ms_push = m < (int)c->tune_ms_push[dt].size() ? c->tune_ms_push[dt][m] : 0.0;
  if (ms_pull) *ms_pull = m < (int)c->tune_ms_pull[dt].size() ? c->tune_ms_pull[dt][m] : 0.0;
  if (fused_coarse) *fused_coarse = c->tail_choice[dt];
  if (ms_vcycle_fused) *ms_vcycle_fused = c->tune_ms_tail[dt][1];
  if (ms_vcycle_levels) *ms_vcycle_levels = c->tune_ms_tail[dt][0];
  return GMG_OK;
}

gmg_status gmg_vcycle(gmg_ctx* c, int dt, void* e, const void* r, const gmg_params* pp) {
  if (!c) return GMG_ERR_BAD_INPUT;
  gmg_params p;
  gmg_default_params(&p);
  if (pp) p = *pp;
  gmg_status st = check_level(c, 0, dt);
  if (st) return st;
  if ((st = build_coefs(c))) return st;
  if ((st = ensure_flow_lag(c, p))) return st;
  const size_t n = dt_size(dt) * (size_t)c->L[0].nelem;
  launch_copy_to_rhs(dt, c->dev[0], r, c->buf[0].r[dt], c->stream);
  vcycle(c, dt, 0, p, c->stream);
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(e, c->buf[0].e[dt], n, cudaMemcpyDeviceToDevice, c->stream));
  return take_dev_err(c, c->stream);
}

gmg_status gmg_apply(gmg_ctx* c, void* const* out, void* const* phi) {
  if (!c || !out || !phi || !out[0] || !phi[0]) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if ((st = build_coefs(c))) return st;
  cudaStream_t s = c->stream;
  if (c->amr) {
    double *x[GMG_MAX_AMR_LEVELS], *y[GMG_MAX_AMR_LEVELS];
    for (int l = 0; l < namr(c); ++l) {
      if (!out[l] || !phi[l]) SETERR(c, GMG_ERR_BAD_INPUT, "composite context: pass an array for every AMR level");
      x[l] = (double*)phi[l];
      y[l] = (double*)out[l];
    }
    comp_apply_n(c, x, y, s);
    CK(c, cudaGetLastError());
    return GMG_OK;
  }
  // out = -(0 - A phi): the residual pass with a zero right-hand side, negated
  launch_fill(DT_F64, c->dev[0], phi[0], -1, 0, s);
  CK(c, cudaMemsetAsync(c->tmp0, 0, 8 * (size_t)c->L[0].nelem, s));
  launch_residual(DT_F64, DT_F64, c->dev[0], phi[0], c->tmp0, coefs64(c, 0), out[0], nullptr, nullptr, s);
  launch_scale_valid(c->dev[0], (double*)out[0], -1.0, s);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_solve(gmg_ctx* c, void* const* phiv, const void* const* rhsv, double tol_rel, double tol_abs,
                     const gmg_params* pp, gmg_solve_info* info) {
  if (!c || !phiv || !rhsv || !phiv[0] || !rhsv[0]) return GMG_ERR_BAD_INPUT;
  gmg_params p;
  gmg_default_params(&p);
  if (pp) p = *pp;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if (c->ns() != 1) SETERR(c, GMG_ERR_BAD_INPUT, "context holds several problems: use gmg_batch_solve");
  if ((st = params_ok(c, p))) return st;
  if ((st = ensure_flow_lag(c, p))) return st;
  if ((st = build_coefs(c))) return st;
  if (c->amr) {
    double* x[GMG_MAX_AMR_LEVELS];
    const double* b[GMG_MAX_AMR_LEVELS];
    for (int l = 0; l < namr(c); ++l) {
      if (!phiv[l] || !rhsv[l]) SETERR(c, GMG_ERR_BAD_INPUT, "composite context: pass arrays for every AMR level");
      x[l] = (double*)phiv[l];
      b[l] = (const double*)rhsv[l];
    }
    if (p.precision != GMG_FP64) SETERR(c, GMG_ERR_BAD_INPUT, "the composite solve runs in FP64");
    if (p.krylov) SETERR(c, GMG_ERR_BAD_INPUT, "krylov: one-level contexts only");
    return solve_amr_n(c, x, b, tol_rel, tol_abs, p, info);
  }
  if (p.krylov) return krylov_solve(c, (double*)phiv[0], (const double*)rhsv[0], tol_rel, tol_abs, p, info);
  return solve_impl(c, (double*)phiv[0], (const double*)rhsv[0], tol_rel, tol_abs, p, info);
}

gmg_status gmg_batch_solve(gmg_ctx* c, void* phi, const void* rhs, double tol_rel, double tol_abs,
                           const gmg_params* pp, gmg_solve_info* infos) {
  if (!c || !phi || !rhs) return GMG_ERR_BAD_INPUT;
  gmg_params p;
  gmg_default_params(&p);
  if (pp) p = *pp;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if ((st = params_ok(c, p))) return st;
  if ((st = ensure_flow_lag(c, p))) return st;
  if ((st = build_coefs(c))) return st;
  return solve_impl(c, (double*)phi, (const double*)rhs, tol_rel, tol_abs, p, infos);
}

gmg_status gmg_apply_transpose(gmg_ctx* c, void* const* out, void* const* y) {
  if (!c || !out || !y || !out[0] || !y[0]) return GMG_ERR_BAD_INPUT;
  if (!c->amr && !any_quad(c)) return gmg_apply(c, out, y);  // one level, linear walls: A is symmetric
  if (!c->amr) {
    gmg_status st = check_level(c, 0, DT_F64);
    if (st) return st;
    if (c->ns() != 1) SETERR(c, GMG_ERR_BAD_INPUT, "transpose with quadratic walls: single-problem contexts only");
    if ((st = build_coefs(c))) return st;
    apply_transpose_one(c, (double*)y[0], (double*)out[0], c->stream);
    CK(c, cudaGetLastError());
    return GMG_OK;
  }
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if ((st = build_coefs(c))) return st;
  double *yy[GMG_MAX_AMR_LEVELS], *oo[GMG_MAX_AMR_LEVELS];
  for (int l = 0; l < namr(c); ++l) {
    if (!out[l] || !y[l]) SETERR(c, GMG_ERR_BAD_INPUT, "composite context: pass arrays for every AMR level");
    yy[l] = (double*)y[l];
    oo[l] = (double*)out[l];
  }
  if ((st = adjoint_layout_ok(c))) return st;
  comp_apply_transpose_n(c, yy, oo, c->stream);
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_solve_adjoint(gmg_ctx* c, void* const* lambda, const void* const* g, double tol_rel,
                             const gmg_params* pp, gmg_solve_info* info) {
  if (!c || !lambda || !g || !lambda[0] || !g[0]) return GMG_ERR_BAD_INPUT;
  gmg_params p;
  gmg_default_params(&p);
  if (pp) p = *pp;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if (c->ns() != 1) SETERR(c, GMG_ERR_BAD_INPUT, "adjoint: single-problem contexts only");
  if ((st = params_ok(c, p))) return st;
  if ((st = ensure_flow_lag(c, p))) return st;
  if ((st = build_coefs(c))) return st;
  if (!c->amr && any_quad(c)) {  // non-symmetric operator: BiCGStab on A^T
    p.krylov = 1;
    return krylov_solve(c, (double*)lambda[0], (const double*)g[0], tol_rel, 0.0, p, info, true);
  }
  if (!c->amr) {  // symmetric operator: the adjoint solve is a forward solve (mean projected)
    p.project_mean = 1;
    return solve_impl(c, (double*)lambda[0], (const double*)g[0], tol_rel, 0.0, p, info);
  }
  double* lam[GMG_MAX_AMR_LEVELS];
  const double* gg[GMG_MAX_AMR_LEVELS];
  for (int l = 0; l < namr(c); ++l) {
    if (!lambda[l] || !g[l]) SETERR(c, GMG_ERR_BAD_INPUT, "composite context: pass arrays for every AMR level");
    lam[l] = (double*)lambda[l];
    gg[l] = (const double*)g[l];
  }
  if ((st = adjoint_layout_ok(c))) return st;
  p.precision = GMG_FP64;
  return solve_adjoint_amr_n(c, lam, gg, tol_rel, p, info);
}

gmg_status gmg_beta_grad(gmg_ctx* c, void* const* dbeta, void* const* phi, void* const* lambda) {
  return gmg_beta_grad_walls(c, dbeta, phi, lambda, nullptr);
}

gmg_status gmg_beta_grad_walls(gmg_ctx* c, void* const* dbeta, void* const* phi, void* const* lambda,
                               const void* const* values) {
  if (!c || !dbeta || !phi || !lambda || !dbeta[0] || !phi[0] || !lambda[0]) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if ((st = build_coefs(c))) return st;
  if (c->ns() != 1) SETERR(c, GMG_ERR_BAD_INPUT, "beta gradient: single-problem contexts only");
  if (values && (st = wall_values_check(c, values))) return st;
  cudaStream_t s = c->stream;
  double* pc = (double*)phi[0];
  double* lc = (double*)lambda[0];
  if (c->amr) {
    // level l's faces: its own rows, the reflux rows of level l - 1 on its coarse/fine faces
    // (lambda of level l - 1), none under level l + 1 (covered cells: 0)
    const int L = namr(c);
    double *ph[GMG_MAX_AMR_LEVELS], *la[GMG_MAX_AMR_LEVELS];
    for (int l = 0; l < L; ++l) {
      if (!dbeta[l] || !phi[l] || !lambda[l]) SETERR(c, GMG_ERR_BAD_INPUT, "composite context: pass every AMR level");
      ph[l] = (double*)phi[l];
      la[l] = (double*)lambda[l];
    }
    if ((st = adjoint_layout_ok(c))) return st;
    for (int l = 0; l + 1 < L; ++l) launch_zero_covered(c->amrl[l].A, la[l], s);
    for (int l = L - 1; l >= 1; --l) {
      level_fill(c, l, ph[l], ph[l - 1], CF_INTERP, s);
      launch_fill(DT_F64, adev(c, l), la[l], -1, 0, s);
    }
    launch_fill(DT_F64, c->dev[0], pc, -1, 0, s);
    launch_fill(DT_F64, c->dev[0], lc, -1, 0, s);
    for (int l = L - 1; l >= 0; --l) {
      const AmrDev* below = l > 0 ? &c->amrl[l - 1].A : nullptr;  // pair (l - 1, l)
      const AmrDev* above = l + 1 < L ? &c->amrl[l].A : nullptr;  // pair (l, l + 1)
      launch_grad_beta(adev(c, l), ph[l], la[l], l == 0 ? c->betac_cell : c->amrl[l - 1].beta_cell, c->b,
                       below ? below->cfidx : nullptr, below ? below->cf : nullptr, l > 0 ? la[l - 1] : nullptr,
                       below ? below->hf_over_hc : 0.5, above ? above->covered : nullptr, (double*)dbeta[l], s);
    }
  } else {
    launch_fill(DT_F64, c->dev[0], pc, -1, 0, s);
    launch_fill(DT_F64, c->dev[0], lc, -1, 0, s);
    if (values && (st = wall_values_pass(c, values, 1, pc, nullptr, nullptr))) return st;
    launch_grad_beta(c->dev[0], pc, lc, c->betac_cell, c->b, nullptr, nullptr, nullptr, 0.5, nullptr,
                     (double*)dbeta[0], s);
  }
  CK(c, cudaGetLastError());
  return GMG_OK;
}

gmg_status gmg_wall_values_rhs(gmg_ctx* c, void* out, const void* rhs, const void* const* values) {
  if (!c || !out || !rhs || !values) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if ((st = build_coefs(c))) return st;
  if ((st = wall_values_check(c, values))) return st;
  if (out != rhs)
    CK(c, cudaMemcpyAsync(out, rhs, 8 * (size_t)c->L[0].nelem, cudaMemcpyDeviceToDevice, c->stream));
  return wall_values_pass(c, values, 0, (double*)out, nullptr, nullptr);
}

gmg_status gmg_wall_values_grad(gmg_ctx* c, const void* lambda, void* const* dvalues) {
  if (!c || !lambda || !dvalues) return GMG_ERR_BAD_INPUT;
  gmg_status st = check_level(c, 0, DT_F64);
  if (st) return st;
  if ((st = build_coefs(c))) return st;
  if ((st = wall_values_check(c, (const void* const*)dvalues))) return st;
  return wall_values_pass(c, (const void* const*)dvalues, 2, nullptr, (const double*)lambda, dvalues);
}

}  // extern "C"
