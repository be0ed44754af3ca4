// meta.cpp -- multigrid hierarchy and cached exchange tables (host).
#include "meta.h"

#include <algorithm>
#include <map>
#include <tuple>
#include <cstdio>
#include <functional>

namespace gmg {

Box intersect(const Box& a, const Box& b) {
  Box r;
  for (int d = 0; d < 3; ++d) {
    r.lo[d] = std::max(a.lo[d], b.lo[d]);
    r.hi[d] = std::min(a.hi[d], b.hi[d]);
  }
  return r;
}

Box shifted(const Box& a, int d, int s) {
  Box r = a;
  r.lo[d] += s;
  r.hi[d] += s;
  return r;
}

static int pmod2(int a) { return ((a % 2) + 2) % 2; }

std::string validate_boxes(const std::vector<Box>& boxes, const Box& domain, bool must_cover) {
  int64_t vol = 0;
  for (size_t b = 0; b < boxes.size(); ++b) {
    const Box& B = boxes[b];
    if (B.empty()) return "empty box " + std::to_string(b);
    for (int d = 0; d < 3; ++d)
      if (B.lo[d] < domain.lo[d] || B.hi[d] > domain.hi[d]) return "box " + std::to_string(b) + " outside the domain";
    vol += B.volume();
  }
  // pairwise disjointness: sort by lo.x and sweep
  std::vector<int> idx(boxes.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return boxes[a].lo[0] < boxes[b].lo[0]; });
  for (size_t a = 0; a < idx.size(); ++a)
    for (size_t b = a + 1; b < idx.size(); ++b) {
      if (boxes[idx[b]].lo[0] > boxes[idx[a]].hi[0]) break;
      if (!intersect(boxes[idx[a]], boxes[idx[b]]).empty())
        return "boxes " + std::to_string(idx[a]) + " and " + std::to_string(idx[b]) + " overlap";
    }
  if (must_cover && vol != domain.volume()) return "boxes do not cover the domain";
  return "";
}

std::vector<Box> chop(const Box& dom, int mgs) {
  std::vector<std::pair<int, int>> cuts[3];
  for (int d = 0; d < 3; ++d)
    for (int s = dom.lo[d]; s <= dom.hi[d]; s += mgs) cuts[d].push_back({s, std::min(s + mgs - 1, dom.hi[d])});
  std::vector<Box> out;
  for (auto& z : cuts[2])
    for (auto& y : cuts[1])
      for (auto& x : cuts[0]) {
        Box b;
        b.lo[0] = x.first; b.hi[0] = x.second;
        b.lo[1] = y.first; b.hi[1] = y.second;
        b.lo[2] = z.first; b.hi[2] = z.second;
        out.push_back(b);
      }
  return out;
}

// Face ghost rectangles of every box (Sec. "Operations on a level").  For each face slab
// of each box, the slab is intersected with every box of the same solve (and with its
// periodic images along the face normal); the part outside a wall becomes a reflection
// rectangle: minus the adjacent interior value at a Dirichlet wall, plus it at a Neumann
// wall (the homogeneous wall rules; wall values enter the right-hand side).  Edge and corner ghosts are not needed by the 7-point stencil.
static std::string build_ghosts(LevelMeta& L) {
  L.ghosts.clear();
  L.cf_slabs.clear();
  const int nb = (int)L.boxes.size();
  // boxes per solve
  std::vector<std::vector<int>> members(L.geoms.size());
  for (int b = 0; b < nb; ++b) members[L.box_solve[b]].push_back(b);
  for (int b = 0; b < nb; ++b) {
    const Box& B = L.boxes[b];
    const SolveGeom& G = L.geoms[L.box_solve[b]];
    for (int d = 0; d < 3; ++d) {
      int d1 = (d == 0) ? 1 : 0;
      int d2 = (d == 2) ? 1 : 2;
      for (int side = 0; side < 2; ++side) {
        Box slab = B;
        int gd = side ? B.hi[d] + 1 : B.lo[d] - 1;
        slab.lo[d] = slab.hi[d] = gd;
        bool outside = gd < G.domain.lo[d] || gd > G.domain.hi[d];
        int bc = side ? G.bchi[d] : G.bclo[d];
        if (outside && bc != 0) {
          GhostRect r{};
          r.dst_box = r.src_box = b;
          for (int q = 0; q < 3; ++q) r.dst[q] = r.src[q] = 0;
          r.dst[d] = side ? B.n(d) : -1;
          r.src[d] = side ? B.n(d) - 1 : 0;
          r.d1 = d1; r.d2 = d2;
          r.n1 = B.n(d1); r.n2 = B.n(d2);
          r.sign = bc == 2 ? 1 : -1;
          r.par0 = pmod2(B.lo[0] + B.lo[1] + B.lo[2] + r.dst[0] + r.dst[1] + r.dst[2]);
          r.kind = 1;
          if (bc == 1 && (side ? G.qhi[d] : G.qlo[d]) && B.n(d) >= 2) {
            // quadratic rule: ghost = -2 phi_0 + phi_1 / 3; the rectangle fills phi_1 / 3 and
            // the diagonal takes the -2 phi_0 part (so the ghost holds no value of the cell
            // next to it, and the row of that cell stays exact under Gauss-Seidel)
            r.src[d] = side ? B.n(d) - 2 : 1;
            r.sign = 1;
            r.kind = 2;
          }
          L.ghosts.push_back(r);
          continue;
        }
        int64_t covered = 0;
        int len = G.domain.n(d);
        int shifts[3] = {0, 0, 0};
        int nsh = 1;
        if (G.periodic(d)) { shifts[1] = len; shifts[2] = -len; nsh = 3; }
        for (int ob : members[L.box_solve[b]]) {
          for (int s = 0; s < nsh; ++s) {
            Box img = shifted(L.boxes[ob], d, shifts[s]);
            Box I = intersect(slab, img);
            if (I.empty()) continue;
            GhostRect r{};
            r.dst_box = b;
            r.src_box = ob;
            for (int q = 0; q < 3; ++q) {
              r.dst[q] = I.lo[q] - B.lo[q];
              r.src[q] = I.lo[q] - img.lo[q];
            }
            r.d1 = d1; r.d2 = d2;
            r.n1 = I.n(d1); r.n2 = I.n(d2);
            r.sign = 1;
            r.par0 = pmod2(I.lo[0] + I.lo[1] + I.lo[2]);
            r.kind = 0;
            L.ghosts.push_back(r);
            covered += I.volume();
          }
        }
        if (covered != slab.volume()) {
          if (L.allow_cf && covered == 0) {  // a whole face on the coarse/fine boundary
            L.cf_slabs.push_back({b, d, side});
            continue;
          }
          return "ghost cells of box " + std::to_string(b) +
                 (L.allow_cf ? " are partly covered by other boxes of the level (not supported)"
                             : " are not covered by the level (coarse/fine boundary)");
        }
      }
    }
  }
  L.ghost_chunks.clear();
  for (int g = 0; g < (int)L.ghosts.size(); ++g) {
    int n = L.ghosts[g].n1 * L.ghosts[g].n2;
    for (int s = 0; s < n; s += GHOST_CHUNK) L.ghost_chunks.push_back({g, s});
  }
  return "";
}

static void build_bottom(LevelMeta& L) {
  L.bot_cells.clear();
  L.bot_ghosts.clear();
  L.bot_descs.clear();
  for (int s = 0; s < (int)L.geoms.size(); ++s) {
    if (!L.solve_present[s] || !L.solve_bottom[s]) continue;
    BotDesc D{};
    D.cell0 = (int)L.bot_cells.size();
    D.ghost0 = (int)L.bot_ghosts.size();
    D.solve = s;
    for (int b = 0; b < (int)L.boxes.size(); ++b) {
      if (L.box_solve[b] != s) continue;
      const DevBox& B = L.dbox[b];
      for (int k = 0; k < B.nz; ++k)
        for (int j = 0; j < B.ny; ++j)
          for (int i = 0; i < B.nx; ++i) L.bot_cells.push_back({elem_index(B, i, j, k), B.sy, B.sx, 0});
    }
    for (const GhostRect& g : L.ghosts) {
      if (L.box_solve[g.dst_box] != s) continue;
      const DevBox& Bd = L.dbox[g.dst_box];
      const DevBox& Bs = L.dbox[g.src_box];
      for (int v = 0; v < g.n2; ++v)
        for (int u = 0; u < g.n1; ++u) {
          int dl[3] = {g.dst[0], g.dst[1], g.dst[2]};
          int sl[3] = {g.src[0], g.src[1], g.src[2]};
          dl[g.d1] += u; dl[g.d2] += v;
          sl[g.d1] += u; sl[g.d2] += v;
          L.bot_ghosts.push_back({elem_index(Bd, dl[0], dl[1], dl[2]), elem_index(Bs, sl[0], sl[1], sl[2]), ghost_factor(g)});
        }
    }
    D.ncell = (int)L.bot_cells.size() - D.cell0;
    D.nghost = (int)L.bot_ghosts.size() - D.ghost0;
    D.singular = 0;  // set from the operator's scalars at coefficient time
    L.bot_descs.push_back(D);
  }
}

// Tables of the dataflow sweep (flow.cu).  Per independent problem the level's z extent is
// cut into slabs of whole planes (about FLOW_SLAB_CELLS cells, 1 to 16 planes); every
// smoothed box is cut into items of its full x extent and about FLOW_ITEM_CELLS cells
// (a range of rows of one plane, or whole planes), inside the planes it shares with one slab.  An item of phase c waits for phase
// c - 1 in slabs s - 1, s, s + 1 (periodic in z where the problem is): a colour phase on
// planes Q reads the other colour on planes Q - 1, Q and Q + 1 (the 7-point stencil), as the
// previous phase left them, and overwrites values that the previous phase read there.
static void build_flow(LevelMeta& L) {
  L.flow_items.clear();
  L.flow_slabs.clear();
  for (auto& o : L.flow_order) o.clear();
  L.vc_flow_skip.assign(L.geoms.size(), 0);
  if (L.allow_cf || !L.push_ok) return;
  const int nb = (int)L.boxes.size();
  const int ns = (int)L.geoms.size();
  int64_t cells = 0;
  for (int b = 0; b < nb; ++b)
    if (!L.solve_bottom[L.box_solve[b]]) cells += L.boxes[b].volume();
  if (cells < FLOW_MIN_CELLS) return;
  std::vector<FlowItem> items;
  std::vector<FlowSlab> slabs;
  for (int q = 0; q < ns; ++q) {
    if (!L.solve_present[q] || L.solve_bottom[q]) continue;
    const Box& dom = L.geoms[q].domain;
    const int nzd = dom.n(2);
    const int64_t area = (int64_t)dom.n(0) * dom.n(1);
    const int planes = (int)std::max<int64_t>(1, std::min<int64_t>(16, FLOW_SLAB_CELLS / std::max<int64_t>(1, area)));
    const int nsl = (nzd + planes - 1) / planes;
    const int base = (int)slabs.size();
    for (int sl = 0; sl < nsl; ++sl) {
      FlowSlab S{};
      S.first = (int)items.size();
      S.solve = q;
      const int g0 = dom.lo[2] + sl * planes, g1 = std::min(g0 + planes, dom.lo[2] + nzd);
      for (int b = 0; b < nb; ++b) {
        if (L.box_solve[b] != q) continue;
        const Box& B = L.boxes[b];
        const int z0 = std::max(g0, B.lo[2]) - B.lo[2], z1 = std::min(g1, B.hi[2] + 1) - B.lo[2];
        if (z1 <= z0) continue;
        const int nx = B.n(0), ny = B.n(1);
        if (nx * ny >= FLOW_ITEM_CELLS) {  // items of one plane and a range of rows
          const int rows = std::max(1, FLOW_ITEM_CELLS / nx);
          for (int z = z0; z < z1; ++z)
            for (int y0 = 0; y0 < ny; y0 += rows) items.push_back({b, base + sl, z, z + 1, y0, std::min(ny, y0 + rows)});
        } else {  // items of whole planes
          const int np = std::max(1, FLOW_ITEM_CELLS / (nx * ny));
          for (int z = z0; z < z1; z += np) items.push_back({b, base + sl, z, std::min(z1, z + np), 0, ny});
        }
      }
      S.count = (int)items.size() - S.first;
      int k = 0;
      for (int d = -1; d <= 1; ++d) {
        int t = sl + d;
        if (t < 0 || t >= nsl) {
          if (!L.geoms[q].periodic(2)) continue;
          t = (t + nsl) % nsl;
        }
        bool dup = false;
        for (int u = 0; u < k; ++u) dup |= S.dep[u] == base + t;
        if (!dup) S.dep[k++] = base + t;
      }
      for (; k < 3; ++k) S.dep[k] = -1;
      slabs.push_back(S);
    }
  }
  if (items.empty() || slabs.size() >= (1u << 24)) return;
  L.flow_items = items;
  L.flow_slabs = slabs;
  build_flow_order(L, FLOW_LAG_CELLS);
}

static int g_wave_capacity = 8 * 152;
void set_wave_capacity(int blocks) { g_wave_capacity = std::max(1, blocks); }
int wave_capacity() { return g_wave_capacity; }

// Wavefront tables.  Face f = 2 d + side of box b is described by its one ghost rectangle:
// a wall, or a copy from box Y whose face matches b's (same extents and offsets across the
// face, so b's row bands and planes are Y's).  Marching directions come from a union-find
// with parity over the boxes (x and y neighbours: same direction; z neighbours: opposite);
// a contradiction -- an odd number of boxes around a periodic z, one box periodic in z --
// leaves the level without tables.
void build_wave(LevelMeta& L, int max_resident) {
  L.wave_tiles.clear();
  L.wave_ppt = 0;
  L.wave_max_solve_tiles = 0;
  L.wave_layer_cells = 0;
  if (L.allow_cf || !L.push_ok) return;
  const int nb = (int)L.boxes.size();
  std::vector<char> sm(nb, 0);
  int max_npx = 0, max_ny = 1, nsm = 0;
  for (int b = 0; b < nb; ++b) {
    if (L.solve_bottom[L.box_solve[b]]) continue;
    const Box& B = L.boxes[b];
    if (B.n(0) % 2 != 0 || B.n(0) < 2 || B.n(2) > WAVE_MAX_PLANES) return;
    sm[b] = 1;
    ++nsm;
    max_npx = std::max(max_npx, B.n(0) / 2);
    max_ny = std::max(max_ny, B.n(1));
  }
  if (!nsm) return;
  struct Face {
    int count = 0, kind = -1, box = -1;
  };
  std::vector<Face> face((size_t)nb * 6);
  for (const GhostRect& g : L.ghosts) {
    const int X = g.dst_box;
    if (!sm[X]) continue;
    const int d = 3 - g.d1 - g.d2;
    const Box& BX = L.boxes[X];
    const int side = g.dst[d] < 0 ? 0 : 1;
    Face& F = face[(size_t)X * 6 + 2 * d + side];
    F.count++;
    F.kind = g.kind;
    F.box = g.src_box;
    if (g.kind == 2) return;
    if (g.n1 != BX.n(g.d1) || g.n2 != BX.n(g.d2) || g.dst[g.d1] != 0 || g.dst[g.d2] != 0) return;
    if (g.kind == 0) {
      const Box& BY = L.boxes[g.src_box];
      if (!sm[g.src_box] || g.src[g.d1] != 0 || g.src[g.d2] != 0 || BY.n(g.d1) != BX.n(g.d1) ||
          BY.n(g.d2) != BX.n(g.d2))
        return;
    }
  }
  for (int b = 0; b < nb; ++b)
    if (sm[b])
      for (int f = 0; f < 6; ++f)
        if (face[(size_t)b * 6 + f].count != 1) return;
  // marching directions
  std::vector<int> up(nb), rel(nb, 0);
  for (int b = 0; b < nb; ++b) up[b] = b;
  std::function<int(int)> find = [&](int x) {
    if (up[x] == x) return x;
    const int r = find(up[x]);
    rel[x] ^= rel[up[x]];
    up[x] = r;
    return r;
  };
  for (int b = 0; b < nb; ++b) {
    if (!sm[b]) continue;
    for (int f = 0; f < 6; ++f) {
      const Face& F = face[(size_t)b * 6 + f];
      if (F.kind != 0) continue;
      const int want = f >= 4 ? 1 : 0;  // z neighbours march the other way
      const int ra = find(b), rb = find(F.box);
      if (ra == rb) {
        if ((rel[b] ^ rel[F.box]) != want) return;
      } else {
        up[ra] = rb;
        rel[ra] = rel[b] ^ rel[F.box] ^ want;
      }
    }
  }
  std::vector<int> dir(nb, 0);
  for (int b = 0; b < nb; ++b)
    if (sm[b]) {
      find(b);
      dir[b] = rel[b];
    }
  // tile height: the fewest cell pairs per thread with every problem's tiles resident at once
  const int ns = (int)L.geoms.size();
  int ppt = 0, ty = 0, most = 0;
  for (int cand : {1, 2, 4}) {
    if (max_npx > WAVE_BLOCK * cand) continue;
    const int h = std::max(1, std::min(max_ny, WAVE_BLOCK * cand / max_npx));
    std::vector<int> per(ns, 0);
    for (int b = 0; b < nb; ++b)
      if (sm[b]) per[L.box_solve[b]] += (L.boxes[b].n(1) + h - 1) / h;
    const int mx = *std::max_element(per.begin(), per.end());
    if (mx <= max_resident) {
      ppt = cand;
      ty = h;
      most = mx;
      break;
    }
  }
  if (!ppt) return;
  std::vector<int> first(nb, -1), count(nb, 0);
  std::vector<WaveTile> tiles;
  for (int b = 0; b < nb; ++b) {  // (boxes are stored problem by problem)
    if (!sm[b]) continue;
    first[b] = (int)tiles.size();
    const int ny = L.boxes[b].n(1);
    for (int y0 = 0; y0 < ny; y0 += ty) {
      WaveTile t{};
      t.box = b;
      t.y0 = y0;
      t.y1 = std::min(ny, y0 + ty);
      t.dir = dir[b];
      t.solve = L.box_solve[b];
      tiles.push_back(t);
    }
    count[b] = (int)tiles.size() - first[b];
  }
  for (int b = 0; b < nb; ++b) {
    if (!sm[b]) continue;
    const int nzb = L.boxes[b].n(2);
    (void)nzb;
    for (int u = 0; u < count[b]; ++u) {
      WaveTile& t = tiles[first[b] + u];
      const Face* F = &face[(size_t)b * 6];
      for (int side = 0; side < 2; ++side)  // x: the band of the same rows in the neighbour
        t.nb[side] = F[side].kind == 0 ? first[F[side].box] + u : -1;
      t.nb[2] = u > 0 ? first[b] + u - 1 : (F[2].kind == 0 ? first[F[2].box] + count[F[2].box] - 1 : -1);
      t.nb[3] = u + 1 < count[b] ? first[b] + u + 1 : (F[3].kind == 0 ? first[F[3].box] : -1);
      for (int side = 0; side < 2; ++side) {
        const Face& G = F[4 + side];
        if (G.kind != 0) {
          t.zb[side] = -1;
          t.zneed[side] = 0;
          continue;
        }
        const int Y = G.box;
        t.zb[side] = first[Y] + u;
        const int nzy = L.boxes[Y].n(2);
        // the plane of Y next to this face: its last (z-) or first (z+) plane
        const bool y_last_plane = side == 0;
        const bool y_marches_up = dir[Y] == 0;
        t.zneed[side] = (y_last_plane == y_marches_up) ? nzy : 1;
      }
    }
  }
  L.wave_tiles = tiles;
  L.wave_ppt = ppt;
  L.wave_max_solve_tiles = most;
  L.wave_layer_cells = 0;
  for (int b = 0; b < nb; ++b)
    if (sm[b]) L.wave_layer_cells += (int64_t)L.boxes[b].n(0) * L.boxes[b].n(1);
}

// The dispense order: (phase, slab) groups sorted by a position tau, in cells of the whole
// level: tau(0, s) = the level's cells times the fraction of its problem's slabs up to and
// including s (every problem advances at the same pace), tau(c, s) = lag + the largest
// tau(c - 1, .) of the slabs it waits for.  Every item comes after the items it waits for.
void build_flow_order(LevelMeta& L, int64_t lag) {
  for (auto& o : L.flow_order) o.clear();
  const int nsl = (int)L.flow_slabs.size();
  if (!nsl) return;
  L.flow_lag = lag;
  int64_t total = 0;
  std::vector<int> nsl_of(L.geoms.size(), 0), first_of(L.geoms.size(), -1);
  for (int s = 0; s < nsl; ++s) {
    const FlowSlab& S = L.flow_slabs[s];
    if (first_of[S.solve] < 0) first_of[S.solve] = s;
    nsl_of[S.solve]++;
  }
  for (const FlowItem& it : L.flow_items) {
    const DevBox& B = L.dbox[it.box];
    total += (int64_t)B.nx * (it.y1 - it.y0) * (it.z1 - it.z0);
  }
  std::vector<double> tau(nsl), prev(nsl);
  for (int n = 1; n <= FLOW_MAX_PHASES; ++n) {
    struct G { double t; int c, s; };
    std::vector<G> groups;
    for (int s = 0; s < nsl; ++s) {
      const FlowSlab& S = L.flow_slabs[s];
      tau[s] = (double)total * (double)(s - first_of[S.solve] + 1) / (double)nsl_of[S.solve];
    }
    for (int c = 0; c < n; ++c) {
      if (c > 0) {
        prev = tau;
        for (int s = 0; s < nsl; ++s) {
          double m = 0;
          for (int u = 0; u < 3; ++u)
            if (L.flow_slabs[s].dep[u] >= 0) m = std::max(m, prev[L.flow_slabs[s].dep[u]]);
          tau[s] = m + (double)std::max<int64_t>(lag, 1);
        }
      }
      for (int s = 0; s < nsl; ++s) groups.push_back({tau[s], c, s});
    }
    std::stable_sort(groups.begin(), groups.end(), [](const G& x, const G& y) {
      return x.t != y.t ? x.t < y.t : (x.c != y.c ? x.c < y.c : x.s < y.s);
    });
    std::vector<FlowChunk>& o = L.flow_order[n - 1];
    for (const G& g : groups) {
      const FlowSlab& S = L.flow_slabs[g.s];
      for (int i = S.first; i < S.first + S.count; ++i) {
        const FlowItem& I = L.flow_items[i];
        o.push_back({(g.c << 24) | g.s, I.box, I.z0, I.z1, I.y0, I.y1});
      }
    }
  }
}

void build_ec_ghosts(LevelMeta& L) {
  L.ec_ghosts.clear();
  L.ec_built = true;
  const int nb = (int)L.boxes.size();
  // per solve: buckets of side S (the largest box edge of the solve) holding the boxes that
  // overlap them, so the owner of a cell is found among a few boxes
  const int ns = (int)L.geoms.size();
  std::vector<int> side(ns, 1);
  for (int b = 0; b < nb; ++b)
    for (int d = 0; d < 3; ++d) side[L.box_solve[b]] = std::max(side[L.box_solve[b]], L.boxes[b].n(d));
  std::map<std::tuple<int, int, int, int>, std::vector<int>> buckets;
  auto bucket_of = [&](int s, const int g[3], int* k) {
    for (int d = 0; d < 3; ++d) k[d] = (g[d] - L.geoms[s].domain.lo[d]) / side[s];
  };
  for (int b = 0; b < nb; ++b) {
    const int s = L.box_solve[b];
    int k0[3], k1[3];
    bucket_of(s, L.boxes[b].lo, k0);
    bucket_of(s, L.boxes[b].hi, k1);
    for (int z = k0[2]; z <= k1[2]; ++z)
      for (int y = k0[1]; y <= k1[1]; ++y)
        for (int x = k0[0]; x <= k1[0]; ++x) buckets[std::make_tuple(s, x, y, z)].push_back(b);
  }
  for (int b = 0; b < nb; ++b) {
    const Box& B = L.boxes[b];
    const int s = L.box_solve[b];
    const SolveGeom& G = L.geoms[s];
    const DevBox& Db = L.dbox[b];
    for (int k = -1; k <= B.n(2); ++k)
      for (int j = -1; j <= B.n(1); ++j)
        for (int i = -1; i <= B.n(0); ++i) {
          const int loc[3] = {i, j, k};
          int out = 0;
          for (int d = 0; d < 3; ++d) out += (loc[d] < 0 || loc[d] >= B.n(d));
          if (out < 2) continue;  // valid cells and face ghosts
          int g[3];
          double sign = 1.0;
          for (int d = 0; d < 3; ++d) {
            const int n = G.domain.n(d);
            int rel = B.lo[d] + loc[d] - G.domain.lo[d];
            if (rel < 0 || rel >= n) {
              const int bc = rel < 0 ? G.bclo[d] : G.bchi[d];
              if (bc == 0) {
                rel = ((rel % n) + n) % n;
              } else {
                rel = rel < 0 ? -1 - rel : 2 * n - 1 - rel;
                if (bc == 1) sign = -sign;
              }
            }
            g[d] = G.domain.lo[d] + rel;
          }
          int kb[3];
          bucket_of(s, g, kb);
          int src = -1;
          auto it = buckets.find(std::make_tuple(s, kb[0], kb[1], kb[2]));
          if (it != buckets.end())
            for (int c : it->second) {
              const Box& C = L.boxes[c];
              if (g[0] >= C.lo[0] && g[0] <= C.hi[0] && g[1] >= C.lo[1] && g[1] <= C.hi[1] && g[2] >= C.lo[2] &&
                  g[2] <= C.hi[2]) {
                src = c;
                break;
              }
            }
          if (src < 0) continue;  // (boxes cover every solve's domain on a multigrid level)
          const DevBox& Ds = L.dbox[src];
          const Box& S = L.boxes[src];
          L.ec_ghosts.push_back({elem_index(Db, i, j, k),
                                 elem_index(Ds, g[0] - S.lo[0], g[1] - S.lo[1], g[2] - S.lo[2]), sign});
        }
  }
}

std::string finalize_level(LevelMeta& L) {
  const int nb = (int)L.boxes.size();
  L.dbox.resize(nb);
  int64_t off = 0;
  L.ncells = 0;
  for (int b = 0; b < nb; ++b) {
    const Box& B = L.boxes[b];
    DevBox& D = L.dbox[b];
    D.nx = B.n(0); D.ny = B.n(1); D.nz = B.n(2);
    D.sx = ((GX + D.nx + 1 + ROW_ALIGN - 1) / ROW_ALIGN) * ROW_ALIGN;
    D.sy = (int64_t)D.sx * (D.ny + 2);
    for (int d = 0; d < 3; ++d) D.lo[d] = B.lo[d];
    D.solve = L.box_solve[b];
    D.off = off;
    off += ((D.sy * (D.nz + 2) + BOX_ALIGN - 1) / BOX_ALIGN) * BOX_ALIGN;
    L.ncells += B.volume();
  }
  L.nelem = off;
  if (L.parent.size() != (size_t)nb) L.parent.assign(nb, -1);
  std::string err = build_ghosts(L);
  if (!err.empty()) return err;
  // push faces: each ghost rectangle copies one face of its source box (its source layer is
  // the box's first or last layer along the normal) to a translate in the destination box
  L.push_faces.assign((size_t)nb * 6, PushFace{-1, 1, 0, 0, 0, 0, 0, 0, 0});
  L.push_ok = true;
  for (const GhostRect& g : L.ghosts) {
    const int d = 3 - g.d1 - g.d2;
    const DevBox& S = L.dbox[g.src_box];
    const int n[3] = {S.nx, S.ny, S.nz};
    if (g.kind == 2) {  // a quadratic wall's source is not on the box face
      L.push_ok = false;
      continue;
    }
    if (n[d] < 2 || (g.src[d] != 0 && g.src[d] != n[d] - 1) || g.n1 != n[g.d1] || g.n2 != n[g.d2] ||
        g.src[g.d1] != 0 || g.src[g.d2] != 0) {
      L.push_ok = false;  // a face split over several rectangles, or a one-cell-thick box
      continue;
    }
    PushFace& P = L.push_faces[(size_t)g.src_box * 6 + 2 * d + (g.src[d] == 0 ? 0 : 1)];
    if (P.box >= 0) L.push_ok = false;  // two rectangles from one face
    P.box = g.dst_box;
    P.sign = g.sign;
    P.dx = g.dst[0] - g.src[0];
    P.dy = g.dst[1] - g.src[1];
    P.dz = g.dst[2] - g.src[2];
    const DevBox& Dd = L.dbox[g.dst_box];
    P.direct = (Dd.sx == S.sx && Dd.sy == S.sy) ? 1 : 0;
    P.delta = elem_index(Dd, g.dst[0], g.dst[1], g.dst[2]) - elem_index(S, g.src[0], g.src[1], g.src[2]);
    P.wall = g.kind == 1 ? 1 : 0;
  }
  for (int q = 0; q < (int)L.geoms.size(); ++q)
    if (L.solve_present[q])
      for (int d = 0; d < 3; ++d)
        if (L.geoms[q].periodic(d) && L.geoms[q].domain.n(d) % 2 != 0) L.push_ok = false;
  L.pair_chunks.clear();
  L.quad_chunks.clear();
  L.pair_all_chunks.clear();
  L.cell_chunks.clear();
  L.quad_ok = true;
  for (int b = 0; b < nb; ++b) {
    const DevBox& D = L.dbox[b];
    int64_t ncell = (int64_t)D.nx * D.ny * D.nz;
    for (int64_t s = 0; s < ncell; s += BLOCK) L.cell_chunks.push_back({b, (int)s});
    int64_t npair = (int64_t)((D.nx + 1) / 2) * D.ny * D.nz;
    for (int64_t s = 0; s < npair; s += BLOCK) L.pair_all_chunks.push_back({b, (int)s});
    if (L.solve_bottom[L.box_solve[b]]) continue;
    for (int64_t s = 0; s < npair; s += BLOCK) L.pair_chunks.push_back({b, (int)s});
    if (D.nx % 4 != 0) L.quad_ok = false;
    const int64_t nquad = (int64_t)(D.nx / 4) * D.ny * D.nz;
    for (int64_t s = 0; s < nquad; s += BLOCK) L.quad_chunks.push_back({b, (int)s});
  }
  if (!L.quad_ok) L.quad_chunks.clear();
  // boxes are stored solve by solve, so each solve's cell chunks are contiguous
  const int ns = (int)L.geoms.size();
  L.solve_chunk_range.assign(ns + 1, 0);
  std::vector<int64_t> cells(ns, 0);
  for (const Chunk& ch : L.cell_chunks) L.solve_chunk_range[L.box_solve[ch.item] + 1]++;
  for (int q = 0; q < ns; ++q) L.solve_chunk_range[q + 1] += L.solve_chunk_range[q];
  for (int b = 0; b < nb; ++b) cells[L.box_solve[b]] += L.boxes[b].volume();
  L.inv_count.assign(ns, 0.0);
  for (int q = 0; q < ns; ++q) L.inv_count[q] = cells[q] ? 1.0 / (double)cells[q] : 0.0;
  L.coarse_chunks.clear();
  for (int b = 0; b < nb; ++b) {
    if (L.parent[b] < 0) continue;
    const DevBox& D = L.dbox[b];
    int64_t nc = (int64_t)(D.nx / 2) * (D.ny / 2) * (D.nz / 2);
    for (int64_t s = 0; s < nc; s += BLOCK) L.coarse_chunks.push_back({b, (int)s});
  }
  build_bottom(L);
  build_flow(L);
  build_wave(L, g_wave_capacity);
  return "";
}

bool make_coarse(LevelMeta& f, LevelMeta& c) {
  const int nb = (int)f.boxes.size();
  const int ns = (int)f.geoms.size();
  f.parent.assign(nb, -1);
  f.solve_bottom.assign(ns, 0);
  c = LevelMeta();
  c.geoms = f.geoms;
  c.solve_present.assign(ns, 0);
  c.solve_bottom.assign(ns, 0);
  bool any = false;
  for (int s = 0; s < ns; ++s) {
    if (!f.solve_present[s]) continue;
    std::vector<int> mem;
    for (int b = 0; b < nb; ++b)
      if (f.box_solve[b] == s) mem.push_back(b);
    bool per_box = true, evenly = true;
    int64_t vol = 0;
    for (int b : mem) {
      const Box& B = f.boxes[b];
      vol += B.volume();
      for (int d = 0; d < 3; ++d) {
        if (pmod2(B.lo[d]) != 0 || B.n(d) % 2 != 0) { evenly = false; per_box = false; }
        if (B.n(d) < 4) per_box = false;
      }
    }
    const SolveGeom& G = f.geoms[s];
    bool agg = false;
    if (!per_box && evenly && vol == G.domain.volume()) {
      agg = true;
      for (int d = 0; d < 3; ++d)
        if (G.domain.n(d) % 2 != 0 || G.domain.n(d) < 4 || pmod2(G.domain.lo[d]) != 0) agg = false;
    }
    if (!per_box && !agg) {
      f.solve_bottom[s] = 1;
      continue;
    }
    any = true;
    c.solve_present[s] = 1;
    SolveGeom& CG = c.geoms[s];
    for (int d = 0; d < 3; ++d) {
      CG.domain.lo[d] = G.domain.lo[d] / 2;
      CG.domain.hi[d] = (G.domain.hi[d] + 1) / 2 - 1;
      CG.h[d] = 2.0 * G.h[d];
    }
    if (per_box) {
      for (int b : mem) {
        Box cb;
        for (int d = 0; d < 3; ++d) {
          cb.lo[d] = f.boxes[b].lo[d] / 2;
          cb.hi[d] = (f.boxes[b].hi[d] + 1) / 2 - 1;
        }
        f.parent[b] = (int)c.boxes.size();
        c.boxes.push_back(cb);
        c.box_solve.push_back(s);
      }
    } else {
      int P = (int)c.boxes.size();
      c.boxes.push_back(CG.domain);
      c.box_solve.push_back(s);
      for (int b : mem) f.parent[b] = P;
    }
  }
  return any;
}

std::string build_tail(std::vector<LevelMeta>& L, TailHost& T) {
  T = TailHost();
  const int n = (int)L.size();
  const int ns = n ? (int)L[0].geoms.size() : 0;
  T.first_at.assign(n, 0);
  T.count_at.assign(n, 0);
  T.tail_from.assign(ns, -1);
  // per solve: cells per level, bottom level; the tail starts at the first level >= 1 with
  // at most TAIL_MAX_CELLS cells (sizes only shrink going down)
  std::vector<int> bottom(ns, -1);
  for (int s = 0; s < ns; ++s) {
    for (int m = 0; m < n; ++m)
      if (L[m].solve_present[s] && L[m].solve_bottom[s]) bottom[s] = m;
    if (bottom[s] < 1 || bottom[s] >= TAIL_MAXLEV) continue;
    for (int m = 1; m <= bottom[s]; ++m) {
      int64_t cells = 0;
      for (int b = 0; b < (int)L[m].boxes.size(); ++b)
        if (L[m].box_solve[b] == s) cells += L[m].boxes[b].volume();
      if (cells <= TAIL_MAX_CELLS) {
        T.tail_from[s] = m;
        break;
      }
    }
  }
  std::vector<int> order;
  for (int s = 0; s < ns; ++s)
    if (T.tail_from[s] >= 0) order.push_back(s);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return T.tail_from[a] < T.tail_from[b]; });
  for (int s : order) {
    TailDesc D{};
    D.solve = s;
    D.m0 = T.tail_from[s];
    D.mb = bottom[s];
    D.lev0 = (int)T.levels.size();
    D.singular = 0;  // set from the operator's scalars at coefficient time
    // bounding box of the problem's boxes on level m; false unless they tile it
    auto bbox = [&](int m, int lo[3], int hi[3]) {
      int64_t vol = 0;
      bool first = true;
      for (int d = 0; d < 3; ++d) lo[d] = 0, hi[d] = -1;
      for (int b = 0; b < (int)L[m].boxes.size(); ++b) {
        if (L[m].box_solve[b] != s) continue;
        const Box& B = L[m].boxes[b];
        for (int d = 0; d < 3; ++d) {
          lo[d] = first ? B.lo[d] : std::min(lo[d], B.lo[d]);
          hi[d] = first ? B.hi[d] : std::max(hi[d], B.hi[d]);
        }
        first = false;
        vol += B.volume();
      }
      const int64_t bv = (int64_t)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
      return !first && vol == bv && bv <= (1 << 24);
    };
    D.dense = 1;
    for (int m = D.m0; m <= D.mb; ++m) {
      const LevelMeta& M = L[m];
      TailLevel TL{};
      // the dense form: the problem's boxes of this level must tile their bounding box
      int dlo[3], dhi[3];
      if (!bbox(m, dlo, dhi)) D.dense = 0;
      const int dn[3] = {dhi[0] - dlo[0] + 1, dhi[1] - dlo[1] + 1, dhi[2] - dlo[2] + 1};
      TL.dsx = dn[0] + 2;
      TL.dsy = (dn[0] + 2) * (dn[1] + 2);
      TL.dne = D.dense ? TL.dsy * (dn[2] + 2) : 0;
      // dense slot of global cell (gi, gj, gk); cells outside the domain's ghost layer: -1
      auto dslot = [&](int gi, int gj, int gk) -> int {
        const int u = gi - dlo[0] + 1, v = gj - dlo[1] + 1, w = gk - dlo[2] + 1;
        if (!D.dense || u < 0 || v < 0 || w < 0 || u > dn[0] + 1 || v > dn[1] + 1 || w > dn[2] + 1) return -1;
        return u + TL.dsx * v + TL.dsy * w;
      };
      auto inside = [&](int gi, int gj, int gk) {
        return gi >= dlo[0] && gi <= dhi[0] && gj >= dlo[1] && gj <= dhi[1] && gk >= dlo[2] && gk <= dhi[2];
      };
      TL.cell0 = (int)T.cells.size();
      for (int colour = 0; colour < 2; ++colour) {
        const int c0 = (int)T.cells.size();
        for (int b = 0; b < (int)M.boxes.size(); ++b) {
          if (M.box_solve[b] != s) continue;
          const DevBox& B = M.dbox[b];
          for (int k = 0; k < B.nz; ++k)
            for (int j = 0; j < B.ny; ++j)
              for (int i = 0; i < B.nx; ++i)
                if (pmod2(B.lo[0] + B.lo[1] + B.lo[2] + i + j + k) == colour) {
                  const int gi = B.lo[0] + i, gj = B.lo[1] + j, gk = B.lo[2] + k;
                  int slot = std::max(0, dslot(gi, gj, gk));
                  if (gi == dhi[0]) slot |= TAIL_HI_X;
                  if (gj == dhi[1]) slot |= TAIL_HI_Y;
                  if (gk == dhi[2]) slot |= TAIL_HI_Z;
                  if (gi == dlo[0]) slot |= TAIL_LO_X;
                  if (gj == dlo[1]) slot |= TAIL_LO_Y;
                  if (gk == dlo[2]) slot |= TAIL_LO_Z;
                  T.cells.push_back({elem_index(B, i, j, k), B.sy, B.sx, slot});
                }
        }
        TL.ncell[colour] = (int)T.cells.size() - c0;
      }
      TL.ghost0 = (int)T.ghosts.size();
      TL.dghost0 = (int)T.dghosts.size();
      for (int parity = 0; parity < 2; ++parity) {
        const int g0 = (int)T.ghosts.size();
        const int dg0 = (int)T.dghosts.size();
        for (const GhostRect& g : M.ghosts) {
          if (M.box_solve[g.dst_box] != s) continue;
          const DevBox& Bd = M.dbox[g.dst_box];
          const DevBox& Bs = M.dbox[g.src_box];
          for (int v = 0; v < g.n2; ++v)
            for (int u = 0; u < g.n1; ++u) {
              if (pmod2(g.par0 + u + v) != parity) continue;
              int dl[3] = {g.dst[0], g.dst[1], g.dst[2]};
              int sl[3] = {g.src[0], g.src[1], g.src[2]};
              dl[g.d1] += u; dl[g.d2] += v;
              sl[g.d1] += u; sl[g.d2] += v;
              T.ghosts.push_back({elem_index(Bd, dl[0], dl[1], dl[2]), elem_index(Bs, sl[0], sl[1], sl[2]),
                                  ghost_factor(g)});
              // dense form: only the ghosts outside the domain (a ghost between two boxes is
              // the neighbouring cell itself there)
              const int gd[3] = {Bd.lo[0] + dl[0], Bd.lo[1] + dl[1], Bd.lo[2] + dl[2]};
              const int gs[3] = {Bs.lo[0] + sl[0], Bs.lo[1] + sl[1], Bs.lo[2] + sl[2]};
              if (D.dense && !inside(gd[0], gd[1], gd[2])) {
                const int a = dslot(gd[0], gd[1], gd[2]), b2 = dslot(gs[0], gs[1], gs[2]);
                if (a < 0 || b2 < 0 || !inside(gs[0], gs[1], gs[2])) D.dense = 0;
                else T.dghosts.push_back({a, b2, ghost_factor(g)});
                // the face's rule: a wall copies the cell inward, a periodic image the cell
                // at the other end (one cell across: both readings give the same copy)
                int ax = -1;
                for (int d = 0; d < 3; ++d)
                  if (gd[d] < dlo[d] || gd[d] > dhi[d]) ax = ax < 0 ? d : 3;
                if (ax < 0 || ax > 2) {
                  D.dense = 0;
                } else {
                  const int side = gd[ax] < dlo[ax] ? 0 : 1;
                  const int inward = side ? dhi[ax] : dlo[ax], across = side ? dlo[ax] : dhi[ax];
                  const int sg = ghost_factor(g) < 0 ? -1 : 1;
                  int rule = 0;
                  if (gs[ax] == inward && (sg < 0 || dn[ax] > 1)) rule = sg;
                  else if (gs[ax] == across && sg > 0) rule = 2;
                  for (int d = 0; d < 3; ++d)
                    if (d != ax && gs[d] != gd[d]) rule = 0;
                  // (a smoothed level pushes values into periodic images: an odd period
                  // would make a cell's image the other colour's neighbour)
                  if (rule == 2 && m < D.mb && (dn[ax] & 1)) rule = 0;
                  int& f = TL.face[2 * ax + side];
                  if (rule == 0 || (f != 0 && f != rule)) D.dense = 0;
                  else f = rule;
                }
              }
            }
        }
        TL.nghost[parity] = (int)T.ghosts.size() - g0;
        TL.ndghost[parity] = (int)T.dghosts.size() - dg0;
      }
      TL.xfer0 = (int)T.xfer.size();
      if (m < D.mb) {
        const LevelMeta& Cm = L[m + 1];
        int clo[3], chi[3];
        if (!bbox(m + 1, clo, chi)) D.dense = 0;
        const int csx = chi[0] - clo[0] + 3, csy = csx * (chi[1] - clo[1] + 3);
        for (int b = 0; b < (int)M.boxes.size(); ++b) {
          if (M.box_solve[b] != s) continue;
          if (M.parent[b] < 0) return "tail: a box without a coarse parent above the bottom (internal error)";
          const DevBox& F = M.dbox[b];
          const DevBox& P = Cm.dbox[M.parent[b]];
          for (int ck = 0; ck < F.nz / 2; ++ck)
            for (int cj = 0; cj < F.ny / 2; ++cj)
              for (int ci = 0; ci < F.nx / 2; ++ci) {
                TailXfer x{};
                x.qc = elem_index(P, (F.lo[0] >> 1) + ci - P.lo[0], (F.lo[1] >> 1) + cj - P.lo[1],
                                  (F.lo[2] >> 1) + ck - P.lo[2]);
                x.qf = elem_index(F, 2 * ci, 2 * cj, 2 * ck);
                x.sx = F.sx;
                x.sy = (int)F.sy;
                if (D.dense) {
                  const int g[3] = {(F.lo[0] >> 1) + ci, (F.lo[1] >> 1) + cj, (F.lo[2] >> 1) + ck};
                  x.dqc = (g[0] - clo[0] + 1) + csx * (g[1] - clo[1] + 1) + csy * (g[2] - clo[2] + 1);
                  const int f[3] = {F.lo[0] + 2 * ci, F.lo[1] + 2 * cj, F.lo[2] + 2 * ck};
                  x.dqf = dslot(f[0], f[1], f[2]);
                  if (x.dqf < 0) D.dense = 0;
                  x.dfl = (f[0] == dlo[0] ? TAIL_LO_X : 0) | (f[1] == dlo[1] ? TAIL_LO_Y : 0) |
                          (f[2] == dlo[2] ? TAIL_LO_Z : 0) | (f[0] + 1 == dhi[0] ? TAIL_HI_X : 0) |
                          (f[1] + 1 == dhi[1] ? TAIL_HI_Y : 0) | (f[2] + 1 == dhi[2] ? TAIL_HI_Z : 0);
                }
                T.xfer.push_back(x);
              }
        }
      }
      TL.nxfer = (int)T.xfer.size() - TL.xfer0;
      T.levels.push_back(TL);
    }
    {
      const LevelMeta& M = L[D.mb];
      int64_t lo = -1, hi = 0;
      for (int b = 0; b < (int)M.boxes.size(); ++b) {
        if (M.box_solve[b] != s) continue;
        const DevBox& B = M.dbox[b];
        if (lo < 0 || B.off < lo) lo = B.off;
        hi = std::max(hi, B.off + B.sy * (B.nz + 2));
      }
      D.bot_base = lo;
      D.bot_span = (int)std::min<int64_t>(hi - lo, 1 << 30);
    }
    if (T.count_at[D.m0]++ == 0) T.first_at[D.m0] = (int)T.descs.size();
    T.descs.push_back(D);
  }
  // the grid launches of the V-cycle skip what the tails do
  for (int m = 0; m < n; ++m) {
    LevelMeta& M = L[m];
    auto in_tail = [&](int solve) { return T.tail_from[solve] >= 0 && T.tail_from[solve] <= m; };
    M.vc_ghost_chunks.clear();
    for (const Chunk& ch : M.ghost_chunks)
      if (!in_tail(M.box_solve[M.ghosts[ch.item].dst_box])) M.vc_ghost_chunks.push_back(ch);
    M.vc_pair_chunks.clear();
    for (const Chunk& ch : M.pair_chunks)
      if (!in_tail(M.box_solve[ch.item])) M.vc_pair_chunks.push_back(ch);
    M.vc_quad_chunks.clear();
    for (const Chunk& ch : M.quad_chunks)
      if (!in_tail(M.box_solve[ch.item])) M.vc_quad_chunks.push_back(ch);
    M.vc_coarse_chunks.clear();
    for (const Chunk& ch : M.coarse_chunks)
      if (!in_tail(M.box_solve[ch.item])) M.vc_coarse_chunks.push_back(ch);
    M.vc_bot_descs.clear();
    for (const BotDesc& d : M.bot_descs)
      if (!in_tail(d.solve)) M.vc_bot_descs.push_back(d);
    M.vc_flow_skip.assign(M.geoms.size(), 0);
    for (int q = 0; q < (int)M.geoms.size(); ++q) M.vc_flow_skip[q] = in_tail(q) ? 1 : 0;
  }
  return "";
}

}  // namespace gmg
