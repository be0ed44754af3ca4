// amr_meta.cpp -- host tables of the two-level composite operator (built once per layout).
//
// Sec. "Operations between levels": the fine level's ghost cells on the coarse/fine
// boundary are interpolated from coarse data; coarse cells next to the fine level take the
// averaged fine fluxes (refluxing); coarse cells under the fine level are covered.
#include "amr_meta.h"

#include <map>

namespace gmg {

namespace {

int pmod(int a, int m) {
  int r = a % m;
  return r < 0 ? r + m : r;
}

// element offset of the (periodically wrapped) global cell g on a level, or -1
int64_t cell_elem(const LevelMeta& L, const int g_in[3], int* box_out = nullptr) {
  const SolveGeom& G = L.geoms[0];
  int g[3] = {g_in[0], g_in[1], g_in[2]};
  for (int d = 0; d < 3; ++d)
    if (G.periodic(d)) g[d] = G.domain.lo[d] + pmod(g[d] - G.domain.lo[d], G.domain.n(d));
  for (int b = 0; b < (int)L.boxes.size(); ++b) {
    const Box& B = L.boxes[b];
    if (g[0] < B.lo[0] || g[0] > B.hi[0] || g[1] < B.lo[1] || g[1] > B.hi[1] || g[2] < B.lo[2] || g[2] > B.hi[2])
      continue;
    if (box_out) *box_out = b;
    return elem_index(L.dbox[b], g[0] - B.lo[0], g[1] - B.lo[1], g[2] - B.lo[2]);
  }
  return -1;
}

}  // namespace

std::string build_amr(const LevelMeta& C, LevelMeta& F, AmrHost& A) {
  A = AmrHost();
  // covered coarse cells: below a fine cell
  A.covered.assign(C.nelem, 0);
  for (int b = 0; b < (int)C.boxes.size(); ++b) {
    const Box& B = C.boxes[b];
    for (int k = B.lo[2]; k <= B.hi[2]; ++k)
      for (int j = B.lo[1]; j <= B.hi[1]; ++j)
        for (int i = B.lo[0]; i <= B.hi[0]; ++i) {
          int gf[3] = {2 * i, 2 * j, 2 * k};
          if (cell_elem(F, gf) >= 0) {
            int64_t q = elem_index(C.dbox[b], i - B.lo[0], j - B.lo[1], k - B.lo[2]);
            A.covered[q] = 1;
            A.covered_list.push_back(q);
          }
        }
  }
  // ghost elements of the coarse level take the covered flag of the cell they copy, so a
  // kernel that looks at a neighbour across a coarse box face sees whether it is covered
  for (const GhostRect& g : C.ghosts) {
    if (g.kind != 0) continue;
    const DevBox& Dd = C.dbox[g.dst_box];
    const DevBox& Ds = C.dbox[g.src_box];
    for (int v = 0; v < g.n2; ++v)
      for (int u = 0; u < g.n1; ++u) {
        int dl[3] = {g.dst[0], g.dst[1], g.dst[2]}, sl[3] = {g.src[0], g.src[1], g.src[2]};
        dl[g.d1] += u; dl[g.d2] += v;
        sl[g.d1] += u; sl[g.d2] += v;
        A.covered[elem_index(Dd, dl[0], dl[1], dl[2])] = A.covered[elem_index(Ds, sl[0], sl[1], sl[2])];
      }
  }
  // coarse/fine ghosts of the fine level
  A.cfidx.assign(F.nelem, -1);
  for (const CfSlab& S : F.cf_slabs) {
    const Box& B = F.boxes[S.box];
    const DevBox& D = F.dbox[S.box];
    const int d = S.d, d1 = (d == 0) ? 1 : 0, d2 = (d == 2) ? 1 : 2;
    const int n[3] = {B.n(0), B.n(1), B.n(2)};
    if (n[d] < 2) return "fine boxes must be at least 2 cells wide";
    for (int v = 0; v < n[d2]; ++v)
      for (int u = 0; u < n[d1]; ++u) {
        int loc[3];
        loc[d] = S.side ? n[d] : -1;
        loc[d1] = u;
        loc[d2] = v;
        int in1[3] = {loc[0], loc[1], loc[2]}, in2[3] = {loc[0], loc[1], loc[2]};
        in1[d] = S.side ? n[d] - 1 : 0;
        in2[d] = S.side ? n[d] - 2 : 1;
        CfGhost G{};
        G.dst = elem_index(D, loc[0], loc[1], loc[2]);
        G.f1 = elem_index(D, in1[0], in1[1], in1[2]);
        G.f2 = elem_index(D, in2[0], in2[1], in2[2]);
        G.fslot = S.side ? G.dst : G.f1;  // face slot i holds the face at i - 1/2
        G.d = d;
        int g[3], Cc[3];
        double s[3];
        for (int q = 0; q < 3; ++q) {
          g[q] = B.lo[q] + loc[q];
          Cc[q] = (g[q] - pmod(g[q], 2)) / 2;
          s[q] = pmod(g[q], 2) == 0 ? -0.25 : 0.25;
        }
        G.cq[0] = cell_elem(C, Cc);
        G.cw[0] = 1.0;
        const int t[2] = {d1, d2};
        for (int e = 0; e < 2; ++e) {
          int Cp[3] = {Cc[0], Cc[1], Cc[2]}, Cm[3] = {Cc[0], Cc[1], Cc[2]};
          Cp[t[e]] += 1;
          Cm[t[e]] -= 1;
          const double st = s[t[e]];
          G.cq[1 + 2 * e] = cell_elem(C, Cp);
          G.cq[2 + 2 * e] = cell_elem(C, Cm);
          G.cw[1 + 2 * e] = 0.5 * st + 0.5 * st * st;
          G.cw[2 + 2 * e] = -0.5 * st + 0.5 * st * st;
          G.cw[0] -= st * st;
        }
        for (int e = 0; e < 5; ++e)
          if (G.cq[e] < 0 || A.covered[G.cq[e]])
            return "coarse/fine interpolation needs uncovered coarse neighbours (fine level too close to another fine box "
                   "or to a wall)";
        A.cfidx[G.dst] = (int)A.cf.size();
        A.cf.push_back(G);
      }
  }
  // reflux: faces between an uncovered coarse cell and a covered one
  std::map<int64_t, std::vector<RefluxFace>> per_cell;
  for (int b = 0; b < (int)C.boxes.size(); ++b) {
    const Box& B = C.boxes[b];
    const DevBox& D = C.dbox[b];
    for (int k = B.lo[2]; k <= B.hi[2]; ++k)
      for (int j = B.lo[1]; j <= B.hi[1]; ++j)
        for (int i = B.lo[0]; i <= B.hi[0]; ++i) {
          const int gl[3] = {i, j, k};
          const int64_t I = elem_index(D, i - B.lo[0], j - B.lo[1], k - B.lo[2]);
          if (A.covered[I]) continue;
          for (int d = 0; d < 3; ++d) {
            const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
            const int64_t sd = d == 0 ? 1 : (d == 1 ? (int64_t)D.sx : D.sy);
            for (int side = 0; side < 2; ++side) {
              int gn[3] = {gl[0], gl[1], gl[2]};
              gn[d] += side ? 1 : -1;
              const int64_t N = cell_elem(C, gn);
              if (N < 0 || !A.covered[N]) continue;
              RefluxFace R{};
              R.N = N;
              R.cslot = side ? I + sd : I;
              R.d = d;
              int q = 0;
              for (int v = 0; v < 2; ++v)
                for (int u = 0; u < 2; ++u, ++q) {
                  int fg[3];
                  fg[d] = side ? 2 * gn[d] : 2 * gn[d] + 1;
                  fg[d1] = 2 * gl[d1] + u;
                  fg[d2] = 2 * gl[d2] + v;
                  int fb = -1;
                  const int64_t fq = cell_elem(F, fg, &fb);
                  if (fq < 0) return "reflux face without fine cells (internal error)";
                  const int64_t fsd = d == 0 ? 1 : (d == 1 ? (int64_t)F.dbox[fb].sx : F.dbox[fb].sy);
                  const int64_t gq = side ? fq - fsd : fq + fsd;
                  if (A.cfidx[gq] < 0) return "reflux face whose fine ghost is not a coarse/fine ghost (internal error)";
                  R.f[q] = fq;
                  R.g[q] = gq;
                  R.fslot[q] = side ? fq : gq;
                  R.cf[q] = A.cfidx[gq];
                }
              per_cell[I].push_back(R);
            }
          }
        }
  }
  for (auto& kv : per_cell) {
    RefluxCell rc{};
    rc.I = kv.first;
    rc.face0 = (int)A.rfaces.size();
    rc.nface = (int)kv.second.size();
    for (auto& f : kv.second) A.rfaces.push_back(f);
    A.rcells.push_back(rc);
  }
  // coefficient restriction onto level 0 under the fine level (Sec. "Operations between
  // levels"): every level-0 face slot with a covered cell on either side, and every covered
  // cell.  The composite operator reads none of these; the coarse correction operator does.
  auto is_covered = [&](const int g[3]) {
    const int gf[3] = {2 * g[0], 2 * g[1], 2 * g[2]};
    return cell_elem(F, gf) >= 0;
  };
  for (int b = 0; b < (int)C.boxes.size(); ++b) {
    const Box& B = C.boxes[b];
    const DevBox& D = C.dbox[b];
    for (int d = 0; d < 3; ++d) {
      const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      int ext[3] = {B.n(0), B.n(1), B.n(2)};
      ext[d] += 1;
      for (int k = 0; k < ext[2]; ++k)
        for (int j = 0; j < ext[1]; ++j)
          for (int i = 0; i < ext[0]; ++i) {
            const int G[3] = {B.lo[0] + i, B.lo[1] + j, B.lo[2] + k};
            int Gl[3] = {G[0], G[1], G[2]};
            Gl[d] -= 1;
            if (!is_covered(G) && !is_covered(Gl)) continue;
            // the fine face at 2G (its tangential low corner), from the box of the fine cell
            // above it, else from the box of the fine cell below it (slot n of that box)
            int fg[3] = {2 * G[0], 2 * G[1], 2 * G[2]};
            int fb = -1;
            int64_t f0 = cell_elem(F, fg, &fb);
            if (f0 < 0) {
              fg[d] -= 1;
              f0 = cell_elem(F, fg, &fb);
              if (f0 < 0) return "covered face without fine faces (internal error)";
              f0 += d == 0 ? 1 : (d == 1 ? (int64_t)F.dbox[fb].sx : F.dbox[fb].sy);
            }
            const DevBox& FD = F.dbox[fb];
            const int64_t st[3] = {1, FD.sx, FD.sy};
            AvgFace a{};
            a.cslot = elem_index(D, i, j, k);
            a.f0 = f0;
            a.s1 = (int)st[d1];
            a.s2 = (int)st[d2];
            a.d = d;
            A.avg_faces.push_back(a);
          }
    }
    for (int k = 0; k < B.n(2); ++k)
      for (int j = 0; j < B.n(1); ++j)
        for (int i = 0; i < B.n(0); ++i) {
          const int64_t q = elem_index(D, i, j, k);
          if (!A.covered[q]) continue;
          const int gf[3] = {2 * (B.lo[0] + i), 2 * (B.lo[1] + j), 2 * (B.lo[2] + k)};
          int fb = -1;
          AvgCell a{};
          a.cq = q;
          a.f0 = cell_elem(F, gf, &fb);
          a.sx = F.dbox[fb].sx;
          a.sy = (int)F.dbox[fb].sy;
          A.avg_cells.push_back(a);
        }
  }
  // each fine box's coarsened image must lie in one coarse box (transfers use it)
  F.parent.assign(F.boxes.size(), -1);
  for (int b = 0; b < (int)F.boxes.size(); ++b) {
    const Box& B = F.boxes[b];
    for (int d = 0; d < 3; ++d)
      if (pmod(B.lo[d], 2) || pmod(B.hi[d] + 1, 2)) return "fine boxes must be aligned to the refinement ratio 2";
    int lo[3] = {B.lo[0] / 2, B.lo[1] / 2, B.lo[2] / 2}, hi[3] = {(B.hi[0] + 1) / 2 - 1, (B.hi[1] + 1) / 2 - 1,
                                                                    (B.hi[2] + 1) / 2 - 1};
    for (int cb = 0; cb < (int)C.boxes.size(); ++cb) {
      const Box& P = C.boxes[cb];
      if (lo[0] >= P.lo[0] && hi[0] <= P.hi[0] && lo[1] >= P.lo[1] && hi[1] <= P.hi[1] && lo[2] >= P.lo[2] &&
          hi[2] <= P.hi[2])
        F.parent[b] = cb;
    }
    if (F.parent[b] < 0) return "each fine box, coarsened, must lie inside one coarse box";
  }
  F.coarse_chunks.clear();
  for (int b = 0; b < (int)F.boxes.size(); ++b) {
    const DevBox& D = F.dbox[b];
    const int64_t nc = (int64_t)(D.nx / 2) * (D.ny / 2) * (D.nz / 2);
    for (int64_t s = 0; s < nc; s += BLOCK) F.coarse_chunks.push_back({b, (int)s});
  }
  return "";
}

}  // namespace gmg
