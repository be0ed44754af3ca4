// walls.cu -- nonzero values on the physical walls of level 0 (Sec. "Linear Solvers": the
// operator equation with its boundary conditions; Sec. "Basic data structures": BCRec).
//
// Inside the solver every wall is homogeneous: a Dirichlet ghost is minus the adjacent
// interior value, a Neumann ghost equals it.  A wall value g makes the ghost affine --
// Dirichlet (phi = g on the face): ghost = 2g - interior; Neumann (outward normal
// derivative g): ghost = interior + h g -- and the part that does not depend on phi is a
// constant that moves to the right-hand side.  In the row of the cell next to the face,
// -w (ghost - phi) with w = b beta_face / h^2 contributes -w 2g (Dirichlet) or -w h g
// (Neumann); so rhs - A_g(0) = rhs + c g with c = 2w or w h, and solving A_0 phi =
// rhs - A_g(0) with homogeneous walls gives the solution with the wall values.
//
// A quadratic Dirichlet side (kind 3; boxes of two or more cells along the normal) has the
// ghost 8g/3 - 2 phi_0 + phi_1 / 3: the constant is 8g/3 and c = 8w/3.  Its homogeneous
// part puts the entry -w/3 on phi_1 into the wall cell's row, which the transpose moves
// into phi_1's row.
//
// One kernel does the four uses of that map, one launch per wall face (faces in the order
// x-, x+, y-, y+, z-, z+, so a corner cell's sum has a fixed order):
//   mode 0: f[q] += c g             (fold the values into a right-hand side)
//   mode 1: f[ghost] += (2, 8/3 or h) g (complete homogeneous ghosts of phi to the affine rule)
//   mode 2: dg = c lambda[q]         (the transpose: dL/dg for an adjoint lambda)
//   mode 3: f[q1] -= (w / 3) lam[q]  (quadratic sides: the transposed operator's entry, q1 the
//                                     cell next to q inward; f = A^T lam without it)
// A block row (blockIdx.y) takes one box; boxes without a face on the wall return at once.
#include "kernels.h"

namespace gmg {
namespace {

constexpr int WT = 256;

__global__ void __launch_bounds__(WT)
    k_wall_values(const DevBox* __restrict__ boxes, const DevGeom* __restrict__ geoms, int face, int kind, double h,
                  const double* __restrict__ w, const double* __restrict__ g, int mode, double* f,
                  const double* __restrict__ lam, double* dg) {
  const DevBox B = boxes[blockIdx.y];
  const DevGeom G = geoms[B.solve];
  const int d = face >> 1, side = face & 1;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const int n[3] = {B.nx, B.ny, B.nz};
  if (side == 0 ? B.lo[d] != G.dlo[d] : B.lo[d] + n[d] - 1 != G.dhi[d]) return;
  const int nf = n[t1] * n[t2];
  const int64_t sd = d == 0 ? 1 : (d == 1 ? (int64_t)B.sx : B.sy);
  const int64_t nt1 = G.dhi[t1] - G.dlo[t1] + 1;
  for (int e = blockIdx.x * WT + threadIdx.x; e < nf; e += gridDim.x * WT) {
    int loc[3];
    loc[t1] = e % n[t1];
    loc[t2] = e / n[t1];
    loc[d] = side ? n[d] - 1 : 0;
    const int64_t q = elem_index(B, loc[0], loc[1], loc[2]);
    const int64_t qf = side ? q + sd : q;  // the wall face's slot (slot i holds face i - 1/2)
    const int64_t qg = side ? q + sd : q - sd;
    const int64_t tt = (int64_t)(B.lo[t1] + loc[t1] - G.dlo[t1]) + nt1 * (int64_t)(B.lo[t2] + loc[t2] - G.dlo[t2]);
    const bool quad = kind == 3 && n[d] >= 2;
    const double gf = kind == 2 ? h : (quad ? 8.0 / 3.0 : 2.0);  // ghost = homogeneous part + gf g
    if (mode == 0) {
      f[q] += (kind == 2 ? w[qf] * h : gf * w[qf]) * g[tt];
    } else if (mode == 1) {
      f[qg] += gf * g[tt];
    } else if (mode == 2) {
      dg[tt] = (kind == 2 ? w[qf] * h : gf * w[qf]) * lam[q];
    } else if (quad) {
      f[side ? q - sd : q + sd] -= (w[qf] / 3.0) * lam[q];
    }
  }
}

}  // namespace

void launch_wall_values(const LevelDev& L, int nboxes, int max_face_cells, int face, int kind, double h,
                        const double* w, const double* g, int mode, double* f, const double* lam, double* dg,
                        cudaStream_t s) {
  if (nboxes <= 0 || max_face_cells <= 0) return;
  count_launches(1);
  const dim3 grid((unsigned)((max_face_cells + WT - 1) / WT), (unsigned)nboxes);
  k_wall_values<<<grid, WT, 0, s>>>(L.boxes, L.geoms, face, kind, h, w, g, mode, f, lam, dg);
}

}  // namespace gmg
