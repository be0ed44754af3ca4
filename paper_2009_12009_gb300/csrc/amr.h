// amr.h -- two-level composite (coarse level 0 + ratio-2 fine level 1) tables and kernels.
#pragma once

#include "kernels.h"

namespace gmg {

// modes of the coarse/fine ghost fill
enum { CF_INTERP = 0, CF_COPY = 1, CF_ZERO = 2 };

// one fine ghost cell on the coarse/fine boundary
struct CfGhost {
  int64_t dst;     // ghost element (fine layout)
  int64_t f1, f2;  // first and second fine cells inward
  int64_t cq[5];   // coarse cells C, C+t1, C-t1, C+t2, C-t2 (coarse level-0 layout)
  double cw[5];    // tangential quadratic weights of phi_c*
  int64_t fslot;   // face slot (fine layout) of the face between f1 and the ghost
  int d;           // normal direction
  int pad;
};

// one coarse face shared by an uncovered coarse cell I and a covered cell N
struct RefluxFace {
  int64_t N;       // covered coarse neighbour (coarse layout)
  int64_t cslot;   // coarse face slot (coarse layout)
  int64_t f[4];    // fine cells next to the face (fine layout)
  int64_t g[4];    // fine ghosts on I's side (fine layout)
  int64_t fslot[4];// fine face slots
  int cf[4];       // their CfGhost indices
  int d;
  int pad;
};

// an uncovered coarse cell with coarse/fine faces
struct RefluxCell {
  int64_t I;
  int face0, nface;
};

// a level-0 face tiled by 4 fine faces: its coefficient is their mean (restriction of the
// coefficients between AMR levels, as between multigrid levels)
struct AvgFace {
  int64_t cslot;   // coarse face slot (coarse layout)
  int64_t f0;      // first fine face slot (fine layout); the others at +s1, +s2, +s1+s2
  int s1, s2;      // fine element strides along the two tangential directions
  int d;           // face direction
  int pad;
};

// a covered coarse cell and its 8 fine children (f0 + {0,1} + sx*{0,1} + sy*{0,1})
struct AvgCell {
  int64_t cq;
  int64_t f0;
  int sx, sy;
};

struct AmrDev {
  const CfGhost* cf = nullptr;
  int ncf = 0;
  const RefluxCell* rcells = nullptr;
  int nrcell = 0;
  const RefluxFace* rfaces = nullptr;
  const int64_t* covered_list = nullptr;  // covered coarse elements
  int ncov = 0;
  const unsigned char* covered = nullptr; // coarse layout: 1 where covered
  const int* cfidx = nullptr;             // fine layout: C/F ghost index or -1
  double hf_over_hc = 0.5;
  const AvgFace* avg_faces = nullptr;
  int navg_face = 0;
  const AvgCell* avg_cells = nullptr;
  int navg_cell = 0;
};

void launch_cf_fill(const AmrDev& A, double* f, const double* c, int mode, cudaStream_t s);
// out = in + std_part * (coarse faces' w (c_I - c_N)) - reflux of the fine field
void launch_reflux(const AmrDev& A, const Coefs& coarse, const Coefs& fine, const double* c, const double* f,
                   const double* in, double* out, int std_part, cudaStream_t s);
// level-0 coefficients under the fine level from the fine ones: tiled faces' w = (sum of the
// 4 fine w) / 16 (w = b beta / h^2, h doubling), covered cells' a*alpha = mean of 8 children
void launch_avgdown_coefs(const AmrDev& A, const double* facoef, const double* fwx, const double* fwy,
                          const double* fwz, double* cacoef, double* cwx, double* cwy, double* cwz, cudaStream_t s);
void launch_zero_covered(const AmrDev& A, double* c, cudaStream_t s);
// outc/outf += transpose of the ghost-interpolation and reflux couplings applied to y
void launch_composite_transpose_couplings(const AmrDev& A, const Coefs& coarse, const Coefs& fine, const double* yc,
                                          const double* yf, double* outc, double* outf, cudaStream_t s);
void launch_grad_beta(const LevelDev& L, const double* phi, const double* lam, const double* beta, double b,
                      const int* cfidx, const CfGhost* cfg, const double* lamc, double hf_over_hc,
                      const unsigned char* covered, double* out, cudaStream_t s);

// sum over valid cells of x*y (deterministic: per-block partials, one block adds them)
void launch_dot(const LevelDev& L, const double* x, const double* y, double* partials, double* out, cudaStream_t s);
// out = a x + b y over n elements (ghosts included)
void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s);

}  // namespace gmg
