/*
 * gmg_oracle.c -- plain, slow FP64 CPU reference for the cell-centred geometric
 * multigrid solve of
 *
 *      a*alpha*phi - b*div(beta grad phi) = rhs            (operator equation, Sec. "Linear Solvers")
 *
 * on a BoxArray (Sec. "Basic data structures").  TEST INFRASTRUCTURE ONLY: this file
 * is the oracle that the CUDA path is checked against.  It is used by tests/, by the
 * smoke check and by the benchmark's CPU-baseline leg, never by the product path.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything here is written for clarity, not speed: single thread, one ghosted
 * array per box (Sec. "Containers for mesh data": the FAB's array includes its
 * ghost cells), brute-force box intersections for the ghost-cell exchange, and the
 * V-cycle steps in the order the method states them.
 *
 * Readings of the paper used here (the paper names the components but not their
 * exact form):
 *   - operator: 7-point finite-volume form of the operator equation; face beta is the
 *     harmonic mean of the two cell values; at a physical wall the face takes the
 *     interior cell's beta;
 *   - ghost cells (Sec. "Operations on a level"): copied from the box at the same level
 *     that owns the cell (periodic images included); at a homogeneous Dirichlet wall the
 *     ghost is minus the adjacent interior value (the wall value 0 sits on the face);
 *   - smoother: red-black Gauss-Seidel, colour = parity of i+j+k in the level's global
 *     index, ghosts refreshed before every colour, red first;
 *   - restriction (Sec. "Operations between levels": average of fine data): mean of the
 *     8 children; coarse alpha = mean of children; coarse face beta = mean of the 4 fine
 *     faces on the coarse face;
 *   - prolongation (Sec. "Operations between levels": interpolation): piecewise
 *     constant, added to the fine correction;
 *   - aggregation (Sec. "Linear Solvers"): when the boxes of a level can no longer be
 *     coarsened one by one, merge them into a single box and keep coarsening while the
 *     domain allows;
 *   - bottom solve (Sec. "Linear Solvers": Krylov bottom solver): unpreconditioned
 *     BiCGStab (van der Vorst 1992) from x0 = 0;
 *   - outer loop: phi += Vcycle(r); r = rhs - A phi; stop at ||r||_inf <= tol*||rhs||_inf.
 *   - singular problems (all periodic, a = 0): rhs, bottom rhs and the result are
 *     projected onto zero mean.
 *
 * Parity pins: every function here is pinned by tests in tests/test_oracle_*.py
 * (closed-form discrete eigen-solutions, second-order convergence on a manufactured
 * solution, dense direct solves, box-layout invariance, symmetry and conservation
 * identities, restriction/prolongation identities).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PERIODIC 0
#define ORC_DIRICHLET 1
#define ORC_MAXLEV 32

typedef struct {
  int nb;
  int *lo, *hi;          /* 3*nb, inclusive cell indices in this level's index space */
  int dlo[3], dhi[3];    /* domain box at this level, inclusive */
  int bclo[3], bchi[3];  /* boundary condition per side */
  double h[3];           /* cell size */
  int64_t *off;          /* offset of box b's ghosted array inside a level field */
  int64_t ntot;          /* total length of a level field */
  /* ghost map: field[gdst] = gfac * field[gsrc]; gsrc < 0 means "not filled here"
     (a coarse/fine ghost) */
  int64_t ng;
  int64_t *gdst, *gsrc;
  double *gfac;
  int *parent;           /* box on the next coarser level that contains coarsen(box), or NULL */
  /* coefficients on this level (ghosted layout; face slot i holds the face at i-1/2) */
  double *alpha, *bx, *by, *bz;
  /* work vectors for the V-cycle */
  double *e, *r, *t;
} olev;

typedef struct {
  int nlev;
  olev L[ORC_MAXLEV];
  double a, b;
  int singular;
  int nu1, nu2, bot_maxit;
  double bot_tol;
  int last_bottom_iters;
} oprob;

/* ------------------------------------------------------------------ layout */

static int bn(const olev* l, int b, int d) { return l->hi[3 * b + d] - l->lo[3 * b + d] + 1; }

/* flat index of local cell (i,j,k), each in [-1, n] */
static int64_t IX(const olev* l, int b, int i, int j, int k) {
  int64_t nx = bn(l, b, 0) + 2, ny = bn(l, b, 1) + 2;
  return l->off[b] + (int64_t)(i + 1) + nx * ((int64_t)(j + 1) + ny * (int64_t)(k + 1));
}

static int pmod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

static int inbox(const olev* l, int b, const int g[3]) {
  for (int d = 0; d < 3; ++d)
    if (g[d] < l->lo[3 * b + d] || g[d] > l->hi[3 * b + d]) return 0;
  return 1;
}

static int find_box(const olev* l, const int g[3]) {
  for (int b = 0; b < l->nb; ++b)
    if (inbox(l, b, g)) return b;
  return -1;
}

static void level_alloc(olev* l) {
  l->off = (int64_t*)malloc(sizeof(int64_t) * (l->nb + 1));
  int64_t o = 0;
  for (int b = 0; b < l->nb; ++b) {
    l->off[b] = o;
    o += (int64_t)(bn(l, b, 0) + 2) * (bn(l, b, 1) + 2) * (bn(l, b, 2) + 2);
  }
  l->off[l->nb] = o;
  l->ntot = o;
  l->alpha = (double*)calloc(o, sizeof(double));
  l->bx = (double*)calloc(o, sizeof(double));
  l->by = (double*)calloc(o, sizeof(double));
  l->bz = (double*)calloc(o, sizeof(double));
  l->e = (double*)calloc(o, sizeof(double));
  l->r = (double*)calloc(o, sizeof(double));
  l->t = (double*)calloc(o, sizeof(double));
}

/* Ghost map, built by brute force: for every face ghost cell of every box, look for
   the box at this level that owns the (periodically wrapped) cell.  Edge and corner
   ghosts are never read by the 7-point stencil and are left alone. */
static void build_ghost_map(olev* l) {
  int64_t cap = 0;
  for (int b = 0; b < l->nb; ++b)
    for (int d = 0; d < 3; ++d) {
      int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      cap += 2 * (int64_t)bn(l, b, d1) * bn(l, b, d2);
    }
  l->gdst = (int64_t*)malloc(sizeof(int64_t) * (cap + 1));
  l->gsrc = (int64_t*)malloc(sizeof(int64_t) * (cap + 1));
  l->gfac = (double*)malloc(sizeof(double) * (cap + 1));
  int64_t n = 0;
  for (int b = 0; b < l->nb; ++b) {
    for (int d = 0; d < 3; ++d) {
      int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      for (int side = 0; side < 2; ++side) {
        for (int u = 0; u < bn(l, b, d1); ++u) {
          for (int v = 0; v < bn(l, b, d2); ++v) {
            int loc[3];
            loc[d] = side ? bn(l, b, d) : -1;
            loc[d1] = u;
            loc[d2] = v;
            int g[3];
            for (int q = 0; q < 3; ++q) g[q] = l->lo[3 * b + q] + loc[q];
            int64_t dst = IX(l, b, loc[0], loc[1], loc[2]);
            int outside = (g[d] < l->dlo[d] || g[d] > l->dhi[d]);
            int bc = side ? l->bchi[d] : l->bclo[d];
            if (outside && bc == ORC_PERIODIC) {
              int len = l->dhi[d] - l->dlo[d] + 1;
              g[d] = l->dlo[d] + pmod(g[d] - l->dlo[d], len);
              outside = 0;
            }
            if (outside) {
              /* homogeneous Dirichlet: ghost = -(adjacent interior cell) */
              int in[3] = {loc[0], loc[1], loc[2]};
              in[d] = side ? bn(l, b, d) - 1 : 0;
              l->gdst[n] = dst;
              l->gsrc[n] = IX(l, b, in[0], in[1], in[2]);
              l->gfac[n] = -1.0;
            } else {
              int ob = find_box(l, g);
              l->gdst[n] = dst;
              if (ob < 0) {
                l->gsrc[n] = -1; /* coarse/fine ghost: not filled from this level */
                l->gfac[n] = 0.0;
              } else {
                l->gsrc[n] = IX(l, ob, g[0] - l->lo[3 * ob], g[1] - l->lo[3 * ob + 1],
                                g[2] - l->lo[3 * ob + 2]);
                l->gfac[n] = 1.0;
              }
            }
            ++n;
          }
        }
      }
    }
  }
  l->ng = n;
}

/* Sec. "Operations on a level": fill ghost cells from the owning box at the same level
   (or the physical boundary condition). */
static void fill_ghosts(const olev* l, double* f) {
  for (int64_t q = 0; q < l->ng; ++q)
    if (l->gsrc[q] >= 0) f[l->gdst[q]] = l->gfac[q] * f[l->gsrc[q]];
}

static int covers_domain(const olev* l) {
  int64_t vol = 0, dvol = 1;
  for (int b = 0; b < l->nb; ++b) vol += (int64_t)bn(l, b, 0) * bn(l, b, 1) * bn(l, b, 2);
  for (int d = 0; d < 3; ++d) dvol *= (l->dhi[d] - l->dlo[d] + 1);
  return vol == dvol; /* boxes are disjoint and inside the domain (checked at creation) */
}

/* ------------------------------------------------------------- hierarchy */

static void free_level(olev* l) {
  free(l->lo); free(l->hi); free(l->off); free(l->gdst); free(l->gsrc); free(l->gfac);
  free(l->parent); free(l->alpha); free(l->bx); free(l->by); free(l->bz);
  free(l->e); free(l->r); free(l->t);
  memset(l, 0, sizeof(*l));
}

/* Multigrid hierarchy (Sec. "Linear Solvers", with aggregation):
   - if every box has even lo, even size and size >= 4 in all directions, the coarse
     level holds each box coarsened by 2 (its parent is the box itself);
   - otherwise, if every box has even lo and even size, the boxes cover the domain and
     every domain edge is even and >= 4, the coarse level is the coarsened domain as a
     single box (aggregation);
   - otherwise this level is the bottom. */
static int make_coarse(const olev* f, olev* c) {
  int nb = f->nb;
  int per_box = 1, evenly = 1;
  for (int b = 0; b < nb; ++b)
    for (int d = 0; d < 3; ++d) {
      int lo = f->lo[3 * b + d], n = bn(f, b, d);
      if (pmod(lo, 2) != 0 || n % 2 != 0) { evenly = 0; per_box = 0; }
      if (n < 4) per_box = 0;
    }
  int agg = 0;
  if (!per_box && evenly && covers_domain(f)) {
    agg = 1;
    for (int d = 0; d < 3; ++d) {
      int n = f->dhi[d] - f->dlo[d] + 1;
      if (n % 2 != 0 || n < 4 || pmod(f->dlo[d], 2) != 0) agg = 0;
    }
  }
  if (!per_box && !agg) return 0;
  memset(c, 0, sizeof(*c));
  for (int d = 0; d < 3; ++d) {
    c->dlo[d] = f->dlo[d] / 2;
    c->dhi[d] = (f->dhi[d] + 1) / 2 - 1;
    c->bclo[d] = f->bclo[d];
    c->bchi[d] = f->bchi[d];
    c->h[d] = 2.0 * f->h[d];
  }
  c->nb = per_box ? nb : 1;
  c->lo = (int*)malloc(sizeof(int) * 3 * c->nb);
  c->hi = (int*)malloc(sizeof(int) * 3 * c->nb);
  ((olev*)f)->parent = (int*)malloc(sizeof(int) * nb);
  if (per_box) {
    for (int b = 0; b < nb; ++b) {
      for (int d = 0; d < 3; ++d) {
        c->lo[3 * b + d] = f->lo[3 * b + d] / 2;
        c->hi[3 * b + d] = (f->hi[3 * b + d] + 1) / 2 - 1;
      }
      f->parent[b] = b;
    }
  } else {
    for (int d = 0; d < 3; ++d) { c->lo[d] = c->dlo[d]; c->hi[d] = c->dhi[d]; }
    for (int b = 0; b < nb; ++b) f->parent[b] = 0;
  }
  level_alloc(c);
  build_ghost_map(c);
  return 1;
}

void* orc_create(const int* dlo, const int* dhi, const int* bclo, const int* bchi,
                 const double* plo, const double* phi_, int nb, const int* boxes) {
  oprob* p = (oprob*)calloc(1, sizeof(oprob));
  olev* l = &p->L[0];
  l->nb = nb;
  l->lo = (int*)malloc(sizeof(int) * 3 * nb);
  l->hi = (int*)malloc(sizeof(int) * 3 * nb);
  for (int b = 0; b < nb; ++b)
    for (int d = 0; d < 3; ++d) {
      l->lo[3 * b + d] = boxes[6 * b + d];
      l->hi[3 * b + d] = boxes[6 * b + 3 + d];
    }
  for (int d = 0; d < 3; ++d) {
    l->dlo[d] = dlo[d];
    l->dhi[d] = dhi[d];
    l->bclo[d] = bclo[d];
    l->bchi[d] = bchi[d];
    l->h[d] = (phi_[d] - plo[d]) / (double)(dhi[d] - dlo[d] + 1);
  }
  /* validity: boxes inside the domain and pairwise disjoint; periodic on both sides */
  for (int d = 0; d < 3; ++d)
    if ((bclo[d] == ORC_PERIODIC) != (bchi[d] == ORC_PERIODIC)) { free(l->lo); free(l->hi); free(p); return NULL; }
  for (int b = 0; b < nb; ++b) {
    for (int d = 0; d < 3; ++d)
      if (l->lo[3 * b + d] < dlo[d] || l->hi[3 * b + d] > dhi[d] || l->lo[3 * b + d] > l->hi[3 * b + d]) {
        free(l->lo); free(l->hi); free(p); return NULL;
      }
    for (int c = 0; c < b; ++c) {
      int overlap = 1;
      for (int d = 0; d < 3; ++d)
        if (l->hi[3 * b + d] < l->lo[3 * c + d] || l->hi[3 * c + d] < l->lo[3 * b + d]) overlap = 0;
      if (overlap) { free(l->lo); free(l->hi); free(p); return NULL; }
    }
  }
  level_alloc(l);
  build_ghost_map(l);
  p->nlev = 1;
  while (p->nlev < ORC_MAXLEV && make_coarse(&p->L[p->nlev - 1], &p->L[p->nlev])) p->nlev++;
  p->a = 0.0;
  p->b = 1.0;
  p->nu1 = 2;
  p->nu2 = 2;
  p->bot_maxit = 200;
  p->bot_tol = 1e-4;
  int allper = 1;
  for (int d = 0; d < 3; ++d) allper &= (bclo[d] == ORC_PERIODIC);
  p->singular = allper; /* until a != 0 is set */
  return p;
}

void orc_destroy(void* vp) {
  oprob* p = (oprob*)vp;
  if (!p) return;
  for (int m = 0; m < p->nlev; ++m) free_level(&p->L[m]);
  free(p);
}

int orc_nlevels(void* vp) { return ((oprob*)vp)->nlev; }
int orc_level_nboxes(void* vp, int m) { return ((oprob*)vp)->L[m].nb; }
int64_t orc_level_size(void* vp, int m) { return ((oprob*)vp)->L[m].ntot; }
void orc_level_boxes(void* vp, int m, int* out) {
  olev* l = &((oprob*)vp)->L[m];
  for (int b = 0; b < l->nb; ++b)
    for (int d = 0; d < 3; ++d) {
      out[6 * b + d] = l->lo[3 * b + d];
      out[6 * b + 3 + d] = l->hi[3 * b + d];
    }
}
void orc_level_domain(void* vp, int m, int* out) {
  olev* l = &((oprob*)vp)->L[m];
  for (int d = 0; d < 3; ++d) { out[d] = l->dlo[d]; out[3 + d] = l->dhi[d]; }
}
/* parent box of each box on the next coarser level (-1 at the bottom) */
void orc_level_parents(void* vp, int m, int* out) {
  olev* l = &((oprob*)vp)->L[m];
  for (int b = 0; b < l->nb; ++b) out[b] = l->parent ? l->parent[b] : -1;
}
void orc_set_params(void* vp, int nu1, int nu2, int bot_maxit, double bot_tol) {
  oprob* p = (oprob*)vp;
  p->nu1 = nu1; p->nu2 = nu2; p->bot_maxit = bot_maxit; p->bot_tol = bot_tol;
}
int orc_last_bottom_iters(void* vp) { return ((oprob*)vp)->last_bottom_iters; }

/* dense array over the level's domain (x fastest) <-> ghosted per-box layout */
void orc_dense_to_boxed(void* vp, int m, const double* dense, double* boxed) {
  olev* l = &((oprob*)vp)->L[m];
  int64_t nx = l->dhi[0] - l->dlo[0] + 1, ny = l->dhi[1] - l->dlo[1] + 1;
  memset(boxed, 0, sizeof(double) * l->ntot);
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) {
          int64_t gi = l->lo[3 * b] + i - l->dlo[0], gj = l->lo[3 * b + 1] + j - l->dlo[1],
                  gk = l->lo[3 * b + 2] + k - l->dlo[2];
          boxed[IX(l, b, i, j, k)] = dense[gi + nx * (gj + ny * gk)];
        }
}
void orc_boxed_to_dense(void* vp, int m, const double* boxed, double* dense) {
  olev* l = &((oprob*)vp)->L[m];
  int64_t nx = l->dhi[0] - l->dlo[0] + 1, ny = l->dhi[1] - l->dlo[1] + 1;
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) {
          int64_t gi = l->lo[3 * b] + i - l->dlo[0], gj = l->lo[3 * b + 1] + j - l->dlo[1],
                  gk = l->lo[3 * b + 2] + k - l->dlo[2];
          dense[gi + nx * (gj + ny * gk)] = boxed[IX(l, b, i, j, k)];
        }
}

/* ---------------------------------------------------------- coefficients */

/* Level-0 coefficients from cell-centred alpha and beta (dense over the domain).
   Face beta = harmonic mean of the two adjacent cells (periodic images across a
   periodic boundary); at a wall face, the interior cell's beta. */
static double dense_at(const olev* l, const double* dense, const int g[3]) {
  int64_t nx = l->dhi[0] - l->dlo[0] + 1, ny = l->dhi[1] - l->dlo[1] + 1;
  return dense[(g[0] - l->dlo[0]) + nx * ((g[1] - l->dlo[1]) + ny * (int64_t)(g[2] - l->dlo[2]))];
}

static void coarsen_coeffs(const olev* f, olev* c);

int orc_set_coeffs(void* vp, double a, double bsc, const double* alpha_dense, const double* beta_dense) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  p->a = a;
  p->b = bsc;
  int allper = 1;
  for (int d = 0; d < 3; ++d) allper &= (l->bclo[d] == ORC_PERIODIC);
  p->singular = allper && (a == 0.0);
  memset(l->alpha, 0, sizeof(double) * l->ntot);
  memset(l->bx, 0, sizeof(double) * l->ntot);
  memset(l->by, 0, sizeof(double) * l->ntot);
  memset(l->bz, 0, sizeof(double) * l->ntot);
  double* face[3] = {l->bx, l->by, l->bz};
  for (int b = 0; b < l->nb; ++b) {
    int n[3] = {bn(l, b, 0), bn(l, b, 1), bn(l, b, 2)};
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          int g[3] = {l->lo[3 * b] + i, l->lo[3 * b + 1] + j, l->lo[3 * b + 2] + k};
          l->alpha[IX(l, b, i, j, k)] = alpha_dense ? dense_at(l, alpha_dense, g) : 1.0;
        }
    for (int d = 0; d < 3; ++d) {
      int ext[3] = {n[0], n[1], n[2]};
      ext[d] += 1; /* faces 0..n along d */
      for (int k = 0; k < ext[2]; ++k)
        for (int j = 0; j < ext[1]; ++j)
          for (int i = 0; i < ext[0]; ++i) {
            int loc[3] = {i, j, k};
            int gR[3], gL[3];
            for (int q = 0; q < 3; ++q) gR[q] = gL[q] = l->lo[3 * b + q] + loc[q];
            gL[d] -= 1;
            double val;
            if (!beta_dense) {
              val = 1.0;
            } else {
              int Lout = gL[d] < l->dlo[d], Rout = gR[d] > l->dhi[d];
              int per = (l->bclo[d] == ORC_PERIODIC);
              int len = l->dhi[d] - l->dlo[d] + 1;
              if (per) {
                gL[d] = l->dlo[d] + pmod(gL[d] - l->dlo[d], len);
                gR[d] = l->dlo[d] + pmod(gR[d] - l->dlo[d], len);
                Lout = Rout = 0;
              }
              if (Lout) val = dense_at(l, beta_dense, gR);
              else if (Rout) val = dense_at(l, beta_dense, gL);
              else {
                double bl = dense_at(l, beta_dense, gL), br = dense_at(l, beta_dense, gR);
                val = 2.0 * bl * br / (bl + br);
              }
            }
            face[d][IX(l, b, loc[0], loc[1], loc[2])] = val;
          }
    }
  }
  for (int m = 0; m + 1 < p->nlev; ++m) coarsen_coeffs(&p->L[m], &p->L[m + 1]);
  return 0;
}

/* Sec. "Operations between levels" (average of fine data): coarse alpha is the mean of
   the 8 children; a coarse face takes the mean of the 4 fine faces that tile it. */
static void coarsen_coeffs(const olev* f, olev* c) {
  memset(c->alpha, 0, sizeof(double) * c->ntot);
  memset(c->bx, 0, sizeof(double) * c->ntot);
  memset(c->by, 0, sizeof(double) * c->ntot);
  memset(c->bz, 0, sizeof(double) * c->ntot);
  double* ff[3] = {f->bx, f->by, f->bz};
  double* cf[3] = {c->bx, c->by, c->bz};
  for (int fb = 0; fb < f->nb; ++fb) {
    int P = f->parent[fb];
    int clo[3], chi[3];
    for (int d = 0; d < 3; ++d) {
      clo[d] = f->lo[3 * fb + d] / 2;
      chi[d] = (f->hi[3 * fb + d] + 1) / 2 - 1;
    }
    for (int K = clo[2]; K <= chi[2]; ++K)
      for (int J = clo[1]; J <= chi[1]; ++J)
        for (int I = clo[0]; I <= chi[0]; ++I) {
          double s = 0.0;
          for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
              for (int di = 0; di < 2; ++di)
                s += f->alpha[IX(f, fb, 2 * I + di - f->lo[3 * fb], 2 * J + dj - f->lo[3 * fb + 1],
                                 2 * K + dk - f->lo[3 * fb + 2])];
          c->alpha[IX(c, P, I - c->lo[3 * P], J - c->lo[3 * P + 1], K - c->lo[3 * P + 2])] = s / 8.0;
        }
    for (int d = 0; d < 3; ++d) {
      int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      int ehi[3] = {chi[0], chi[1], chi[2]};
      ehi[d] += 1;
      for (int K = clo[2]; K <= ehi[2]; ++K)
        for (int J = clo[1]; J <= ehi[1]; ++J)
          for (int I = clo[0]; I <= ehi[0]; ++I) {
            int C[3] = {I, J, K};
            double s = 0.0;
            for (int u = 0; u < 2; ++u)
              for (int v = 0; v < 2; ++v) {
                int F[3];
                F[d] = 2 * C[d];
                F[d1] = 2 * C[d1] + u;
                F[d2] = 2 * C[d2] + v;
                s += ff[d][IX(f, fb, F[0] - f->lo[3 * fb], F[1] - f->lo[3 * fb + 1], F[2] - f->lo[3 * fb + 2])];
              }
            cf[d][IX(c, P, I - c->lo[3 * P], J - c->lo[3 * P + 1], K - c->lo[3 * P + 2])] = s / 4.0;
          }
    }
  }
}

void orc_get_coeffs(void* vp, int m, double* alpha, double* bx, double* by, double* bz) {
  olev* l = &((oprob*)vp)->L[m];
  if (alpha) memcpy(alpha, l->alpha, sizeof(double) * l->ntot);
  if (bx) memcpy(bx, l->bx, sizeof(double) * l->ntot);
  if (by) memcpy(by, l->by, sizeof(double) * l->ntot);
  if (bz) memcpy(bz, l->bz, sizeof(double) * l->ntot);
}

/* ----------------------------------------------------------- level steps */

/* (A phi) at one valid cell, operator equation of Sec. "Linear Solvers":
   a*alpha*phi - b * sum_d h_d^-2 [ beta_{+}(phi_{+} - phi) - beta_{-}(phi - phi_{-}) ] */
static double op_cell(const oprob* p, const olev* l, const double* f, int b, int i, int j, int k) {
  double c = f[IX(l, b, i, j, k)];
  double hx2 = l->h[0] * l->h[0], hy2 = l->h[1] * l->h[1], hz2 = l->h[2] * l->h[2];
  double fx = (l->bx[IX(l, b, i + 1, j, k)] * (f[IX(l, b, i + 1, j, k)] - c) -
               l->bx[IX(l, b, i, j, k)] * (c - f[IX(l, b, i - 1, j, k)])) / hx2;
  double fy = (l->by[IX(l, b, i, j + 1, k)] * (f[IX(l, b, i, j + 1, k)] - c) -
               l->by[IX(l, b, i, j, k)] * (c - f[IX(l, b, i, j - 1, k)])) / hy2;
  double fz = (l->bz[IX(l, b, i, j, k + 1)] * (f[IX(l, b, i, j, k + 1)] - c) -
               l->bz[IX(l, b, i, j, k)] * (c - f[IX(l, b, i, j, k - 1)])) / hz2;
  return p->a * l->alpha[IX(l, b, i, j, k)] * c - p->b * (fx + fy + fz);
}

/* out = A phi on MG level m (ghosts of phi refreshed first) */
void orc_apply_level(void* vp, int m, double* phi, double* out) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[m];
  fill_ghosts(l, phi);
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) out[IX(l, b, i, j, k)] = op_cell(p, l, phi, b, i, j, k);
}

void orc_fill_ghosts(void* vp, int m, double* f) { fill_ghosts(&((oprob*)vp)->L[m], f); }

/* One colour of red-black Gauss-Seidel: refresh ghosts, then for every cell whose
   global (i+j+k) parity equals `colour`, solve its row for phi using the current
   neighbour values:
     phi = (rhs + b*sum_f h_f^-2 beta_f phi_nbr) / (a*alpha + b*sum_f h_f^-2 beta_f),
   faces taken in the order x-, x+, y-, y+, z-, z+. */
void orc_smooth_colour(void* vp, int m, double* phi, const double* rhs, int colour) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[m];
  fill_ghosts(l, phi);
  double ihx2 = 1.0 / (l->h[0] * l->h[0]), ihy2 = 1.0 / (l->h[1] * l->h[1]), ihz2 = 1.0 / (l->h[2] * l->h[2]);
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) {
          int gs = l->lo[3 * b] + i + l->lo[3 * b + 1] + j + l->lo[3 * b + 2] + k;
          if (pmod(gs, 2) != colour) continue;
          double wxm = ihx2 * l->bx[IX(l, b, i, j, k)], wxp = ihx2 * l->bx[IX(l, b, i + 1, j, k)];
          double wym = ihy2 * l->by[IX(l, b, i, j, k)], wyp = ihy2 * l->by[IX(l, b, i, j + 1, k)];
          double wzm = ihz2 * l->bz[IX(l, b, i, j, k)], wzp = ihz2 * l->bz[IX(l, b, i, j, k + 1)];
          double num = wxm * phi[IX(l, b, i - 1, j, k)] + wxp * phi[IX(l, b, i + 1, j, k)] +
                       wym * phi[IX(l, b, i, j - 1, k)] + wyp * phi[IX(l, b, i, j + 1, k)] +
                       wzm * phi[IX(l, b, i, j, k - 1)] + wzp * phi[IX(l, b, i, j, k + 1)];
          double den = wxm + wxp + wym + wyp + wzm + wzp;
          phi[IX(l, b, i, j, k)] =
              (rhs[IX(l, b, i, j, k)] + p->b * num) / (p->a * l->alpha[IX(l, b, i, j, k)] + p->b * den);
        }
}

/* r = rhs - A phi */
void orc_residual(void* vp, int m, double* phi, const double* rhs, double* r) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[m];
  fill_ghosts(l, phi);
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i)
          r[IX(l, b, i, j, k)] = rhs[IX(l, b, i, j, k)] - op_cell(p, l, phi, b, i, j, k);
}

/* Average-down restriction, level m -> m+1: coarse value = mean of its 8 children. */
void orc_restrict(void* vp, int m, const double* fine, double* coarse) {
  oprob* p = (oprob*)vp;
  olev* f = &p->L[m];
  olev* c = &p->L[m + 1];
  for (int fb = 0; fb < f->nb; ++fb) {
    int P = f->parent[fb];
    for (int K = f->lo[3 * fb + 2] / 2; K <= (f->hi[3 * fb + 2] + 1) / 2 - 1; ++K)
      for (int J = f->lo[3 * fb + 1] / 2; J <= (f->hi[3 * fb + 1] + 1) / 2 - 1; ++J)
        for (int I = f->lo[3 * fb] / 2; I <= (f->hi[3 * fb] + 1) / 2 - 1; ++I) {
          double s = 0.0;
          for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
              for (int di = 0; di < 2; ++di)
                s += fine[IX(f, fb, 2 * I + di - f->lo[3 * fb], 2 * J + dj - f->lo[3 * fb + 1],
                             2 * K + dk - f->lo[3 * fb + 2])];
          coarse[IX(c, P, I - c->lo[3 * P], J - c->lo[3 * P + 1], K - c->lo[3 * P + 2])] = s / 8.0;
        }
  }
}

/* Piecewise-constant prolongation of a coarse correction, added to the fine one. */
void orc_prolong_add(void* vp, int m, const double* coarse, double* fine) {
  oprob* p = (oprob*)vp;
  olev* f = &p->L[m];
  olev* c = &p->L[m + 1];
  for (int fb = 0; fb < f->nb; ++fb) {
    int P = f->parent[fb];
    for (int k = 0; k < bn(f, fb, 2); ++k)
      for (int j = 0; j < bn(f, fb, 1); ++j)
        for (int i = 0; i < bn(f, fb, 0); ++i) {
          int I = (f->lo[3 * fb] + i) / 2, J = (f->lo[3 * fb + 1] + j) / 2, K = (f->lo[3 * fb + 2] + k) / 2;
          fine[IX(f, fb, i, j, k)] += coarse[IX(c, P, I - c->lo[3 * P], J - c->lo[3 * P + 1], K - c->lo[3 * P + 2])];
        }
  }
}

/* ------------------------------------------------ reductions on a level */

static double lev_dot(const olev* l, const double* x, const double* y) {
  double s = 0.0;
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) s += x[IX(l, b, i, j, k)] * y[IX(l, b, i, j, k)];
  return s;
}

static double lev_norminf(const olev* l, const double* x) {
  double s = 0.0;
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) {
          double v = fabs(x[IX(l, b, i, j, k)]);
          if (v > s || v != v) s = v;
        }
  return s;
}

static double lev_sum(const olev* l, const double* x) {
  double s = 0.0;
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) s += x[IX(l, b, i, j, k)];
  return s;
}

static int64_t lev_ncells(const olev* l) {
  int64_t n = 0;
  for (int b = 0; b < l->nb; ++b) n += (int64_t)bn(l, b, 0) * bn(l, b, 1) * bn(l, b, 2);
  return n;
}

static void lev_add_const(const olev* l, double* x, double c) {
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) x[IX(l, b, i, j, k)] += c;
}

double orc_level_dot(void* vp, int m, const double* x, const double* y) { return lev_dot(&((oprob*)vp)->L[m], x, y); }
double orc_level_norminf(void* vp, int m, const double* x) { return lev_norminf(&((oprob*)vp)->L[m], x); }

/* ----------------------------------------------------------- bottom solve */

/* Unpreconditioned BiCGStab (van der Vorst 1992) for A x = rhs on the bottom level,
   x0 = 0.  Stops when ||r||_inf <= bot_tol * ||r0||_inf, after bot_maxit iterations,
   or on breakdown (|rho| or |(rhat, v)| below 1e-300, or (t,t) = 0), keeping the
   current iterate.  For a singular problem the right-hand side is first projected onto
   zero mean and so is the result.  Returns the number of iterations taken. */
int orc_bottom(void* vp, const double* rhs_in, double* x) {
  oprob* p = (oprob*)vp;
  int m = p->nlev - 1;
  olev* l = &p->L[m];
  int64_t n = l->ntot;
  double* r = (double*)calloc(n, sizeof(double));
  double* rh = (double*)calloc(n, sizeof(double));
  double* pp = (double*)calloc(n, sizeof(double));
  double* v = (double*)calloc(n, sizeof(double));
  double* s = (double*)calloc(n, sizeof(double));
  double* t = (double*)calloc(n, sizeof(double));
  memcpy(r, rhs_in, sizeof(double) * n);
  if (p->singular) lev_add_const(l, r, -lev_sum(l, r) / (double)lev_ncells(l));
  memset(x, 0, sizeof(double) * n);
  memcpy(rh, r, sizeof(double) * n);
  double r0 = lev_norminf(l, r);
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0;
  if (r0 > 0.0) {
    for (it = 1; it <= p->bot_maxit; ++it) {
      double rho = lev_dot(l, rh, r);
      if (fabs(rho) < 1e-300) { it--; break; }
      double beta = (rho / rho_old) * (alpha / omega);
      for (int64_t q = 0; q < n; ++q) pp[q] = r[q] + beta * (pp[q] - omega * v[q]);
      orc_apply_level(vp, m, pp, v);
      double rv = lev_dot(l, rh, v);
      if (fabs(rv) < 1e-300) { it--; break; }
      alpha = rho / rv;
      for (int64_t q = 0; q < n; ++q) s[q] = r[q] - alpha * v[q];
      if (lev_norminf(l, s) <= p->bot_tol * r0) {
        for (int64_t q = 0; q < n; ++q) x[q] += alpha * pp[q];
        break;
      }
      orc_apply_level(vp, m, s, t);
      double tt = lev_dot(l, t, t);
      if (tt == 0.0) {
        for (int64_t q = 0; q < n; ++q) x[q] += alpha * pp[q];
        break;
      }
      omega = lev_dot(l, t, s) / tt;
      for (int64_t q = 0; q < n; ++q) {
        x[q] += alpha * pp[q] + omega * s[q];
        r[q] = s[q] - omega * t[q];
      }
      if (lev_norminf(l, r) <= p->bot_tol * r0) break;
      rho_old = rho;
    }
    if (it > p->bot_maxit) it = p->bot_maxit;
  }
  if (p->singular) lev_add_const(l, x, -lev_sum(l, x) / (double)lev_ncells(l));
  /* ghosts of x are left as computed; callers only read valid cells */
  free(r); free(rh); free(pp); free(v); free(s); free(t);
  p->last_bottom_iters = it;
  return it;
}

/* --------------------------------------------------------------- V-cycle */

/* V-cycle on the correction equation A_m e = r at MG level m, e = 0 on entry:
   nu1 smoothing sweeps, residual, restriction, recursion, prolongation, nu2 sweeps. */
void orc_vcycle(void* vp, int m, double* e, const double* r) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[m];
  memset(e, 0, sizeof(double) * l->ntot);
  if (m == p->nlev - 1) {
    orc_bottom(vp, r, e);
    return;
  }
  for (int s = 0; s < p->nu1; ++s) {
    orc_smooth_colour(vp, m, e, r, 0);
    orc_smooth_colour(vp, m, e, r, 1);
  }
  orc_residual(vp, m, e, r, l->t);
  olev* c = &p->L[m + 1];
  memset(c->r, 0, sizeof(double) * c->ntot);
  orc_restrict(vp, m, l->t, c->r);
  orc_vcycle(vp, m + 1, c->e, c->r);
  orc_prolong_add(vp, m, c->e, e);
  for (int s = 0; s < p->nu2; ++s) {
    orc_smooth_colour(vp, m, e, r, 0);
    orc_smooth_colour(vp, m, e, r, 1);
  }
}

/* ------------------------------------------------------------ outer loop */

/* Solve A phi = rhs (dense arrays over the level-0 domain) from phi = 0:
   phi += Vcycle(r), r = rhs - A phi, until ||r||_inf <= max(tol_rel*||rhs||_inf, tol_abs)
   or maxit iterations.  hist[0..iters] receives ||r||_inf after each iteration.
   status: 0 converged, -1 bad input (nonzero-mean rhs of a singular problem without
   project_mean), -2 not converged, -3 diverged (non-finite residual). */
int orc_solve(void* vp, const double* rhs_dense, double* phi_dense, double tol_rel, double tol_abs, int maxit,
              int project_mean, double* hist, int* status) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  int64_t n = l->ntot;
  double* rhs = (double*)calloc(n, sizeof(double));
  double* phi = (double*)calloc(n, sizeof(double));
  double* r = (double*)calloc(n, sizeof(double));
  double* e = (double*)calloc(n, sizeof(double));
  orc_dense_to_boxed(vp, 0, rhs_dense, rhs);
  double rhsnorm = lev_norminf(l, rhs);
  *status = 0;
  if (p->singular) {
    double mean = lev_sum(l, rhs) / (double)lev_ncells(l);
    if (fabs(mean) > 1e-12 * rhsnorm && !project_mean) {
      *status = -1;
      free(rhs); free(phi); free(r); free(e);
      return 0;
    }
    lev_add_const(l, rhs, -mean);
  }
  memcpy(r, rhs, sizeof(double) * n);
  double target = tol_rel * rhsnorm;
  if (tol_abs > target) target = tol_abs;
  double rn = lev_norminf(l, r);
  if (hist) hist[0] = rn;
  int it = 0;
  while (!(rn <= target) && it < maxit) {
    orc_vcycle(vp, 0, e, r);
    for (int64_t q = 0; q < n; ++q) phi[q] += e[q];
    orc_residual(vp, 0, phi, rhs, r);
    rn = lev_norminf(l, r);
    ++it;
    if (hist) hist[it] = rn;
    if (!(rn == rn) || isinf(rn)) { *status = -3; break; }
  }
  if (*status == 0 && !(rn <= target)) *status = -2;
  if (p->singular) lev_add_const(l, phi, -lev_sum(l, phi) / (double)lev_ncells(l));
  orc_boxed_to_dense(vp, 0, phi, phi_dense);
  free(rhs); free(phi); free(r); free(e);
  return it;
}

/* out = A phi for dense level-0 arrays */
void orc_apply(void* vp, const double* phi_dense, double* out_dense) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  double* phi = (double*)calloc(l->ntot, sizeof(double));
  double* out = (double*)calloc(l->ntot, sizeof(double));
  orc_dense_to_boxed(vp, 0, phi_dense, phi);
  orc_apply_level(vp, 0, phi, out);
  orc_boxed_to_dense(vp, 0, out, out_dense);
  free(phi); free(out);
}
