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
 * Everything here is written for clarity, not speed: one ghosted array per box (Sec.
 * "Containers for mesh data": the FAB's array includes its ghost cells), brute-force box
 * intersections for the ghost-cell exchange, and the V-cycle steps in the order the method
 * states them.  By default one thread; orc_set_threads(n) lets the loops over boxes whose
 * iterations write disjoint cells and compute each cell exactly as one thread does (colour
 * sweeps, residuals, operator applications, restriction, interpolation, ghost copies,
 * max-norms) run on n OpenMP threads -- the results are bitwise those of one thread.  Sums
 * stay sequential.
 *
 * Readings of the paper used here (the paper names the components but not their
 * exact form):
 *   - operator: 7-point finite-volume form of the operator equation; face beta is the
 *     harmonic mean of the two cell values; at a physical wall the face takes the
 *     interior cell's beta;
 *   - ghost cells (Sec. "Operations on a level"): copied from the box at the same level
 *     that owns the cell (periodic images included); at a Dirichlet wall the ghost is
 *     2g minus the adjacent interior value (the wall value g sits on the face: linear
 *     extrapolation), at a Neumann wall the interior value plus h*g (g the outward normal
 *     derivative); g = 0 (homogeneous walls) unless wall values are given, and always 0
 *     in the correction equations of the V-cycle;
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
 *   - outer loop: r0 = rhs - A(0) (nonzero only through wall values); phi += Vcycle(r);
 *     r = rhs - A phi with the wall values; stop at ||r||_inf <= tol*||r0||_inf.
 *   - singular problems (no Dirichlet wall, a = 0): the initial residual, the bottom rhs
 *     and the result are projected onto zero mean.
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
#define ORC_NEUMANN 2
#define ORC_DIRICHLET_QUAD 3 /* accepted by orc_create: a Dirichlet side whose ghosts take the quadratic rule */
#define ORC_MAXLEV 32

typedef struct {
  int nb;
  int *lo, *hi;          /* 3*nb, inclusive cell indices in this level's index space */
  int dlo[3], dhi[3];    /* domain box at this level, inclusive */
  int bclo[3], bchi[3];  /* boundary condition per side */
  int qlo[3], qhi[3];    /* 1: that Dirichlet side extrapolates quadratically (ghost_quad) */
  double h[3];           /* cell size */
  int64_t *off;          /* offset of box b's ghosted array inside a level field */
  int64_t ntot;          /* total length of a level field */
  /* ghost map: field[gdst] = gfac * field[gsrc]; gsrc < 0 means "not filled here"
     (a coarse/fine ghost) */
  int64_t ng;
  int64_t *gdst, *gsrc;
  double *gfac;
  /* quadratic Dirichlet ghosts: the second interior cell inward (the ghost is
     -2 f[gsrc] + f[gsrc2] / 3); -1 for every other entry */
  int64_t *gsrc2;
  int64_t *ginv;         /* element -> ghost-map entry (-1: none), built on first use */
  /* per ghost-map entry at a physical wall: the wall face (2*d + side) and the index of
     the ghost's tangential position in that face's value array; gwall = -1 elsewhere */
  int *gwall;
  int64_t *gtan;
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
  double* bcval[6];  /* level-0 wall values per face (2*d + side), or NULL (g = 0) */
  int bot_cg;        /* bottom solver: 0 BiCGStab, 1 conjugate gradients */
  int post_rev;      /* post-smoothing colour order: 0 red then black, 1 black then red */
  int prolong;       /* interpolation of the coarse correction: 0 piecewise constant, 1 trilinear */
} oprob;

/* ------------------------------------------------------------------ layout */

/* OpenMP threads of the box loops (1: sequential) */
static int g_threads = 1;
void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return g_threads; }

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
  l->gwall = (int*)malloc(sizeof(int) * (cap + 1));
  l->gtan = (int64_t*)malloc(sizeof(int64_t) * (cap + 1));
  l->gsrc2 = (int64_t*)malloc(sizeof(int64_t) * (cap + 1));
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
            l->gwall[n] = -1;
            l->gtan[n] = 0;
            l->gsrc2[n] = -1;
            if (outside) {
              /* wall: ghost = -(adjacent interior cell) at a Dirichlet wall, +(adjacent
                 interior cell) at a Neumann wall; the wall value's part is added by
                 fill_ghosts_bc.  Tangential axes of the face in increasing order, the
                 lower one fastest. */
              int in[3] = {loc[0], loc[1], loc[2]};
              int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
              in[d] = side ? bn(l, b, d) - 1 : 0;
              l->gdst[n] = dst;
              l->gsrc[n] = IX(l, b, in[0], in[1], in[2]);
              l->gfac[n] = bc == ORC_NEUMANN ? 1.0 : -1.0;
              l->gwall[n] = 2 * d + side;
              l->gtan[n] = (int64_t)(g[t1] - l->dlo[t1]) + (int64_t)(l->dhi[t1] - l->dlo[t1] + 1) * (g[t2] - l->dlo[t2]);
              if (bc == ORC_DIRICHLET && (side ? l->qhi[d] : l->qlo[d]) && bn(l, b, d) >= 2) {
                /* quadratic rule: the parabola through the wall value (on the face) and the
                   two interior cell centres, read at the ghost's centre */
                in[d] = side ? bn(l, b, d) - 2 : 1;
                l->gsrc2[n] = IX(l, b, in[0], in[1], in[2]);
                l->gfac[n] = -2.0;
              }
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
  #pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (int64_t q = 0; q < l->ng; ++q) {
    if (l->gsrc2[q] >= 0)
      f[l->gdst[q]] = -2.0 * f[l->gsrc[q]] + f[l->gsrc2[q]] / 3.0;
    else if (l->gsrc[q] >= 0)
      f[l->gdst[q]] = l->gfac[q] * f[l->gsrc[q]];
  }
}

/* Dirichlet wall order, per side: the homogeneous ghost of a box's wall cell phi_0 is
   -phi_0 (linear: the line through phi_0 and 0 on the face), or, where the side is quadratic
   and the box has two cells along the wall normal, -2 phi_0 + phi_1 / 3 (the parabola
   through 0 on the face, phi_0 and the next cell inward phi_1, read half a cell outside
   the face).  A wall value g adds 2 g (linear) or 8 g / 3 (quadratic). */
static int quad_face(const olev* l, int b, const int c[3], int d, int side) {
  int n = bn(l, b, d);
  if (n < 2 || c[d] != (side ? n - 1 : 0)) return 0;
  int g = l->lo[3 * b + d] + c[d] + (side ? 1 : -1);
  if (g >= l->dlo[d] && g <= l->dhi[d]) return 0;
  return (side ? l->bchi[d] : l->bclo[d]) == ORC_DIRICHLET && (side ? l->qhi[d] : l->qlo[d]);
}

/* a level with no Dirichlet wall has the constants in the null space of A when a = 0 */
static int has_dirichlet(const olev* l) {
  for (int d = 0; d < 3; ++d)
    if (l->bclo[d] == ORC_DIRICHLET || l->bchi[d] == ORC_DIRICHLET) return 1;
  return 0;
}

static int covers_domain(const olev* l) {
  int64_t vol = 0, dvol = 1;
  for (int b = 0; b < l->nb; ++b) vol += (int64_t)bn(l, b, 0) * bn(l, b, 1) * bn(l, b, 2);
  for (int d = 0; d < 3; ++d) dvol *= (l->dhi[d] - l->dlo[d] + 1);
  return vol == dvol; /* boxes are disjoint and inside the domain (checked at creation) */
}

/* ------------------------------------------------------------- hierarchy */

static void free_level(olev* l) {
  free(l->lo); free(l->hi); free(l->off); free(l->gdst); free(l->gsrc); free(l->gfac); free(l->gwall); free(l->gtan);
  free(l->gsrc2); free(l->ginv);
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
    c->qlo[d] = f->qlo[d];
    c->qhi[d] = f->qhi[d];
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
    l->qlo[d] = bclo[d] == ORC_DIRICHLET_QUAD;
    l->qhi[d] = bchi[d] == ORC_DIRICHLET_QUAD;
    l->bclo[d] = l->qlo[d] ? ORC_DIRICHLET : bclo[d];
    l->bchi[d] = l->qhi[d] ? ORC_DIRICHLET : bchi[d];
    l->h[d] = (phi_[d] - plo[d]) / (double)(dhi[d] - dlo[d] + 1);
  }
  /* validity: boxes inside the domain and pairwise disjoint; periodic on both sides */
  for (int d = 0; d < 3; ++d)
    if ((bclo[d] == ORC_PERIODIC) != (bchi[d] == ORC_PERIODIC) || bclo[d] < 0 || bclo[d] > 3 || bchi[d] < 0 ||
        bchi[d] > 3) {
      free(l->lo); free(l->hi); free(p); return NULL;
    }
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
  p->singular = !has_dirichlet(l); /* until a != 0 is set */
  return p;
}

void orc_destroy(void* vp) {
  oprob* p = (oprob*)vp;
  if (!p) return;
  for (int m = 0; m < p->nlev; ++m) free_level(&p->L[m]);
  for (int f = 0; f < 6; ++f) free(p->bcval[f]);
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
/* bottom_cg: the bottom solve by conjugate gradients instead of BiCGStab; post_reverse: the
   post-smoothing sweeps take black before red, the reverse of the pre-smoothing order, which
   makes the V-cycle a symmetric operator when A is (the preconditioner of the top-level
   conjugate gradients) */
void orc_set_cycle(void* vp, int bottom_cg, int post_reverse) {
  oprob* p = (oprob*)vp;
  p->bot_cg = bottom_cg;
  p->post_rev = post_reverse;
}

/* Interpolation of the coarse correction (Sec. "Operations between levels": the paper names
   interpolation without fixing its order): 0 piecewise constant (default), 1 trilinear. */
void orc_set_prolong(void* vp, int mode) { ((oprob*)vp)->prolong = mode; }

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
  p->singular = !has_dirichlet(l) && (a == 0.0);
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
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1)
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
   faces taken in the order x-, x+, y-, y+, z-, z+.  A face on a quadratic Dirichlet wall is
   taken into the row exactly: its ghost -2 phi + phi_1 / 3 depends on the cell itself, so
   the face adds w_f phi_1 / 3 to the numerator and (1 - (-2)) w_f = 3 w_f to the
   denominator (the cell's row solved exactly, as Gauss-Seidel does; the linear wall's
   ghost -phi is taken from the ghost fill, as every other neighbour). */
void orc_smooth_colour(void* vp, int m, double* phi, const double* rhs, int colour) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[m];
  fill_ghosts(l, phi);
  double ihx2 = 1.0 / (l->h[0] * l->h[0]), ihy2 = 1.0 / (l->h[1] * l->h[1]), ihz2 = 1.0 / (l->h[2] * l->h[2]);
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1)
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
          const int c[3] = {i, j, k};
          int quad = 0;
          for (int d = 0; d < 3; ++d) quad |= quad_face(l, b, c, d, 0) | quad_face(l, b, c, d, 1);
          if (quad) { /* face by face, in the same order */
            const double w[6] = {wxm, wxp, wym, wyp, wzm, wzp};
            num = 0.0;
            den = 0.0;
            for (int f = 0; f < 6; ++f) {
              int d = f / 2, side = f % 2, nb[3] = {i, j, k}, in2[3] = {i, j, k};
              nb[d] += side ? 1 : -1;
              if (quad_face(l, b, c, d, side)) {
                in2[d] += side ? -1 : 1;
                num += w[f] * (phi[IX(l, b, in2[0], in2[1], in2[2])] / 3.0);
                den += 3.0 * w[f];
              } else {
                num += w[f] * phi[IX(l, b, nb[0], nb[1], nb[2])];
                den += w[f];
              }
            }
          }
          phi[IX(l, b, i, j, k)] =
              (rhs[IX(l, b, i, j, k)] + p->b * num) / (p->a * l->alpha[IX(l, b, i, j, k)] + p->b * den);
        }
}

/* r = rhs - A phi */
void orc_residual(void* vp, int m, double* phi, const double* rhs, double* r) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[m];
  fill_ghosts(l, phi);
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1)
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
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1)
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

/* Value of a coarse-level field at global cell index G, which may lie one cell beyond the
   domain: the correction's homogeneous boundary rule extends it -- a periodic axis wraps, a
   wall mirrors the index into the domain (ghost -1 <-> cell 0) with the factor -1 for a
   Dirichlet wall and +1 for a Neumann wall, one factor per axis crossed. */
static double coarse_value(const olev* c, const double* e, const int G[3]) {
  int g[3];
  double sign = 1.0;
  for (int d = 0; d < 3; ++d) {
    int n = c->dhi[d] - c->dlo[d] + 1, rel = G[d] - c->dlo[d];
    if (rel < 0 || rel >= n) {
      int bc = rel < 0 ? c->bclo[d] : c->bchi[d];
      if (bc == ORC_PERIODIC) {
        rel = pmod(rel, n);
      } else {
        rel = rel < 0 ? -1 - rel : 2 * n - 1 - rel;
        if (bc == ORC_DIRICHLET) sign = -sign;
      }
    }
    g[d] = c->dlo[d] + rel;
  }
  int b = find_box(c, g);
  return sign * e[IX(c, b, g[0] - c->lo[3 * b], g[1] - c->lo[3 * b + 1], g[2] - c->lo[3 * b + 2])];
}

/* Trilinear interpolation at fine cell g: the fine centre lies a quarter of a coarse cell from
   its parent's centre along each axis, towards the side s_d = +1 (odd g_d) or -1 (even g_d);
   the weights are 3/4 on the parent's coordinate and 1/4 on the neighbour's, per axis, and
   the eight products are summed z outermost, then y, then x. */
static double trilinear_at(const olev* c, const double* e, const int g[3]) {
  static const double w[2] = {0.75, 0.25};
  int G[3], s[3];
  for (int d = 0; d < 3; ++d) {
    G[d] = g[d] >= 0 ? g[d] / 2 : -((1 - g[d]) / 2);
    s[d] = (g[d] - 2 * G[d]) ? 1 : -1;
  }
  double v = 0.0;
  for (int cz = 0; cz < 2; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        int H[3] = {G[0] + cx * s[0], G[1] + cy * s[1], G[2] + cz * s[2]};
        v += (w[cx] * w[cy] * w[cz]) * coarse_value(c, e, H);
      }
  return v;
}

/* Prolongation of a coarse correction, added to the fine one: piecewise constant (every
   fine cell takes its parent's value) or trilinear (orc_set_prolong). */
void orc_prolong_add(void* vp, int m, const double* coarse, double* fine) {
  oprob* p = (oprob*)vp;
  olev* f = &p->L[m];
  olev* c = &p->L[m + 1];
  if (p->prolong == 1) {
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1)
    for (int fb = 0; fb < f->nb; ++fb)
      for (int k = 0; k < bn(f, fb, 2); ++k)
        for (int j = 0; j < bn(f, fb, 1); ++j)
          for (int i = 0; i < bn(f, fb, 0); ++i) {
            int g[3] = {f->lo[3 * fb] + i, f->lo[3 * fb + 1] + j, f->lo[3 * fb + 2] + k};
            fine[IX(f, fb, i, j, k)] += trilinear_at(c, coarse, g);
          }
    return;
  }
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1)
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
  int nan = 0;
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1) reduction(max : s) reduction(| : nan)
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) {
          double v = fabs(x[IX(l, b, i, j, k)]);
          if (v != v) nan = 1;
          else if (v > s) s = v;
        }
  return nan ? NAN : s;
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
static int bottom_cg(oprob* p, const double* rhs_in, double* x);

int orc_bottom(void* vp, const double* rhs_in, double* x) {
  oprob* p = (oprob*)vp;
  if (p->bot_cg) return bottom_cg(p, rhs_in, x);
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

/* Conjugate gradients (Hestenes and Stiefel 1952) for A x = rhs on the bottom level (A
   symmetric positive definite, or semi-definite with the constants as null space for a
   singular problem), x0 = 0:  p = r;  alpha = (r,r)/(p,Ap);  x += alpha p;  r -= alpha Ap;
   beta = (r',r')/(r,r);  p = r' + beta p.  Stops when ||r||_inf <= bot_tol * ||r0||_inf,
   after bot_maxit iterations, or on breakdown ((p,Ap) not positive), keeping the current
   iterate.  Singular problems: rhs and result projected onto zero mean, as for BiCGStab. */
static int bottom_cg(oprob* p, const double* rhs_in, double* x) {
  int m = p->nlev - 1;
  olev* l = &p->L[m];
  int64_t n = l->ntot;
  double* r = (double*)calloc(n, sizeof(double));
  double* pp = (double*)calloc(n, sizeof(double));
  double* q = (double*)calloc(n, sizeof(double));
  memcpy(r, rhs_in, sizeof(double) * n);
  if (p->singular) lev_add_const(l, r, -lev_sum(l, r) / (double)lev_ncells(l));
  memset(x, 0, sizeof(double) * n);
  double r0 = lev_norminf(l, r);
  int it = 0;
  if (r0 > 0.0) {
    memcpy(pp, r, sizeof(double) * n);
    double rho = lev_dot(l, r, r);
    for (it = 1; it <= p->bot_maxit; ++it) {
      orc_apply_level(p, m, pp, q);
      double pq = lev_dot(l, pp, q);
      if (!(pq > 0.0)) { it--; break; }
      double alpha = rho / pq;
      for (int64_t k = 0; k < n; ++k) {
        x[k] += alpha * pp[k];
        r[k] -= alpha * q[k];
      }
      if (lev_norminf(l, r) <= p->bot_tol * r0) break;
      double rho_new = lev_dot(l, r, r);
      double beta = rho_new / rho;
      rho = rho_new;
      for (int64_t k = 0; k < n; ++k) pp[k] = r[k] + beta * pp[k];
    }
    if (it > p->bot_maxit) it = p->bot_maxit;
  }
  if (p->singular) lev_add_const(l, x, -lev_sum(l, x) / (double)lev_ncells(l));
  free(r); free(pp); free(q);
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
    orc_smooth_colour(vp, m, e, r, p->post_rev ? 1 : 0);
    orc_smooth_colour(vp, m, e, r, p->post_rev ? 0 : 1);
  }
}

/* ------------------------------------------------------------ wall values */

/* Values g on a level-0 wall face (face = 2*d + side): phi on the face for a Dirichlet
   wall, the outward normal derivative for a Neumann wall.  `values` is a dense array over
   the face's two tangential axes in increasing order, the lower one fastest (NULL: g = 0).
   Returns -1 for a periodic face or a bad face index. */
int orc_set_bc_values(void* vp, int face, const double* values) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  if (face < 0 || face > 5) return -1;
  int d = face / 2, side = face % 2;
  int bc = side ? l->bchi[d] : l->bclo[d];
  if (bc == ORC_PERIODIC) return -1;
  free(p->bcval[face]);
  p->bcval[face] = NULL;
  if (!values) return 0;
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  int64_t n = (int64_t)(l->dhi[t1] - l->dlo[t1] + 1) * (l->dhi[t2] - l->dlo[t2] + 1);
  p->bcval[face] = (double*)malloc(sizeof(double) * n);
  memcpy(p->bcval[face], values, sizeof(double) * n);
  return 0;
}

/* level-0 ghosts with the wall values: the homogeneous ghost plus 2g (Dirichlet: the
   line through the interior value and g on the face; 8g/3 for the parabola of the
   quadratic rule) or h*g (Neumann: the one-sided difference across the face equals g) */
static void fill_ghosts_bc(const oprob* p, double* f) {
  const olev* l = &p->L[0];
  fill_ghosts(l, f);
  for (int64_t q = 0; q < l->ng; ++q) {
    int w = l->gwall[q];
    if (w < 0 || !p->bcval[w]) continue;
    int d = w / 2, side = w % 2;
    double g = p->bcval[w][l->gtan[q]];
    int bc = side ? l->bchi[d] : l->bclo[d];
    f[l->gdst[q]] += bc == ORC_NEUMANN ? l->h[d] * g : (l->gsrc2[q] >= 0 ? 8.0 * g / 3.0 : 2.0 * g);
  }
}

/* r = rhs - A phi on level 0 with the wall values in the ghosts */
static void residual_bc(oprob* p, double* phi, const double* rhs, double* r) {
  olev* l = &p->L[0];
  fill_ghosts_bc(p, phi);
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1)
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i)
          r[IX(l, b, i, j, k)] = rhs[IX(l, b, i, j, k)] - op_cell(p, l, phi, b, i, j, k);
}

/* out = A phi with the wall values (an affine map unless every g is 0), dense arrays */
void orc_apply_bc(void* vp, const double* phi_dense, double* out_dense) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  double* phi = (double*)calloc(l->ntot, sizeof(double));
  double* out = (double*)calloc(l->ntot, sizeof(double));
  orc_dense_to_boxed(vp, 0, phi_dense, phi);
  fill_ghosts_bc(p, phi);
  #pragma omp parallel for schedule(dynamic) num_threads(g_threads) if (g_threads > 1)
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) out[IX(l, b, i, j, k)] = op_cell(p, l, phi, b, i, j, k);
  orc_boxed_to_dense(vp, 0, out, out_dense);
  free(phi); free(out);
}

/* ------------------------------------------------- gradients (one level) */

/* Gradient of a loss L(phi) with respect to the cell-centred beta of level 0, given the
   solution phi of A phi = rhs (wall values in A) and the adjoint lambda (A^T lambda =
   dL/dphi).  dL/dbeta = lambda^T d(rhs - A phi)/dbeta: the row of cell q holds, per face
   f, -b beta_f (phi_nbr - phi_q) / h^2, so face f adds lambda_q b (phi_nbr - phi_q) / h^2
   for each of its (one or two) rows, with phi_nbr the neighbour or, at a wall, the ghost
   of the wall rule (wall values included; the quadratic rule's ghost where it applies).  The face sum then goes to the cells through
   the rule that made beta_f: harmonic mean 2 bL bR / (bL + bR), derivative 2 bR^2 /
   (bL + bR)^2 for bL; a wall face takes the interior cell's beta, derivative 1.
   Dense arrays over the domain (x fastest); beta_dense is the cell beta given to
   orc_set_coeffs (NULL: beta = 1). */
void orc_grad_beta_cells(void* vp, const double* phi_dense, const double* lam_dense, const double* beta_dense,
                         double* out_dense) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  int n[3] = {l->dhi[0] - l->dlo[0] + 1, l->dhi[1] - l->dlo[1] + 1, l->dhi[2] - l->dlo[2] + 1};
  int64_t N = (int64_t)n[0] * n[1] * n[2];
  for (int64_t q = 0; q < N; ++q) out_dense[q] = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int c[3] = {i, j, k};
        int64_t q = i + (int64_t)n[0] * (j + (int64_t)n[1] * k);
        double bq = beta_dense ? beta_dense[q] : 1.0;
        for (int d = 0; d < 3; ++d) {
          double w = p->b / (l->h[d] * l->h[d]);
          int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
          for (int side = 0; side < 2; ++side) {
            int nb[3] = {c[0], c[1], c[2]};
            nb[d] += side ? 1 : -1;
            int outside = nb[d] < 0 || nb[d] >= n[d];
            int bc = side ? l->bchi[d] : l->bclo[d];
            if (outside && bc == ORC_PERIODIC) {
              nb[d] = pmod(nb[d], n[d]);
              outside = 0;
            }
            if (outside) {
              double ghost = bc == ORC_NEUMANN ? phi_dense[q] : -phi_dense[q];
              int gc[3] = {l->dlo[0] + c[0], l->dlo[1] + c[1], l->dlo[2] + c[2]}, bx = find_box(l, gc), lc[3];
              for (int e = 0; e < 3; ++e) lc[e] = gc[e] - l->lo[3 * bx + e];
              const int quad = quad_face(l, bx, lc, d, side);
              if (quad) {
                int in[3] = {c[0], c[1], c[2]};
                in[d] += side ? -1 : 1;
                ghost = -2.0 * phi_dense[q] + phi_dense[in[0] + (int64_t)n[0] * (in[1] + (int64_t)n[1] * in[2])] / 3.0;
              }
              const double* gv = p->bcval[2 * d + side];
              if (gv) {
                double g = gv[(int64_t)c[t1] + (int64_t)n[t1] * c[t2]];
                ghost += bc == ORC_NEUMANN ? l->h[d] * g : (quad ? 8.0 * g / 3.0 : 2.0 * g);
              }
              out_dense[q] += lam_dense[q] * w * (ghost - phi_dense[q]);
              continue;
            }
            int64_t r = nb[0] + (int64_t)n[0] * (nb[1] + (int64_t)n[1] * nb[2]);
            double br = beta_dense ? beta_dense[r] : 1.0;
            double s = bq + br;
            /* this row's share of face f, passed to both cells of the face */
            double gf = lam_dense[q] * w * (phi_dense[r] - phi_dense[q]);
            out_dense[q] += gf * 2.0 * br * br / (s * s);
            out_dense[r] += gf * 2.0 * bq * bq / (s * s);
          }
        }
      }
}

/* dL/dg on wall face `face` (= 2*d + side): the wall values enter rhs - A 0 of the wall
   cell q as +2 b beta_f g / h^2 (Dirichlet; 8/3 in place of 2 under the quadratic rule) or
   +b beta_f g / h (Neumann), so
   dL/dg = lambda_q times that factor.  out: the face's value layout (tangential axes in
   increasing order, the lower one fastest). */
int orc_grad_wall_values(void* vp, const double* lam_dense, int face, double* out) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  if (face < 0 || face > 5) return -1;
  int d = face / 2, side = face % 2;
  int bc = side ? l->bchi[d] : l->bclo[d];
  if (bc == ORC_PERIODIC) return -1;
  int n[3] = {l->dhi[0] - l->dlo[0] + 1, l->dhi[1] - l->dlo[1] + 1, l->dhi[2] - l->dlo[2] + 1};
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  double* fa = d == 0 ? l->bx : (d == 1 ? l->by : l->bz);
  for (int v = 0; v < n[t2]; ++v)
    for (int u = 0; u < n[t1]; ++u) {
      int c[3], fl[3];
      c[d] = side ? n[d] - 1 : 0;
      c[t1] = u;
      c[t2] = v;
      int g[3] = {l->dlo[0] + c[0], l->dlo[1] + c[1], l->dlo[2] + c[2]};
      int b = find_box(l, g);
      for (int e = 0; e < 3; ++e) fl[e] = g[e] - l->lo[3 * b + e];
      if (side) fl[d] += 1; /* the wall face's slot */
      double beta_f = fa[IX(l, b, fl[0], fl[1], fl[2])];
      double h = l->h[d];
      int lc[3] = {g[0] - l->lo[3 * b], g[1] - l->lo[3 * b + 1], g[2] - l->lo[3 * b + 2]};
      double wg = quad_face(l, b, lc, d, side) ? 8.0 / 3.0 : 2.0;
      double fac = bc == ORC_NEUMANN ? p->b * beta_f / h : wg * p->b * beta_f / (h * h);
      out[u + (int64_t)n[t1] * v] = lam_dense[c[0] + (int64_t)n[0] * (c[1] + (int64_t)n[1] * c[2])] * fac;
    }
  return 0;
}

/* ------------------------------------------------------------ outer loop */

/* Solve A phi = rhs (dense arrays over the level-0 domain, wall values in A) from
   phi = 0: r0 = rhs - A 0; phi += Vcycle(r), r = rhs - A phi, until
   ||r||_inf <= max(tol_rel*||r0||_inf, tol_abs) or maxit iterations (without wall values
   r0 = rhs).  The V-cycle solves the correction equation with homogeneous walls.  hist[0..iters] receives ||r||_inf after each iteration.
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
  residual_bc(p, phi, rhs, r); /* r0 = rhs - A 0 */
  double rhsnorm = lev_norminf(l, r);
  *status = 0;
  if (p->singular) {
    double mean = lev_sum(l, r) / (double)lev_ncells(l);
    if (fabs(mean) > 1e-12 * rhsnorm && !project_mean) {
      *status = -1;
      free(rhs); free(phi); free(r); free(e);
      return 0;
    }
    lev_add_const(l, rhs, -mean);
    lev_add_const(l, r, -mean);
  }
  double target = tol_rel * rhsnorm;
  if (tol_abs > target) target = tol_abs;
  double rn = lev_norminf(l, r);
  if (hist) hist[0] = rn;
  int it = 0;
  while (!(rn <= target) && it < maxit) {
    orc_vcycle(vp, 0, e, r);
    #pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (int64_t q = 0; q < n; ++q) phi[q] += e[q];
    residual_bc(p, phi, rhs, r);
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

/* ------------------------------------------------- Krylov-accelerated multigrid */

/* z = M v: one V-cycle on the correction equation A e = v from e = 0 (the multigrid
   preconditioner); singular problems: z projected onto zero mean */
static void mg_precond(oprob* p, const double* v, double* z) {
  olev* l = &p->L[0];
  orc_vcycle(p, 0, z, v);
  if (p->singular) lev_add_const(l, z, -lev_sum(l, z) / (double)lev_ncells(l));
}

/* q = A v on level 0 with homogeneous walls (v's ghosts refreshed) */
static void apply0(oprob* p, double* v, double* q) { orc_apply_level(p, 0, v, q); }

/* Solve A phi = rhs from phi = 0 by a Krylov method preconditioned with one V-cycle per
   application (Sec. "Linear Solvers": native Krylov solvers next to multigrid):
     method 1: BiCGStab (van der Vorst 1992) preconditioned on the right, x += alpha M p +
               omega M s;
     method 2: conjugate gradients preconditioned by M (use orc_set_cycle(.., 1) for a
               symmetric V-cycle).
   The wall values enter as for orc_solve: b = rhs - A_g(0), solve A_0 x = b.  Stops when the
   recursive residual ||r||_inf <= max(tol_rel ||b||_inf, tol_abs), after maxit iterations,
   or on breakdown.  hist[0..it]: ||r||_inf.  status as orc_solve.  Singular problems: b
   and every preconditioned vector projected onto zero mean, phi returned with zero mean. */
int orc_solve_krylov(void* vp, const double* rhs_dense, double* phi_dense, double tol_rel, double tol_abs, int maxit,
                     int method, int project_mean, double* hist, int* status) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  int64_t n = l->ntot;
  double* V[10];
  for (int k = 0; k < 10; ++k) V[k] = (double*)calloc(n, sizeof(double));
  double *x = V[0], *b = V[1], *r = V[2], *rh = V[3], *pp = V[4], *v = V[5], *y = V[6], *sv = V[7], *t = V[8],
         *z = V[9];
  double* rhs = (double*)calloc(n, sizeof(double));
  orc_dense_to_boxed(vp, 0, rhs_dense, rhs);
  residual_bc(p, x, rhs, b); /* b = rhs - A_g 0 */
  double bnorm = lev_norminf(l, b);
  *status = 0;
  int it = 0;
  if (p->singular) {
    double mean = lev_sum(l, b) / (double)lev_ncells(l);
    if (fabs(mean) > 1e-12 * bnorm && !project_mean) {
      *status = -1;
      goto done;
    }
    lev_add_const(l, b, -mean);
  }
  {
    double target = tol_rel * bnorm;
    if (tol_abs > target) target = tol_abs;
    memcpy(r, b, sizeof(double) * n);
    double rn = lev_norminf(l, r);
    if (hist) hist[0] = rn;
    if (method == 1) {
      memcpy(rh, r, sizeof(double) * n);
      double rho_old = 1.0, alpha = 1.0, omega = 1.0;
      while (!(rn <= target) && it < maxit) {
        ++it;
        double rho = lev_dot(l, rh, r);
        if (fabs(rho) < 1e-300) { --it; break; }
        double beta = (rho / rho_old) * (alpha / omega);
        for (int64_t k = 0; k < n; ++k) pp[k] = r[k] + beta * (pp[k] - omega * v[k]);
        mg_precond(p, pp, y);
        apply0(p, y, v);
        double rv = lev_dot(l, rh, v);
        if (fabs(rv) < 1e-300) { --it; break; }
        alpha = rho / rv;
        for (int64_t k = 0; k < n; ++k) sv[k] = r[k] - alpha * v[k];
        double sn = lev_norminf(l, sv);
        if (sn <= target) {
          for (int64_t k = 0; k < n; ++k) x[k] += alpha * y[k];
          memcpy(r, sv, sizeof(double) * n);
          rn = sn;
          if (hist) hist[it] = rn;
          break;
        }
        mg_precond(p, sv, z);
        apply0(p, z, t);
        double tt = lev_dot(l, t, t);
        if (tt == 0.0) { --it; break; }
        omega = lev_dot(l, t, sv) / tt;
        for (int64_t k = 0; k < n; ++k) {
          x[k] += alpha * y[k] + omega * z[k];
          r[k] = sv[k] - omega * t[k];
        }
        rn = lev_norminf(l, r);
        if (hist) hist[it] = rn;
        if (!(rn == rn) || isinf(rn)) { *status = -3; break; }
        rho_old = rho;
      }
    } else {
      mg_precond(p, r, z);
      memcpy(pp, z, sizeof(double) * n);
      double rho = lev_dot(l, r, z);
      while (!(rn <= target) && it < maxit) {
        ++it;
        apply0(p, pp, v);
        double pv = lev_dot(l, pp, v);
        if (!(pv > 0.0)) { --it; break; }
        double alpha = rho / pv;
        for (int64_t k = 0; k < n; ++k) {
          x[k] += alpha * pp[k];
          r[k] -= alpha * v[k];
        }
        rn = lev_norminf(l, r);
        if (hist) hist[it] = rn;
        if (!(rn == rn) || isinf(rn)) { *status = -3; break; }
        if (rn <= target) break;
        mg_precond(p, r, z);
        double rho_new = lev_dot(l, r, z);
        double beta = rho_new / rho;
        rho = rho_new;
        for (int64_t k = 0; k < n; ++k) pp[k] = z[k] + beta * pp[k];
      }
    }
    if (*status == 0 && !(rn <= target)) *status = -2;
  }
  if (p->singular) lev_add_const(l, x, -lev_sum(l, x) / (double)lev_ncells(l));
  orc_boxed_to_dense(vp, 0, x, phi_dense);
done:
  for (int k = 0; k < 10; ++k) free(V[k]);
  free(rhs);
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

/* ghost-map entry that fills element e of level l, or -1 (a valid cell, or an edge or corner
   ghost) */
static int64_t ghost_entry(olev* l, int64_t e) {
  if (!l->ginv) {
    l->ginv = (int64_t*)malloc(sizeof(int64_t) * (l->ntot + 1));
    for (int64_t q = 0; q < l->ntot; ++q) l->ginv[q] = -1;
    for (int64_t q = 0; q < l->ng; ++q) l->ginv[l->gdst[q]] = q;
  }
  return l->ginv[e];
}

/* x = A^T y on level 0 with homogeneous walls, dense arrays.  Straight from the definition
   (A^T y)_c = sum_r A[r][c] y_r: every row r of the operator (the 7-point stencil of
   op_cell) is expanded into its matrix entries -- a neighbour that is a ghost cell stands
   for the cells the ghost map fills it from, with the map's factors (a linear Dirichlet
   wall's ghost -phi_0 lands on the diagonal, the quadratic rule's -2 phi_0 + phi_1 / 3 on
   the diagonal and on the next cell inward) -- and y_r times each entry is added to x at
   the entry's column.  Sequential (the scatter crosses boxes). */
void orc_apply_transpose(void* vp, const double* y_dense, double* x_dense) {
  oprob* p = (oprob*)vp;
  olev* l = &p->L[0];
  double* y = (double*)calloc(l->ntot, sizeof(double));
  double* x = (double*)calloc(l->ntot, sizeof(double));
  orc_dense_to_boxed(vp, 0, y_dense, y);
  for (int b = 0; b < l->nb; ++b)
    for (int k = 0; k < bn(l, b, 2); ++k)
      for (int j = 0; j < bn(l, b, 1); ++j)
        for (int i = 0; i < bn(l, b, 0); ++i) {
          const int64_t r = IX(l, b, i, j, k);
          const double yr = y[r];
          double diag = p->a * l->alpha[r];
          for (int d = 0; d < 3; ++d) {
            const double* bf = d == 0 ? l->bx : (d == 1 ? l->by : l->bz);
            for (int side = 0; side < 2; ++side) {
              int nb[3] = {i, j, k}, up[3] = {i, j, k};
              nb[d] += side ? 1 : -1;
              up[d] += side ? 1 : 0; /* face slot: the face at i - 1/2 is stored at i */
              const double w = p->b * bf[IX(l, b, up[0], up[1], up[2])] / (l->h[d] * l->h[d]);
              diag += w; /* -b * (-beta_f phi_r) / h^2 */
              const int64_t e = IX(l, b, nb[0], nb[1], nb[2]);
              const int inside = nb[d] >= 0 && nb[d] < bn(l, b, d);
              if (inside) {
                x[e] -= w * yr;
                continue;
              }
              const int64_t g = ghost_entry(l, e);
              if (g < 0 || l->gsrc[g] < 0) continue; /* not filled from this level */
              if (l->gsrc2[g] >= 0) {
                x[l->gsrc[g]] -= w * (-2.0) * yr;
                x[l->gsrc2[g]] -= w * (1.0 / 3.0) * yr;
              } else {
                x[l->gsrc[g]] -= w * l->gfac[g] * yr;
              }
            }
          }
          x[r] += diag * yr;
        }
  orc_boxed_to_dense(vp, 0, x, x_dense);
  free(y); free(x);
}

/* =====================================================================
 * Two-level composite problem (Sec. "Operations between levels", Sec. "Linear
 * Solvers": multi-AMR-level geometric multigrid).  Level 0 (coarse) covers the domain;
 * level 1 (fine, refinement ratio 2) covers part of it.  The unknowns are the fine cells
 * and the coarse cells NOT covered by fine cells.
 *
 * Readings used (the paper names interpolation, restriction and refluxing but gives no
 * formulas):
 *   - a fine ghost g across a coarse/fine face normal to d is the quadratic through the
 *     coarse value interpolated tangentially to g's position (phi_c*, at the coarse cell
 *     centre one fine cell beyond g) and the first two fine cells inward:
 *       phi_g = 8/15 phi_c* + 2/3 phi_f1 - 1/5 phi_f2,
 *       phi_c* = phi_C + sum over the two tangential axes t of
 *                s_t (phi_{C+t} - phi_{C-t}) / 2 + s_t^2 (phi_{C+t} - 2 phi_C + phi_{C-t}) / 2,
 *     with s_t = +-1/4 the ghost's offset from the coarse centre in coarse cells;
 *   - a fine face on the coarse/fine boundary takes the adjacent fine cell's beta;
 *   - refluxing (Sec. "Operations between levels"): an uncovered coarse cell uses, on a
 *     face shared with a covered cell, the mean of the 4 fine fluxes through that face
 *     instead of its own coarse flux;
 *   - covered coarse values are the average of their 8 fine children.
 * The operator is written row by row as (unknown, coefficient) terms, each coefficient
 * that carries a face beta tagged with that face, so that the same row code gives
 * A x, A^T y and the derivative lambda^T (dA/dbeta) phi.
 * ===================================================================== */

typedef struct {
  int64_t dst;       /* ghost slot in the fine boxed layout */
  int64_t f1, f2;    /* first and second fine cells inward */
  int64_t cq[5];     /* coarse cells C, C+t1, C-t1, C+t2, C-t2 (coarse boxed layout) */
  double cw[5];      /* weights of phi_c* */
} ocfghost;

typedef struct {
  oprob* C;          /* coarse level + its multigrid hierarchy */
  oprob* F;          /* fine level (its own hierarchy is not used) */
  char* covered;     /* coarse boxed layout: 1 where fine cells lie above */
  int64_t ncf;
  ocfghost* cf;      /* coarse/fine ghosts of the fine level */
  int64_t* cfidx;    /* fine boxed layout -> index into cf, or -1 */
  int64_t* gentry;   /* fine boxed layout -> fine ghost-map entry, or -1 */
  double a, b;
  int nu1, nu2;
} oamr;

static int64_t coarse_at(const olev* c, const int g_in[3]) {
  int g[3] = {g_in[0], g_in[1], g_in[2]};
  for (int d = 0; d < 3; ++d)
    if (c->bclo[d] == ORC_PERIODIC) {
      int len = c->dhi[d] - c->dlo[d] + 1;
      g[d] = c->dlo[d] + pmod(g[d] - c->dlo[d], len);
    }
  int b = find_box(c, g);
  if (b < 0) return -1;
  return IX(c, b, g[0] - c->lo[3 * b], g[1] - c->lo[3 * b + 1], g[2] - c->lo[3 * b + 2]);
}

static int box_of_index(const olev* l, int64_t q) {
  int b = 0;
  while (!(q >= l->off[b] && q < l->off[b + 1])) ++b;
  return b;
}

/* Tables of a coarse/fine pair (A->C level 0 coarse, A->F level 0 fine, ratio 2): covered
   coarse cells, the fine ghost-map entry of every fine ghost slot, and the coarse/fine ghosts
   of the fine level with their interpolation stencils.  Returns -1 when the fine boxes are
   not ratio-2 aligned and at least 2 cells wide, or when a coarse/fine ghost's stencil
   needs a coarse cell that the coarse level lacks or that is covered. */
static int amr_build_pair(oamr* A) {
  olev* c = &A->C->L[0];
  olev* f = &A->F->L[0];
  for (int b = 0; b < f->nb; ++b)
    for (int d = 0; d < 3; ++d)
      if (pmod(f->lo[3 * b + d], 2) || pmod(f->hi[3 * b + d] + 1, 2) || bn(f, b, d) < 2) return -1;
  A->covered = (char*)calloc(c->ntot, 1);
  for (int b = 0; b < c->nb; ++b)
    for (int k = 0; k < bn(c, b, 2); ++k)
      for (int j = 0; j < bn(c, b, 1); ++j)
        for (int i = 0; i < bn(c, b, 0); ++i) {
          int g[3] = {2 * (c->lo[3 * b] + i), 2 * (c->lo[3 * b + 1] + j), 2 * (c->lo[3 * b + 2] + k)};
          A->covered[IX(c, b, i, j, k)] = find_box(f, g) >= 0;
        }
  A->gentry = (int64_t*)malloc(sizeof(int64_t) * f->ntot);
  A->cfidx = (int64_t*)malloc(sizeof(int64_t) * f->ntot);
  for (int64_t q = 0; q < f->ntot; ++q) A->gentry[q] = A->cfidx[q] = -1;
  for (int64_t e = 0; e < f->ng; ++e) A->gentry[f->gdst[e]] = e;
  /* coarse/fine ghosts: the fine ghost-map entries that no fine box fills */
  A->cf = (ocfghost*)calloc(f->ng + 1, sizeof(ocfghost));
  int64_t n = 0;
  for (int64_t e = 0; e < f->ng; ++e) {
    if (f->gsrc[e] >= 0) continue;
    int64_t gq = f->gdst[e];
    int b = box_of_index(f, gq);
    int64_t nx = bn(f, b, 0) + 2, ny = bn(f, b, 1) + 2;
    int64_t rel = gq - f->off[b];
    int loc[3] = {(int)(rel % nx) - 1, (int)((rel / nx) % ny) - 1, (int)(rel / (nx * ny)) - 1};
    int d = -1, side = 0;
    for (int q = 0; q < 3; ++q) {
      if (loc[q] < 0) { d = q; side = 0; }
      if (loc[q] >= bn(f, b, q)) { d = q; side = 1; }
    }
    int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    ocfghost* G = &A->cf[n];
    G->dst = gq;
    int in1[3] = {loc[0], loc[1], loc[2]}, in2[3] = {loc[0], loc[1], loc[2]};
    in1[d] = side ? bn(f, b, d) - 1 : 0;
    in2[d] = side ? bn(f, b, d) - 2 : 1;
    G->f1 = IX(f, b, in1[0], in1[1], in1[2]);
    G->f2 = IX(f, b, in2[0], in2[1], in2[2]);
    int g[3], C[3];
    double s[3];
    for (int q = 0; q < 3; ++q) {
      g[q] = f->lo[3 * b + q] + loc[q];
      C[q] = (g[q] - pmod(g[q], 2)) / 2;
      s[q] = (pmod(g[q], 2) == 0) ? -0.25 : 0.25;
    }
    int t[2] = {d1, d2};
    G->cq[0] = coarse_at(c, C);
    G->cw[0] = 1.0;
    for (int e2 = 0; e2 < 2; ++e2) {
      int Cp[3] = {C[0], C[1], C[2]}, Cm[3] = {C[0], C[1], C[2]};
      Cp[t[e2]] += 1;
      Cm[t[e2]] -= 1;
      double st = s[t[e2]];
      G->cq[1 + 2 * e2] = coarse_at(c, Cp);
      G->cq[2 + 2 * e2] = coarse_at(c, Cm);
      G->cw[1 + 2 * e2] = 0.5 * st + 0.5 * st * st;
      G->cw[2 + 2 * e2] = -0.5 * st + 0.5 * st * st;
      G->cw[0] -= st * st;
    }
    for (int e2 = 0; e2 < 5; ++e2)
      if (G->cq[e2] < 0 || A->covered[G->cq[e2]]) return -1; /* interpolation must use uncovered coarse cells */
    A->cfidx[gq] = n;
    ++n;
  }
  A->ncf = n;
  return 0;
}

static void amr_free_tables(oamr* A) {
  free(A->covered); free(A->cf); free(A->cfidx); free(A->gentry);
  A->covered = NULL; A->cf = NULL; A->cfidx = NULL; A->gentry = NULL;
}

void* orc_amr_create(const int* dlo, const int* dhi, const int* bclo, const int* bchi, const double* plo,
                     const double* phi_, int nbc, const int* cboxes, int nbf, const int* fboxes) {
  for (int d = 0; d < 3; ++d) /* composite operators take the linear Dirichlet rule only */
    if (bclo[d] == ORC_DIRICHLET_QUAD || bchi[d] == ORC_DIRICHLET_QUAD) return NULL;
  oamr* A = (oamr*)calloc(1, sizeof(oamr));
  A->C = (oprob*)orc_create(dlo, dhi, bclo, bchi, plo, phi_, nbc, cboxes);
  int fdlo[3], fdhi[3];
  for (int d = 0; d < 3; ++d) { fdlo[d] = 2 * dlo[d]; fdhi[d] = 2 * dhi[d] + 1; }
  A->F = A->C ? (oprob*)orc_create(fdlo, fdhi, bclo, bchi, plo, phi_, nbf, fboxes) : NULL;
  if (!A->C || !A->F || amr_build_pair(A) != 0) {
    orc_destroy(A->C); orc_destroy(A->F); amr_free_tables(A); free(A);
    return NULL;
  }
  A->a = 0.0;
  A->b = 1.0;
  A->nu1 = 2;
  A->nu2 = 2;
  return A;
}

void orc_amr_destroy(void* vp) {
  oamr* A = (oamr*)vp;
  if (!A) return;
  orc_destroy(A->C);
  orc_destroy(A->F);
  amr_free_tables(A);
  free(A);
}

void* orc_amr_coarse(void* vp) { return ((oamr*)vp)->C; }
void* orc_amr_fine(void* vp) { return ((oamr*)vp)->F; }
int64_t orc_amr_ncf(void* vp) { return ((oamr*)vp)->ncf; }
void orc_amr_covered(void* vp, char* out) { memcpy(out, ((oamr*)vp)->covered, ((oamr*)vp)->C->L[0].ntot); }

/* Coefficients: dense cell alpha/beta over the coarse domain and over the FINE domain
   (only the fine boxes' cells are read).  Fine faces on the coarse/fine boundary take the
   adjacent fine cell's beta. */
/* fine cell g wrapped into the fine domain along periodic directions */
static void wrap_periodic(const olev* l, int g[3]) {
  for (int d = 0; d < 3; ++d)
    if (l->bclo[d] == ORC_PERIODIC) g[d] = l->dlo[d] + pmod(g[d] - l->dlo[d], l->dhi[d] - l->dlo[d] + 1);
}

/* beta of the fine face at fine index g[d] - 1/2 along d, read from a fine box holding the
   cell on its high side or on its low side; 0 when neither cell is a fine cell */
static int fine_face_beta(const olev* f, int d, const int g_in[3], double* out) {
  const double* ff = d == 0 ? f->bx : (d == 1 ? f->by : f->bz);
  int g[3] = {g_in[0], g_in[1], g_in[2]};
  wrap_periodic(f, g);
  int b = find_box(f, g);
  if (b >= 0) {
    *out = ff[IX(f, b, g[0] - f->lo[3 * b], g[1] - f->lo[3 * b + 1], g[2] - f->lo[3 * b + 2])];
    return 1;
  }
  int gl[3] = {g_in[0], g_in[1], g_in[2]};
  gl[d] -= 1;
  wrap_periodic(f, gl);
  b = find_box(f, gl);
  if (b < 0) return 0;
  int loc[3] = {gl[0] - f->lo[3 * b], gl[1] - f->lo[3 * b + 1], gl[2] - f->lo[3 * b + 2]};
  loc[d] += 1; /* the face above the low cell: slot n of that box */
  *out = ff[IX(f, b, loc[0], loc[1], loc[2])];
  return 1;
}

/* Sec. "Operations between levels" (average of fine data onto the coarse level) applied to
   the face coefficients: a level-0 face tiled by fine faces (a face of a covered cell)
   takes the mean of its 4 fine faces, the same rule as between multigrid levels.  The
   composite operator never reads these faces (covered cells have no rows, and refluxing
   replaces the coarse flux on the coarse/fine boundary): they shape only the coarse
   correction operator of the composite iteration, which then sees the fine coefficients
   instead of a coarse re-discretisation of them.  The coarser multigrid levels of level 0
   are rebuilt from the result. */
static void amr_average_down_faces(oamr* A) {
  olev* c = &A->C->L[0];
  const olev* f = &A->F->L[0];
  double* cf[3] = {c->bx, c->by, c->bz};
  for (int b = 0; b < c->nb; ++b)
    for (int d = 0; d < 3; ++d) {
      int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
      int ext[3] = {bn(c, b, 0), bn(c, b, 1), bn(c, b, 2)};
      ext[d] += 1;
      for (int k = 0; k < ext[2]; ++k)
        for (int j = 0; j < ext[1]; ++j)
          for (int i = 0; i < ext[0]; ++i) {
            int G[3] = {c->lo[3 * b] + i, c->lo[3 * b + 1] + j, c->lo[3 * b + 2] + k};
            double s = 0.0, v;
            int found = 1;
            for (int t1 = 0; t1 < 2 && found; ++t1)
              for (int t2 = 0; t2 < 2 && found; ++t2) {
                int g[3] = {2 * G[0], 2 * G[1], 2 * G[2]};
                g[d1] += t1;
                g[d2] += t2;
                found = fine_face_beta(f, d, g, &v);
                s += v;
              }
            if (found) cf[d][IX(c, b, i, j, k)] = 0.25 * s;
          }
    }
  /* and a covered cell's alpha is the mean of its 8 children's */
  for (int b = 0; b < c->nb; ++b)
    for (int k = 0; k < bn(c, b, 2); ++k)
      for (int j = 0; j < bn(c, b, 1); ++j)
        for (int i = 0; i < bn(c, b, 0); ++i) {
          int64_t q = IX(c, b, i, j, k);
          if (!A->covered[q]) continue;
          double s = 0.0;
          for (int e = 0; e < 8; ++e) {
            int g[3] = {2 * (c->lo[3 * b] + i) + (e & 1), 2 * (c->lo[3 * b + 1] + j) + ((e >> 1) & 1),
                        2 * (c->lo[3 * b + 2] + k) + (e >> 2)};
            int fb = find_box(f, g);
            s += f->alpha[IX(f, fb, g[0] - f->lo[3 * fb], g[1] - f->lo[3 * fb + 1], g[2] - f->lo[3 * fb + 2])];
          }
          c->alpha[q] = 0.125 * s;
        }
  for (int m = 0; m + 1 < A->C->nlev; ++m) coarsen_coeffs(&A->C->L[m], &A->C->L[m + 1]);
}

int orc_amr_set_coeffs(void* vp, double a, double bsc, const double* alpha_c, const double* beta_c,
                       const double* alpha_f, const double* beta_f) {
  oamr* A = (oamr*)vp;
  A->a = a;
  A->b = bsc;
  orc_set_coeffs(A->C, a, bsc, alpha_c, beta_c);
  orc_set_coeffs(A->F, a, bsc, alpha_f, beta_f);
  olev* f = &A->F->L[0];
  double* face[3] = {f->bx, f->by, f->bz};
  for (int64_t q = 0; q < A->ncf; ++q) {
    const ocfghost* G = &A->cf[q];
    int b = box_of_index(f, G->dst);
    int64_t nx = bn(f, b, 0) + 2, ny = bn(f, b, 1) + 2;
    int64_t diff = G->f1 - G->dst;
    int d = (diff == 1 || diff == -1) ? 0 : ((diff == nx || diff == -nx) ? 1 : 2);
    int64_t slot = diff > 0 ? G->f1 : G->dst; /* face slot i holds the face at i - 1/2 */
    int64_t rel = G->f1 - f->off[b];
    int g[3] = {f->lo[3 * b] + (int)(rel % nx) - 1, f->lo[3 * b + 1] + (int)((rel / nx) % ny) - 1,
                f->lo[3 * b + 2] + (int)(rel / (nx * ny)) - 1};
    face[d][slot] = beta_f ? dense_at(f, beta_f, g) : 1.0;
  }
  amr_average_down_faces(A);
  return 0;
}

/* ------------------------------------------------------------------ rows */

typedef struct {
  int mode;               /* 0: apply, 1: transpose, 2: beta gradient */
  const double *xc, *xf;  /* apply / gradient: the vector A acts on */
  double *yc, *yf;        /* transpose: output */
  double yrow;            /* transpose / gradient: the row's value of y (lambda) */
  double acc;             /* apply: the row value */
  double *gc[3], *gf[3];  /* gradient: per-face accumulators, coarse and fine */
} orow;

/* a term coef * x[which][q] with coef = c * beta(face) when fw >= 0 (fw: 0 coarse, 1 fine
   face array of direction fd, slot fs), else coef = c */
static void term(const oamr* A, orow* R, int which, int64_t q, double c, int fw, int fd, int64_t fs) {
  double beta = 1.0;
  if (fw >= 0) {
    const olev* l = fw ? &A->F->L[0] : &A->C->L[0];
    const double* fa = fd == 0 ? l->bx : (fd == 1 ? l->by : l->bz);
    beta = fa[fs];
  }
  if (R->mode == 0) {
    R->acc += c * beta * (which ? R->xf[q] : R->xc[q]);
  } else if (R->mode == 1) {
    if (which) R->yf[q] += c * beta * R->yrow;
    else R->yc[q] += c * beta * R->yrow;
  } else if (fw >= 0) {
    double* g = fw ? R->gf[fd] : R->gc[fd];
    g[fs] -= R->yrow * c * (which ? R->xf[q] : R->xc[q]);
  }
}

/* the value of fine ghost slot gq as terms, scaled by c (face tag passed through) */
static void fine_ghost_terms(const oamr* A, orow* R, int64_t gq, double c, int fw, int fd, int64_t fs) {
  const olev* f = &A->F->L[0];
  int64_t cfi = A->cfidx[gq];
  if (cfi >= 0) {
    const ocfghost* G = &A->cf[cfi];
    for (int e = 0; e < 5; ++e) term(A, R, 0, G->cq[e], c * (8.0 / 15.0) * G->cw[e], fw, fd, fs);
    term(A, R, 1, G->f1, c * (2.0 / 3.0), fw, fd, fs);
    term(A, R, 1, G->f2, c * (-0.2), fw, fd, fs);
    return;
  }
  int64_t e = A->gentry[gq];
  term(A, R, 1, f->gsrc[e], c * f->gfac[e], fw, fd, fs);
}

/* fine row: a alpha phi - b sum_d [beta+(phi+ - phi) - beta-(phi - phi-)] / h_d^2 */
static void fine_row(const oamr* A, orow* R, int b, int i, int j, int k) {
  const olev* f = &A->F->L[0];
  int64_t q = IX(f, b, i, j, k);
  int loc[3] = {i, j, k};
  term(A, R, 1, q, A->a * f->alpha[q], -1, 0, 0);
  for (int d = 0; d < 3; ++d) {
    double ih2 = A->b / (f->h[d] * f->h[d]);
    for (int side = 0; side < 2; ++side) {
      int nl[3] = {loc[0], loc[1], loc[2]};
      nl[d] += side ? 1 : -1;
      int fl[3] = {loc[0], loc[1], loc[2]};
      if (side) fl[d] += 1;
      int64_t fs = IX(f, b, fl[0], fl[1], fl[2]);
      term(A, R, 1, q, ih2, 1, d, fs);
      int64_t nq = IX(f, b, nl[0], nl[1], nl[2]);
      if (nl[d] >= 0 && nl[d] < bn(f, b, d)) term(A, R, 1, nq, -ih2, 1, d, fs);
      else fine_ghost_terms(A, R, nq, -ih2, 1, d, fs);
    }
  }
}

/* coarse row of an uncovered coarse cell; on a face shared with a covered cell the flux is
   the mean of the 4 fine fluxes beta_f (phi_fine - phi_ghost) / h_f through that face */
static void coarse_row(const oamr* A, orow* R, int b, int i, int j, int k) {
  const olev* c = &A->C->L[0];
  const olev* f = &A->F->L[0];
  int64_t q = IX(c, b, i, j, k);
  int loc[3] = {i, j, k};
  term(A, R, 0, q, A->a * c->alpha[q], -1, 0, 0);
  for (int d = 0; d < 3; ++d) {
    double hc = c->h[d], hf = f->h[d];
    int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    int gl[3] = {c->lo[3 * b] + i, c->lo[3 * b + 1] + j, c->lo[3 * b + 2] + k};
    for (int side = 0; side < 2; ++side) {
      int gn[3] = {gl[0], gl[1], gl[2]};
      gn[d] += side ? 1 : -1;
      int64_t nq = coarse_at(c, gn);
      if (nq >= 0 && A->covered[nq]) {
        for (int u = 0; u < 2; ++u)
          for (int v = 0; v < 2; ++v) {
            int fg[3];
            fg[d] = side ? 2 * gn[d] : 2 * gn[d] + 1; /* fine cell next to the face */
            fg[d1] = 2 * gl[d1] + u;
            fg[d2] = 2 * gl[d2] + v;
            for (int t = 0; t < 3; ++t)
              if (f->bclo[t] == ORC_PERIODIC) {
                int len = f->dhi[t] - f->dlo[t] + 1;
                fg[t] = f->dlo[t] + pmod(fg[t] - f->dlo[t], len);
              }
            int fb = find_box(f, fg);
            int fl[3] = {fg[0] - f->lo[3 * fb], fg[1] - f->lo[3 * fb + 1], fg[2] - f->lo[3 * fb + 2]};
            int64_t fq = IX(f, fb, fl[0], fl[1], fl[2]);
            int ghl[3] = {fl[0], fl[1], fl[2]};
            ghl[d] += side ? -1 : 1;
            int64_t gq = IX(f, fb, ghl[0], ghl[1], ghl[2]);
            int sl[3] = {fl[0], fl[1], fl[2]};
            if (!side) sl[d] += 1;
            int64_t fs = IX(f, fb, sl[0], sl[1], sl[2]);
            /* high side: -b F / hc with F = beta (phi_f - phi_g) / hf;
               low side:  +b F / hc with F = beta (phi_g - phi_f) / hf: the same terms */
            double cf = A->b * 0.25 / (hf * hc);
            term(A, R, 1, fq, -cf, 1, d, fs);
            fine_ghost_terms(A, R, gq, cf, 1, d, fs);
          }
        continue;
      }
      int fl[3] = {loc[0], loc[1], loc[2]};
      if (side) fl[d] += 1;
      int64_t fs = IX(c, b, fl[0], fl[1], fl[2]);
      double w = A->b / (hc * hc);
      term(A, R, 0, q, w, 0, d, fs);
      if (nq < 0) { /* wall: ghost = -phi (homogeneous Dirichlet) or +phi (homogeneous Neumann) */
        int bc = side ? c->bchi[d] : c->bclo[d];
        term(A, R, 0, q, bc == ORC_NEUMANN ? -w : w, 0, d, fs);
      } else {
        term(A, R, 0, nq, -w, 0, d, fs);
      }
    }
  }
}

typedef void (*row_fn)(const oamr*, orow*, int, int, int, int);

static void amr_sweep(const oamr* A, orow* R, double* yc, double* yf, const double* ycin, const double* yfin) {
  const olev* c = &A->C->L[0];
  const olev* f = &A->F->L[0];
  for (int b = 0; b < f->nb; ++b)
    for (int k = 0; k < bn(f, b, 2); ++k)
      for (int j = 0; j < bn(f, b, 1); ++j)
        for (int i = 0; i < bn(f, b, 0); ++i) {
          int64_t q = IX(f, b, i, j, k);
          R->acc = 0.0;
          if (yfin) R->yrow = yfin[q];
          fine_row(A, R, b, i, j, k);
          if (yf) yf[q] = R->acc;
        }
  for (int b = 0; b < c->nb; ++b)
    for (int k = 0; k < bn(c, b, 2); ++k)
      for (int j = 0; j < bn(c, b, 1); ++j)
        for (int i = 0; i < bn(c, b, 0); ++i) {
          int64_t q = IX(c, b, i, j, k);
          if (A->covered[q]) continue;
          R->acc = 0.0;
          if (ycin) R->yrow = ycin[q];
          coarse_row(A, R, b, i, j, k);
          if (yc) yc[q] = R->acc;
        }
}

/* y = A x (composite), boxed layouts; covered coarse entries of y are 0 */
void orc_amr_apply_boxed(void* vp, const double* xc, const double* xf, double* yc, double* yf) {
  oamr* A = (oamr*)vp;
  orow R;
  memset(&R, 0, sizeof(R));
  R.mode = 0;
  R.xc = xc;
  R.xf = xf;
  memset(yc, 0, sizeof(double) * A->C->L[0].ntot);
  memset(yf, 0, sizeof(double) * A->F->L[0].ntot);
  amr_sweep(A, &R, yc, yf, NULL, NULL);
}

/* x = A^T y; covered coarse entries of y are ignored */
void orc_amr_apply_transpose_boxed(void* vp, const double* yc, const double* yf, double* xc, double* xf) {
  oamr* A = (oamr*)vp;
  orow R;
  memset(&R, 0, sizeof(R));
  R.mode = 1;
  R.yc = xc;
  R.yf = xf;
  memset(xc, 0, sizeof(double) * A->C->L[0].ntot);
  memset(xf, 0, sizeof(double) * A->F->L[0].ntot);
  amr_sweep(A, &R, NULL, NULL, yc, yf);
}

/* dL/dbeta_face = -lambda^T (dA/dbeta_face) phi for every coarse and fine face (boxed
   face layouts, zeroed first) */
void orc_amr_grad_faces(void* vp, const double* phic, const double* phif, const double* lamc, const double* lamf,
                        double* gcx, double* gcy, double* gcz, double* gfx, double* gfy, double* gfz) {
  oamr* A = (oamr*)vp;
  orow R;
  memset(&R, 0, sizeof(R));
  R.mode = 2;
  R.xc = phic;
  R.xf = phif;
  double* gc[3] = {gcx, gcy, gcz};
  double* gf[3] = {gfx, gfy, gfz};
  for (int d = 0; d < 3; ++d) {
    R.gc[d] = gc[d];
    R.gf[d] = gf[d];
    memset(gc[d], 0, sizeof(double) * A->C->L[0].ntot);
    memset(gf[d], 0, sizeof(double) * A->F->L[0].ntot);
  }
  amr_sweep(A, &R, NULL, NULL, lamc, lamf);
}

/* ------------------------------------------------------------------ solve */

/* coarse/fine ghosts of the fine field from coarse values cx (NULL: zero) */
static void amr_fill_cf(const oamr* A, double* fx, const double* cx) {
  for (int64_t q = 0; q < A->ncf; ++q) {
    const ocfghost* G = &A->cf[q];
    double cs = 0.0;
    if (cx)
      for (int e = 0; e < 5; ++e) cs += G->cw[e] * cx[G->cq[e]];
    fx[G->dst] = (8.0 / 15.0) * cs + (2.0 / 3.0) * fx[G->f1] - 0.2 * fx[G->f2];
  }
}

/* covered coarse cells := mean of their 8 fine children */
static void amr_average_down(const oamr* A, const double* fx, double* cx) {
  const olev* c = &A->C->L[0];
  const olev* f = &A->F->L[0];
  for (int b = 0; b < f->nb; ++b)
    for (int K = f->lo[3 * b + 2] / 2; K <= (f->hi[3 * b + 2] + 1) / 2 - 1; ++K)
      for (int J = f->lo[3 * b + 1] / 2; J <= (f->hi[3 * b + 1] + 1) / 2 - 1; ++J)
        for (int I = f->lo[3 * b] / 2; I <= (f->hi[3 * b] + 1) / 2 - 1; ++I) {
          double s = 0.0;
          for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
              for (int di = 0; di < 2; ++di)
                s += fx[IX(f, b, 2 * I + di - f->lo[3 * b], 2 * J + dj - f->lo[3 * b + 1], 2 * K + dk - f->lo[3 * b + 2])];
          int G[3] = {I, J, K};
          cx[coarse_at(c, G)] = s / 8.0;
        }
}

/* one red-black colour on the fine level, coarse/fine ghosts from cx */
static void amr_fine_colour(oamr* A, double* ef, const double* rf, const double* cx, int colour) {
  amr_fill_cf(A, ef, cx);
  orc_smooth_colour(A->F, 0, ef, rf, colour); /* fills the fine/fine ghosts, keeps the C/F ones */
}

/* volume-weighted composite sum and volume (fine cells h_f^3, uncovered coarse h_c^3) */
static void amr_vsum(const oamr* A, const double* xc, const double* xf, double* s, double* v) {
  const olev* c = &A->C->L[0];
  const olev* f = &A->F->L[0];
  double vc = c->h[0] * c->h[1] * c->h[2], vf = f->h[0] * f->h[1] * f->h[2];
  *s = 0.0;
  *v = 0.0;
  for (int b = 0; b < f->nb; ++b)
    for (int k = 0; k < bn(f, b, 2); ++k)
      for (int j = 0; j < bn(f, b, 1); ++j)
        for (int i = 0; i < bn(f, b, 0); ++i) { *s += vf * xf[IX(f, b, i, j, k)]; *v += vf; }
  for (int b = 0; b < c->nb; ++b)
    for (int k = 0; k < bn(c, b, 2); ++k)
      for (int j = 0; j < bn(c, b, 1); ++j)
        for (int i = 0; i < bn(c, b, 0); ++i) {
          int64_t q = IX(c, b, i, j, k);
          if (A->covered[q]) continue;
          *s += vc * xc[q];
          *v += vc;
        }
}

static void amr_add_const(const oamr* A, double* xc, double* xf, double k) {
  lev_add_const(&A->C->L[0], xc, k);
  lev_add_const(&A->F->L[0], xf, k);
}

static double amr_norminf(const oamr* A, const double* xc, const double* xf) {
  const olev* c = &A->C->L[0];
  double m = lev_norminf(&A->F->L[0], xf);
  for (int b = 0; b < c->nb; ++b)
    for (int k = 0; k < bn(c, b, 2); ++k)
      for (int j = 0; j < bn(c, b, 1); ++j)
        for (int i = 0; i < bn(c, b, 0); ++i) {
          int64_t q = IX(c, b, i, j, k);
          if (A->covered[q]) continue;
          double v = fabs(xc[q]);
          if (v > m || v != v) m = v;
        }
  return m;
}

/* composite residual r = rhs - A phi (covered coarse entries 0) */
static void amr_residual(oamr* A, const double* rc_in, const double* rf_in, const double* pc, const double* pf,
                         double* rc, double* rf) {
  olev* c = &A->C->L[0];
  olev* f = &A->F->L[0];
  orc_amr_apply_boxed(A, pc, pf, rc, rf);
  for (int64_t q = 0; q < f->ntot; ++q) rf[q] = rf_in[q] - rf[q];
  for (int64_t q = 0; q < c->ntot; ++q) rc[q] = A->covered[q] ? 0.0 : rc_in[q] - rc[q];
}

/* Composite multigrid solve (the two-level iteration of the multi-level solver):
   1. r = composite residual;
   2. fine correction e_f from 0 by nu1 red-black sweeps with homogeneous coarse/fine
      ghosts (coarse correction 0);
   3. coarse right-hand side: on covered cells the average of the fine correction
      residual r_f - A_f e_f, on uncovered cells r_c minus the change of their composite
      row by e_f (the fine correction's reflux);
   4. one V-cycle of the coarse level's own hierarchy gives e_c;
   5. e_f += piecewise-constant interpolation of e_c;
   6. nu2 fine sweeps with coarse/fine ghosts interpolated from e_c;
   7. covered e_c := average of e_f; phi += e.
   Stops at ||r||_inf <= max(tol_rel ||rhs||_inf, tol_abs) over the composite unknowns.
   Singular (all periodic, a = 0): rhs projected to zero volume-weighted mean; phi returned
   with zero volume-weighted mean.  Dense arrays: coarse over the coarse domain, fine over
   the fine domain (cells outside fine boxes ignored; covered coarse cells of phi_c hold the
   average of the fine solution on return). */
int orc_amr_solve(void* vp, const double* rhsc_d, const double* rhsf_d, double* phic_d, double* phif_d, double tol_rel,
                  double tol_abs, int maxit, double* hist, int* status) {
  oamr* A = (oamr*)vp;
  olev* c = &A->C->L[0];
  olev* f = &A->F->L[0];
  int64_t nc = c->ntot, nf = f->ntot;
  double *rhc = calloc(nc, 8), *rhf = calloc(nf, 8), *pc = calloc(nc, 8), *pf = calloc(nf, 8);
  double *rc = calloc(nc, 8), *rf = calloc(nf, 8), *ec = calloc(nc, 8), *ef = calloc(nf, 8);
  double *yc = calloc(nc, 8), *yf = calloc(nf, 8), *cr = calloc(nc, 8);
  orc_dense_to_boxed(A->C, 0, rhsc_d, rhc);
  orc_dense_to_boxed(A->F, 0, rhsf_d, rhf);
  for (int64_t q = 0; q < nc; ++q)
    if (A->covered[q]) rhc[q] = 0.0;
  double rn0 = amr_norminf(A, rhc, rhf);
  int sing = A->C->singular;
  if (sing) {
    double s, v;
    amr_vsum(A, rhc, rhf, &s, &v);
    amr_add_const(A, rhc, rhf, -s / v);
    for (int64_t q = 0; q < nc; ++q)
      if (A->covered[q]) rhc[q] = 0.0;
  }
  double target = tol_rel * rn0 > tol_abs ? tol_rel * rn0 : tol_abs;
  amr_residual(A, rhc, rhf, pc, pf, rc, rf);
  double rn = amr_norminf(A, rc, rf);
  if (hist) hist[0] = rn;
  int it = 0;
  *status = 0;
  while (!(rn <= target) && it < maxit) {
    memset(ef, 0, 8 * nf);
    memset(ec, 0, 8 * nc);
    for (int s = 0; s < A->nu1; ++s) {
      amr_fine_colour(A, ef, rf, NULL, 0);
      amr_fine_colour(A, ef, rf, NULL, 1);
    }
    orc_amr_apply_boxed(A, ec, ef, yc, yf); /* A(0, e_f): fine rows and the reflux change */
    memset(cr, 0, 8 * nc);
    for (int64_t q = 0; q < nf; ++q) yf[q] = rf[q] - yf[q];
    amr_average_down(A, yf, cr);
    for (int64_t q = 0; q < nc; ++q)
      if (!A->covered[q]) cr[q] = rc[q] - yc[q];
    orc_vcycle(A->C, 0, ec, cr);
    /* piecewise-constant interpolation of e_c into e_f */
    for (int b = 0; b < f->nb; ++b)
      for (int k = 0; k < bn(f, b, 2); ++k)
        for (int j = 0; j < bn(f, b, 1); ++j)
          for (int i = 0; i < bn(f, b, 0); ++i) {
            int G[3] = {(f->lo[3 * b] + i) >> 1, (f->lo[3 * b + 1] + j) >> 1, (f->lo[3 * b + 2] + k) >> 1};
            ef[IX(f, b, i, j, k)] += ec[coarse_at(c, G)];
          }
    for (int s = 0; s < A->nu2; ++s) {
      amr_fine_colour(A, ef, rf, ec, 0);
      amr_fine_colour(A, ef, rf, ec, 1);
    }
    amr_average_down(A, ef, ec);
    for (int64_t q = 0; q < nf; ++q) pf[q] += ef[q];
    for (int64_t q = 0; q < nc; ++q) pc[q] += ec[q];
    amr_average_down(A, pf, pc);
    amr_residual(A, rhc, rhf, pc, pf, rc, rf);
    rn = amr_norminf(A, rc, rf);
    ++it;
    if (hist) hist[it] = rn;
    if (!(rn == rn) || isinf(rn)) { *status = -3; break; }
  }
  if (*status == 0 && !(rn <= target)) *status = -2;
  if (sing) {
    double s, v;
    amr_vsum(A, pc, pf, &s, &v);
    amr_add_const(A, pc, pf, -s / v);
    amr_average_down(A, pf, pc);
  }
  orc_boxed_to_dense(A->C, 0, pc, phic_d);
  orc_boxed_to_dense(A->F, 0, pf, phif_d);
  free(rhc); free(rhf); free(pc); free(pf); free(rc); free(rf); free(ec); free(ef); free(yc); free(yf); free(cr);
  return it;
}

/* dense wrappers (coarse dense over the coarse domain, fine dense over the fine domain) */
void orc_amr_apply(void* vp, const double* xc_d, const double* xf_d, double* yc_d, double* yf_d, int transpose) {
  oamr* A = (oamr*)vp;
  int64_t nc = A->C->L[0].ntot, nf = A->F->L[0].ntot;
  double *xc = calloc(nc, 8), *xf = calloc(nf, 8), *yc = calloc(nc, 8), *yf = calloc(nf, 8);
  orc_dense_to_boxed(A->C, 0, xc_d, xc);
  orc_dense_to_boxed(A->F, 0, xf_d, xf);
  if (transpose) orc_amr_apply_transpose_boxed(A, xc, xf, yc, yf);
  else orc_amr_apply_boxed(A, xc, xf, yc, yf);
  orc_boxed_to_dense(A->C, 0, yc, yc_d);
  orc_boxed_to_dense(A->F, 0, yf, yf_d);
  free(xc); free(xf); free(yc); free(yf);
}

/* dL/dbeta at the cells of one level (dense, zeroed first) from its per-face gradients g[d]
   (boxed face slots): a face between two cells of the level took the harmonic mean
   2 bL bR / (bL + bR) (d/dbL = 2 bR^2 / (bL + bR)^2); a wall face, or a face on the
   level's coarse/fine boundary, took the one adjacent cell's beta (d = 1). */
static void face_grads_to_cells(const olev* l, double* const* g, const double* beta_dl, double* out_dl) {
  int64_t nx = l->dhi[0] - l->dlo[0] + 1, ny = l->dhi[1] - l->dlo[1] + 1, nz = l->dhi[2] - l->dlo[2] + 1;
  memset(out_dl, 0, sizeof(double) * nx * ny * nz);
  for (int b = 0; b < l->nb; ++b)
    for (int d = 0; d < 3; ++d) {
      int ext[3] = {bn(l, b, 0), bn(l, b, 1), bn(l, b, 2)};
      ext[d] += 1;
      for (int k = 0; k < ext[2]; ++k)
        for (int j = 0; j < ext[1]; ++j)
          for (int i = 0; i < ext[0]; ++i) {
            int loc[3] = {i, j, k};
            double gface = g[d][IX(l, b, i, j, k)];
            if (gface == 0.0) continue;
            /* a face shared by two boxes has a slot in each; each slot carries the part
               of dL/dbeta of the rows that read it, so every slot is mapped to its cells */
            int gR[3], gL[3];
            for (int q = 0; q < 3; ++q) gR[q] = gL[q] = l->lo[3 * b + q] + loc[q];
            gL[d] -= 1;
            int per = l->bclo[d] == ORC_PERIODIC;
            int len = l->dhi[d] - l->dlo[d] + 1;
            int Lw[3] = {gL[0], gL[1], gL[2]}, Rw[3] = {gR[0], gR[1], gR[2]};
            if (per) {
              Lw[d] = l->dlo[d] + pmod(Lw[d] - l->dlo[d], len);
              Rw[d] = l->dlo[d] + pmod(Rw[d] - l->dlo[d], len);
            }
            int Lin = (per || (gL[d] >= l->dlo[d])) && find_box(l, Lw) >= 0;
            int Rin = (per || (gR[d] <= l->dhi[d])) && find_box(l, Rw) >= 0;
            int64_t iL = (Lw[0] - l->dlo[0]) + nx * ((Lw[1] - l->dlo[1]) + ny * (int64_t)(Lw[2] - l->dlo[2]));
            int64_t iR = (Rw[0] - l->dlo[0]) + nx * ((Rw[1] - l->dlo[1]) + ny * (int64_t)(Rw[2] - l->dlo[2]));
            if (Lin && Rin) {
              double bl = beta_dl[iL], br = beta_dl[iR], s2 = (bl + br) * (bl + br);
              out_dl[iL] += gface * 2.0 * br * br / s2;
              out_dl[iR] += gface * 2.0 * bl * bl / s2;
            } else if (Rin) {
              out_dl[iR] += gface;
            } else if (Lin) {
              out_dl[iL] += gface;
            }
            (void)nz;
          }
    }
}

/* dL/dbeta at cells (dense) from the face gradients: a face between two cells of the same
   level took the harmonic mean 2 bL bR / (bL + bR) (d/dbL = 2 bR^2 / (bL + bR)^2); a wall
   face or a coarse/fine fine face took the one adjacent cell's beta (d = 1). */
void orc_amr_grad_beta_cells(void* vp, const double* phic_d, const double* phif_d, const double* lamc_d,
                             const double* lamf_d, const double* betac_d, const double* betaf_d, double* gc_d,
                             double* gf_d) {
  oamr* A = (oamr*)vp;
  oprob* P[2] = {A->C, A->F};
  int64_t nn[2] = {A->C->L[0].ntot, A->F->L[0].ntot};
  double* v[2][2];
  double* g[2][3];
  for (int w = 0; w < 2; ++w) {
    v[w][0] = calloc(nn[w], 8);
    v[w][1] = calloc(nn[w], 8);
    for (int d = 0; d < 3; ++d) g[w][d] = calloc(nn[w], 8);
  }
  orc_dense_to_boxed(A->C, 0, phic_d, v[0][0]);
  orc_dense_to_boxed(A->C, 0, lamc_d, v[0][1]);
  orc_dense_to_boxed(A->F, 0, phif_d, v[1][0]);
  orc_dense_to_boxed(A->F, 0, lamf_d, v[1][1]);
  /* lambda is zero on covered coarse cells (not unknowns) */
  for (int64_t q = 0; q < nn[0]; ++q)
    if (A->covered[q]) v[0][1][q] = 0.0;
  orc_amr_grad_faces(A, v[0][0], v[1][0], v[0][1], v[1][1], g[0][0], g[0][1], g[0][2], g[1][0], g[1][1], g[1][2]);
  const double* beta_d[2] = {betac_d, betaf_d};
  double* out_d[2] = {gc_d, gf_d};
  for (int w = 0; w < 2; ++w) face_grads_to_cells(&P[w]->L[0], g[w], beta_d[w], out_d[w]);
  for (int w = 0; w < 2; ++w) {
    free(v[w][0]);
    free(v[w][1]);
    for (int d = 0; d < 3; ++d) free(g[w][d]);
  }
}

/* =====================================================================
 * Several AMR levels (Sec. "Linear Solvers": multi-AMR-level geometric multigrid; Sec.
 * "Operations between levels").  Level 0 covers the domain; level l (1 <= l < L) is a
 * BoxArray at ratio 2 to level l-1, properly nested in it (its coarse/fine interpolation
 * stencils find uncovered level-(l-1) cells).  The unknowns are the cells of every level
 * not covered by the next finer one.  A cell's row is the level's 7-point operator with:
 * neighbours in the level's own boxes or its periodic images; wall ghosts by the wall rule;
 * coarse/fine ghosts interpolated from the next coarser level (the quadratic of the
 * two-level form); and, on a face shared with a cell covered by the next finer level, the
 * mean of the 4 fine fluxes through it (refluxing).  Each consecutive pair of levels keeps
 * the two-level tables (oamr, built by amr_build_pair, not owning its levels).
 * ===================================================================== */

#define ORC_MAXAMR 4

typedef struct {
  int L;
  oprob* P[ORC_MAXAMR];            /* level l as a one-level problem on its BoxArray */
  oamr pair[ORC_MAXAMR - 1];       /* pair[l]: C = P[l], F = P[l+1] */
  int64_t* gentry[ORC_MAXAMR];     /* level l's ghost slot -> its ghost-map entry, or -1 */
  double a, b;
  int nu1, nu2;
} omlv;

void orc_mlv_destroy(void* vp) {
  omlv* M = (omlv*)vp;
  if (!M) return;
  for (int l = 0; l + 1 < M->L; ++l) amr_free_tables(&M->pair[l]);
  for (int l = 0; l < M->L; ++l) {
    orc_destroy(M->P[l]);
    free(M->gentry[l]);
  }
  free(M);
}

/* L levels; nboxes[l] boxes of level l at boxes[6 * (sum of earlier nboxes) ...] in level
   l's index space (lo[3], hi[3] inclusive).  NULL when a level's boxes are invalid or not
   properly nested. */
void* orc_mlv_create(const int* dlo, const int* dhi, const int* bclo, const int* bchi, const double* plo,
                     const double* phi_, int L, const int* nboxes, const int* boxes) {
  if (L < 1 || L > ORC_MAXAMR) return NULL;
  for (int d = 0; d < 3; ++d) /* composite operators take the linear Dirichlet rule only */
    if (bclo[d] == ORC_DIRICHLET_QUAD || bchi[d] == ORC_DIRICHLET_QUAD) return NULL;
  omlv* M = (omlv*)calloc(1, sizeof(omlv));
  M->L = L;
  int off = 0;
  int ok = 1;
  for (int l = 0; l < L && ok; ++l) {
    int ldlo[3], ldhi[3];
    for (int d = 0; d < 3; ++d) {
      ldlo[d] = dlo[d] << l;
      ldhi[d] = ((dhi[d] + 1) << l) - 1;
    }
    M->P[l] = (oprob*)orc_create(ldlo, ldhi, bclo, bchi, plo, phi_, nboxes[l], boxes + 6 * off);
    off += nboxes[l];
    if (!M->P[l]) ok = 0;
  }
  for (int l = 0; l + 1 < L && ok; ++l) {
    M->pair[l].C = M->P[l];
    M->pair[l].F = M->P[l + 1];
    if (amr_build_pair(&M->pair[l]) != 0) ok = 0;
  }
  if (!ok) {
    orc_mlv_destroy(M);
    return NULL;
  }
  for (int l = 0; l < L; ++l) {
    olev* f = &M->P[l]->L[0];
    M->gentry[l] = (int64_t*)malloc(sizeof(int64_t) * f->ntot);
    for (int64_t q = 0; q < f->ntot; ++q) M->gentry[l][q] = -1;
    for (int64_t e = 0; e < f->ng; ++e) M->gentry[l][f->gdst[e]] = e;
  }
  M->a = 0.0;
  M->b = 1.0;
  M->nu1 = 2;
  M->nu2 = 2;
  return M;
}

int orc_mlv_nlevels(void* vp) { return ((omlv*)vp)->L; }
void* orc_mlv_level(void* vp, int l) { return ((omlv*)vp)->P[l]; }
/* covered flags of level l (boxed), l < L - 1 */
void orc_mlv_covered(void* vp, int l, char* out) {
  omlv* M = (omlv*)vp;
  memcpy(out, M->pair[l].covered, M->P[l]->L[0].ntot);
}

/* Coefficients per level (dense over each level's domain; NULL alpha: 1; NULL beta: 1).  A
   face of level l on its coarse/fine boundary takes its fine cell's beta; then, from the
   finest pair down, the faces and alphas of level l under level l + 1 are averaged from it
   (the coefficient restriction of the two-level form). */
int orc_mlv_set_coeffs(void* vp, double a, double bsc, const double* const* alpha, const double* const* beta) {
  omlv* M = (omlv*)vp;
  M->a = a;
  M->b = bsc;
  for (int l = 0; l < M->L; ++l) orc_set_coeffs(M->P[l], a, bsc, alpha ? alpha[l] : NULL, beta ? beta[l] : NULL);
  for (int l = 1; l < M->L; ++l) {  /* coarse/fine faces of level l: the fine cell's beta */
    oamr* A = &M->pair[l - 1];
    olev* f = &A->F->L[0];
    double* face[3] = {f->bx, f->by, f->bz};
    const double* bf = beta ? beta[l] : NULL;
    for (int64_t q = 0; q < A->ncf; ++q) {
      const ocfghost* G = &A->cf[q];
      int b = box_of_index(f, G->dst);
      int64_t nx = bn(f, b, 0) + 2, ny = bn(f, b, 1) + 2;
      int64_t diff = G->f1 - G->dst;
      int d = (diff == 1 || diff == -1) ? 0 : ((diff == nx || diff == -nx) ? 1 : 2);
      int64_t slot = diff > 0 ? G->f1 : G->dst;
      int64_t rel = G->f1 - f->off[b];
      int g[3] = {f->lo[3 * b] + (int)(rel % nx) - 1, f->lo[3 * b + 1] + (int)((rel / nx) % ny) - 1,
                  f->lo[3 * b + 2] + (int)(rel / (nx * ny)) - 1};
      face[d][slot] = bf ? dense_at(f, bf, g) : 1.0;
    }
  }
  for (int l = M->L - 2; l >= 0; --l) amr_average_down_faces(&M->pair[l]);
  return 0;
}

/* value of level l's ghost slot gq for the level fields x: a coarse/fine ghost by the
   interpolation from level l - 1, a wall ghost by the wall rule, a copy from its source */
static double mlv_ghost_value(const omlv* M, const double* const* x, int l, int64_t gq) {
  if (l > 0) {
    const oamr* A = &M->pair[l - 1];
    int64_t cfi = A->cfidx[gq];
    if (cfi >= 0) {
      const ocfghost* G = &A->cf[cfi];
      double cs = 0.0;
      for (int e = 0; e < 5; ++e) cs += G->cw[e] * x[l - 1][G->cq[e]];
      return (8.0 / 15.0) * cs + (2.0 / 3.0) * x[l][G->f1] - 0.2 * x[l][G->f2];
    }
  }
  const olev* f = &M->P[l]->L[0];
  int64_t e = M->gentry[l][gq];
  return f->gfac[e] * x[l][f->gsrc[e]];
}

/* (A x) at valid cell (b; i, j, k) of level l, an uncovered cell */
static double mlv_row(const omlv* M, const double* const* x, int l, int b, int i, int j, int k) {
  const olev* f = &M->P[l]->L[0];
  const int64_t q = IX(f, b, i, j, k);
  const int loc[3] = {i, j, k};
  double v = M->a * f->alpha[q] * x[l][q];
  for (int d = 0; d < 3; ++d) {
    const double* fa = d == 0 ? f->bx : (d == 1 ? f->by : f->bz);
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    for (int side = 0; side < 2; ++side) {
      int nl[3] = {loc[0], loc[1], loc[2]};
      nl[d] += side ? 1 : -1;
      const int inside = nl[d] >= 0 && nl[d] < bn(f, b, d);
      const int64_t nq = IX(f, b, nl[0], nl[1], nl[2]);
      int64_t src = -1; /* the level-l cell behind the neighbour slot, if it is one */
      if (inside) {
        src = nq;
      } else {
        int64_t e = M->gentry[l][nq];
        if (f->gsrc[e] >= 0 && f->gwall[e] < 0) src = f->gsrc[e];
      }
      if (l + 1 < M->L && src >= 0 && M->pair[l].covered[src]) {
        /* reflux: the mean of the 4 fine fluxes through this face, b beta_f (x_f - x_g) / h_f
           over h_c, the fine ghost x_g interpolated from this level */
        const olev* fn = &M->P[l + 1]->L[0];
        int gl[3] = {f->lo[3 * b] + i, f->lo[3 * b + 1] + j, f->lo[3 * b + 2] + k};
        int gn[3] = {gl[0], gl[1], gl[2]};
        gn[d] += side ? 1 : -1;
        double cf = M->b * 0.25 / (fn->h[d] * f->h[d]);
        const double* fna = d == 0 ? fn->bx : (d == 1 ? fn->by : fn->bz);
        for (int u = 0; u < 2; ++u)
          for (int w = 0; w < 2; ++w) {
            int fg[3];
            fg[d] = side ? 2 * gn[d] : 2 * gn[d] + 1;
            fg[d1] = 2 * gl[d1] + u;
            fg[d2] = 2 * gl[d2] + w;
            wrap_periodic(fn, fg);
            int fb = find_box(fn, fg);
            int fl[3] = {fg[0] - fn->lo[3 * fb], fg[1] - fn->lo[3 * fb + 1], fg[2] - fn->lo[3 * fb + 2]};
            int ghl[3] = {fl[0], fl[1], fl[2]};
            ghl[d] += side ? -1 : 1;
            int sl[3] = {fl[0], fl[1], fl[2]};
            if (!side) sl[d] += 1;
            double beta = fna[IX(fn, fb, sl[0], sl[1], sl[2])];
            double xf = x[l + 1][IX(fn, fb, fl[0], fl[1], fl[2])];
            double xg = mlv_ghost_value(M, x, l + 1, IX(fn, fb, ghl[0], ghl[1], ghl[2]));
            v += cf * beta * (xg - xf);
          }
        continue;
      }
      int fl[3] = {loc[0], loc[1], loc[2]};
      if (side) fl[d] += 1;
      const double w = M->b * fa[IX(f, b, fl[0], fl[1], fl[2])] / (f->h[d] * f->h[d]);
      const double xn = inside ? x[l][nq] : mlv_ghost_value(M, x, l, nq);
      v += w * (x[l][q] - xn);
    }
  }
  return v;
}

static int mlv_covered(const omlv* M, int l, int64_t q) { return l + 1 < M->L && M->pair[l].covered[q]; }

/* The row of an uncovered cell written as terms coef * x[level][q] (the row mlv_row
   evaluates, term by term), so that one walk over the rows gives A x (mode 0), scatters
   A^T y (mode 1: each term of row r adds coef * y_r to its column) or the face gradient
   dL/dbeta_face = -sum_r y_r (d coef / d beta_face) x_q (mode 2).  A term whose coefficient
   is b beta_face / h^2 names that face: level fw, direction fd, boxed slot fs (fw < 0:
   none). */
typedef struct {
  int mode;
  const double* const* x;   /* modes 0 and 2 */
  double* const* y;         /* mode 1: output */
  double yrow, acc;
  double* g[ORC_MAXAMR][3]; /* mode 2: output */
  int bad;                  /* modes 1 and 2: a term read a covered cell */
} mterm;

static void mlv_term(const omlv* M, mterm* R, int lx, int64_t q, double c, int fw, int fd, int64_t fs) {
  double beta = 1.0;
  if (fw >= 0) {
    const olev* f = &M->P[fw]->L[0];
    beta = (fd == 0 ? f->bx : (fd == 1 ? f->by : f->bz))[fs];
  }
  if (R->mode != 0 && mlv_covered(M, lx, q)) R->bad = 1;
  if (R->mode == 0) R->acc += c * beta * R->x[lx][q];
  else if (R->mode == 1) R->y[lx][q] += c * beta * R->yrow;
  else if (fw >= 0) R->g[fw][fd][fs] -= R->yrow * c * R->x[lx][q];
}

/* the value of level l's ghost slot gq as terms, scaled by c (face tag passed through) */
static void mlv_ghost_terms(const omlv* M, mterm* R, int l, int64_t gq, double c, int fw, int fd, int64_t fs) {
  if (l > 0) {
    const oamr* A = &M->pair[l - 1];
    int64_t cfi = A->cfidx[gq];
    if (cfi >= 0) {
      const ocfghost* G = &A->cf[cfi];
      for (int e = 0; e < 5; ++e) mlv_term(M, R, l - 1, G->cq[e], c * (8.0 / 15.0) * G->cw[e], fw, fd, fs);
      mlv_term(M, R, l, G->f1, c * (2.0 / 3.0), fw, fd, fs);
      mlv_term(M, R, l, G->f2, c * (-0.2), fw, fd, fs);
      return;
    }
  }
  const olev* f = &M->P[l]->L[0];
  int64_t e = M->gentry[l][gq];
  mlv_term(M, R, l, f->gsrc[e], c * f->gfac[e], fw, fd, fs);
}

static void mlv_row_terms(const omlv* M, mterm* R, int l, int b, int i, int j, int k) {
  const olev* f = &M->P[l]->L[0];
  const int64_t q = IX(f, b, i, j, k);
  const int loc[3] = {i, j, k};
  mlv_term(M, R, l, q, M->a * f->alpha[q], -1, 0, 0);
  for (int d = 0; d < 3; ++d) {
    const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
    for (int side = 0; side < 2; ++side) {
      int nl[3] = {loc[0], loc[1], loc[2]};
      nl[d] += side ? 1 : -1;
      const int inside = nl[d] >= 0 && nl[d] < bn(f, b, d);
      const int64_t nq = IX(f, b, nl[0], nl[1], nl[2]);
      int64_t src = -1;
      if (inside) {
        src = nq;
      } else {
        int64_t e = M->gentry[l][nq];
        if (f->gsrc[e] >= 0 && f->gwall[e] < 0) src = f->gsrc[e];
      }
      if (l + 1 < M->L && src >= 0 && M->pair[l].covered[src]) {
        /* reflux: b / h_c times the mean of the 4 fine fluxes beta_f (x_g - x_f) / h_f */
        const olev* fn = &M->P[l + 1]->L[0];
        int gl[3] = {f->lo[3 * b] + i, f->lo[3 * b + 1] + j, f->lo[3 * b + 2] + k};
        int gn[3] = {gl[0], gl[1], gl[2]};
        gn[d] += side ? 1 : -1;
        double cf = M->b * 0.25 / (fn->h[d] * f->h[d]);
        for (int u = 0; u < 2; ++u)
          for (int w = 0; w < 2; ++w) {
            int fg[3];
            fg[d] = side ? 2 * gn[d] : 2 * gn[d] + 1;
            fg[d1] = 2 * gl[d1] + u;
            fg[d2] = 2 * gl[d2] + w;
            wrap_periodic(fn, fg);
            int fb = find_box(fn, fg);
            int fl[3] = {fg[0] - fn->lo[3 * fb], fg[1] - fn->lo[3 * fb + 1], fg[2] - fn->lo[3 * fb + 2]};
            int ghl[3] = {fl[0], fl[1], fl[2]};
            ghl[d] += side ? -1 : 1;
            int sl[3] = {fl[0], fl[1], fl[2]};
            if (!side) sl[d] += 1;
            int64_t fs = IX(fn, fb, sl[0], sl[1], sl[2]);
            mlv_term(M, R, l + 1, IX(fn, fb, fl[0], fl[1], fl[2]), -cf, l + 1, d, fs);
            mlv_ghost_terms(M, R, l + 1, IX(fn, fb, ghl[0], ghl[1], ghl[2]), cf, l + 1, d, fs);
          }
        continue;
      }
      int fl[3] = {loc[0], loc[1], loc[2]};
      if (side) fl[d] += 1;
      const int64_t fs = IX(f, b, fl[0], fl[1], fl[2]);
      const double w = M->b / (f->h[d] * f->h[d]);
      mlv_term(M, R, l, q, w, l, d, fs);
      if (inside) mlv_term(M, R, l, nq, -w, l, d, fs);
      else mlv_ghost_terms(M, R, l, nq, -w, l, d, fs);
    }
  }
}

/* every uncovered row once; mode 0 stores the row value in yout, modes 1 and 2 take the
   row's weight from yin */
static void mlv_walk(const omlv* M, mterm* R, double* const* yout, double* const* yin) {
  for (int l = 0; l < M->L; ++l) {
    const olev* f = &M->P[l]->L[0];
    for (int b = 0; b < f->nb; ++b)
      for (int k = 0; k < bn(f, b, 2); ++k)
        for (int j = 0; j < bn(f, b, 1); ++j)
          for (int i = 0; i < bn(f, b, 0); ++i) {
            int64_t q = IX(f, b, i, j, k);
            if (mlv_covered(M, l, q)) continue;
            R->acc = 0.0;
            if (yin) R->yrow = yin[l][q];
            mlv_row_terms(M, R, l, b, i, j, k);
            if (yout) yout[l][q] = R->acc;
          }
  }
}

/* y = A x over all levels (boxed); covered entries of y are 0 */
static void mlv_apply(const omlv* M, const double* const* x, double* const* y) {
  for (int l = 0; l < M->L; ++l) {
    const olev* f = &M->P[l]->L[0];
    memset(y[l], 0, sizeof(double) * f->ntot);
    for (int b = 0; b < f->nb; ++b)
      for (int k = 0; k < bn(f, b, 2); ++k)
        for (int j = 0; j < bn(f, b, 1); ++j)
          for (int i = 0; i < bn(f, b, 0); ++i) {
            int64_t q = IX(f, b, i, j, k);
            if (!mlv_covered(M, l, q)) y[l][q] = mlv_row(M, x, l, b, i, j, k);
          }
  }
}

static double mlv_norminf(const omlv* M, double* const* x) {
  double m = 0.0;
  for (int l = 0; l < M->L; ++l) {
    const olev* f = &M->P[l]->L[0];
    for (int b = 0; b < f->nb; ++b)
      for (int k = 0; k < bn(f, b, 2); ++k)
        for (int j = 0; j < bn(f, b, 1); ++j)
          for (int i = 0; i < bn(f, b, 0); ++i) {
            int64_t q = IX(f, b, i, j, k);
            if (mlv_covered(M, l, q)) continue;
            double v = fabs(x[l][q]);
            if (v > m || v != v) m = v;
          }
  }
  return m;
}

/* volume-weighted sum over the composite cells, and their volume */
static void mlv_vsum(const omlv* M, double* const* x, double* s, double* vol) {
  *s = 0.0;
  *vol = 0.0;
  for (int l = 0; l < M->L; ++l) {
    const olev* f = &M->P[l]->L[0];
    double v = f->h[0] * f->h[1] * f->h[2];
    for (int b = 0; b < f->nb; ++b)
      for (int k = 0; k < bn(f, b, 2); ++k)
        for (int j = 0; j < bn(f, b, 1); ++j)
          for (int i = 0; i < bn(f, b, 0); ++i) {
            int64_t q = IX(f, b, i, j, k);
            if (mlv_covered(M, l, q)) continue;
            *s += v * x[l][q];
            *vol += v;
          }
  }
}

/* r = rhs - A phi on the composite cells (covered 0) */
static void mlv_residual(const omlv* M, double* const* rhs, double* const* phi, double* const* r) {
  mlv_apply(M, (const double* const*)phi, r);
  for (int l = 0; l < M->L; ++l) {
    int64_t n = M->P[l]->L[0].ntot;
    for (int64_t q = 0; q < n; ++q) r[l][q] = mlv_covered(M, l, q) ? 0.0 : rhs[l][q] - r[l][q];
  }
}

/* covered cells of levels L-2 .. 0 := mean of their children, finest pair first */
static void mlv_average_down(const omlv* M, double* const* x) {
  for (int l = M->L - 1; l >= 1; --l) amr_average_down(&M->pair[l - 1], x[l], x[l - 1]);
}

/* one red-black colour on level l >= 1, coarse/fine ghosts from cx (NULL: 0) */
static void mlv_colour(omlv* M, int l, double* e, const double* r, const double* cx, int colour) {
  amr_fill_cf(&M->pair[l - 1], e, cx);
  orc_smooth_colour(M->P[l], 0, e, r, colour);
}

/* Composite multigrid solve over L levels (the multi-level form of the two-level iteration):
   r = composite residual; then, from e = 0 on every level:
   down, for l = L-1 .. 1: nu1 red-black sweeps of e_l on the correction equation of level
     l (right-hand side rr_l; coarse/fine ghosts with a zero coarse correction); the level's
     correction residual s_l = rr_l - A_l e_l; the right-hand side of level l-1: on cells
     covered by level l the average of s_l, elsewhere its composite residual minus the change
     of its composite rows by e_l (the correction's reflux);
   level 0: one V-cycle of its own hierarchy;
   up, for l = 1 .. L-1: e_l += piecewise-constant interpolation of e_(l-1); nu2 sweeps with
     coarse/fine ghosts interpolated from e_(l-1);
   covered corrections := averages of their children (finest pair first); phi += e; covered
   phi := averages.  With L = 2 these are the steps of orc_amr_solve.  Stops at
   ||r||_inf <= max(tol_rel ||rhs||_inf, tol_abs) over the composite cells.  Singular (no
   Dirichlet wall, a = 0): rhs projected to zero volume-weighted mean, phi returned so.
   rhs_d[l], phi_d[l]: dense over level l's domain (cells outside its boxes ignored). */
int orc_mlv_solve(void* vp, const double* const* rhs_d, double* const* phi_d, double tol_rel, double tol_abs, int maxit,
                  double* hist, int* status) {
  omlv* M = (omlv*)vp;
  const int L = M->L;
  double *rhs[ORC_MAXAMR], *phi[ORC_MAXAMR], *r[ORC_MAXAMR], *e[ORC_MAXAMR], *rr[ORC_MAXAMR], *y[ORC_MAXAMR],
      *s[ORC_MAXAMR], *zero[ORC_MAXAMR];
  for (int l = 0; l < L; ++l) {
    int64_t n = M->P[l]->L[0].ntot;
    rhs[l] = calloc(n, 8); phi[l] = calloc(n, 8); r[l] = calloc(n, 8); e[l] = calloc(n, 8);
    rr[l] = calloc(n, 8); y[l] = calloc(n, 8); s[l] = calloc(n, 8); zero[l] = calloc(n, 8);
    orc_dense_to_boxed(M->P[l], 0, rhs_d[l], rhs[l]);
    for (int64_t q = 0; q < n; ++q)
      if (mlv_covered(M, l, q)) rhs[l][q] = 0.0;
  }
  double rn0 = mlv_norminf(M, rhs);
  int sing = M->P[0]->singular;
  if (sing) {
    double sm, v;
    mlv_vsum(M, rhs, &sm, &v);
    for (int l = 0; l < L; ++l) {
      lev_add_const(&M->P[l]->L[0], rhs[l], -sm / v);
      int64_t n = M->P[l]->L[0].ntot;
      for (int64_t q = 0; q < n; ++q)
        if (mlv_covered(M, l, q)) rhs[l][q] = 0.0;
    }
  }
  double target = tol_rel * rn0 > tol_abs ? tol_rel * rn0 : tol_abs;
  mlv_residual(M, rhs, phi, r);
  double rn = mlv_norminf(M, r);
  if (hist) hist[0] = rn;
  int it = 0;
  *status = 0;
  while (!(rn <= target) && it < maxit) {
    for (int l = 0; l < L; ++l) memset(e[l], 0, 8 * M->P[l]->L[0].ntot);
    memcpy(rr[L - 1], r[L - 1], 8 * M->P[L - 1]->L[0].ntot);
    for (int l = L - 1; l >= 1; --l) {
      for (int sw = 0; sw < M->nu1; ++sw) {
        mlv_colour(M, l, e[l], rr[l], NULL, 0);
        mlv_colour(M, l, e[l], rr[l], NULL, 1);
      }
      amr_fill_cf(&M->pair[l - 1], e[l], NULL);
      orc_residual(M->P[l], 0, e[l], rr[l], s[l]);
      /* composite rows of level l-1 applied to (0 below l, e_l on l) */
      const double* xs[ORC_MAXAMR];
      for (int q = 0; q < L; ++q) xs[q] = (q == l) ? e[l] : zero[q];
      mlv_apply(M, xs, y);
      int64_t nc = M->P[l - 1]->L[0].ntot;
      memset(rr[l - 1], 0, 8 * nc);
      amr_average_down(&M->pair[l - 1], s[l], rr[l - 1]);
      for (int64_t q = 0; q < nc; ++q)
        if (!M->pair[l - 1].covered[q]) rr[l - 1][q] = r[l - 1][q] - y[l - 1][q];
    }
    orc_vcycle(M->P[0], 0, e[0], rr[0]);
    for (int l = 1; l < L; ++l) {
      const olev* f = &M->P[l]->L[0];
      const olev* c = &M->P[l - 1]->L[0];
      for (int b = 0; b < f->nb; ++b)
        for (int k = 0; k < bn(f, b, 2); ++k)
          for (int j = 0; j < bn(f, b, 1); ++j)
            for (int i = 0; i < bn(f, b, 0); ++i) {
              int G[3] = {(f->lo[3 * b] + i) >> 1, (f->lo[3 * b + 1] + j) >> 1, (f->lo[3 * b + 2] + k) >> 1};
              e[l][IX(f, b, i, j, k)] += e[l - 1][coarse_at(c, G)];
            }
      for (int sw = 0; sw < M->nu2; ++sw) {
        mlv_colour(M, l, e[l], rr[l], e[l - 1], 0);
        mlv_colour(M, l, e[l], rr[l], e[l - 1], 1);
      }
    }
    mlv_average_down(M, e);
    for (int l = 0; l < L; ++l) {
      int64_t n = M->P[l]->L[0].ntot;
      for (int64_t q = 0; q < n; ++q) phi[l][q] += e[l][q];
    }
    mlv_average_down(M, phi);
    mlv_residual(M, rhs, phi, r);
    rn = mlv_norminf(M, r);
    ++it;
    if (hist) hist[it] = rn;
    if (!(rn == rn) || isinf(rn)) { *status = -3; break; }
  }
  if (*status == 0 && !(rn <= target)) *status = -2;
  if (sing) {
    double sm, v;
    mlv_vsum(M, phi, &sm, &v);
    for (int l = 0; l < L; ++l) lev_add_const(&M->P[l]->L[0], phi[l], -sm / v);
    mlv_average_down(M, phi);
  }
  for (int l = 0; l < L; ++l) {
    orc_boxed_to_dense(M->P[l], 0, phi[l], phi_d[l]);
    free(rhs[l]); free(phi[l]); free(r[l]); free(e[l]); free(rr[l]); free(y[l]); free(s[l]); free(zero[l]);
  }
  return it;
}

/* y = A x for dense level arrays (covered entries of y are 0) */
void orc_mlv_apply(void* vp, const double* const* x_d, double* const* y_d) {
  omlv* M = (omlv*)vp;
  double *x[ORC_MAXAMR], *y[ORC_MAXAMR];
  for (int l = 0; l < M->L; ++l) {
    int64_t n = M->P[l]->L[0].ntot;
    x[l] = calloc(n, 8);
    y[l] = calloc(n, 8);
    orc_dense_to_boxed(M->P[l], 0, x_d[l], x[l]);
  }
  mlv_apply(M, (const double* const*)x, y);
  for (int l = 0; l < M->L; ++l) {
    orc_boxed_to_dense(M->P[l], 0, y[l], y_d[l]);
    free(x[l]); free(y[l]);
  }
}

/* y = A x through the term walk (the same rows as orc_mlv_apply, summed term by term) */
void orc_mlv_apply_terms(void* vp, const double* const* x_d, double* const* y_d) {
  omlv* M = (omlv*)vp;
  double *x[ORC_MAXAMR], *y[ORC_MAXAMR];
  for (int l = 0; l < M->L; ++l) {
    int64_t n = M->P[l]->L[0].ntot;
    x[l] = calloc(n, 8);
    y[l] = calloc(n, 8);
    orc_dense_to_boxed(M->P[l], 0, x_d[l], x[l]);
  }
  mterm R;
  memset(&R, 0, sizeof(R));
  R.mode = 0;
  R.x = (const double* const*)x;
  mlv_walk(M, &R, y, NULL);
  for (int l = 0; l < M->L; ++l) {
    orc_boxed_to_dense(M->P[l], 0, y[l], y_d[l]);
    free(x[l]); free(y[l]);
  }
}

/* x = A^T y for dense level arrays (covered entries of y are ignored, those of x are 0).
   Returns 0, or -1 when a term reads a cell covered by a finer level (a level closer than
   two cells to the coarse/fine boundary of the level it refines): the covered values are
   then averages of finer ones, and A is not a matrix over the unknowns alone. */
int orc_mlv_apply_transpose(void* vp, const double* const* y_d, double* const* x_d) {
  omlv* M = (omlv*)vp;
  double *x[ORC_MAXAMR], *y[ORC_MAXAMR];
  for (int l = 0; l < M->L; ++l) {
    int64_t n = M->P[l]->L[0].ntot;
    x[l] = calloc(n, 8);
    y[l] = calloc(n, 8);
    orc_dense_to_boxed(M->P[l], 0, y_d[l], y[l]);
  }
  mterm R;
  memset(&R, 0, sizeof(R));
  R.mode = 1;
  R.y = x;
  mlv_walk(M, &R, NULL, y);
  for (int l = 0; l < M->L; ++l) {
    orc_boxed_to_dense(M->P[l], 0, x[l], x_d[l]);
    free(x[l]); free(y[l]);
  }
  return R.bad ? -1 : 0;
}

/* dL/dbeta at the cells of every level (dense; covered cells 0) for L = lambda^T (rhs - A phi):
   -lambda^T (dA/dbeta_face) phi per face (lambda's covered entries are ignored), then through
   the face rule of each level (face_grads_to_cells).  Faces under a finer level shape only
   the correction operator, so they take no gradient.  Returns 0 or -1 (as the transpose). */
int orc_mlv_grad_beta_cells(void* vp, const double* const* phi_d, const double* const* lam_d,
                            const double* const* beta_d, double* const* out_d) {
  omlv* M = (omlv*)vp;
  double *phi[ORC_MAXAMR], *lam[ORC_MAXAMR];
  mterm R;
  memset(&R, 0, sizeof(R));
  R.mode = 2;
  for (int l = 0; l < M->L; ++l) {
    int64_t n = M->P[l]->L[0].ntot;
    phi[l] = calloc(n, 8);
    lam[l] = calloc(n, 8);
    orc_dense_to_boxed(M->P[l], 0, phi_d[l], phi[l]);
    orc_dense_to_boxed(M->P[l], 0, lam_d[l], lam[l]);
    for (int d = 0; d < 3; ++d) R.g[l][d] = calloc(n, 8);
  }
  R.x = (const double* const*)phi;
  mlv_walk(M, &R, NULL, lam);
  for (int l = 0; l < M->L; ++l) {
    face_grads_to_cells(&M->P[l]->L[0], R.g[l], beta_d[l], out_d[l]);
    free(phi[l]); free(lam[l]);
    for (int d = 0; d < 3; ++d) free(R.g[l][d]);
  }
  return R.bad ? -1 : 0;
}
