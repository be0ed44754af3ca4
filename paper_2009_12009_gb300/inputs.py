"""Seeded synthetic inputs for the multigrid workloads.

This module is shared by the oracle checks and the CUDA path and therefore holds none of
the solver's arithmetic: only grid generation (max_grid_size chopping, Sec. "Regridding")
and the random coefficient / right-hand-side fields.  Dense arrays are float64 with shape
(nz, ny, nx), x fastest.

Workload shapes follow the solver study of Sec. "Linear Solvers" (a variable-coefficient
alpha/beta problem with 256^3 cells on each node):

  poisson32   32^3 periodic, 8 boxes of 16^3, beta = 1, rhs = sin(2 pi x) sin(2 pi y) sin(2 pi z)
  abec256     256^3 Dirichlet, 64 boxes of 64^3, beta log-normal smoothed, rhs N(0,1)
  abec512     512^3 Dirichlet, 64 boxes of 128^3, same recipe
  batch64     64 solves with edges drawn from {32,48,64,96,128,160}, boxes of at most 32^3
  amr2        two-level composite: 128^3 periodic + ratio-2 patch over coarse [32,96)^3
"""
from __future__ import annotations

import numpy as np

PERIODIC = 0
DIRICHLET = 1
NEUMANN = 2
DIRICHLET_QUAD = 3  # Dirichlet side whose ghosts take the quadratic rule

SEEDS = {"poisson32": 12010, "abec256": 12011, "abec512": 12012, "batch64": 12013, "amr2": 12014,
         "walls256": 12015, "contrast256": 12016, "amr3": 12017}
BATCH_EDGES = (32, 48, 64, 96, 128, 160)


def chop(lo, hi, max_grid_size):
    """Cut the box [lo, hi] into chunks of max_grid_size cells per axis from the low end,
    the remainder last (48 -> 32 + 16 for max_grid_size 32).  Box order: x fastest."""
    cuts = []
    for d in range(3):
        c = []
        s = lo[d]
        while s <= hi[d]:
            e = min(s + max_grid_size - 1, hi[d])
            c.append((s, e))
            s = e + 1
        cuts.append(c)
    boxes = []
    for (zl, zh) in cuts[2]:
        for (yl, yh) in cuts[1]:
            for (xl, xh) in cuts[0]:
                boxes.append(((xl, yl, zl), (xh, yh, zh)))
    return boxes


def cell_centres(n, lo=0.0, hi=1.0):
    h = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * h


def sin_product(shape, mode=(2, 2, 2), kind="periodic"):
    """prod_d sin(m_d * pi * x_d) at cell centres of the unit cube (kind='dirichlet'),
    or prod_d sin(2 pi x_d) (kind='periodic', mode ignored)."""
    nz, ny, nx = shape
    xs = [cell_centres(nx), cell_centres(ny), cell_centres(nz)]
    if kind == "periodic":
        fx, fy, fz = (np.sin(2 * np.pi * x) for x in xs)
    else:
        fx, fy, fz = (np.sin(m * np.pi * x) for m, x in zip(mode, xs))
    return fz[:, None, None] * fy[None, :, None] * fx[None, None, :]


def box_mean_filter(a, periodic):
    """3x3x3 mean of a cell field: periodic wrap, or a window truncated at the domain edge
    (mean over the in-domain neighbours only).  Applied separably."""
    out = np.array(a, dtype=np.float64, copy=True)
    cnt = np.ones_like(out) if not periodic else None
    for ax in range(3):
        if periodic:
            out = np.roll(out, 1, axis=ax) + out + np.roll(out, -1, axis=ax)
        else:
            s = out.copy()
            c = cnt.copy()
            sl_lo = [slice(None)] * 3
            sl_hi = [slice(None)] * 3
            sl_lo[ax] = slice(0, -1)
            sl_hi[ax] = slice(1, None)
            s[tuple(sl_hi)] += out[tuple(sl_lo)]
            s[tuple(sl_lo)] += out[tuple(sl_hi)]
            c[tuple(sl_hi)] += cnt[tuple(sl_lo)]
            c[tuple(sl_lo)] += cnt[tuple(sl_hi)]
            out, cnt = s, c
    return out / 27.0 if periodic else out / cnt


def lognormal_beta(rng, shape, periodic):
    """beta = exp(N(0,1)) per cell, smoothed by one 3x3x3 mean filter."""
    return box_mean_filter(np.exp(rng.standard_normal(shape)), periodic)


def poisson32():
    n = 32
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    return dict(name="poisson32", domain=dom, boxes=chop(*dom, 16), bc_lo=[PERIODIC] * 3, bc_hi=[PERIODIC] * 3,
                a=0.0, b=1.0, alpha=None, beta=None, rhs=sin_product((n, n, n), kind="periodic"))


def abec(n, max_grid_size, seed, bc=DIRICHLET, name=None):
    """Variable-beta problem (a = 0, b = 1) on n^3: log-normal smoothed beta, N(0,1) rhs."""
    rng = np.random.default_rng(seed)
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    shape = (n, n, n)
    beta = lognormal_beta(rng, shape, periodic=(bc == PERIODIC))
    rhs = rng.standard_normal(shape)
    if bc == PERIODIC:
        rhs -= rhs.mean()
    return dict(name=name or f"abec{n}", domain=dom, boxes=chop(*dom, max_grid_size), bc_lo=[bc] * 3,
                bc_hi=[bc] * 3, a=0.0, b=1.0, alpha=None, beta=beta, rhs=rhs)


def abec256():
    return abec(256, 64, SEEDS["abec256"], name="abec256")


def abec512():
    return abec(512, 128, SEEDS["abec512"], name="abec512")


def contrast256():
    """The abec256 recipe with a high-contrast coefficient: beta = exp(3 N(0,1)) before the
    3x3x3 mean filter (spans ~8 decades), where the multigrid iteration alone needs ~150
    V-cycles and Krylov acceleration pays."""
    n = 256
    rng = np.random.default_rng(SEEDS["contrast256"])
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    shape = (n, n, n)
    beta = box_mean_filter(np.exp(3.0 * rng.standard_normal(shape)), False)
    rhs = rng.standard_normal(shape)
    return dict(name="contrast256", domain=dom, boxes=chop(*dom, 64), bc_lo=[DIRICHLET] * 3, bc_hi=[DIRICHLET] * 3,
                a=0.0, b=1.0, alpha=None, beta=beta, rhs=rhs)


def face_shape(domain, face):
    """(n_t2, n_t1) of a wall face (2*d + side): its tangential axes in increasing order, the
    lower one fastest."""
    d = face // 2
    t1, t2 = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
    lo, hi = domain
    return (hi[t2] - lo[t2] + 1, hi[t1] - lo[t1] + 1)


def walls256():
    """The abec256 recipe with mixed walls and nonzero wall values: x- Neumann, x+ Dirichlet,
    y- Dirichlet, y+ Neumann, z- Neumann, z+ Dirichlet; every wall face carries N(0,1) values
    (Dirichlet: phi on the face; Neumann: the outward normal derivative)."""
    cfg = abec(256, 64, SEEDS["walls256"], name="walls256")
    cfg["bc_lo"] = [NEUMANN, DIRICHLET, NEUMANN]
    cfg["bc_hi"] = [DIRICHLET, NEUMANN, DIRICHLET]
    rng = np.random.default_rng(SEEDS["walls256"] + 1)
    cfg["wall_values"] = {f: rng.standard_normal(face_shape(cfg["domain"], f)) for f in range(6)}
    return cfg


def batch_sizes(nsolves=64, seed=None):
    rng = np.random.default_rng(SEEDS["batch64"] if seed is None else seed)
    return [tuple(int(v) for v in rng.choice(BATCH_EDGES, size=3)) for _ in range(nsolves)]


def batch_problem(size, index, seed=None, max_grid_size=32):
    """One member of the batched workload: edges size=(nx, ny, nz), Dirichlet walls."""
    base = SEEDS["batch64"] if seed is None else seed
    rng = np.random.default_rng(base + 1 + index)
    nx, ny, nz = size
    dom = ((0, 0, 0), (nx - 1, ny - 1, nz - 1))
    shape = (nz, ny, nx)
    beta = lognormal_beta(rng, shape, periodic=False)
    rhs = rng.standard_normal(shape)
    return dict(name=f"batch{index}", domain=dom, boxes=chop(*dom, max_grid_size), bc_lo=[DIRICHLET] * 3,
                bc_hi=[DIRICHLET] * 3, a=0.0, b=1.0, alpha=None, beta=beta, rhs=rhs,
                prob_hi=(nx / 64.0, ny / 64.0, nz / 64.0))


def batch64(nsolves=64, seed=None):
    return [batch_problem(s, i, seed) for i, s in enumerate(batch_sizes(nsolves, seed))]


def amr2(n=128, seed=None):
    """Two-level composite workload: level 0 n^3 periodic in boxes of (n/2)^3; level 1 at ratio
    2 over the central half of the coarse domain ([n/4, 3n/4)^3 coarse -> (n)^3 fine cells in 8
    boxes of (n/2)^3).  beta log-normal smoothed (periodic wrap on level 0, window truncated at
    the patch edge on level 1, drawn independently), coarse cells under the patch take the
    average of their fine children; rhs N(0,1) on the composite cells minus its
    volume-weighted mean; phi_target N(0,1).  Fine arrays span the patch (n^3)."""
    rng = np.random.default_rng(SEEDS["amr2"] if seed is None else seed)
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    lo, hi = n // 2, 3 * n // 2 - 1
    fdom = ((lo, lo, lo), (hi, hi, hi))
    cshape, fshape = (n, n, n), (n, n, n)
    beta_c = lognormal_beta(rng, cshape, periodic=True)
    beta_f = lognormal_beta(rng, fshape, periodic=False)
    q = n // 4
    avg = beta_f.reshape(n // 2, 2, n // 2, 2, n // 2, 2).mean(axis=(1, 3, 5))
    beta_c[q:3 * q, q:3 * q, q:3 * q] = avg
    covered = np.zeros(cshape, dtype=bool)
    covered[q:3 * q, q:3 * q, q:3 * q] = True
    rhs_c = rng.standard_normal(cshape) * ~covered
    rhs_f = rng.standard_normal(fshape)
    vc, vf = 1.0, 1.0 / 8.0
    mean = (vc * rhs_c.sum() + vf * rhs_f.sum()) / (vc * (~covered).sum() + vf * rhs_f.size)
    rhs_c = (rhs_c - mean) * ~covered
    rhs_f = rhs_f - mean
    return dict(name="amr2", domain=dom, coarse_boxes=chop(*dom, n // 2), fine_boxes=chop(*fdom, n // 2),
                fine_slice=(lo, hi), bc_lo=[PERIODIC] * 3, bc_hi=[PERIODIC] * 3, a=0.0, b=1.0, beta_c=beta_c,
                beta_f=beta_f, rhs_c=rhs_c, rhs_f=rhs_f, covered=covered,
                target_c=rng.standard_normal(cshape) * ~covered, target_f=rng.standard_normal(fshape))


def amr3(n=128, seed=None):
    """Three-level composite workload: level 0 n^3 periodic in boxes of (n/2)^3; level 1 at
    ratio 2 over level-0 cells [n/4, 3n/4)^3 (level-1 cells [n/2, 3n/2)^3, 8 boxes of
    (n/2)^3); level 2 at ratio 2 over level-1 cells [5n/8, 9n/8)^3, off the centre of level 1
    (level-2 cells [5n/4, 9n/4)^3, 64 boxes of (n/4)^3, so that each lies, coarsened, inside
    one level-1 box).  beta log-normal smoothed per level
    (periodic wrap on level 0, window truncated at the patch edge above), cells under a finer
    level take the average of their children, finest pair first; rhs N(0,1) on the composite
    cells minus its volume-weighted mean.  Arrays of level l span its patch (n^3 each);
    `level_lo` is the patch's low corner in level l's index space."""
    rng = np.random.default_rng(SEEDS["amr3"] if seed is None else seed)
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    los = [0, n // 2, 5 * n // 4]
    level_boxes = [chop((lo,) * 3, (lo + n - 1,) * 3, n // 2 if l < 2 else n // 4) for l, lo in enumerate(los)]
    shape = (n, n, n)
    betas = [lognormal_beta(rng, shape, periodic=(l == 0)) for l in range(3)]
    covered = [np.zeros(shape, dtype=bool) for _ in range(3)]
    for l in (1, 0):
        # the finer patch's footprint in level l's patch-relative indices
        a = los[l + 1] // 2 - los[l]
        m = n // 2
        avg = betas[l + 1].reshape(m, 2, m, 2, m, 2).mean(axis=(1, 3, 5))
        betas[l][a:a + m, a:a + m, a:a + m] = avg
        covered[l][a:a + m, a:a + m, a:a + m] = True
    rhss = [rng.standard_normal(shape) * ~c for c in covered]
    vol = [8.0 ** (-l) for l in range(3)]
    mean = sum(v * r.sum() for v, r in zip(vol, rhss)) / sum(v * (~c).sum() for v, c in zip(vol, covered))
    rhss = [(r - mean) * ~c for r, c in zip(rhss, covered)]
    return dict(name="amr3", domain=dom, level_boxes=level_boxes, level_lo=[(lo,) * 3 for lo in los],
                bc_lo=[PERIODIC] * 3, bc_hi=[PERIODIC] * 3, a=0.0, b=1.0, betas=betas, rhss=rhss, covered=covered)
