"""ctypes shim over the plain FP64 CPU multigrid oracle (gmg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the benchmark's
CPU-baseline leg.  The product path never imports it.

Dense arrays are numpy float64 of shape (nz, ny, nx) over a level's domain (x fastest).
"Boxed" arrays are the oracle's own layout: one ghosted (nx+2)(ny+2)(nz+2) array per
box, concatenated in box order.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SOURCES = ["gmg_oracle.c"]
LIB = os.path.join(BUILD, "liboracle.so")

PERIODIC = 0
DIRICHLET = 1
NEUMANN = 2

# status codes of orc_solve
OK, BAD_INPUT, NOT_CONVERGED, DIVERGED = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


def set_threads(n: int) -> None:
    """OpenMP threads of the oracle's box loops (1: sequential; results are bitwise the same)."""
    lib().orc_set_threads(int(n))


def threads() -> int:
    return lib().orc_get_threads()


_i32p = C.POINTER(C.c_int)
_f64p = C.POINTER(C.c_double)


def _declare(L):
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_set_prolong.argtypes = [C.c_void_p, C.c_int]
    L.orc_get_threads.restype = C.c_int
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [_i32p, _i32p, _i32p, _i32p, _f64p, _f64p, C.c_int, _i32p]
    L.orc_destroy.argtypes = [C.c_void_p]
    for name in ["orc_nlevels"]:
        getattr(L, name).argtypes = [C.c_void_p]
        getattr(L, name).restype = C.c_int
    L.orc_level_nboxes.argtypes = [C.c_void_p, C.c_int]
    L.orc_level_nboxes.restype = C.c_int
    L.orc_level_size.argtypes = [C.c_void_p, C.c_int]
    L.orc_level_size.restype = C.c_int64
    L.orc_level_boxes.argtypes = [C.c_void_p, C.c_int, _i32p]
    L.orc_level_domain.argtypes = [C.c_void_p, C.c_int, _i32p]
    L.orc_level_parents.argtypes = [C.c_void_p, C.c_int, _i32p]
    L.orc_set_params.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double]
    L.orc_last_bottom_iters.argtypes = [C.c_void_p]
    L.orc_last_bottom_iters.restype = C.c_int
    L.orc_dense_to_boxed.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p]
    L.orc_boxed_to_dense.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p]
    L.orc_set_coeffs.argtypes = [C.c_void_p, C.c_double, C.c_double, _f64p, _f64p]
    L.orc_set_coeffs.restype = C.c_int
    L.orc_get_coeffs.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p, _f64p, _f64p]
    L.orc_apply_level.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p]
    L.orc_fill_ghosts.argtypes = [C.c_void_p, C.c_int, _f64p]
    L.orc_smooth_colour.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p, C.c_int]
    L.orc_residual.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p, _f64p]
    L.orc_restrict.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p]
    L.orc_prolong_add.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p]
    L.orc_level_dot.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p]
    L.orc_level_dot.restype = C.c_double
    L.orc_level_norminf.argtypes = [C.c_void_p, C.c_int, _f64p]
    L.orc_level_norminf.restype = C.c_double
    L.orc_bottom.argtypes = [C.c_void_p, _f64p, _f64p]
    L.orc_bottom.restype = C.c_int
    L.orc_vcycle.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p]
    L.orc_solve.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_double, C.c_int, C.c_int, _f64p, _i32p]
    L.orc_solve.restype = C.c_int
    L.orc_apply.argtypes = [C.c_void_p, _f64p, _f64p]
    L.orc_apply_transpose.argtypes = [C.c_void_p, _f64p, _f64p]
    L.orc_set_cycle.argtypes = [C.c_void_p, C.c_int, C.c_int]
    L.orc_solve_krylov.argtypes = [C.c_void_p, _f64p, _f64p, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int,
                                   _f64p, _i32p]
    L.orc_solve_krylov.restype = C.c_int
    L.orc_apply_bc.argtypes = [C.c_void_p, _f64p, _f64p]
    L.orc_set_bc_values.argtypes = [C.c_void_p, C.c_int, _f64p]
    L.orc_set_bc_values.restype = C.c_int
    L.orc_grad_beta_cells.argtypes = [C.c_void_p, _f64p, _f64p, _f64p, _f64p]
    L.orc_grad_wall_values.argtypes = [C.c_void_p, _f64p, C.c_int, _f64p]
    L.orc_grad_wall_values.restype = C.c_int


def _ip(a):
    return a.ctypes.data_as(_i32p)


def _dp(a):
    return a.ctypes.data_as(_f64p) if a is not None else None


def _i32(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


class Problem:
    """Single-level problem on a BoxArray with its multigrid hierarchy.

    domain: (lo[3], hi[3]) inclusive; boxes: list of (lo[3], hi[3]) inclusive;
    bc_lo/bc_hi: PERIODIC, DIRICHLET, NEUMANN or DIRICHLET_QUAD (a Dirichlet side with the
    quadratic ghost rule) per direction; prob_lo/prob_hi: physical extent.  Walls are homogeneous unless set_bc_values gives them values.
    """

    def __init__(self, domain, boxes, bc_lo, bc_hi, prob_lo=(0.0, 0.0, 0.0), prob_hi=(1.0, 1.0, 1.0)):
        L = lib()
        dlo, dhi = _i32(domain[0]), _i32(domain[1])
        bx = _i32([list(b[0]) + list(b[1]) for b in boxes]).reshape(-1)
        self._bclo, self._bchi = _i32(bc_lo), _i32(bc_hi)
        self._plo, self._phi = _f64(prob_lo), _f64(prob_hi)
        self.h = L.orc_create(_ip(dlo), _ip(dhi), _ip(self._bclo), _ip(self._bchi), _dp(self._plo),
                              _dp(self._phi), len(boxes), _ip(bx))
        if not self.h:
            raise ValueError("oracle: invalid domain/boxes/boundary conditions")
        self.domain = (tuple(dlo), tuple(dhi))

    def __del__(self):
        if getattr(self, "h", None) and not getattr(self, "_view", False):
            lib().orc_destroy(self.h)
        self.h = None

    # hierarchy -------------------------------------------------------------
    @property
    def nlevels(self) -> int:
        return lib().orc_nlevels(self.h)

    def level_boxes(self, m):
        nb = lib().orc_level_nboxes(self.h, m)
        out = np.zeros(6 * nb, dtype=np.int32)
        lib().orc_level_boxes(self.h, m, _ip(out))
        out = out.reshape(nb, 6)
        return [(tuple(int(v) for v in r[:3]), tuple(int(v) for v in r[3:])) for r in out]

    def level_domain(self, m):
        out = np.zeros(6, dtype=np.int32)
        lib().orc_level_domain(self.h, m, _ip(out))
        return (tuple(int(v) for v in out[:3]), tuple(int(v) for v in out[3:]))

    def level_parents(self, m):
        nb = lib().orc_level_nboxes(self.h, m)
        out = np.zeros(nb, dtype=np.int32)
        lib().orc_level_parents(self.h, m, _ip(out))
        return [int(v) for v in out]

    def level_shape(self, m):
        lo, hi = self.level_domain(m)
        return (hi[2] - lo[2] + 1, hi[1] - lo[1] + 1, hi[0] - lo[0] + 1)

    def level_size(self, m):
        return int(lib().orc_level_size(self.h, m))

    def set_cycle(self, bottom_cg=False, post_reverse=False):
        """bottom solver CG instead of BiCGStab; post-smoothing black before red (symmetric
        V-cycle)."""
        lib().orc_set_cycle(self.h, int(bottom_cg), int(post_reverse))

    def set_prolong(self, trilinear=False):
        """interpolation of the coarse correction: piecewise constant (default) or trilinear"""
        lib().orc_set_prolong(self.h, int(bool(trilinear)))

    def set_params(self, nu1=2, nu2=2, bot_maxit=200, bot_tol=1e-4):
        lib().orc_set_params(self.h, nu1, nu2, bot_maxit, bot_tol)

    # layout ------------------------------------------------------------------
    def to_boxed(self, m, dense):
        dense = _f64(dense)
        assert dense.shape == self.level_shape(m)
        out = np.zeros(self.level_size(m))
        lib().orc_dense_to_boxed(self.h, m, _dp(dense), _dp(out))
        return out

    def to_dense(self, m, boxed):
        boxed = _f64(boxed)
        out = np.zeros(self.level_shape(m))
        lib().orc_boxed_to_dense(self.h, m, _dp(boxed), _dp(out))
        return out

    def box_view(self, m, boxed, b):
        """View of box b's ghosted array, shape (nz+2, ny+2, nx+2)."""
        boxes = self.level_boxes(m)
        off = 0
        for q, (lo, hi) in enumerate(boxes):
            n = [hi[d] - lo[d] + 3 for d in range(3)]
            size = n[0] * n[1] * n[2]
            if q == b:
                return boxed[off:off + size].reshape(n[2], n[1], n[0])
            off += size
        raise IndexError(b)

    # coefficients --------------------------------------------------------------
    def set_coeffs(self, a=0.0, b=1.0, alpha=None, beta=None):
        self._alpha = None if alpha is None else _f64(alpha)
        self._beta = None if beta is None else _f64(beta)
        lib().orc_set_coeffs(self.h, a, b, _dp(self._alpha), _dp(self._beta))

    def coeffs(self, m):
        n = self.level_size(m)
        al, bx, by, bz = (np.zeros(n) for _ in range(4))
        lib().orc_get_coeffs(self.h, m, _dp(al), _dp(bx), _dp(by), _dp(bz))
        return al, bx, by, bz

    # steps (boxed arrays, modified in place where the C function does) ----------
    def fill_ghosts(self, m, f):
        lib().orc_fill_ghosts(self.h, m, _dp(f))

    def apply_level(self, m, phi):
        out = np.zeros_like(phi)
        lib().orc_apply_level(self.h, m, _dp(phi), _dp(out))
        return out

    def smooth_colour(self, m, phi, rhs, colour):
        lib().orc_smooth_colour(self.h, m, _dp(phi), _dp(_f64(rhs)), colour)

    def residual(self, m, phi, rhs):
        r = np.zeros_like(phi)
        lib().orc_residual(self.h, m, _dp(phi), _dp(_f64(rhs)), _dp(r))
        return r

    def restrict(self, m, fine):
        c = np.zeros(self.level_size(m + 1))
        lib().orc_restrict(self.h, m, _dp(_f64(fine)), _dp(c))
        return c

    def prolong_add(self, m, coarse, fine):
        lib().orc_prolong_add(self.h, m, _dp(_f64(coarse)), _dp(fine))

    def dot(self, m, x, y):
        return lib().orc_level_dot(self.h, m, _dp(_f64(x)), _dp(_f64(y)))

    def norminf(self, m, x):
        return lib().orc_level_norminf(self.h, m, _dp(_f64(x)))

    def bottom(self, rhs):
        x = np.zeros(self.level_size(self.nlevels - 1))
        it = lib().orc_bottom(self.h, _dp(_f64(rhs)), _dp(x))
        return x, it

    def vcycle(self, m, r):
        e = np.zeros(self.level_size(m))
        lib().orc_vcycle(self.h, m, _dp(e), _dp(_f64(r)))
        return e

    # whole solve ------------------------------------------------------------------
    def solve(self, rhs, tol_rel=1e-10, tol_abs=0.0, maxit=100, project_mean=False):
        rhs = _f64(rhs)
        phi = np.zeros(self.level_shape(0))
        hist = np.zeros(maxit + 1)
        status = np.zeros(1, dtype=np.int32)
        it = lib().orc_solve(self.h, _dp(rhs), _dp(phi), tol_rel, tol_abs, maxit, int(project_mean),
                             _dp(hist), _ip(status))
        return phi, int(it), hist[:it + 1].copy(), int(status[0])

    def solve_krylov(self, rhs, method, tol_rel=1e-10, tol_abs=0.0, maxit=100, project_mean=False):
        """Krylov solve preconditioned by one V-cycle per application: method 1 BiCGStab
        (right preconditioned), 2 conjugate gradients.  Returns (phi, iterations,
        recursive-residual history, status)."""
        rhs = _f64(rhs)
        phi = np.zeros(self.level_shape(0))
        hist = np.zeros(maxit + 1)
        status = np.zeros(1, dtype=np.int32)
        it = lib().orc_solve_krylov(self.h, _dp(rhs), _dp(phi), tol_rel, tol_abs, maxit, int(method),
                                    int(project_mean), _dp(hist), _ip(status))
        return phi, int(it), hist[:it + 1].copy(), int(status[0])

    def apply(self, phi):
        """A phi with homogeneous walls (linear)."""
        phi = _f64(phi)
        out = np.zeros(self.level_shape(0))
        lib().orc_apply(self.h, _dp(phi), _dp(out))
        return out

    def apply_transpose(self, y):
        """A^T y with homogeneous walls, from the matrix entries of A's rows (sequential)."""
        y = _f64(y)
        out = np.zeros(self.level_shape(0))
        lib().orc_apply_transpose(self.h, _dp(y), _dp(out))
        return out

    # wall values ----------------------------------------------------------------
    def face_shape(self, face):
        """Shape of face (2*d + side)'s value array: its two tangential axes in increasing
        order, the lower one fastest (numpy shape (n_t2, n_t1))."""
        d = face // 2
        t1, t2 = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
        lo, hi = self.domain
        return (hi[t2] - lo[t2] + 1, hi[t1] - lo[t1] + 1)

    def set_bc_values(self, face, values):
        """Wall values of level-0 face `face` = 2*d + side: phi on the face (Dirichlet) or the
        outward normal derivative (Neumann); None clears them (g = 0)."""
        if values is None:
            st = lib().orc_set_bc_values(self.h, face, None)
        else:
            v = _f64(values)
            if v.shape != self.face_shape(face):
                raise ValueError(f"face {face}: values of shape {v.shape}, expected {self.face_shape(face)}")
            st = lib().orc_set_bc_values(self.h, face, _dp(v))
        if st != 0:
            raise ValueError(f"face {face} is periodic or out of range")

    def grad_beta(self, phi, lam, beta=None):
        """dL/dbeta at the cells (dense) from the solution phi (wall values of this problem)
        and the adjoint lambda; beta: the cell beta of set_coeffs (None: 1)."""
        out = np.zeros(self.level_shape(0))
        b = None if beta is None else _f64(beta)
        lib().orc_grad_beta_cells(self.h, _dp(_f64(phi)), _dp(_f64(lam)), _dp(b), _dp(out))
        return out

    def grad_wall_values(self, lam, face):
        """dL/dg on wall face `face` for the adjoint lambda (dense)."""
        out = np.zeros(self.face_shape(face))
        if lib().orc_grad_wall_values(self.h, _dp(_f64(lam)), face, _dp(out)) != 0:
            raise ValueError(f"face {face} is periodic or out of range")
        return out

    def apply_bc(self, phi):
        """A phi with the wall values in the ghosts (affine in phi)."""
        phi = _f64(phi)
        out = np.zeros(self.level_shape(0))
        lib().orc_apply_bc(self.h, _dp(phi), _dp(out))
        return out


def _declare_amr(L):
    vp = C.c_void_p
    L.orc_amr_create.restype = vp
    L.orc_amr_create.argtypes = [_i32p, _i32p, _i32p, _i32p, _f64p, _f64p, C.c_int, _i32p, C.c_int, _i32p]
    L.orc_amr_destroy.argtypes = [vp]
    L.orc_amr_coarse.restype = vp
    L.orc_amr_coarse.argtypes = [vp]
    L.orc_amr_fine.restype = vp
    L.orc_amr_fine.argtypes = [vp]
    L.orc_amr_ncf.restype = C.c_int64
    L.orc_amr_ncf.argtypes = [vp]
    L.orc_amr_covered.argtypes = [vp, C.c_char_p]
    L.orc_amr_set_coeffs.argtypes = [vp, C.c_double, C.c_double, _f64p, _f64p, _f64p, _f64p]
    L.orc_amr_apply.argtypes = [vp, _f64p, _f64p, _f64p, _f64p, C.c_int]
    L.orc_amr_solve.restype = C.c_int
    L.orc_amr_solve.argtypes = [vp, _f64p, _f64p, _f64p, _f64p, C.c_double, C.c_double, C.c_int, _f64p, _i32p]
    L.orc_amr_grad_beta_cells.argtypes = [vp, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]


class AmrProblem:
    """Two-level composite problem: a coarse level covering the domain and a ratio-2 fine
    level over part of it.  Coarse dense arrays are (nz, ny, nx) over the coarse domain;
    fine dense arrays are over the whole FINE-resolution domain (only cells inside fine
    boxes are used)."""

    def __init__(self, domain, coarse_boxes, fine_boxes, bc_lo, bc_hi, prob_lo=(0.0, 0.0, 0.0),
                 prob_hi=(1.0, 1.0, 1.0)):
        L = lib()
        if not hasattr(L, "_amr_declared"):
            _declare_amr(L)
            L._amr_declared = True
        dlo, dhi = _i32(domain[0]), _i32(domain[1])
        cb = _i32([list(b[0]) + list(b[1]) for b in coarse_boxes]).reshape(-1)
        fb = _i32([list(b[0]) + list(b[1]) for b in fine_boxes]).reshape(-1)
        self._keep = [_i32(bc_lo), _i32(bc_hi), _f64(prob_lo), _f64(prob_hi)]
        self.h = L.orc_amr_create(_ip(dlo), _ip(dhi), _ip(self._keep[0]), _ip(self._keep[1]), _dp(self._keep[2]),
                                  _dp(self._keep[3]), len(coarse_boxes), _ip(cb), len(fine_boxes), _ip(fb))
        if not self.h:
            raise ValueError("oracle: invalid two-level layout")
        self.coarse_shape = tuple(int(dhi[d] - dlo[d] + 1) for d in (2, 1, 0))
        self.fine_shape = tuple(2 * n for n in self.coarse_shape)
        self.fine_boxes = fine_boxes
        self.C = Problem.__new__(Problem)
        self.C.h = L.orc_amr_coarse(self.h)
        self.F = Problem.__new__(Problem)
        self.F.h = L.orc_amr_fine(self.h)
        # masks of the composite unknowns
        self.fine_mask = np.zeros(self.fine_shape, dtype=bool)
        for lo, hi in fine_boxes:
            self.fine_mask[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = True
        cov = self.fine_mask.reshape(self.coarse_shape[0], 2, self.coarse_shape[1], 2, self.coarse_shape[2], 2)
        self.covered = cov.all(axis=(1, 3, 5))
        self.coarse_mask = ~self.covered

    def __del__(self):
        if getattr(self, "h", None):
            # the coarse/fine sub-problems are owned by the composite handle
            self.C.h = None
            self.F.h = None
            lib().orc_amr_destroy(self.h)
            self.h = None

    @property
    def ncf(self):
        return int(lib().orc_amr_ncf(self.h))

    def set_coeffs(self, a=0.0, b=1.0, alpha_c=None, beta_c=None, alpha_f=None, beta_f=None):
        self._coef = [None if x is None else _f64(x) for x in (alpha_c, beta_c, alpha_f, beta_f)]
        lib().orc_amr_set_coeffs(self.h, a, b, *(_dp(x) for x in self._coef))

    def apply(self, xc, xf, transpose=False):
        xc, xf = _f64(xc), _f64(xf)
        yc, yf = np.zeros(self.coarse_shape), np.zeros(self.fine_shape)
        lib().orc_amr_apply(self.h, _dp(xc), _dp(xf), _dp(yc), _dp(yf), int(transpose))
        return yc * self.coarse_mask, yf * self.fine_mask

    def solve(self, rhs_c, rhs_f, tol_rel=1e-10, tol_abs=0.0, maxit=100):
        rc, rf = _f64(rhs_c), _f64(rhs_f)
        pc, pf = np.zeros(self.coarse_shape), np.zeros(self.fine_shape)
        hist = np.zeros(maxit + 1)
        st = np.zeros(1, dtype=np.int32)
        it = lib().orc_amr_solve(self.h, _dp(rc), _dp(rf), _dp(pc), _dp(pf), tol_rel, tol_abs, maxit, _dp(hist),
                                 _ip(st))
        return pc, pf * self.fine_mask, int(it), hist[:it + 1].copy(), int(st[0])

    def grad_beta(self, phi_c, phi_f, lam_c, lam_f, beta_c, beta_f):
        """dL/dbeta at coarse and fine cells from dL/dbeta_face = -lambda^T dA/dbeta_face phi."""
        args = [_f64(x) for x in (phi_c, phi_f, lam_c, lam_f, beta_c, beta_f)]
        gc, gf = np.zeros(self.coarse_shape), np.zeros(self.fine_shape)
        lib().orc_amr_grad_beta_cells(self.h, *(_dp(x) for x in args), _dp(gc), _dp(gf))
        return gc, gf

    # composite-vector helpers ---------------------------------------------------------------
    def pack(self, xc, xf):
        return np.concatenate([np.asarray(xc)[self.coarse_mask], np.asarray(xf)[self.fine_mask]])

    def unpack(self, v):
        nc = int(self.coarse_mask.sum())
        xc, xf = np.zeros(self.coarse_shape), np.zeros(self.fine_shape)
        xc[self.coarse_mask] = v[:nc]
        xf[self.fine_mask] = v[nc:]
        return xc, xf

    def volumes(self):
        nz, ny, nx = self.coarse_shape
        plo, phi = self._keep[2], self._keep[3]
        vc = np.prod([(phi[d] - plo[d]) / n for d, n in zip(range(3), (nx, ny, nz))])
        return self.pack(np.full(self.coarse_shape, vc), np.full(self.fine_shape, vc / 8.0))

    def matrix(self):
        """Dense composite matrix (small problems only), columns = composite unknowns."""
        n = int(self.coarse_mask.sum() + self.fine_mask.sum())
        M = np.zeros((n, n))
        e = np.zeros(n)
        for j in range(n):
            e[:] = 0.0
            e[j] = 1.0
            M[:, j] = self.pack(*self.apply(*self.unpack(e)))
        return M


def _declare_mlv(L):
    vp = C.c_void_p
    pp = C.POINTER(_f64p)
    L.orc_mlv_create.restype = vp
    L.orc_mlv_create.argtypes = [_i32p, _i32p, _i32p, _i32p, _f64p, _f64p, C.c_int, _i32p, _i32p]
    L.orc_mlv_destroy.argtypes = [vp]
    L.orc_mlv_covered.argtypes = [vp, C.c_int, C.c_char_p]
    L.orc_mlv_set_coeffs.argtypes = [vp, C.c_double, C.c_double, pp, pp]
    L.orc_mlv_set_coeffs.restype = C.c_int
    L.orc_mlv_apply.argtypes = [vp, pp, pp]
    L.orc_mlv_solve.argtypes = [vp, pp, pp, C.c_double, C.c_double, C.c_int, _f64p, _i32p]
    L.orc_mlv_solve.restype = C.c_int
    L.orc_mlv_level.restype = vp
    L.orc_mlv_level.argtypes = [vp, C.c_int]
    L.orc_mlv_apply_terms.argtypes = [vp, pp, pp]
    L.orc_mlv_apply_transpose.argtypes = [vp, pp, pp]
    L.orc_mlv_apply_transpose.restype = C.c_int
    L.orc_mlv_grad_beta_cells.argtypes = [vp, pp, pp, pp, pp]
    L.orc_mlv_grad_beta_cells.restype = C.c_int


def _ptrs(arrays):
    a = (_f64p * len(arrays))()
    for i, x in enumerate(arrays):
        a[i] = _dp(x) if x is not None else None
    return a


class MultiLevelProblem:
    """Composite problem over L AMR levels (ratio 2 between consecutive levels): level 0 covers
    the domain, level l is a BoxArray in level l's index space (the domain scaled by 2^l),
    properly nested in level l - 1.  Dense arrays of level l are (nz, ny, nx) over the whole
    level-l domain; only cells inside level l's boxes are used, and of those only the ones
    not covered by level l + 1 are unknowns."""

    def __init__(self, domain, level_boxes, bc_lo, bc_hi, prob_lo=(0.0, 0.0, 0.0), prob_hi=(1.0, 1.0, 1.0)):
        L = lib()
        if not hasattr(L, "_mlv_declared"):
            _declare_mlv(L)
            L._mlv_declared = True
        dlo, dhi = _i32(domain[0]), _i32(domain[1])
        nb = _i32([len(b) for b in level_boxes])
        bx = _i32([list(b[0]) + list(b[1]) for lev in level_boxes for b in lev]).reshape(-1)
        self._keep = [_i32(bc_lo), _i32(bc_hi), _f64(prob_lo), _f64(prob_hi)]
        self.h = L.orc_mlv_create(_ip(dlo), _ip(dhi), _ip(self._keep[0]), _ip(self._keep[1]), _dp(self._keep[2]),
                                  _dp(self._keep[3]), len(level_boxes), _ip(nb), _ip(bx))
        if not self.h:
            raise ValueError("oracle: invalid multi-level layout")
        self.L = len(level_boxes)
        base = tuple(int(dhi[d] - dlo[d] + 1) for d in (2, 1, 0))
        self.shapes = [tuple(n << l for n in base) for l in range(self.L)]
        self.level_boxes = level_boxes
        self.inside = []
        for l in range(self.L):
            m = np.zeros(self.shapes[l], dtype=bool)
            for lo, hi in level_boxes[l]:
                m[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] = True
            self.inside.append(m)
        # unknowns: inside level l and not under level l + 1
        self.masks = []
        for l in range(self.L):
            m = self.inside[l].copy()
            if l + 1 < self.L:
                s = self.shapes[l]
                m &= ~self.inside[l + 1].reshape(s[0], 2, s[1], 2, s[2], 2).all(axis=(1, 3, 5))
            self.masks.append(m)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_mlv_destroy(self.h)
            self.h = None

    def level(self, l):
        """level l as a one-level Problem view (owned by this handle)"""
        P = Problem.__new__(Problem)
        P.h = lib().orc_mlv_level(self.h, l)
        P._view = True
        lo = tuple(0 for _ in range(3))
        s = self.shapes[l]
        P.domain = (lo, (s[2] - 1, s[1] - 1, s[0] - 1))
        return P

    def set_coeffs(self, a=0.0, b=1.0, alphas=None, betas=None):
        self._coef = [None if alphas is None else [_f64(x) for x in alphas],
                      None if betas is None else [_f64(x) for x in betas]]
        lib().orc_mlv_set_coeffs(self.h, a, b, _ptrs(self._coef[0]) if alphas is not None else None,
                                 _ptrs(self._coef[1]) if betas is not None else None)

    def apply(self, xs, transpose=False, terms=False):
        """A x (rows evaluated directly; terms=True: the same rows summed term by term), or
        A^T x (scattered term by term; raises ValueError where a term reads a covered cell).
        Entries outside the unknowns are 0."""
        xs = [_f64(x) for x in xs]
        ys = [np.zeros(s) for s in self.shapes]
        if transpose:
            if lib().orc_mlv_apply_transpose(self.h, _ptrs(xs), _ptrs(ys)) != 0:
                raise ValueError("oracle: a coarse/fine term reads a covered cell (nesting closer than two cells)")
        elif terms:
            lib().orc_mlv_apply_terms(self.h, _ptrs(xs), _ptrs(ys))
        else:
            lib().orc_mlv_apply(self.h, _ptrs(xs), _ptrs(ys))
        return [y * m for y, m in zip(ys, self.masks)]

    def grad_beta(self, phis, lams, betas=None):
        """dL/dbeta per level (dense; 0 outside the unknowns) for L = lambda^T (rhs - A(beta) phi),
        betas the cell arrays given to set_coeffs (None: 1)."""
        phis = [_f64(x) for x in phis]
        lams = [_f64(x) for x in lams]
        betas = [_f64(np.ones(s) if betas is None else b) for s, b in zip(self.shapes, betas or [None] * self.L)]
        outs = [np.zeros(s) for s in self.shapes]
        if lib().orc_mlv_grad_beta_cells(self.h, _ptrs(phis), _ptrs(lams), _ptrs(betas), _ptrs(outs)) != 0:
            raise ValueError("oracle: a coarse/fine term reads a covered cell (nesting closer than two cells)")
        return [o * m for o, m in zip(outs, self.masks)]

    def solve(self, rhss, tol_rel=1e-10, tol_abs=0.0, maxit=100):
        rs = [_f64(r) for r in rhss]
        ps = [np.zeros(s) for s in self.shapes]
        hist = np.zeros(maxit + 1)
        st = np.zeros(1, dtype=np.int32)
        it = lib().orc_mlv_solve(self.h, _ptrs(rs), _ptrs(ps), tol_rel, tol_abs, maxit, _dp(hist), _ip(st))
        return [p * m for p, m in zip(ps, self.inside)], int(it), hist[:it + 1].copy(), int(st[0])

    def pack(self, xs):
        return np.concatenate([np.asarray(x)[m] for x, m in zip(xs, self.masks)])

    def unpack(self, v):
        out, o = [], 0
        for s, m in zip(self.shapes, self.masks):
            x = np.zeros(s)
            k = int(m.sum())
            x[m] = v[o:o + k]
            o += k
            out.append(x)
        return out

    def volumes(self):
        return np.concatenate([np.full(int(m.sum()), 8.0 ** (-l)) for l, m in enumerate(self.masks)])

    def matrix(self):
        n = self.pack([np.zeros(s) for s in self.shapes]).size
        A = np.zeros((n, n))
        e = np.zeros(n)
        for j in range(n):
            e[:] = 0.0
            e[j] = 1.0
            A[:, j] = self.pack(self.apply(self.unpack(e)))
        return A
