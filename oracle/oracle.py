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
SOURCES = ["gmg_oracle.c", "gmg_oracle_amr.c"]
LIB = os.path.join(BUILD, "liboracle.so")

PERIODIC = 0
DIRICHLET = 1

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
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
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


_i32p = C.POINTER(C.c_int)
_f64p = C.POINTER(C.c_double)


def _declare(L):
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
    bc_lo/bc_hi: PERIODIC or DIRICHLET per direction; prob_lo/prob_hi: physical extent.
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
        if getattr(self, "h", None):
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

    def apply(self, phi):
        phi = _f64(phi)
        out = np.zeros(self.level_shape(0))
        lib().orc_apply(self.h, _dp(phi), _dp(out))
        return out
