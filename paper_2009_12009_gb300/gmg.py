"""Python binding of the GB300 multigrid library (libgmg.so, C ABI in include/gmg.h).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.
PyTorch supplies device memory (fields and the workspace) and the CUDA stream.  There is
no CPU fallback: if the library cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, BAD_INPUT, NOT_CONVERGED, DIVERGED, CUDA_ERR, DEVICE_TIMEOUT, NO_WORKSPACE, STATE = 0, -1, -2, -3, -4, -5, -6, -7
PERIODIC, DIRICHLET, NEUMANN, DIRICHLET_QUAD = 0, 1, 2, 3
DIRICHLET0 = DIRICHLET
FP64, MIXED_FP32, MIXED_BF16 = 0, 1, 2
DT_F64, DT_F32, DT_BF16 = 0, 1, 2
GX = 8  # first valid cell of a row sits at element GX (16-byte aligned for every type)

PRECISION = {"fp64": FP64, "fp32": MIXED_FP32, "mixed_fp32": MIXED_FP32, "bf16": MIXED_BF16, "mixed_bf16": MIXED_BF16}

# every symbol declared in include/gmg.h
EXPORTS = [
    "gmg_default_params", "gmg_create", "gmg_destroy", "gmg_last_error", "gmg_define_domain", "gmg_define_level",
    "gmg_chop_domain", "gmg_mg_nlevels", "gmg_mg_level_info", "gmg_mg_level_boxes", "gmg_wave_tiles", "gmg_tail_plan", "gmg_mg_layout", "gmg_layout",
    "gmg_pack", "gmg_unpack", "gmg_set_scalars", "gmg_set_acoef", "gmg_set_bcoef_cell", "gmg_set_bcoef_face",
    "gmg_get_coeffs", "gmg_workspace_size", "gmg_set_workspace", "gmg_solve", "gmg_apply", "gmg_fill_boundary",
    "gmg_smooth", "gmg_residual", "gmg_restrict", "gmg_prolong_add", "gmg_prolong_add_trilinear",
    "gmg_bottom_solve", "gmg_vcycle",
    "gmg_box_bicgstab_noalloc", "gmg_define_batch", "gmg_num_solves", "gmg_solve_boxes", "gmg_pack_solve",
    "gmg_unpack_solve", "gmg_batch_solve", "gmg_amr_level_boxes", "gmg_pack_amr", "gmg_unpack_amr",
    "gmg_apply_transpose", "gmg_solve_adjoint", "gmg_beta_grad", "gmg_autotune", "gmg_tuned",
    "gmg_wall_values_rhs", "gmg_wall_values_grad", "gmg_beta_grad_walls", "gmg_dfma_probe",
    "gmg_partition", "gmg_ghost_rects", "gmg_exchange_plan",
]


class Params(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("max_iter", C.c_int), ("bottom_max_iter", C.c_int),
                ("bottom_tol", C.c_double), ("precision", C.c_int), ("project_mean", C.c_int),
                ("use_graph", C.c_int), ("profile", C.c_int), ("fused_coarse", C.c_int),
                ("fused_sweep", C.c_int), ("ghost_push", C.c_int),
                ("vector_smooth", C.c_int), ("pdl", C.c_int), ("fuse_residual_sweep", C.c_int),
                ("krylov", C.c_int), ("bottom_solver", C.c_int), ("post_reverse", C.c_int),
                ("fuse_correction", C.c_int), ("settled_zero", C.c_int), ("flow_warps", C.c_int),
                ("flow_lag_kcells", C.c_int), ("serpentine", C.c_int), ("prolongation", C.c_int),
                ("wave_sweep", C.c_int), ("tail_dense", C.c_int),
                ("fuse_restriction_sweep", C.c_int), ("fuse_prolongation", C.c_int),
                ("fork_bottoms", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("rhs_norm", C.c_double),
                ("initial_resid", C.c_double), ("final_resid", C.c_double), ("hist_len", C.c_int),
                ("resid_hist", C.c_double * 256), ("bottom_iters", C.c_int), ("solve_ms", C.c_double),
                ("kernel_launches", C.c_longlong), ("smooth0_ms", C.c_double), ("smooth0_launches", C.c_int),
                ("resid0_ms", C.c_double), ("resid0_launches", C.c_int), ("smooth0_passes", C.c_int)]

    def history(self):
        return [self.resid_hist[i] for i in range(self.hist_len)]


class GmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gmg status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libgmg.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libgmg.so is missing and could not be built")
        L = C.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    vp, i32p, i64p, f64p = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_double)
    sig = {
        "gmg_default_params": [C.POINTER(Params)],
        "gmg_dfma_probe": [vp, C.c_int, C.c_int, f64p],
        "gmg_prolong_add_trilinear": [vp, C.c_int, C.c_int, vp, vp],
        "gmg_partition": [vp, C.c_int, C.c_int, C.c_longlong, i32p],
        "gmg_ghost_rects": [vp, C.c_int, i32p, i32p],
        "gmg_exchange_plan": [vp, C.c_int, i32p, C.c_int, i32p, i32p, i32p, i32p],
        "gmg_create": [C.POINTER(C.c_void_p), vp],
        "gmg_destroy": [vp],
        "gmg_define_domain": [vp, i32p, i32p, f64p, f64p, i32p, i32p],
        "gmg_define_level": [vp, C.c_int, C.c_int, i32p, C.c_int],
        "gmg_chop_domain": [vp, C.c_int, C.c_int],
        "gmg_mg_nlevels": [vp, i32p],
        "gmg_mg_level_info": [vp, C.c_int, i32p, i32p],
        "gmg_mg_level_boxes": [vp, C.c_int, i32p, i32p],
        "gmg_wave_tiles": [vp, C.c_int, i32p, i32p, i32p, C.c_int],
        "gmg_tail_plan": [vp, C.c_int, C.c_int, i32p, C.POINTER(C.c_longlong)],
        "gmg_mg_layout": [vp, C.c_int, C.c_int, i64p, i64p, i32p],
        "gmg_layout": [vp, C.c_int, i64p, i64p],
        "gmg_pack": [vp, C.c_int, C.c_int, vp, vp],
        "gmg_unpack": [vp, C.c_int, C.c_int, vp, vp],
        "gmg_set_scalars": [vp, C.c_double, C.c_double],
        "gmg_set_acoef": [vp, C.c_int, vp],
        "gmg_set_bcoef_cell": [vp, C.c_int, vp],
        "gmg_set_bcoef_face": [vp, C.c_int, vp, vp, vp],
        "gmg_get_coeffs": [vp, C.c_int, C.c_int, vp, vp, vp, vp],
        "gmg_workspace_size": [vp, C.POINTER(Params), C.POINTER(C.c_size_t)],
        "gmg_set_workspace": [vp, vp, C.c_size_t],
        "gmg_solve": [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_double, C.c_double, C.POINTER(Params),
                      C.POINTER(SolveInfo)],
        "gmg_apply": [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)],
        "gmg_fill_boundary": [vp, C.c_int, C.c_int, vp, C.c_int],
        "gmg_smooth": [vp, C.c_int, C.c_int, vp, vp, C.c_int],
        "gmg_residual": [vp, C.c_int, C.c_int, vp, vp, C.c_int, vp, f64p],
        "gmg_restrict": [vp, C.c_int, C.c_int, vp, vp],
        "gmg_prolong_add": [vp, C.c_int, C.c_int, vp, vp],
        "gmg_bottom_solve": [vp, C.c_int, vp, vp, C.POINTER(Params), i32p],
        "gmg_vcycle": [vp, C.c_int, vp, vp, C.POINTER(Params)],
        "gmg_box_bicgstab_noalloc": [vp, C.c_int, C.c_int, C.c_int, i32p, i32p, C.c_int, vp, vp, vp, vp, vp, vp,
                                     C.c_int, C.c_double, vp],
        "gmg_define_batch": [vp, C.c_int, i32p, f64p, f64p, i32p, i32p, i32p, i32p],
        "gmg_num_solves": [vp, i32p],
        "gmg_solve_boxes": [vp, C.c_int, C.c_int, i32p, i32p],
        "gmg_pack_solve": [vp, C.c_int, C.c_int, C.c_int, vp, vp],
        "gmg_unpack_solve": [vp, C.c_int, C.c_int, C.c_int, vp, vp],
        "gmg_batch_solve": [vp, vp, vp, C.c_double, C.c_double, C.POINTER(Params), C.POINTER(SolveInfo)],
        "gmg_amr_level_boxes": [vp, C.c_int, i32p, i32p, i32p],
        "gmg_pack_amr": [vp, C.c_int, vp, vp],
        "gmg_unpack_amr": [vp, C.c_int, vp, vp],
        "gmg_apply_transpose": [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)],
        "gmg_solve_adjoint": [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_double, C.POINTER(Params),
                              C.POINTER(SolveInfo)],
        "gmg_beta_grad": [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)],
        "gmg_wall_values_rhs": [vp, vp, vp, C.POINTER(C.c_void_p)],
        "gmg_wall_values_grad": [vp, vp, C.POINTER(C.c_void_p)],
        "gmg_beta_grad_walls": [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                C.POINTER(C.c_void_p)],
        "gmg_autotune": [vp, C.c_int, vp, C.POINTER(Params)],
        "gmg_tuned": [vp, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                      C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.gmg_last_error.argtypes = [vp]
    L.gmg_last_error.restype = C.c_char_p


def dfma_probe(stream, blocks_per_sm=8, iters=1 << 15):
    """Enqueue the FP64 throughput probe kernel on `stream` (a cudaStream_t as int); returns
    the flops it performs (the caller times it with events on that stream)."""
    f = C.c_double()
    st = lib().gmg_dfma_probe(C.c_void_p(stream or 0), int(blocks_per_sm), int(iters), C.byref(f))
    if st != OK:
        raise GmgError(st, (lib().gmg_last_error(None) or b"").decode())
    return f.value


def default_params(**kw) -> Params:
    p = Params()
    lib().gmg_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        setattr(p, k, v)
    return p


def _arr(vals, ct):
    a = (ct * len(vals))()
    for i, v in enumerate(vals):
        a[i] = v
    return a


def _ptr(t):
    """Device pointer of a torch tensor (or None)."""
    return None if t is None else C.c_void_p(t.data_ptr())


_TORCH_DT = {}


def torch_dtype(dt):
    import torch
    return {DT_F64: torch.float64, DT_F32: torch.float32, DT_BF16: torch.bfloat16}[dt]


class Context:
    """One gmg context: a domain, its BoxArray, the multigrid hierarchy and (after
    allocate()) a torch-owned device workspace."""

    def __init__(self, domain, bc_lo, bc_hi, prob_lo=(0.0, 0.0, 0.0), prob_hi=(1.0, 1.0, 1.0), boxes=None,
                 max_grid_size=None, stream=None):
        self.L = lib()
        h = C.c_void_p()
        self._check(self.L.gmg_create(C.byref(h), C.c_void_p(stream or 0)), None)
        self.h = h
        lo, hi = domain
        self._check(self.L.gmg_define_domain(self.h, _arr(lo, C.c_int), _arr(hi, C.c_int), _arr(prob_lo, C.c_double),
                                             _arr(prob_hi, C.c_double), _arr(bc_lo, C.c_int), _arr(bc_hi, C.c_int)))
        if boxes is not None:
            flat = [v for b in boxes for v in (list(b[0]) + list(b[1]))]
            self._check(self.L.gmg_define_level(self.h, 0, len(boxes), _arr(flat, C.c_int), 1))
        else:
            self._check(self.L.gmg_chop_domain(self.h, 0, int(max_grid_size)))
        self.domain = (tuple(lo), tuple(hi))
        self.workspace = None
        self._keep = []

    def __del__(self):
        if getattr(self, "h", None):
            self.L.gmg_destroy(self.h)
            self.h = None

    def _check(self, st, h=-1):
        if st != OK:
            msg = self.L.gmg_last_error(self.h if h == -1 else h)
            raise GmgError(st, (msg or b"").decode())
        return st

    # ---- hierarchy / layout -------------------------------------------------
    @property
    def nlevels(self):
        n = C.c_int()
        self._check(self.L.gmg_mg_nlevels(self.h, C.byref(n)))
        return n.value

    def level_info(self, m):
        nb = C.c_int()
        dom = (C.c_int * 6)()
        self._check(self.L.gmg_mg_level_info(self.h, m, C.byref(nb), dom))
        return nb.value, (tuple(dom[:3]), tuple(dom[3:]))

    def level_boxes(self, m):
        nb, _ = self.level_info(m)
        lohi = (C.c_int * (6 * nb))()
        par = (C.c_int * nb)()
        self._check(self.L.gmg_mg_level_boxes(self.h, m, lohi, par))
        boxes = [(tuple(lohi[6 * b:6 * b + 3]), tuple(lohi[6 * b + 3:6 * b + 6])) for b in range(nb)]
        return boxes, list(par)

    def wave_tiles(self, m):
        """(cell pairs per thread, int array (ntiles, 13)) of the wavefront sweep on level m:
        box, y0, y1, direction, tiles across x-, x+, y-, y+, z-, z+, the two z waits, problem."""
        n, ppt = C.c_int(), C.c_int()
        self._check(self.L.gmg_wave_tiles(self.h, m, C.byref(n), C.byref(ppt), None, 0))
        out = (C.c_int * max(1, 13 * n.value))()
        self._check(self.L.gmg_wave_tiles(self.h, m, None, None, out, n.value))
        return ppt.value, np.array(out[:13 * n.value], dtype=np.int64).reshape(n.value, 13)

    def tail_plan(self, m, dt=DT_F64):
        """(blocks, dense shared-memory bytes) of the coarse ends starting on level m (fused
        coarse end; bytes 0: the global-memory form)."""
        n, b = C.c_int(), C.c_longlong()
        self._check(self.L.gmg_tail_plan(self.h, m, dt, C.byref(n), C.byref(b)))
        return n.value, b.value

    def layout(self, m, dt=DT_F64):
        nb, _ = self.level_info(m)
        ne = C.c_int64()
        offs = (C.c_int64 * nb)()
        sx = (C.c_int * nb)()
        self._check(self.L.gmg_mg_layout(self.h, m, dt, C.byref(ne), offs, sx))
        return ne.value, list(offs), list(sx)

    def level_shape(self, m):
        _, (lo, hi) = self.level_info(m)
        return (hi[2] - lo[2] + 1, hi[1] - lo[1] + 1, hi[0] - lo[0] + 1)

    # ---- workspace ------------------------------------------------------------
    def workspace_bytes(self, precision=FP64, krylov=False):
        n = C.c_size_t()
        p = default_params(precision=precision, krylov=int(bool(krylov)))
        self._check(self.L.gmg_workspace_size(self.h, C.byref(p), C.byref(n)))
        return n.value

    def allocate(self, precision=FP64, device="cuda", krylov=False):
        """Workspace for solves in `precision` (mixed sizes also serve FP64); krylov=True adds
        the top-level Krylov vectors (params krylov = 1 or 2)."""
        import torch
        nbytes = self.workspace_bytes(precision, krylov)
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = ws.data_ptr()
        off = (-base) % 256
        self._check(self.L.gmg_set_workspace(self.h, C.c_void_p(base + off), C.c_size_t(nbytes)))
        self.workspace = ws
        return self

    def field(self, m=0, dt=DT_F64, device="cuda"):
        import torch
        ne, _, _ = self.layout(m, dt)
        return torch.zeros(ne, dtype=torch_dtype(dt), device=device)

    def box_views(self, buf, m=0):
        """Ghosted (nz+2, ny+2, nx+2) views of every box of a boxed-layout tensor."""
        boxes, _ = self.level_boxes(m)
        _, offs, sxs = self.layout(m)
        out = []
        for (lo, hi), off, sx in zip(boxes, offs, sxs):
            n = [hi[d] - lo[d] + 1 for d in range(3)]
            blk = buf[off:off + sx * (n[1] + 2) * (n[2] + 2)].view(n[2] + 2, n[1] + 2, sx)
            out.append(blk[:, :, GX - 1:GX + n[0] + 1])
        return out

    # ---- sharding plan (host tables; the solves run on one GPU) ---------------------
    def partition(self, m, nranks, min_cells_per_rank=0):
        """owner rank of every box of MG level m (Morton curve cut by cell counts)"""
        nb, _ = self.level_info(m)
        own = (C.c_int * nb)()
        self._check(self.L.gmg_partition(self.h, m, nranks, int(min_cells_per_rank), own))
        return list(own)

    def ghost_rects(self, m):
        """face-ghost rectangles of MG level m: list of dicts (see gmg_ghost_rects)"""
        n = C.c_int()
        self._check(self.L.gmg_ghost_rects(self.h, m, C.byref(n), None))
        raw = (C.c_int * (14 * n.value))()
        self._check(self.L.gmg_ghost_rects(self.h, m, C.byref(n), raw))
        keys = ("dst_box", "src_box", "dst", "src", "d1", "d2", "n1", "n2", "sign", "kind")
        out = []
        for r in range(n.value):
            v = raw[14 * r:14 * r + 14]
            out.append(dict(zip(keys, (v[0], v[1], tuple(v[2:5]), tuple(v[5:8]), v[8], v[9], v[10], v[11], v[12],
                                       v[13]))))
        return out

    def exchange_plan(self, m, owner, rank):
        """(send, recv): lists of (peer, rectangle index) for this rank under owner[]"""
        own = (C.c_int * len(owner))(*owner)
        ns, nr = C.c_int(), C.c_int()
        self._check(self.L.gmg_exchange_plan(self.h, m, own, rank, C.byref(ns), None, C.byref(nr), None))
        s, r = (C.c_int * (2 * ns.value))(), (C.c_int * (2 * nr.value))()
        self._check(self.L.gmg_exchange_plan(self.h, m, own, rank, C.byref(ns), s, C.byref(nr), r))
        return ([(s[2 * i], s[2 * i + 1]) for i in range(ns.value)], [(r[2 * i], r[2 * i + 1]) for i in range(nr.value)])

    # ---- dense <-> boxed --------------------------------------------------------
    def pack(self, dense, m=0, dt=DT_F64, out=None):
        import torch
        dense = torch.as_tensor(dense, dtype=torch.float64, device="cuda").contiguous()
        assert tuple(dense.shape) == self.level_shape(m), (dense.shape, self.level_shape(m))
        out = self.field(m, dt) if out is None else out
        self._check(self.L.gmg_pack(self.h, m, dt, _ptr(dense), _ptr(out)))
        self._keep = [dense]
        return out

    def unpack(self, boxed, m=0, dt=DT_F64):
        import torch
        out = torch.zeros(self.level_shape(m), dtype=torch.float64, device=boxed.device)
        self._check(self.L.gmg_unpack(self.h, m, dt, _ptr(boxed), _ptr(out)))
        return out

    # ---- coefficients -------------------------------------------------------------
    def set_scalars(self, a, b):
        self._check(self.L.gmg_set_scalars(self.h, float(a), float(b)))

    def set_alpha(self, alpha_dense):
        buf = self.pack(alpha_dense)
        self._check(self.L.gmg_set_acoef(self.h, 0, _ptr(buf)))

    def set_beta(self, beta_dense=None):
        import torch
        if beta_dense is None:
            beta_dense = torch.ones(self.level_shape(0), dtype=torch.float64)
        buf = self.pack(beta_dense)
        self._check(self.L.gmg_set_bcoef_cell(self.h, 0, _ptr(buf)))

    def set_beta_faces(self, bx, by, bz):
        self._check(self.L.gmg_set_bcoef_face(self.h, 0, _ptr(bx), _ptr(by), _ptr(bz)))

    def coeffs(self, m, dt=DT_F64):
        wx, wy, wz, d = (self.field(m, dt) for _ in range(4))
        self._check(self.L.gmg_get_coeffs(self.h, m, dt, _ptr(wx), _ptr(wy), _ptr(wz), _ptr(d)))
        return wx, wy, wz, d

    # ---- solve ------------------------------------------------------------------------
    def solve(self, rhs, phi=None, tol_rel=1e-10, tol_abs=0.0, raise_on_error=True, wall_values=None, **params):
        """rhs, phi: FP64 boxed-layout tensors of level 0.  wall_values: nonzero wall values
        (see wall_values_rhs), folded into a copy of rhs first (one buffer per context, so
        repeated solves reuse one captured graph).  Returns (phi, info)."""
        if wall_values is not None:
            if getattr(self, "_wall_rhs", None) is None:
                self._wall_rhs = self.field(0)
            rhs = self.wall_values_rhs(rhs, wall_values, out=self._wall_rhs)
        phi = self.field(0) if phi is None else phi
        p = default_params(**params)
        info = SolveInfo()
        pa = (C.c_void_p * 1)(phi.data_ptr())
        ra = (C.c_void_p * 1)(rhs.data_ptr())
        st = self.L.gmg_solve(self.h, pa, ra, tol_rel, tol_abs, C.byref(p), C.byref(info))
        if st not in (OK, NOT_CONVERGED) and raise_on_error:
            self._check(st)
        return phi, info

    def apply(self, phi, out=None, transpose=False):
        """A phi with homogeneous walls, or A^T phi (transpose; phi's ghosts are overwritten)."""
        out = self.field(0) if out is None else out
        pa = (C.c_void_p * 1)(phi.data_ptr())
        oa = (C.c_void_p * 1)(out.data_ptr())
        fn = self.L.gmg_apply_transpose if transpose else self.L.gmg_apply
        self._check(fn(self.h, oa, pa))
        return out

    def solve_adjoint(self, g, tol_rel=1e-10, **params):
        lam = self.field(0)
        p = default_params(**params)
        info = SolveInfo()
        st = self.L.gmg_solve_adjoint(self.h, _pp(lam), _pp(g), tol_rel, C.byref(p), C.byref(info))
        if st not in (OK, NOT_CONVERGED):
            self._check(st)
        return lam, info

    def beta_grad(self, phi, lam, wall_values=None):
        d = self.field(0)
        if wall_values is None:
            self._check(self.L.gmg_beta_grad(self.h, _pp(d), _pp(phi), _pp(lam)))
        else:
            arr, keep = self._wall_ptrs(wall_values)
            self._check(self.L.gmg_beta_grad_walls(self.h, _pp(d), _pp(phi), _pp(lam), arr))
        return d

    # ---- wall values ----------------------------------------------------------------
    def face_shape(self, face):
        """Shape (n_t2, n_t1) of face `face` (= 2*d + side)'s value array: its tangential axes
        in increasing order, the lower one fastest."""
        d = face // 2
        t1, t2 = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
        lo, hi = self.domain
        return (hi[t2] - lo[t2] + 1, hi[t1] - lo[t1] + 1)

    def _wall_ptrs(self, values):
        """values: dict face -> array, or a sequence of 6 (None: g = 0).  Returns the pointer
        array and the FP64 device tensors it points into."""
        import torch
        arr = (C.c_void_p * 6)()
        keep = []
        for f in range(6):
            v = values.get(f) if isinstance(values, dict) else values[f]
            if v is None:
                continue
            t = torch.as_tensor(v, dtype=torch.float64, device="cuda").contiguous()
            if tuple(t.shape) != self.face_shape(f):
                raise ValueError(f"face {f}: values of shape {tuple(t.shape)}, expected {self.face_shape(f)}")
            arr[f] = t.data_ptr()
            keep.append(t)
        return arr, keep

    def wall_values_rhs(self, rhs, values, out=None):
        """rhs - A_g(0): rhs with the flux the wall values drive into the wall cells."""
        out = self.field(0) if out is None else out
        arr, keep = self._wall_ptrs(values)
        self._check(self.L.gmg_wall_values_rhs(self.h, _ptr(out), _ptr(rhs), arr))
        return out

    def wall_values_grad(self, lam, faces):
        """dL/dg on the given faces for the adjoint lam: {face: (n_t2, n_t1) tensor}."""
        import torch
        arr = (C.c_void_p * 6)()
        out = {}
        for f in faces:
            out[f] = torch.zeros(self.face_shape(f), dtype=torch.float64, device="cuda")
            arr[f] = out[f].data_ptr()
        self._check(self.L.gmg_wall_values_grad(self.h, _ptr(lam), arr))
        return out

    # ---- individual steps ----------------------------------------------------------------
    def fill_boundary(self, f, m=0, dt=DT_F64, colour=-1):
        self._check(self.L.gmg_fill_boundary(self.h, m, dt, _ptr(f), colour))

    def smooth(self, phi, rhs, m=0, dt=DT_F64, colour=0):
        self._check(self.L.gmg_smooth(self.h, m, dt, _ptr(phi), _ptr(rhs), colour))

    def residual(self, phi, rhs, m=0, dt=DT_F64, rdt=None, norm=False):
        rdt = dt if rdt is None else rdt
        r = self.field(m, rdt)
        nv = C.c_double()
        self._check(self.L.gmg_residual(self.h, m, dt, _ptr(phi), _ptr(rhs), rdt, _ptr(r),
                                        C.byref(nv) if norm else None))
        return (r, nv.value) if norm else r

    def restrict(self, fine, m=0, dt=DT_F64):
        c = self.field(m + 1, dt)
        self._check(self.L.gmg_restrict(self.h, m, dt, _ptr(fine), _ptr(c)))
        return c

    def prolong_add(self, coarse, fine, m=0, dt=DT_F64):
        self._check(self.L.gmg_prolong_add(self.h, m, dt, _ptr(coarse), _ptr(fine)))

    def bottom_solve(self, rhs, dt=DT_F64, **params):
        x = self.field(self.nlevels - 1, dt)
        p = default_params(**params)
        it = C.c_int()
        self._check(self.L.gmg_bottom_solve(self.h, dt, _ptr(rhs), _ptr(x), C.byref(p), C.byref(it)))
        return x, it.value

    def autotune(self, rhs, precision=FP64, **params):
        """Time the sweep variants per level (ghost push / exchange, 2- / 4-cell threads) and
        the fused coarse end (gmg_autotune) for this precision; later solves with the default
        params use the fastest.  Returns {"levels": [(variant bits, best ms with push, best ms
        with exchange), ...], "fused_coarse": f, "vcycle_ms": (fused, per-level)}."""
        if isinstance(precision, str):
            precision = PRECISION[precision]
        p = default_params(**params)
        self._check(self.L.gmg_autotune(self.h, precision, _ptr(rhs), C.byref(p)))
        out = []
        f = C.c_int()
        vf, vl = C.c_double(), C.c_double()
        for m in range(self.nlevels):
            ps = C.c_int()
            a, b = C.c_double(), C.c_double()
            self._check(self.L.gmg_tuned(self.h, precision, m, C.byref(ps), C.byref(a), C.byref(b), C.byref(f),
                                         C.byref(vf), C.byref(vl)))
            out.append((ps.value, a.value, b.value))
        return {"levels": out, "fused_coarse": f.value, "vcycle_ms": (vf.value, vl.value)}

    def vcycle(self, r, dt=DT_F64, **params):
        e = self.field(0, dt)
        p = default_params(**params)
        self._check(self.L.gmg_vcycle(self.h, dt, _ptr(e), _ptr(r), C.byref(p)))
        return e


def _pp(*tensors):
    """array of device pointers (level 0, level 1, ...)"""
    return (C.c_void_p * len(tensors))(*[t.data_ptr() for t in tensors])


class AmrContext(Context):
    """Two-level composite problem: level 0 covers the domain, level 1 (ratio 2) covers the
    fine boxes.  Dense fine arrays span the bounding box of the fine boxes."""

    def __init__(self, domain, coarse_boxes, fine_boxes, bc_lo, bc_hi, prob_lo=(0.0, 0.0, 0.0),
                 prob_hi=(1.0, 1.0, 1.0), stream=None):
        super().__init__(domain, bc_lo, bc_hi, prob_lo, prob_hi, boxes=coarse_boxes, stream=stream)
        flat = [v for b in fine_boxes for v in (list(b[0]) + list(b[1]))]
        self._check(self.L.gmg_define_level(self.h, 1, len(fine_boxes), _arr(flat, C.c_int), 2))
        self.fine_boxes = list(fine_boxes)
        lo = [min(b[0][d] for b in fine_boxes) for d in range(3)]
        hi = [max(b[1][d] for b in fine_boxes) for d in range(3)]
        self.fine_lo = tuple(lo)
        self.fine_shape = tuple(hi[d] - lo[d] + 1 for d in (2, 1, 0))
        self.coarse_shape = self.level_shape(0)
        import numpy as np
        cov = np.zeros(self.coarse_shape, dtype=bool)
        for b in fine_boxes:
            cov[b[0][2] // 2:(b[1][2] + 1) // 2, b[0][1] // 2:(b[1][1] + 1) // 2, b[0][0] // 2:(b[1][0] + 1) // 2] = True
        self.covered = cov

    def nelem(self, lev):
        ne = C.c_int64()
        self._check(self.L.gmg_layout(self.h, lev, C.byref(ne), None))
        return ne.value

    def level_field(self, lev):
        import torch
        return torch.zeros(self.nelem(lev), dtype=torch.float64, device="cuda")

    def pack_level(self, lev, dense, out=None):
        import torch
        dense = torch.as_tensor(dense, dtype=torch.float64, device="cuda").contiguous()
        out = self.level_field(lev) if out is None else out
        self._check(self.L.gmg_pack_amr(self.h, lev, _ptr(dense), _ptr(out)))
        self._keep.append(dense)
        return out

    def unpack_level(self, lev, boxed):
        import torch
        shape = self.coarse_shape if lev == 0 else self.fine_shape
        out = torch.zeros(shape, dtype=torch.float64, device=boxed.device)
        self._check(self.L.gmg_unpack_amr(self.h, lev, _ptr(boxed), _ptr(out)))
        return out

    def set_coeffs(self, a=0.0, b=1.0, alpha_c=None, beta_c=None, alpha_f=None, beta_f=None):
        import torch
        self._keep = []
        self.set_scalars(a, b)
        if alpha_c is not None:
            self._check(self.L.gmg_set_acoef(self.h, 0, _ptr(self.pack_level(0, alpha_c))))
        if alpha_f is not None:
            self._check(self.L.gmg_set_acoef(self.h, 1, _ptr(self.pack_level(1, alpha_f))))
        if beta_c is None:
            beta_c = torch.ones(self.coarse_shape, dtype=torch.float64)
        if beta_f is None:
            beta_f = torch.ones(self.fine_shape, dtype=torch.float64)
        self._check(self.L.gmg_set_bcoef_cell(self.h, 0, _ptr(self.pack_level(0, beta_c))))
        self._check(self.L.gmg_set_bcoef_cell(self.h, 1, _ptr(self.pack_level(1, beta_f))))

    def solve2(self, rhs_c, rhs_f, tol_rel=1e-10, tol_abs=0.0, **params):
        pc, pf = self.level_field(0), self.level_field(1)
        p = default_params(**params)
        info = SolveInfo()
        st = self.L.gmg_solve(self.h, _pp(pc, pf), _pp(rhs_c, rhs_f), tol_rel, tol_abs, C.byref(p), C.byref(info))
        if st not in (OK, NOT_CONVERGED):
            self._check(st)
        return pc, pf, info

    def apply2(self, xc, xf, transpose=False):
        oc, of = self.level_field(0), self.level_field(1)
        fn = self.L.gmg_apply_transpose if transpose else self.L.gmg_apply
        self._check(fn(self.h, _pp(oc, of), _pp(xc, xf)))
        return oc, of

    def solve_adjoint2(self, gc, gf, tol_rel=1e-10, **params):
        lc, lf = self.level_field(0), self.level_field(1)
        p = default_params(**params)
        info = SolveInfo()
        st = self.L.gmg_solve_adjoint(self.h, _pp(lc, lf), _pp(gc, gf), tol_rel, C.byref(p), C.byref(info))
        if st not in (OK, NOT_CONVERGED):
            self._check(st)
        return lc, lf, info

    def beta_grad2(self, pc, pf, lc, lf):
        dc, df = self.level_field(0), self.level_field(1)
        self._check(self.L.gmg_beta_grad(self.h, _pp(dc, df), _pp(pc, pf), _pp(lc, lf)))
        return dc, df


def covered_masks(level_boxes, level_lo, level_shape):
    """Per AMR level, the cells of its dense array (shape level_shape[l], low corner
    level_lo[l] in level l's index space) under a box of level l + 1 (ratio 2)."""
    out = []
    for lev, shape in enumerate(level_shape):
        cov = np.zeros(shape, dtype=bool)
        if lev + 1 < len(level_shape):
            o = level_lo[lev]
            for blo, bhi in level_boxes[lev + 1]:
                cov[tuple(slice(blo[d] // 2 - o[d], (bhi[d] + 1) // 2 - o[d]) for d in (2, 1, 0))] = True
        out.append(cov)
    return out


class MultiLevelContext(Context):
    """Composite problem over several AMR levels: level 0 covers the domain, level l
    (ratio 2 to level l - 1) is a BoxArray in level l's index space, properly nested.  Dense
    arrays of level l >= 1 span the bounding box of its boxes.  Forward solve and operator,
    transpose, adjoint solve and beta gradient (these three need every level at least two
    cells inside the coarse/fine boundary of the level it refines)."""

    def __init__(self, domain, level_boxes, bc_lo, bc_hi, prob_lo=(0.0, 0.0, 0.0), prob_hi=(1.0, 1.0, 1.0),
                 stream=None):
        super().__init__(domain, bc_lo, bc_hi, prob_lo, prob_hi, boxes=level_boxes[0], stream=stream)
        self.nlev_amr = len(level_boxes)
        self.level_boxes = [list(b) for b in level_boxes]
        self.level_lo, self.level_shape_ = [(0, 0, 0)], [self.level_shape(0)]
        for lev in range(1, self.nlev_amr):
            boxes = level_boxes[lev]
            flat = [v for b in boxes for v in (list(b[0]) + list(b[1]))]
            self._check(self.L.gmg_define_level(self.h, lev, len(boxes), _arr(flat, C.c_int), 2))
            lo = [min(b[0][d] for b in boxes) for d in range(3)]
            hi = [max(b[1][d] for b in boxes) for d in range(3)]
            self.level_lo.append(tuple(lo))
            self.level_shape_.append(tuple(hi[d] - lo[d] + 1 for d in (2, 1, 0)))
        self.covered = covered_masks(level_boxes, self.level_lo, self.level_shape_)

    def nelem(self, lev):
        ne = C.c_int64()
        self._check(self.L.gmg_layout(self.h, lev, C.byref(ne), None))
        return ne.value

    def level_field(self, lev):
        import torch
        return torch.zeros(self.nelem(lev), dtype=torch.float64, device="cuda")

    def pack_level(self, lev, dense, out=None):
        import torch
        dense = torch.as_tensor(dense, dtype=torch.float64, device="cuda").contiguous()
        out = self.level_field(lev) if out is None else out
        self._check(self.L.gmg_pack_amr(self.h, lev, _ptr(dense), _ptr(out)))
        self._keep.append(dense)
        return out

    def unpack_level(self, lev, boxed):
        import torch
        out = torch.zeros(self.level_shape_[lev], dtype=torch.float64, device=boxed.device)
        self._check(self.L.gmg_unpack_amr(self.h, lev, _ptr(boxed), _ptr(out)))
        return out

    def set_coeffs(self, a=0.0, b=1.0, alphas=None, betas=None):
        """alphas / betas: per-level dense arrays (level 0 over the domain, level l over its
        bounding box) or None (1)."""
        import torch
        self._keep = []
        self.set_scalars(a, b)
        for lev in range(self.nlev_amr):
            if alphas is not None:
                self._check(self.L.gmg_set_acoef(self.h, lev, _ptr(self.pack_level(lev, alphas[lev]))))
        for lev in range(self.nlev_amr):
            beta = betas[lev] if betas is not None else torch.ones(self.level_shape_[lev], dtype=torch.float64)
            self._check(self.L.gmg_set_bcoef_cell(self.h, lev, _ptr(self.pack_level(lev, beta))))

    def solve_levels(self, rhss, tol_rel=1e-10, tol_abs=0.0, **params):
        """rhss: boxed FP64 right-hand sides per level.  Returns (phis, info)."""
        phis = [self.level_field(lev) for lev in range(self.nlev_amr)]
        p = default_params(**params)
        info = SolveInfo()
        st = self.L.gmg_solve(self.h, _pp(*phis), _pp(*rhss), tol_rel, tol_abs, C.byref(p), C.byref(info))
        if st not in (OK, NOT_CONVERGED):
            self._check(st)
        return phis, info

    def apply_levels(self, xs, transpose=False):
        """A x, or A^T x (transpose: x's ghosts are overwritten, its covered entries cleared)."""
        outs = [self.level_field(lev) for lev in range(self.nlev_amr)]
        fn = self.L.gmg_apply_transpose if transpose else self.L.gmg_apply
        self._check(fn(self.h, _pp(*outs), _pp(*xs)))
        return outs

    def solve_adjoint_levels(self, gs, tol_rel=1e-10, **params):
        """A^T lambda = g over every level.  Returns (lambdas, info)."""
        lams = [self.level_field(lev) for lev in range(self.nlev_amr)]
        p = default_params(**params)
        info = SolveInfo()
        st = self.L.gmg_solve_adjoint(self.h, _pp(*lams), _pp(*gs), tol_rel, C.byref(p), C.byref(info))
        if st not in (OK, NOT_CONVERGED):
            self._check(st)
        return lams, info

    def beta_grad_levels(self, phis, lams):
        """dL/dbeta per level (boxed) for L = lambda^T (rhs - A(beta) phi); the ghosts of phi
        and lambda are overwritten."""
        outs = [self.level_field(lev) for lev in range(self.nlev_amr)]
        self._check(self.L.gmg_beta_grad(self.h, _pp(*outs), _pp(*phis), _pp(*lams)))
        return outs


class BatchContext(Context):
    """Several independent problems solved together (one launch per step covers them all).

    problems: list of dicts with keys domain ((lo), (hi)), boxes [(lo, hi), ...], bc_lo, bc_hi
    and optional prob_lo / prob_hi."""

    def __init__(self, problems, stream=None):
        self.L = lib()
        h = C.c_void_p()
        self._check(self.L.gmg_create(C.byref(h), C.c_void_p(stream or 0)), None)
        self.h = h
        n = len(problems)
        dom, plo, phi, bl, bh, nb, bx = [], [], [], [], [], [], []
        for p in problems:
            dom += list(p["domain"][0]) + list(p["domain"][1])
            plo += list(p.get("prob_lo", (0.0, 0.0, 0.0)))
            phi += list(p.get("prob_hi", (1.0, 1.0, 1.0)))
            bl += list(p["bc_lo"])
            bh += list(p["bc_hi"])
            nb.append(len(p["boxes"]))
            for b in p["boxes"]:
                bx += list(b[0]) + list(b[1])
        self._check(self.L.gmg_define_batch(self.h, n, _arr(dom, C.c_int), _arr(plo, C.c_double),
                                            _arr(phi, C.c_double), _arr(bl, C.c_int), _arr(bh, C.c_int),
                                            _arr(nb, C.c_int), _arr(bx, C.c_int)))
        self.problems = problems
        self.nsolves = n
        self.workspace = None
        self._keep = []

    def solve_shape(self, s, m=0):
        lo, hi = self.problems[s]["domain"]
        f = 2 ** m
        return tuple((hi[d] - lo[d] + 1) // f for d in (2, 1, 0))

    def pack_solve(self, s, dense, out, m=0, dt=DT_F64):
        import torch
        dense = torch.as_tensor(dense, dtype=torch.float64, device="cuda").contiguous()
        self._check(self.L.gmg_pack_solve(self.h, m, dt, s, _ptr(dense), _ptr(out)))
        self._keep.append(dense)
        return out

    def unpack_solve(self, s, boxed, m=0, dt=DT_F64):
        import torch
        out = torch.zeros(self.solve_shape(s, m), dtype=torch.float64, device=boxed.device)
        self._check(self.L.gmg_unpack_solve(self.h, m, dt, s, _ptr(boxed), _ptr(out)))
        return out

    def pack_all(self, dense_list, m=0, dt=DT_F64):
        out = self.field(m, dt)
        self._keep = []
        for s, d in enumerate(dense_list):
            self.pack_solve(s, d, out, m, dt)
        return out

    def set_beta_all(self, betas):
        buf = self.pack_all(betas)
        self._check(self.L.gmg_set_bcoef_cell(self.h, 0, _ptr(buf)))

    def batch_solve(self, rhs, phi=None, tol_rel=1e-10, tol_abs=0.0, **params):
        phi = self.field(0) if phi is None else phi
        p = default_params(**params)
        infos = (SolveInfo * self.nsolves)()
        st = self.L.gmg_batch_solve(self.h, _ptr(phi), _ptr(rhs), tol_rel, tol_abs, C.byref(p), infos)
        if st not in (OK, NOT_CONVERGED):
            self._check(st)
        return phi, list(infos)


class Poisson:
    """Convenience front end for dense problems: a*alpha*phi - b*div(beta grad phi) = rhs
    on an (nz, ny, nx) grid chopped into boxes of at most max_grid_size cells."""

    def __init__(self, shape_xyz, bc="dirichlet", max_grid_size=64, boxes=None, prob_hi=None, precision="fp64",
                 a=0.0, b=1.0, alpha=None, beta=None):
        import torch
        nx, ny, nz = shape_xyz
        bcv = PERIODIC if bc == "periodic" else DIRICHLET0
        self.ctx = Context(((0, 0, 0), (nx - 1, ny - 1, nz - 1)), [bcv] * 3, [bcv] * 3,
                           prob_hi=prob_hi or (1.0, 1.0, 1.0), boxes=boxes, max_grid_size=max_grid_size,
                           stream=torch.cuda.current_stream().cuda_stream)
        self.precision = PRECISION[precision] if isinstance(precision, str) else precision
        self.ctx.allocate(self.precision)
        self.ctx.set_scalars(a, b)
        if alpha is not None:
            self.ctx.set_alpha(alpha)
        self.ctx.set_beta(beta)

    def solve(self, rhs_dense, tol_rel=1e-10, **params):
        rhs = self.ctx.pack(rhs_dense)
        params.setdefault("precision", self.precision)
        phi, info = self.ctx.solve(rhs, tol_rel=tol_rel, **params)
        return self.ctx.unpack(phi), info
