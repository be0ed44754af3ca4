"""Differentiable solves: torch.autograd.Function wrappers of the library's solve.

Forward:  phi = A(beta)^-1 rhs by the multigrid solve (one level, or the composite form
          over two or more AMR levels of Sec. "Operations between levels").
Backward: lambda = A^-T dL/dphi by the adjoint solve (gmg_solve_adjoint), then
          dL/drhs = lambda and dL/dbeta = -lambda^T (dA/dbeta) phi by the face-flux gradient
          kernel (gmg_beta_grad), through the harmonic face mean to the cell beta; with
          wall values g (one level), dL/dg = lambda^T d(rhs - A_g 0)/dg (gmg_wall_values_grad).
Both run in the library's kernels; this module only marshals tensors.

Singular problems (no Dirichlet wall, a = 0): the forward projects rhs onto the operator's range
and returns phi with zero (volume-weighted) mean; the backward projects accordingly, so the
gradients are those of that projected map.  Several levels: phi on cells under a finer
level is returned as 0 (those cells are not unknowns of the composite problem), and the
rhs and beta of those cells do not influence phi (their gradients are 0).
"""
from __future__ import annotations

import torch

from . import gmg


class _AmrSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, rhs_c, rhs_f, beta_c, beta_f):
        C = solver.ctx
        C.set_coeffs(solver.a, solver.b, beta_c=beta_c.detach(), beta_f=beta_f.detach())
        rc = C.pack_level(0, rhs_c.detach())
        rf = C.pack_level(1, rhs_f.detach())
        pc, pf, info = C.solve2(rc, rf, tol_rel=solver.tol, max_iter=solver.max_iter, project_mean=1)
        if info.status != gmg.OK:
            raise gmg.GmgError(info.status, "forward solve did not converge")
        ctx.solver = solver
        ctx.state = (pc, pf)
        mask = torch.as_tensor(~C.covered, device=rhs_c.device, dtype=torch.float64)
        ctx.mask = mask
        solver.last_info = info
        return C.unpack_level(0, pc) * mask, C.unpack_level(1, pf)

    @staticmethod
    def backward(ctx, g_c, g_f):
        solver = ctx.solver
        C = solver.ctx
        pc, pf = ctx.state
        gc = C.pack_level(0, (g_c * ctx.mask).contiguous())
        gf = C.pack_level(1, g_f.contiguous())
        lc, lf, info = C.solve_adjoint2(gc, gf, tol_rel=solver.tol, max_iter=solver.max_iter)
        if info.status != gmg.OK:
            raise gmg.GmgError(info.status, "adjoint solve did not converge")
        solver.last_adjoint_info = info
        dc, df = C.beta_grad2(pc, pf, lc, lf)
        lam_c = C.unpack_level(0, lc) * ctx.mask
        lam_f = C.unpack_level(1, lf)
        return None, lam_c, lam_f, C.unpack_level(0, dc), C.unpack_level(1, df)


class AmrSolve:
    """phi_c, phi_f = AmrSolve(...)(rhs_c, rhs_f, beta_c, beta_f), differentiable in rhs and
    beta.  Dense float64 CUDA tensors: coarse over the level-0 domain (nz, ny, nx), fine over
    the bounding box of the fine boxes."""

    def __init__(self, domain, coarse_boxes, fine_boxes, bc_lo, bc_hi, prob_lo=(0.0, 0.0, 0.0),
                 prob_hi=(1.0, 1.0, 1.0), a=0.0, b=1.0, tol=1e-10, max_iter=100):
        self.ctx = gmg.AmrContext(domain, coarse_boxes, fine_boxes, bc_lo, bc_hi, prob_lo, prob_hi,
                                  stream=torch.cuda.current_stream().cuda_stream)
        self.ctx.allocate(gmg.FP64)
        self.a, self.b, self.tol, self.max_iter = a, b, tol, max_iter

    def __call__(self, rhs_c, rhs_f, beta_c, beta_f):
        return _AmrSolve.apply(self, rhs_c, rhs_f, beta_c, beta_f)


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, rhs, beta, *walls):
        C = solver.ctx
        C.set_beta(beta.detach())
        wv = None if all(w is None for w in walls) else [None if w is None else w.detach() for w in walls]
        phi, info = C.solve(C.pack(rhs.detach()), tol_rel=solver.tol, max_iter=solver.max_iter, project_mean=1,
                            wall_values=wv)
        if info.status != gmg.OK:
            raise gmg.GmgError(info.status, "forward solve did not converge")
        ctx.solver = solver
        ctx.phi = phi
        ctx.wv = wv
        return C.unpack(phi)

    @staticmethod
    def backward(ctx, g):
        solver = ctx.solver
        C = solver.ctx
        lam, info = C.solve_adjoint(C.pack(g.contiguous()), tol_rel=solver.tol, max_iter=solver.max_iter)
        if info.status != gmg.OK:
            raise gmg.GmgError(info.status, "adjoint solve did not converge")
        d = C.beta_grad(ctx.phi, lam, wall_values=ctx.wv)
        dwalls = [None] * 6
        if ctx.wv is not None:
            faces = [f for f in range(6) if ctx.wv[f] is not None and ctx.needs_input_grad[3 + f]]
            if faces:
                got = C.wall_values_grad(lam, faces)
                for f in faces:
                    dwalls[f] = got[f]
        return (None, C.unpack(lam), C.unpack(d), *dwalls)


_BC = {"periodic": gmg.PERIODIC, "dirichlet": gmg.DIRICHLET, "neumann": gmg.NEUMANN,
       "dirichlet_quad": gmg.DIRICHLET_QUAD}


class Solve:
    """phi = Solve(...)(rhs, beta, wall_values) on one level, differentiable in rhs, beta and
    the wall values.  bc: "periodic", "dirichlet", "neumann" or "dirichlet_quad" (the quadratic
    wall rule) on every side, or a pair of
    per-axis lists (bc_lo, bc_hi) of those names or codes.  wall_values: None, or a dict
    face -> (n_t2, n_t1) tensor (face = 2*d + side; see gmg.Context.face_shape)."""

    def __init__(self, shape_xyz, bc="dirichlet", max_grid_size=64, prob_hi=(1.0, 1.0, 1.0), a=0.0, b=1.0,
                 tol=1e-10, max_iter=100):
        nx, ny, nz = shape_xyz
        if isinstance(bc, str):
            lo = hi = [_BC[bc]] * 3
        else:
            lo, hi = ([_BC[v] if isinstance(v, str) else int(v) for v in side] for side in bc)
        self.ctx = gmg.Context(((0, 0, 0), (nx - 1, ny - 1, nz - 1)), lo, hi, prob_hi=prob_hi,
                               max_grid_size=max_grid_size, stream=torch.cuda.current_stream().cuda_stream)
        self.ctx.allocate(gmg.FP64)
        self.ctx.set_scalars(a, b)
        self.tol, self.max_iter = tol, max_iter

    def __call__(self, rhs, beta, wall_values=None):
        walls = [None] * 6
        if wall_values is not None:
            for f, v in wall_values.items():
                walls[f] = v
        return _Solve.apply(self, rhs, beta, *walls)


class _MultiLevelSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, solver, *args):
        C = solver.ctx
        L = C.nlev_amr
        rhss, betas = args[:L], args[L:]
        C.set_coeffs(solver.a, solver.b, betas=[b.detach() for b in betas])
        rs = [C.pack_level(lev, r.detach()) for lev, r in enumerate(rhss)]
        phis, info = C.solve_levels(rs, tol_rel=solver.tol, max_iter=solver.max_iter, project_mean=1)
        if info.status != gmg.OK:
            raise gmg.GmgError(info.status, "forward solve did not converge")
        masks = [torch.as_tensor(~cov, device=rhss[0].device, dtype=torch.float64) for cov in C.covered]
        ctx.solver, ctx.state, ctx.masks = solver, phis, masks
        solver.last_info = info
        return tuple(C.unpack_level(lev, p) * m for lev, (p, m) in enumerate(zip(phis, masks)))

    @staticmethod
    def backward(ctx, *gs):
        solver = ctx.solver
        C = solver.ctx
        g = [C.pack_level(lev, (x * m).contiguous()) for lev, (x, m) in enumerate(zip(gs, ctx.masks))]
        lams, info = C.solve_adjoint_levels(g, tol_rel=solver.tol, max_iter=solver.max_iter)
        if info.status != gmg.OK:
            raise gmg.GmgError(info.status, "adjoint solve did not converge")
        solver.last_adjoint_info = info
        ds = C.beta_grad_levels(ctx.state, lams)
        dr = [C.unpack_level(lev, lam) * m for lev, (lam, m) in enumerate(zip(lams, ctx.masks))]
        return (None, *dr, *[C.unpack_level(lev, d) for lev, d in enumerate(ds)])


class MultiLevelSolve:
    """phis = MultiLevelSolve(...)(rhss, betas): the composite solve over several AMR levels,
    differentiable in every level's rhs and beta.  Dense float64 CUDA tensors per level:
    level 0 over the domain (nz, ny, nx), level l over the bounding box of its boxes."""

    def __init__(self, domain, level_boxes, bc_lo, bc_hi, prob_lo=(0.0, 0.0, 0.0), prob_hi=(1.0, 1.0, 1.0),
                 a=0.0, b=1.0, tol=1e-10, max_iter=100):
        self.ctx = gmg.MultiLevelContext(domain, level_boxes, bc_lo, bc_hi, prob_lo, prob_hi,
                                         stream=torch.cuda.current_stream().cuda_stream)
        self.ctx.allocate(gmg.FP64)
        self.a, self.b, self.tol, self.max_iter = a, b, tol, max_iter

    def __call__(self, rhss, betas):
        return _MultiLevelSolve.apply(self, *rhss, *betas)
