"""Two-level composite form on the GPU against the oracle: composite operator and its
transpose, the composite multigrid solve, the adjoint solve and the beta gradient.

Tolerances: operator applications 1e-12 of scale (FMA and summation-order differences);
solves at a fixed iteration count and to 1e-12 agree to 1e-10 relative (the FP64
requirement); the adjoint lambda matches a LAPACK solve of the oracle's transposed composite
matrix to 1e-9; beta gradients computed from the same phi and lambda agree to 1e-10 of
their scale."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_12009_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def average_down(xf, cshape):
    nz, ny, nx = cshape
    return xf.reshape(nz, 2, ny, 2, nx, 2).mean(axis=(1, 3, 5))


class AmrPair:
    def __init__(self, n=16, patch=(4, 12), bc=P_, seed=7):
        dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
        lo, hi = 2 * patch[0], 2 * patch[1] - 1
        fdom = ((lo, lo, lo), (hi, hi, hi))
        cboxes = I.chop(*dom, n // 2)
        fboxes = I.chop(*fdom, (hi - lo + 1) // 2)
        self.P = O.AmrProblem(dom, cboxes, fboxes, [bc] * 3, [bc] * 3)
        self.C = gmg.AmrContext(dom, cboxes, fboxes, [bc] * 3, [bc] * 3,
                                stream=torch.cuda.current_stream().cuda_stream)
        self.C.allocate(gmg.FP64)
        self.sl = tuple(slice(lo, hi + 1) for _ in range(3))
        rng = np.random.default_rng(seed)
        per = bc == P_
        self.bf = I.box_mean_filter(np.exp(rng.standard_normal(self.P.fine_shape)), per)
        bc_ = I.box_mean_filter(np.exp(rng.standard_normal(self.P.coarse_shape)), per)
        self.bc = np.where(self.P.covered, average_down(self.bf, self.P.coarse_shape), bc_)
        self.P.set_coeffs(0.0, 1.0, beta_c=self.bc, beta_f=self.bf)
        self.C.set_coeffs(0.0, 1.0, beta_c=torch.from_numpy(self.bc), beta_f=torch.from_numpy(self.bf[self.sl]))
        self.rng = rng
        self.singular = bc != D_  # periodic or zero-flux walls with a = 0

    def to_gpu(self, xc, xf):
        return self.C.pack_level(0, torch.from_numpy(xc)), self.C.pack_level(1, torch.from_numpy(xf[self.sl].copy()))

    def from_gpu(self, gc, gf):
        xc = self.C.unpack_level(0, gc).cpu().numpy()
        xf = np.zeros(self.P.fine_shape)
        xf[self.sl] = self.C.unpack_level(1, gf).cpu().numpy()
        return xc, xf

    def rand_composite(self):
        xc = self.rng.standard_normal(self.P.coarse_shape) * self.P.coarse_mask
        xf = self.rng.standard_normal(self.P.fine_shape) * self.P.fine_mask
        return xc, xf

    def rand_rhs(self):
        rc, rf = self.rand_composite()
        if self.singular:
            v = self.P.pack(rc, rf)
            V = self.P.volumes()
            rc, rf = self.P.unpack(v - (V @ v) / V.sum())
        return rc, rf


@pytest.fixture(scope="module", params=[P_, D_, N_], ids=["periodic", "dirichlet", "neumann"])
def amr(request):
    return AmrPair(bc=request.param)


def scale_of(P, x):
    return np.abs(P.pack(*x)).max()


@pytest.mark.parametrize("transpose", [False, True])
def test_composite_apply(amr, transpose):
    xc, xf = amr.rand_composite()
    want = amr.P.apply(xc, xf, transpose=transpose)
    gc, gf = amr.to_gpu(xc, xf)
    oc, of = amr.C.apply2(gc, gf, transpose=transpose)
    got = amr.from_gpu(oc, of)
    got = (got[0] * amr.P.coarse_mask, got[1] * amr.P.fine_mask)
    scale = scale_of(amr.P, want)
    assert np.abs(amr.P.pack(*got) - amr.P.pack(*want)).max() <= 1e-12 * scale


def test_composite_solve_fixed_iterations(amr):
    rc, rf = amr.rand_rhs()
    pc, pf, it, hist, st = amr.P.solve(rc, rf, tol_rel=0.0, maxit=4)
    gc, gf = amr.to_gpu(rc, rf)
    oc, of, info = amr.C.solve2(gc, gf, tol_rel=0.0, max_iter=4)
    got = amr.from_gpu(oc, of)
    assert info.iterations == it == 4
    want = amr.P.pack(pc, pf)
    assert np.abs(amr.P.pack(*got) - want).max() <= 1e-10 * np.abs(want).max()
    np.testing.assert_allclose(info.history(), hist, rtol=1e-6, atol=1e-11 * hist[0])


def test_composite_solve_to_tolerance(amr):
    rc, rf = amr.rand_rhs()
    pc, pf, it, hist, st = amr.P.solve(rc, rf, tol_rel=1e-12, maxit=200)
    gc, gf = amr.to_gpu(rc, rf)
    oc, of, info = amr.C.solve2(gc, gf, tol_rel=1e-12, max_iter=200)
    assert st == 0 and info.status == gmg.OK
    assert abs(info.iterations - it) <= 1
    got = amr.from_gpu(oc, of)
    want = amr.P.pack(pc, pf)
    assert np.abs(amr.P.pack(*got) - want).max() <= 1e-10 * np.abs(want).max()
    # covered coarse cells hold the average of the fine solution
    np.testing.assert_allclose(got[0][amr.P.covered], average_down(got[1], amr.P.coarse_shape)[amr.P.covered],
                               rtol=1e-13, atol=1e-13 * np.abs(want).max())


def test_adjoint_solve_residual(amr):
    """A^T lambda = g (projected for the periodic case), checked with the ORACLE's transposed
    operator, and lambda's sum is zero for the singular problem."""
    gcn, gfn = amr.rand_composite()
    gc, gf = amr.to_gpu(gcn, gfn)
    lc, lf, info = amr.C.solve_adjoint2(gc, gf, tol_rel=1e-11, max_iter=100)
    assert info.status == gmg.OK, (info.status, info.history()[-3:])
    lam = amr.P.pack(*amr.from_gpu(lc, lf))
    g = amr.P.pack(gcn, gfn)
    if amr.singular:
        V = amr.P.volumes()
        g = g - V * g.sum() / V.sum()
        assert abs(lam.sum()) <= 1e-10 * np.abs(lam).sum()
    r = g - amr.P.pack(*amr.P.apply(*amr.P.unpack(lam), transpose=True))
    assert np.abs(r).max() <= 1.01e-11 * np.abs(g).max()


def test_beta_gradient_matches_oracle(amr):
    """Same phi and lambda (the oracle's) on both sides: the cell gradients agree."""
    rc, rf = amr.rand_rhs()
    pc, pf, it, hist, st = amr.P.solve(rc, rf, tol_rel=1e-12, maxit=200)
    lc, lf = amr.rand_composite()
    want_c, want_f = amr.P.grad_beta(pc, pf, lc, lf, amr.bc, amr.bf)
    gpc, gpf = amr.to_gpu(pc, pf)
    glc, glf = amr.to_gpu(lc, lf)
    dc, df = amr.C.beta_grad2(gpc, gpf, glc, glf)
    got_c, got_f = amr.from_gpu(dc, df)
    scale = max(np.abs(want_c).max(), np.abs(want_f).max())
    assert np.abs(got_c - want_c).max() <= 1e-10 * scale
    assert np.abs((got_f - want_f)[amr.P.fine_mask]).max() <= 1e-10 * scale
    assert np.abs(got_c[amr.P.covered]).max() == 0.0


def test_small_adjoint_vs_lapack():
    """lambda from the GPU adjoint solve equals a LAPACK solve of the oracle's assembled
    transposed composite matrix (8^3 coarse cells, 8^3 fine cells)."""
    pair = AmrPair(n=8, patch=(2, 6), bc=D_, seed=3)
    M = pair.P.matrix()
    gcn, gfn = pair.rand_composite()
    g = pair.P.pack(gcn, gfn)
    want = np.linalg.solve(M.T, g)
    lc, lf, info = pair.C.solve_adjoint2(*pair.to_gpu(gcn, gfn), tol_rel=1e-13, max_iter=200)
    assert info.status == gmg.OK
    got = pair.P.pack(*pair.from_gpu(lc, lf))
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()


def test_autograd_gradients_match_oracle_adjoint():
    """torch.autograd through the two-level solve: dL/drhs = lambda and dL/dbeta (coarse and
    fine cells) equal the oracle's LAPACK adjoint and the oracle's beta gradient, for
    L = 0.5 sum over composite cells (phi - phi_t)^2."""
    from paper_2009_12009_gb300.autograd import AmrSolve

    n, patch = 8, (2, 6)
    pair = AmrPair(n=n, patch=patch, bc=D_, seed=11)
    P = pair.P
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    lo, hi = 2 * patch[0], 2 * patch[1] - 1
    solver = AmrSolve(dom, I.chop(*dom, n // 2), I.chop((lo,) * 3, (hi,) * 3, (hi - lo + 1) // 2), [D_] * 3, [D_] * 3,
                      tol=1e-13, max_iter=200)
    rc, rf = pair.rand_rhs()
    tc, tf = pair.rand_composite()
    dev = "cuda"
    t_rc = torch.tensor(rc, device=dev, requires_grad=True)
    t_rf = torch.tensor(rf[pair.sl], device=dev, requires_grad=True)
    t_bc = torch.tensor(pair.bc, device=dev, requires_grad=True)
    t_bf = torch.tensor(pair.bf[pair.sl], device=dev, requires_grad=True)
    pc, pf = solver(t_rc, t_rf, t_bc, t_bf)
    loss = 0.5 * ((pc - torch.tensor(tc, device=dev)) ** 2).sum() + 0.5 * ((pf - torch.tensor(tf[pair.sl], device=dev)) ** 2).sum()
    loss.backward()
    # oracle: phi, lambda (LAPACK on the assembled transposed matrix), beta gradient
    opc, opf, it, hist, st = P.solve(rc, rf, tol_rel=1e-13, maxit=200)
    g = P.pack(opc, opf) - P.pack(tc, tf)
    lam = np.linalg.solve(P.matrix().T, g)
    lc, lf = P.unpack(lam)
    gbc, gbf = P.grad_beta(opc, opf, lc, lf, pair.bc, pair.bf)
    got_lc = t_rc.grad.cpu().numpy()
    got_lf = t_rf.grad.cpu().numpy()
    assert np.abs(got_lc - lc).max() <= 1e-8 * np.abs(lam).max()
    assert np.abs(got_lf - lf[pair.sl]).max() <= 1e-8 * np.abs(lam).max()
    sc = max(np.abs(gbc).max(), np.abs(gbf).max())
    assert np.abs(t_bc.grad.cpu().numpy() - gbc).max() <= 1e-8 * sc
    assert np.abs(t_bf.grad.cpu().numpy() - gbf[pair.sl]).max() <= 1e-8 * sc
