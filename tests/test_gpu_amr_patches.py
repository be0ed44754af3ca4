"""Two-level composite form with several disjoint refined patches on the GPU against the
oracle: the composite operator and its transpose, the composite multigrid solve at a fixed
iteration count and to tolerance, the adjoint solve and the beta gradient (the tolerances of
test_gpu_amr.py)."""
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


LAYOUTS = {
    # two patches far apart, the second split into two fine boxes
    "apart": [((4, 4, 4), (11, 11, 11)), ((20, 4, 16), (23, 11, 23)), ((24, 4, 16), (27, 11, 23))],
    # two patches facing each other across a two-cell coarse gap
    "facing": [((4, 4, 4), (11, 11, 11)), ((16, 4, 4), (19, 11, 11)), ((20, 4, 4), (23, 11, 11))],
}


class PatchPair:
    def __init__(self, layout, bc, seed=21):
        n = 16
        dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
        fb = LAYOUTS[layout]
        cboxes = I.chop(*dom, 8)
        self.P = O.AmrProblem(dom, cboxes, fb, [bc] * 3, [bc] * 3)
        self.C = gmg.AmrContext(dom, cboxes, fb, [bc] * 3, [bc] * 3, stream=torch.cuda.current_stream().cuda_stream)
        self.C.allocate(gmg.FP64)
        lo = [min(b[0][d] for b in fb) for d in range(3)]
        hi = [max(b[1][d] for b in fb) for d in range(3)]
        self.sl = tuple(slice(lo[d], hi[d] + 1) for d in (2, 1, 0))
        rng = np.random.default_rng(seed)
        self.rng = rng
        self.singular = bc != D_
        per = bc == P_
        bf = I.box_mean_filter(np.exp(rng.standard_normal(self.P.fine_shape)), per)
        bc_ = I.box_mean_filter(np.exp(rng.standard_normal(self.P.coarse_shape)), per)
        self.bc = np.where(self.P.covered, average_down(bf, self.P.coarse_shape), bc_)
        self.bf = bf
        self.P.set_coeffs(0.0, 1.0, beta_c=self.bc, beta_f=self.bf)
        self.C.set_coeffs(0.0, 1.0, beta_c=torch.from_numpy(self.bc), beta_f=torch.from_numpy(self.bf[self.sl].copy()))

    def to_gpu(self, xc, xf):
        return self.C.pack_level(0, torch.from_numpy(xc)), self.C.pack_level(1, torch.from_numpy(xf[self.sl].copy()))

    def from_gpu(self, gc, gf):
        xc = self.C.unpack_level(0, gc).cpu().numpy()
        xf = np.zeros(self.P.fine_shape)
        xf[self.sl] = self.C.unpack_level(1, gf).cpu().numpy()
        return xc * self.P.coarse_mask, xf * self.P.fine_mask

    def rand_rhs(self):
        rc = self.rng.standard_normal(self.P.coarse_shape) * self.P.coarse_mask
        rf = self.rng.standard_normal(self.P.fine_shape) * self.P.fine_mask
        if self.singular:
            v = self.P.pack(rc, rf)
            V = self.P.volumes()
            rc, rf = self.P.unpack(v - (V @ v) / V.sum())
        return rc, rf


@pytest.fixture(scope="module", params=[("apart", P_), ("apart", D_), ("facing", N_), ("facing", D_)],
                ids=["apart-periodic", "apart-dirichlet", "facing-neumann", "facing-dirichlet"])
def pp(request):
    return PatchPair(*request.param)


def scale(P, x):
    return np.abs(P.pack(*x)).max()


@pytest.mark.parametrize("transpose", [False, True])
def test_patches_apply(pp, transpose):
    xc = pp.rng.standard_normal(pp.P.coarse_shape) * pp.P.coarse_mask
    xf = pp.rng.standard_normal(pp.P.fine_shape) * pp.P.fine_mask
    want = pp.P.apply(xc, xf, transpose=transpose)
    gc, gf = pp.to_gpu(xc, xf)
    got = pp.from_gpu(*pp.C.apply2(gc, gf, transpose=transpose))
    assert np.abs(pp.P.pack(*got) - pp.P.pack(*want)).max() <= 1e-12 * scale(pp.P, want)


def test_patches_solve_fixed_iterations(pp):
    rc, rf = pp.rand_rhs()
    wc, wf, it, hist, st = pp.P.solve(rc, rf, tol_rel=0.0, maxit=3)
    pc, pf, info = pp.C.solve2(*pp.to_gpu(rc, rf), tol_rel=0.0, max_iter=3)
    assert info.iterations == it == 3
    got = pp.from_gpu(pc, pf)
    assert np.abs(pp.P.pack(*got) - pp.P.pack(wc, wf)).max() <= 1e-10 * scale(pp.P, (wc, wf))


def test_patches_solve_to_tolerance(pp):
    rc, rf = pp.rand_rhs()
    wc, wf, it, hist, st = pp.P.solve(rc, rf, tol_rel=1e-12, maxit=100)
    pc, pf, info = pp.C.solve2(*pp.to_gpu(rc, rf), tol_rel=1e-12, max_iter=100)
    assert st == 0 and info.status == gmg.OK
    got = pp.from_gpu(pc, pf)
    assert np.abs(pp.P.pack(*got) - pp.P.pack(wc, wf)).max() <= 1e-10 * scale(pp.P, (wc, wf))


def test_patches_adjoint_and_gradient(pp):
    """A^T lambda = g solved on the GPU, checked with the oracle's transpose; the beta gradient
    from the oracle's phi and the GPU's lambda against the oracle's gradient of the same."""
    rc, rf = pp.rand_rhs()
    wc, wf, it, hist, st = pp.P.solve(rc, rf, tol_rel=1e-12, maxit=100)
    gc = pp.rng.standard_normal(pp.P.coarse_shape) * pp.P.coarse_mask
    gf = pp.rng.standard_normal(pp.P.fine_shape) * pp.P.fine_mask
    if pp.singular:
        v = pp.P.pack(gc, gf)
        gc, gf = pp.P.unpack(v - (v.sum() / v.size))  # zero plain sum: the range of A^T
    lc, lf, info = pp.C.solve_adjoint2(*pp.to_gpu(gc, gf), tol_rel=1e-11)
    assert info.status == gmg.OK
    lam = pp.from_gpu(lc, lf)
    res = pp.P.pack(gc, gf) - pp.P.pack(*pp.P.apply(*lam, transpose=True))
    if pp.singular:
        res -= res.mean()
    assert np.abs(res).max() <= 1e-10 * np.abs(pp.P.pack(gc, gf)).max()
    want_c, want_f = pp.P.grad_beta(wc, wf, *lam, pp.bc, pp.bf)
    dc, df = pp.C.beta_grad2(*pp.to_gpu(wc, wf), *pp.to_gpu(*lam))
    got_c = pp.C.unpack_level(0, dc).cpu().numpy()
    got_f = np.zeros(pp.P.fine_shape)
    got_f[pp.sl] = pp.C.unpack_level(1, df).cpu().numpy()
    sc = max(np.abs(want_c).max(), np.abs(want_f).max())
    assert np.abs(got_c - want_c).max() <= 1e-10 * sc
    assert np.abs((got_f - want_f) * pp.P.fine_mask).max() <= 1e-10 * sc
