"""Composite form over three AMR levels on the GPU against the oracle (MultiLevelProblem):
the composite operator (1e-12 of scale), the composite multigrid solve at a fixed iteration
count (1e-10, same residual history) and to tolerance (1e-12 on both sides, 1e-10), for
periodic, Dirichlet and Neumann walls."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_12009_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def avg_down(x):
    nz, ny, nx = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))


def three_levels(n=16):
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    l1 = I.chop((n // 2,) * 3, (3 * n // 2 - 1,) * 3, n // 2)
    l2 = I.chop((3 * n // 2,) * 3, (5 * n // 2 - 1,) * 3, n // 2)
    return dom, [I.chop(*dom, n // 2), l1, l2]


class MlvPair:
    def __init__(self, bc, seed=40, n=16):
        dom, lb = three_levels(n)
        self.P = O.MultiLevelProblem(dom, lb, [bc] * 3, [bc] * 3)
        self.C = gmg.MultiLevelContext(dom, lb, [bc] * 3, [bc] * 3, stream=torch.cuda.current_stream().cuda_stream)
        self.C.allocate(gmg.FP64)
        M = self.P
        self.sl = []
        for lev in range(M.L):
            lo = self.C.level_lo[lev]
            sh = self.C.level_shape_[lev]
            self.sl.append(tuple(slice(lo[d], lo[d] + sh[2 - d]) for d in (2, 1, 0)))
        rng = np.random.default_rng(seed)
        self.rng = rng
        per = bc == P_
        betas = [I.box_mean_filter(np.exp(rng.standard_normal(s)), per) for s in M.shapes]
        for l in range(M.L - 2, -1, -1):
            s = M.shapes[l]
            under = M.inside[l + 1].reshape(s[0], 2, s[1], 2, s[2], 2).all(axis=(1, 3, 5))
            betas[l] = np.where(under, avg_down(betas[l + 1]), betas[l])
        self.betas = betas
        M.set_coeffs(0.0, 1.0, betas=betas)
        self.C.set_coeffs(0.0, 1.0, betas=[torch.from_numpy(b[s].copy()) for b, s in zip(betas, self.sl)])
        self.singular = bc != D_

    def to_gpu(self, xs):
        return [self.C.pack_level(l, torch.from_numpy(np.ascontiguousarray(x[s]))) for l, (x, s) in
                enumerate(zip(xs, self.sl))]

    def from_gpu(self, gs):
        out = []
        for l, g in enumerate(gs):
            x = np.zeros(self.P.shapes[l])
            x[self.sl[l]] = self.C.unpack_level(l, g).cpu().numpy()
            out.append(x * self.P.masks[l])
        return out

    def rand_rhs(self):
        rs = [self.rng.standard_normal(s) * m for s, m in zip(self.P.shapes, self.P.masks)]
        if self.singular:
            v = self.P.pack(rs)
            V = self.P.volumes()
            rs = self.P.unpack(v - (V @ v) / V.sum())
        return rs


@pytest.fixture(scope="module", params=[P_, D_, N_], ids=["periodic", "dirichlet", "neumann"])
def mp(request):
    return MlvPair(request.param)


def test_three_level_apply(mp):
    xs = [mp.rng.standard_normal(s) * m for s, m in zip(mp.P.shapes, mp.P.masks)]
    want = mp.P.apply(xs)
    got = mp.from_gpu(mp.C.apply_levels(mp.to_gpu(xs)))
    sc = max(np.abs(w).max() for w in want)
    assert max(np.abs(g - w).max() for g, w in zip(got, want)) <= 1e-12 * sc


def test_three_level_solve_fixed_iterations(mp):
    rs = mp.rand_rhs()
    want, it, hist, st = mp.P.solve(rs, tol_rel=0.0, maxit=3)
    phis, info = mp.C.solve_levels(mp.to_gpu(rs), tol_rel=0.0, max_iter=3)
    assert info.iterations == it == 3
    np.testing.assert_allclose(info.history(), hist, rtol=1e-8)
    got = mp.from_gpu(phis)
    sc = max(np.abs(w * m).max() for w, m in zip(want, mp.P.masks))
    assert max(np.abs((g - w) * m).max() for g, w, m in zip(got, want, mp.P.masks)) <= 1e-10 * sc


def test_three_level_solve_to_tolerance(mp):
    rs = mp.rand_rhs()
    want, it, hist, st = mp.P.solve(rs, tol_rel=1e-12, maxit=100)
    phis, info = mp.C.solve_levels(mp.to_gpu(rs), tol_rel=1e-12, max_iter=100)
    assert st == 0 and info.status == gmg.OK and abs(info.iterations - it) <= 1
    got = mp.from_gpu(phis)
    sc = max(np.abs(w * m).max() for w, m in zip(want, mp.P.masks))
    assert max(np.abs((g - w) * m).max() for g, w, m in zip(got, want, mp.P.masks)) <= 1e-10 * sc
    # the solution's composite residual by the oracle's operator
    r = [rr - a for rr, a in zip(rs, mp.P.apply(got))]
    assert max(np.abs(x).max() for x in r) <= 1.01e-12 * max(np.abs(x).max() for x in rs) * 10


def test_three_levels_refuse_adjoint():
    dom, lb = three_levels(16)
    C = gmg.MultiLevelContext(dom, lb, [D_] * 3, [D_] * 3, stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64)
    C.set_coeffs(0.0, 1.0)
    z = [C.level_field(l) for l in range(3)]
    import ctypes as C_

    arr = (C_.c_void_p * 3)(*[t.data_ptr() for t in z])
    info = gmg.SolveInfo()
    p = gmg.default_params()
    st = C.L.gmg_solve_adjoint(C.h, arr, arr, 1e-10, C_.byref(p), C_.byref(info))
    assert st == gmg.BAD_INPUT
