"""Composite form over three AMR levels on the GPU against the oracle (MultiLevelProblem):
the composite operator and its transpose (1e-12 of scale), the composite multigrid solve at
a fixed iteration count (1e-10, same residual history) and to tolerance (1e-12 on both
sides, 1e-10), the adjoint solve (A^T lambda = g by the oracle's transpose, 1e-10) and the
beta gradient (1e-10 of scale), for periodic, Dirichlet and Neumann walls; and over four
levels (the maximum), periodic and Dirichlet."""
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


def four_levels(n=8):
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    h = n // 2
    return dom, [I.chop(*dom, h)] + [I.chop((lo,) * 3, (lo + n - 1,) * 3, h) for lo in (n // 2, 3 * n // 2, 7 * n // 2)]


class MlvPair:
    def __init__(self, bc, seed=40, n=16, nlev=3):
        dom, lb = three_levels(n) if nlev == 3 else four_levels(n)
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


@pytest.fixture(scope="module", params=[(P_, 3), (D_, 3), (N_, 3), (P_, 4), (D_, 4)],
                ids=["periodic", "dirichlet", "neumann", "periodic-4lev", "dirichlet-4lev"])
def mp(request):
    bc, nlev = request.param
    return MlvPair(bc, nlev=nlev, n=16 if nlev == 3 else 8)


def test_multilevel_apply(mp):
    xs = [mp.rng.standard_normal(s) * m for s, m in zip(mp.P.shapes, mp.P.masks)]
    want = mp.P.apply(xs)
    got = mp.from_gpu(mp.C.apply_levels(mp.to_gpu(xs)))
    sc = max(np.abs(w).max() for w in want)
    assert max(np.abs(g - w).max() for g, w in zip(got, want)) <= 1e-12 * sc


def test_multilevel_solve_fixed_iterations(mp):
    rs = mp.rand_rhs()
    want, it, hist, st = mp.P.solve(rs, tol_rel=0.0, maxit=3)
    phis, info = mp.C.solve_levels(mp.to_gpu(rs), tol_rel=0.0, max_iter=3)
    assert info.iterations == it == 3
    np.testing.assert_allclose(info.history(), hist, rtol=1e-8)
    got = mp.from_gpu(phis)
    sc = max(np.abs(w * m).max() for w, m in zip(want, mp.P.masks))
    assert max(np.abs((g - w) * m).max() for g, w, m in zip(got, want, mp.P.masks)) <= 1e-10 * sc


def test_multilevel_solve_to_tolerance(mp):
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


def test_multilevel_transpose(mp):
    ys = [mp.rng.standard_normal(s) * m for s, m in zip(mp.P.shapes, mp.P.masks)]
    want = mp.P.apply(ys, transpose=True)
    got = mp.from_gpu(mp.C.apply_levels(mp.to_gpu(ys), transpose=True))
    sc = max(np.abs(w).max() for w in want)
    assert max(np.abs(g - w).max() for g, w in zip(got, want)) <= 1e-12 * sc


def test_multilevel_adjoint_and_gradient(mp):
    """A^T lambda = g solved on the GPU, checked with the oracle's transpose; the beta
    gradient from the oracle's phi and the GPU's lambda against the oracle's gradient of the
    same."""
    rs = mp.rand_rhs()
    want, it, hist, st = mp.P.solve(rs, tol_rel=1e-12, maxit=100)
    assert st == 0
    gs = [mp.rng.standard_normal(s) * m for s, m in zip(mp.P.shapes, mp.P.masks)]
    if mp.singular:
        v = mp.P.pack(gs)
        gs = mp.P.unpack(v - v.sum() / v.size)  # zero plain sum: the range of A^T
    lams, info = mp.C.solve_adjoint_levels(mp.to_gpu(gs), tol_rel=1e-11)
    assert info.status == gmg.OK
    lam = mp.from_gpu(lams)
    g = mp.P.pack(gs)
    res = g - mp.P.pack(mp.P.apply(lam, transpose=True))
    if mp.singular:
        res -= res.mean()
        assert abs(mp.P.pack(lam).sum()) <= 1e-10 * np.abs(mp.P.pack(lam)).sum()
    assert np.abs(res).max() <= 1e-10 * np.abs(g).max()
    want_g = mp.P.grad_beta(want, lam, mp.betas)
    outs = mp.C.beta_grad_levels(mp.to_gpu(want), mp.to_gpu(lam))
    got = mp.from_gpu(outs)
    sc = max(np.abs(w).max() for w in want_g)
    assert max(np.abs(gg - w).max() for gg, w in zip(got, want_g)) <= 1e-10 * sc


def test_close_nesting_refuses_transpose():
    """Level 2 one level-1 cell inside level 1's low x edge: a level-1 coarse/fine ghost reads a
    covered cell, so the transpose, the adjoint solve and the gradient refuse; the forward
    operator and solve run."""
    import ctypes as C_

    n = 16
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    lb = [I.chop(*dom, 8), I.chop((8, 8, 8), (23, 23, 23), 8), [((18, 20, 20), (29, 27, 27))]]
    C = gmg.MultiLevelContext(dom, lb, [D_] * 3, [D_] * 3, stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64)
    C.set_coeffs(0.0, 1.0)
    z = [C.level_field(l) for l in range(3)]
    C.apply_levels(z)
    with pytest.raises(gmg.GmgError) as e:
        C.apply_levels(z, transpose=True)
    assert e.value.status == gmg.BAD_INPUT
    arr = (C_.c_void_p * 3)(*[t.data_ptr() for t in z])
    info = gmg.SolveInfo()
    p = gmg.default_params()
    assert C.L.gmg_solve_adjoint(C.h, arr, arr, 1e-10, C_.byref(p), C_.byref(info)) == gmg.BAD_INPUT
    assert C.L.gmg_beta_grad(C.h, arr, arr, arr) == gmg.BAD_INPUT


def test_three_level_autograd_vs_central_differences():
    """dL/d(rhs) and dL/d(beta) of every level from MultiLevelSolve (adjoint solve + beta
    gradient behind torch.autograd) against Richardson-extrapolated central differences of
    GPU forward solves to 1e-12 (eps = 1e-3, 5e-4) in random directions, L = 0.5 sum over
    composite cells (phi - phi_t)^2; periodic (singular) and Dirichlet."""
    from paper_2009_12009_gb300.autograd import MultiLevelSolve

    for bc in (P_, D_):
        dom, lb = three_levels(16)
        solver = MultiLevelSolve(dom, lb, [bc] * 3, [bc] * 3, tol=1e-12, max_iter=100)
        C = solver.ctx
        gen = torch.Generator(device="cpu").manual_seed(9)

        def randn(shape):
            return torch.randn(shape, generator=gen, dtype=torch.float64).cuda()

        keep = [torch.as_tensor(~cov, device="cuda", dtype=torch.float64) for cov in C.covered]
        shapes = C.level_shape_
        vol = [8.0 ** (-l) for l in range(3)]

        def zero_mean(xs):  # composite cells, zero volume-weighted mean (needed if singular)
            xs = [x * k for x, k in zip(xs, keep)]
            if bc == P_:
                m = sum(v * x.sum() for v, x in zip(vol, xs)) / sum(v * k.sum() for v, k in zip(vol, keep))
                xs = [(x - m) * k for x, k in zip(xs, keep)]
            return xs

        r0 = zero_mean([randn(s) for s in shapes])
        b0 = [torch.exp(0.5 * randn(s)) for s in shapes]
        tgt = [randn(s) * k for s, k in zip(shapes, keep)]

        def loss_of(phis):
            return sum(0.5 * (((p - t) * k) ** 2).sum() for p, t, k in zip(phis, tgt, keep))

        rs = [r.clone().requires_grad_(True) for r in r0]
        bs = [b.clone().requires_grad_(True) for b in b0]
        loss_of(solver(rs, bs)).backward()
        assert solver.last_adjoint_info.status == gmg.OK
        dr = zero_mean([randn(s) for s in shapes])
        vb = [0.1 * randn(s) * k for s, k in zip(shapes, keep)]

        def central(solve_at, eps):
            pp, pm = solve_at(eps), solve_at(-eps)
            d = sum(0.5 * ((a - b) * (a + b - 2 * t) * k).sum() for a, b, t, k in zip(pp, pm, tgt, keep))
            return float(d) / (2 * eps)

        def richardson(solve_at):
            return (4 * central(solve_at, 5e-4) - central(solve_at, 1e-3)) / 3

        with torch.no_grad():
            fd_r = richardson(lambda e: solver([r + e * d for r, d in zip(r0, dr)], b0))
            fd_b = richardson(lambda e: solver(r0, [b * (1 + e * v) for b, v in zip(b0, vb)]))
        pred_r = float(sum((r.grad * d).sum() for r, d in zip(rs, dr)))
        pred_b = float(sum((b.grad * b0_ * v).sum() for b, b0_, v in zip(bs, b0, vb)))
        assert abs(fd_r - pred_r) <= 1e-6 * abs(fd_r), (bc, fd_r, pred_r)
        assert abs(fd_b - pred_b) <= 1e-6 * abs(fd_b), (bc, fd_b, pred_b)


def test_multilevel_graph_replay_is_exact(mp):
    """The composite iteration captured once as a CUDA graph and replayed gives bit for bit the
    iterates of direct launches, and later calls (other output arrays) reuse the graph."""
    rs = mp.to_gpu(mp.rand_rhs())
    p1, i1 = mp.C.solve_levels(rs, tol_rel=0.0, max_iter=3, use_graph=1)
    p0, i0 = mp.C.solve_levels(rs, tol_rel=0.0, max_iter=3, use_graph=0)
    p2, i2 = mp.C.solve_levels(rs, tol_rel=0.0, max_iter=3, use_graph=1)
    for a, b, c in zip(p1, p0, p2):
        assert torch.equal(a, b) and torch.equal(a, c)
    assert np.array_equal(i1.history(), i0.history())


def test_multilevel_adjoint_graph_replay(mp):
    """The adjoint solve's preconditioner-and-transpose steps replayed as captured graphs agree
    with direct launches (the transposed couplings add with atomics, so not bit for bit: to
    1e-10 of the solution's scale, same iteration count)."""
    gs = [mp.rng.standard_normal(s) * m for s, m in zip(mp.P.shapes, mp.P.masks)]
    if mp.singular:
        v = mp.P.pack(gs)
        gs = mp.P.unpack(v - v.sum() / v.size)
    g = mp.to_gpu(gs)
    l1, i1 = mp.C.solve_adjoint_levels(g, tol_rel=1e-11, use_graph=1)
    l0, i0 = mp.C.solve_adjoint_levels(g, tol_rel=1e-11, use_graph=0)
    l2, i2 = mp.C.solve_adjoint_levels(g, tol_rel=1e-11, use_graph=1)
    assert i1.iterations == i0.iterations == i2.iterations
    sc = max(float(x.abs().max()) for x in l0)
    for a, b, c in zip(l1, l0, l2):
        assert float((a - b).abs().max()) <= 1e-10 * sc and float((c - b).abs().max()) <= 1e-10 * sc
