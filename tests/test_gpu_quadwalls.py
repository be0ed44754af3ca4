"""Quadratic Dirichlet walls (GMG_BC_DIRICHLET_QUAD) on the GPU against the oracle.

The library keeps every ghost single-source: a quadratic wall's ghost holds a third of the
second cell inward, and the rule's -2 phi_0 sits in the wall cell's diagonal D (so the
smoother's update of that cell solves its row exactly, as the oracle's Gauss-Seidel does).
The oracle writes the full ghost 8g/3 - 2 phi_0 + phi_1 / 3 and folds the self term into its
row solve.  The two agree to rounding: the operator and its transpose to 1e-13 of their
scale, one colour pass to 1e-13, V-cycles to 1e-10 (FP64), 2e-4 (FP32), 6e-2 (BF16), solves
at a fixed iteration count to 1e-10 with the same residual history, solves to 1e-12 to
1e-10.  The adjoint solve (BiCGStab on A^T) meets the oracle's transpose to its tolerance and
LAPACK on a small case; the beta and wall-value gradients agree to 1e-10.  Edge cases: a box
one cell thick at a quadratic wall keeps the linear rule; periodic and Neumann sides next to
quadratic ones; batched problems with different walls; the refusals (conjugate gradients,
trilinear interpolation, composite levels).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_12009_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402

P_, D_, N_, Q_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN, I.DIRICHLET_QUAD
DTS = [gmg.DT_F64, gmg.DT_F32, gmg.DT_BF16]

CASES = {
    # quadratic on all six sides, anisotropic cells, boxes of 16: four levels, 8^3 boxes at
    # level 2 (two-cell boxes along no axis until the bottom)
    "qqq": dict(n=(48, 40, 32), lo=[Q_] * 3, hi=[Q_] * 3, a=0.0, b=1.0, mgs=16, L=(1.2, 1.0, 0.8)),
    # quadratic, linear Dirichlet, Neumann and periodic sides with a*alpha, boxes of 8 (down to
    # boxes of two cells along each axis on level 2)
    "mixed": dict(n=(40, 32, 24), lo=[Q_, P_, N_], hi=[D_, P_, Q_], a=0.6, b=1.3, mgs=8, L=(1.0, 0.9, 0.7)),
    # x extent 17 in boxes of 8: the last box is one cell thick at the high x wall and keeps
    # the linear rule there; odd extents, so level 0 is the bottom level
    "thin": dict(n=(17, 12, 10), lo=[Q_, Q_, D_], hi=[Q_, N_, Q_], a=0.3, b=1.0, mgs=8, L=(1.0, 1.0, 1.0)),
}


class QuadPair:
    def __init__(self, name, seed=21):
        c = CASES[name]
        self.name, self.c = name, c
        n = c["n"]
        self.dom = dom = ((0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1))
        self.boxes = boxes = I.chop(*dom, c["mgs"])
        rng = np.random.default_rng(seed)
        self.shape = shape = (n[2], n[1], n[0])
        self.beta = I.lognormal_beta(rng, shape, periodic=False)
        self.alpha = np.exp(rng.standard_normal(shape)) if c["a"] else None
        self.P = O.Problem(dom, boxes, c["lo"], c["hi"], (0, 0, 0), c["L"])
        self.P.set_coeffs(c["a"], c["b"], alpha=self.alpha, beta=self.beta)
        self.P0 = O.Problem(dom, boxes, c["lo"], c["hi"], (0, 0, 0), c["L"])  # homogeneous walls
        self.P0.set_coeffs(c["a"], c["b"], alpha=self.alpha, beta=self.beta)
        self.C = gmg.Context(dom, c["lo"], c["hi"], prob_hi=c["L"], boxes=boxes,
                             stream=torch.cuda.current_stream().cuda_stream)
        self.C.allocate(gmg.MIXED_FP32)
        self.C.set_scalars(c["a"], c["b"])
        if self.alpha is not None:
            self.C.set_alpha(torch.from_numpy(self.alpha))
        self.C.set_beta(torch.from_numpy(self.beta))
        self.values = {}
        for f in range(6):
            if (c["hi"] if f % 2 else c["lo"])[f // 2] != P_:
                self.values[f] = rng.standard_normal(self.P.face_shape(f))
                self.P.set_bc_values(f, self.values[f])
        self.rhs = rng.standard_normal(shape)
        self.target = rng.standard_normal(shape)
        self.rng = rng

    def gvals(self):
        return {f: torch.from_numpy(v) for f, v in self.values.items()}

    def dev(self, x, m=0, dt=gmg.DT_F64):
        return self.C.pack(torch.from_numpy(np.ascontiguousarray(x)), m, dt)

    def host(self, b, m=0, dt=gmg.DT_F64):
        return self.C.unpack(b, m, dt).cpu().numpy()


@pytest.fixture(scope="module", params=list(CASES))
def qp(request):
    return QuadPair(request.param)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_hierarchy_matches(qp):
    assert qp.C.nlevels == qp.P.nlevels
    assert (qp.C.nlevels == 1) == (qp.name == "thin")


def test_apply_and_transpose_match_oracle(qp):
    x = qp.rng.standard_normal(qp.shape)
    y = qp.rng.standard_normal(qp.shape)
    ax = qp.host(qp.C.apply(qp.dev(x)))
    assert _rel(ax, qp.P.apply(x)) <= 1e-13
    aty = qp.host(qp.C.apply(qp.dev(y), transpose=True))
    assert _rel(aty, qp.P.apply_transpose(y)) <= 1e-13
    # <A x, y> = <x, A^T y>, and A is not symmetric (the wall couplings)
    assert abs(np.sum(ax * y) - np.sum(x * aty)) <= 1e-12 * np.abs(ax).max() * np.abs(y).size
    assert np.abs(aty - qp.host(qp.C.apply(qp.dev(y)))).max() > 1e-6 * np.abs(aty).max()


@pytest.mark.parametrize("colour", [0, 1])
def test_colour_pass_matches_oracle(qp, colour):
    """One colour of Gauss-Seidel on every level (ghosts filled first on both sides)."""
    for m in range(qp.C.nlevels):
        shp = qp.P.level_shape(m)
        phi = qp.rng.standard_normal(shp)
        rhs = qp.rng.standard_normal(shp)
        buf = qp.dev(phi, m)
        qp.C.smooth(buf, qp.dev(rhs, m), m, gmg.DT_F64, colour)
        want = qp.P.to_boxed(m, phi)
        qp.P.smooth_colour(m, want, qp.P.to_boxed(m, rhs), colour)
        assert _rel(qp.host(buf, m), qp.P.to_dense(m, want)) <= 1e-13, m


@pytest.mark.parametrize("dt", DTS)
def test_vcycle_matches_oracle(qp, dt):
    r = qp.rng.standard_normal(qp.shape)
    if dt != gmg.DT_F64:  # the rounded right-hand side on both sides
        r = qp.host(qp.dev(r, 0, dt), 0, dt)
    got = qp.host(qp.C.vcycle(qp.dev(r, 0, dt), dt), 0, dt)
    want = qp.P.to_dense(0, qp.P.vcycle(0, qp.P.to_boxed(0, r)))
    tol = {gmg.DT_F64: 1e-10, gmg.DT_F32: 2e-4, gmg.DT_BF16: 6e-2}[dt]
    assert _rel(got, want) <= tol


@pytest.mark.parametrize("graph", [1, 0])
def test_solve_fixed_iterations_with_values(qp, graph):
    """Four outer iterations with the wall values on both sides: the same iterate and
    residual history.  (A one-level hierarchy is its own BiCGStab bottom, stopped at 1e-4 of
    its start: its iterates depend on rounding at that level, so only the final iterate, by
    then converged, is compared.)"""
    phi, info = qp.C.solve(qp.dev(qp.rhs), tol_rel=0.0, max_iter=4, use_graph=graph, wall_values=qp.gvals())
    want, it, hist, st = qp.P.solve(qp.rhs, tol_rel=0.0, maxit=4)
    assert info.iterations == it == 4
    assert _rel(qp.host(phi), want) <= 1e-10
    if qp.C.nlevels > 1:
        np.testing.assert_allclose(info.history(), hist, rtol=1e-6, atol=1e-11 * hist[0])
    else:
        assert info.history()[0] == pytest.approx(hist[0], rel=1e-13) and info.history()[-1] <= 1e-9 * hist[0]


@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16])
def test_solve_to_tolerance_with_values(qp, prec):
    """To 1e-12 (FP64 outer loop for every precision): within 1e-10 of the oracle's solution,
    and the residual by the oracle's affine operator below 1e-10 of ||rhs - A_g 0||."""
    phi, info = qp.C.solve(qp.dev(qp.rhs), tol_rel=1e-12, max_iter=100, precision=prec, wall_values=qp.gvals())
    assert info.status == gmg.OK
    want, it, hist, st = qp.P.solve(qp.rhs, tol_rel=1e-12, maxit=100)
    assert st == O.OK
    got = qp.host(phi)
    assert _rel(got, want) <= 1e-10
    if prec == gmg.FP64:
        assert abs(info.iterations - it) <= 1
    r0 = qp.rhs - qp.P.apply_bc(np.zeros(qp.shape))
    assert np.abs(qp.rhs - qp.P.apply_bc(got)).max() <= 1e-10 * np.abs(r0).max()


def test_bicgstab_top_level(qp):
    phi, info = qp.C.solve(qp.dev(qp.rhs), tol_rel=1e-12, max_iter=100, krylov=1, wall_values=qp.gvals())
    assert info.status == gmg.OK
    want, it, hist, st = qp.P.solve_krylov(qp.rhs, 1, tol_rel=1e-12, maxit=100)
    assert st == O.OK
    assert _rel(qp.host(phi), want) <= 1e-10


@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32])
def test_adjoint_solve_meets_the_transpose(qp, prec):
    """A^T lambda = g by BiCGStab (preconditioned by the V-cycle of A): the oracle's A^T of the
    result is g to the solve's tolerance."""
    g = qp.rng.standard_normal(qp.shape)
    lam, info = qp.C.solve_adjoint(qp.dev(g), tol_rel=1e-11, precision=prec)
    assert info.status == gmg.OK, info.status
    got = qp.host(lam)
    assert np.abs(qp.P.apply_transpose(got) - g).max() <= 1.05e-11 * np.abs(g).max()
    # not the forward solve: A lambda differs from g
    assert np.abs(qp.P.apply(got) - g).max() > 1e-6 * np.abs(g).max()


def test_adjoint_solve_matches_lapack():
    """12 x 10 x 8 with quadratic walls on five sides: lambda equals LAPACK's solve of the
    transposed assembled matrix."""
    n = (12, 10, 8)
    dom = ((0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1))
    lo, hi = [Q_, Q_, N_], [Q_, Q_, Q_]
    rng = np.random.default_rng(31)
    shape = n[::-1]
    beta = np.exp(rng.standard_normal(shape))
    P = O.Problem(dom, I.chop(*dom, 4), lo, hi)
    P.set_coeffs(0.2, 1.0, alpha=np.ones(shape), beta=beta)
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[:] = 0
        e[j] = 1
        A[:, j] = P.apply(e.reshape(shape)).reshape(-1)
    C = gmg.Context(dom, lo, hi, boxes=I.chop(*dom, 4), stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64)
    C.set_scalars(0.2, 1.0)
    C.set_alpha(torch.ones(shape, dtype=torch.float64))
    C.set_beta(torch.from_numpy(beta))
    g = rng.standard_normal(shape)
    lam, info = C.solve_adjoint(C.pack(torch.from_numpy(g)), tol_rel=1e-13)
    assert info.status == gmg.OK
    want = np.linalg.solve(A.T, g.reshape(-1))
    assert np.abs(C.unpack(lam).cpu().numpy().reshape(-1) - want).max() <= 1e-10 * np.abs(want).max()


def test_gradients_match_oracle(qp):
    """Same phi (the oracle's solution with values) and lambda (LAPACK-free: the oracle's
    transpose checked below) on both sides: dL/dbeta and dL/dg agree."""
    phi, _, _, st = qp.P.solve(qp.rhs, tol_rel=1e-12, maxit=100)
    assert st == O.OK
    lam_t, info = qp.C.solve_adjoint(qp.dev(phi - qp.target), tol_rel=1e-12)
    assert info.status == gmg.OK
    lam = qp.host(lam_t)
    want_b = qp.P.grad_beta(phi, lam, qp.beta)
    got_b = qp.host(qp.C.beta_grad(qp.dev(phi), qp.dev(lam), wall_values=qp.gvals()))
    assert _rel(got_b, want_b) <= 1e-10
    got_g = qp.C.wall_values_grad(qp.dev(lam), list(qp.values))
    for f in qp.values:
        want_g = qp.P.grad_wall_values(lam, f)
        assert _rel(got_g[f].cpu().numpy(), want_g) <= 1e-12, f


def test_autograd_through_quadratic_walls():
    """torch.autograd through the solve: dL/drhs = lambda (A^T lambda = phi - phi_t) and
    dL/dbeta equal the oracle's, with quadratic walls that carry values."""
    from paper_2009_12009_gb300.autograd import Solve

    qp = QuadPair("mixed", seed=22)
    c = qp.c
    S = Solve(c["n"], bc=(c["lo"], c["hi"]), max_grid_size=c["mgs"], prob_hi=c["L"], a=c["a"], b=c["b"], tol=1e-12)
    S.ctx.set_alpha(torch.from_numpy(qp.alpha))
    t_rhs = torch.tensor(qp.rhs, device="cuda", requires_grad=True)
    t_beta = torch.tensor(qp.beta, device="cuda", requires_grad=True)
    t_vals = {f: torch.tensor(v, device="cuda", requires_grad=True) for f, v in qp.values.items()}
    phi = S(t_rhs, t_beta, wall_values=t_vals)
    loss = 0.5 * ((phi - torch.from_numpy(qp.target).cuda()) ** 2).sum()
    loss.backward()
    ophi, _, _, _ = qp.P.solve(qp.rhs, tol_rel=1e-12, maxit=100)
    assert np.abs(phi.detach().cpu().numpy() - ophi).max() <= 1e-10 * np.abs(ophi).max()
    lam = t_rhs.grad.cpu().numpy()
    g = ophi - qp.target
    assert np.abs(qp.P.apply_transpose(lam) - g).max() <= 1e-9 * np.abs(g).max()
    gb = qp.P.grad_beta(ophi, lam, qp.beta)
    assert _rel(t_beta.grad.cpu().numpy(), gb) <= 1e-8
    for f, t in t_vals.items():
        assert _rel(t.grad.cpu().numpy(), qp.P.grad_wall_values(lam, f)) <= 1e-8, f


def test_dataflow_and_push_are_off_on_quadratic_levels(qp):
    """A quadratic wall's ghost is not a face copy: the ghost push and the dataflow sweep that
    needs it stand aside, and asking for them changes nothing."""
    rhs = qp.dev(qp.rhs)
    p1, i1 = qp.C.solve(rhs, tol_rel=0.0, max_iter=3, fused_sweep=1, ghost_push=1)
    a1 = qp.host(p1).copy()
    p0, i0 = qp.C.solve(rhs, tol_rel=0.0, max_iter=3, fused_sweep=0, ghost_push=0)
    assert np.array_equal(a1, qp.host(p0))
    assert i1.history() == i0.history()


def test_batched_problems_with_quadratic_walls():
    """Four problems with different walls in one batched context: every problem's solution and
    iteration count are those of its own oracle solve."""
    walls = [([Q_] * 3, [Q_] * 3), ([D_] * 3, [D_] * 3), ([Q_, N_, D_], [N_, Q_, Q_]), ([P_, Q_, Q_], [P_, D_, N_])]
    sizes = [(32, 24, 16), (16, 16, 32), (24, 32, 16), (32, 16, 24)]
    probs, orcs = [], []
    for i, (sz, (lo, hi)) in enumerate(zip(sizes, walls)):
        p = I.batch_problem(sz, i, seed=777, max_grid_size=8)
        p["bc_lo"], p["bc_hi"] = lo, hi
        probs.append(p)
        P = O.Problem(p["domain"], p["boxes"], lo, hi, (0, 0, 0), p["prob_hi"])
        P.set_coeffs(0.0, 1.0, beta=p["beta"])
        orcs.append(P)
    B = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    B.allocate(gmg.FP64)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    phi, infos = B.batch_solve(B.pack_all([torch.from_numpy(p["rhs"]) for p in probs]), tol_rel=1e-11)
    for s, (p, P) in enumerate(zip(probs, orcs)):
        want, it, hist, st = P.solve(p["rhs"], tol_rel=1e-11, maxit=100)
        assert infos[s].status == gmg.OK and st == O.OK
        assert abs(infos[s].iterations - it) <= 1, s
        got = B.unpack_solve(s, phi).cpu().numpy()
        assert _rel(got, want) <= 1e-9, s


def test_quadratic_walls_refusals():
    qp = QuadPair("qqq")
    rhs = qp.dev(qp.rhs)
    for kw in (dict(krylov=2), dict(bottom_solver=1), dict(prolongation=1)):
        with pytest.raises(gmg.GmgError):
            qp.C.solve(rhs, tol_rel=1e-8, max_iter=5, **kw)
    dom = ((0, 0, 0), (15, 15, 15))
    with pytest.raises((gmg.GmgError, ValueError)):
        gmg.AmrContext(dom, I.chop(*dom, 8), [((8, 8, 8), (23, 23, 23))], [Q_] * 3, [Q_] * 3,
                       stream=torch.cuda.current_stream().cuda_stream)
