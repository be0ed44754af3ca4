"""Neumann walls and nonzero wall values on the GPU against the oracle.

The library folds wall values into the right-hand side (rhs - A_g 0, walls.cu) and solves
with homogeneous walls; the oracle puts the values into its ghost cells at every outer
residual.  The two agree to rounding: the fold to 1e-13 of its scale, solves at a fixed
iteration count to 1e-10 relative with the same residual history, solves to 1e-12 to 1e-10.
Gradients from the same phi and lambda agree to 1e-10 (beta) and 1e-12 (wall values).
Edge cases: a Neumann problem without a Dirichlet wall is singular (projected), wall values
on a periodic face and on multi-problem or two-level contexts are refused.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_12009_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN

CASES = {
    # Dirichlet and Neumann walls with values, y periodic, a*alpha term, boxes of 6 (tails of 2
    # and 4); three levels down to a 6x4x5 bottom (a two-level 24x16x18 hierarchy has an
    # 864-cell BiCGStab bottom whose 1e-4 stop makes the iterates depend on rounding at 1e-6)
    "mixed": dict(n=(24, 16, 20), lo=[N_, P_, D_], hi=[D_, P_, N_], a=0.5, b=1.3, mgs=6, L=(1.2, 0.8, 1.0)),
    # Neumann everywhere with values, a = 0: singular, the fluxes are balanced by projection
    "neumann": dict(n=(16, 16, 16), lo=[N_] * 3, hi=[N_] * 3, a=0.0, b=1.0, mgs=8, L=(1.0, 1.0, 1.0)),
    # Dirichlet everywhere with values (the abec recipe at 32^3)
    "dirichlet": dict(n=(32, 32, 32), lo=[D_] * 3, hi=[D_] * 3, a=0.0, b=1.0, mgs=16, L=(1.0, 1.0, 1.0)),
}


class WallPair:
    def __init__(self, name, seed=11):
        c = CASES[name]
        self.c = c
        n = c["n"]
        dom = ((0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1))
        boxes = I.chop(*dom, c["mgs"])
        rng = np.random.default_rng(seed)
        self.shape = shape = (n[2], n[1], n[0])
        self.beta = I.lognormal_beta(rng, shape, periodic=False)
        self.alpha = np.exp(rng.standard_normal(shape)) if c["a"] else None
        self.P = O.Problem(dom, boxes, c["lo"], c["hi"], (0, 0, 0), c["L"])
        self.P.set_coeffs(c["a"], c["b"], alpha=self.alpha, beta=self.beta)
        self.P0 = O.Problem(dom, boxes, c["lo"], c["hi"], (0, 0, 0), c["L"])  # the same, homogeneous walls
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
        self.singular = D_ not in c["lo"] + c["hi"] and c["a"] == 0.0
        if self.singular:  # make rhs - A_g 0 zero-mean
            self.rhs -= (self.rhs - self.P.apply_bc(np.zeros(shape))).mean()
        self.target = rng.standard_normal(shape)

    def gvals(self):
        return {f: torch.from_numpy(v) for f, v in self.values.items()}


@pytest.fixture(scope="module", params=list(CASES))
def wp(request):
    return WallPair(request.param)


def test_wall_values_rhs_matches_oracle(wp):
    """rhs - A_g(0): the GPU fold against the oracle's affine operator applied to zero."""
    got = wp.C.unpack(wp.C.wall_values_rhs(wp.C.pack(torch.from_numpy(wp.rhs)), wp.gvals())).cpu().numpy()
    want = wp.rhs - wp.P.apply_bc(np.zeros(wp.shape))
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
    # in place gives the same
    buf = wp.C.pack(torch.from_numpy(wp.rhs))
    wp.C.wall_values_rhs(buf, wp.gvals(), out=buf)
    assert np.array_equal(wp.C.unpack(buf).cpu().numpy(), got)


@pytest.mark.parametrize("graph", [1, 0])
def test_solve_with_wall_values_fixed_iterations(wp, graph):
    """Four outer iterations from phi = 0 on both sides: same residual history (the first
    entry is ||rhs - A_g 0||) and iterates within 1e-10."""
    phi, info = wp.C.solve(wp.C.pack(torch.from_numpy(wp.rhs)), tol_rel=0.0, max_iter=4, use_graph=graph,
                           project_mean=1, wall_values=wp.gvals())
    want, it, hist, st = wp.P.solve(wp.rhs, tol_rel=0.0, maxit=4, project_mean=True)
    assert info.iterations == it == 4
    np.testing.assert_allclose(info.history(), hist, rtol=1e-9)
    got = wp.C.unpack(phi).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16])
def test_solve_with_wall_values_to_tolerance(wp, prec):
    """To 1e-12 on both sides (FP64 outer loop for every precision): solutions within 1e-10,
    and the GPU solution's residual by the oracle's affine operator below 1e-10 of ||r0||."""
    phi, info = wp.C.solve(wp.C.pack(torch.from_numpy(wp.rhs)), tol_rel=1e-12, max_iter=100, precision=prec,
                           project_mean=1, wall_values=wp.gvals())
    assert info.status == gmg.OK
    want, it, hist, st = wp.P.solve(wp.rhs, tol_rel=1e-12, maxit=100, project_mean=True)
    assert st == O.OK
    got = wp.C.unpack(phi).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    r0 = wp.rhs - wp.P.apply_bc(np.zeros(wp.shape))
    r = wp.rhs - wp.P.apply_bc(got)
    if wp.singular:
        r -= r.mean()
        r0 -= r0.mean()
    assert np.abs(r).max() <= 1e-10 * np.abs(r0).max()


def test_gradients_with_wall_values_match_oracle(wp):
    """Same phi (the oracle's solution with values) and lambda (the oracle's adjoint, the
    homogeneous operator) on both sides: dL/dbeta and dL/dg agree."""
    phi, _, _, st = wp.P.solve(wp.rhs, tol_rel=1e-12, maxit=100, project_mean=True)
    g = phi - wp.target
    if wp.singular:
        g -= g.mean()
    lam, _, _, st2 = wp.P0.solve(g, tol_rel=1e-12, maxit=100)
    assert st == O.OK and st2 == O.OK
    want_b = wp.P.grad_beta(phi, lam, wp.beta)
    got_b = wp.C.unpack(wp.C.beta_grad(wp.C.pack(torch.from_numpy(phi)), wp.C.pack(torch.from_numpy(lam)),
                                       wall_values=wp.gvals())).cpu().numpy()
    assert np.abs(got_b - want_b).max() <= 1e-10 * np.abs(want_b).max()
    got_g = wp.C.wall_values_grad(wp.C.pack(torch.from_numpy(lam)), list(wp.values))
    for f in wp.values:
        want_g = wp.P.grad_wall_values(lam, f)
        assert np.abs(got_g[f].cpu().numpy() - want_g).max() <= 1e-12 * np.abs(want_g).max(), f


def test_autograd_with_wall_values(wp):
    """torch.autograd through the solve with wall values: dL/drhs, dL/dbeta and dL/dg of
    L = 0.5 ||phi - phi_t||^2 equal the oracle's adjoint gradients."""
    from paper_2009_12009_gb300.autograd import Solve

    c = wp.c
    S = Solve(c["n"], bc=(c["lo"], c["hi"]), max_grid_size=c["mgs"], prob_hi=c["L"], a=c["a"], b=c["b"], tol=1e-12)
    if wp.alpha is not None:
        S.ctx.set_alpha(torch.from_numpy(wp.alpha))
    dev = "cuda"
    t_rhs = torch.tensor(wp.rhs, device=dev, requires_grad=True)
    t_beta = torch.tensor(wp.beta, device=dev, requires_grad=True)
    t_vals = {f: torch.tensor(v, device=dev, requires_grad=True) for f, v in wp.values.items()}
    phi = S(t_rhs, t_beta, wall_values=t_vals)
    loss = 0.5 * ((phi - torch.from_numpy(wp.target).to(dev)) ** 2).sum()
    loss.backward()
    ophi, _, _, _ = wp.P.solve(wp.rhs, tol_rel=1e-12, maxit=100, project_mean=True)
    g = ophi - wp.target
    if wp.singular:
        g -= g.mean()
    lam, _, _, _ = wp.P0.solve(g, tol_rel=1e-12, maxit=100)
    sc = np.abs(lam).max()
    assert np.abs(t_rhs.grad.cpu().numpy() - lam).max() <= 1e-8 * sc
    gb = wp.P.grad_beta(ophi, lam, wp.beta)
    assert np.abs(t_beta.grad.cpu().numpy() - gb).max() <= 1e-8 * np.abs(gb).max()
    for f, t in t_vals.items():
        want = wp.P.grad_wall_values(lam, f)
        assert np.abs(t.grad.cpu().numpy() - want).max() <= 1e-8 * np.abs(want).max(), f


def test_linear_solution_with_wall_values_is_exact():
    """phi = c0 + s.x with matching Dirichlet values and Neumann derivatives is the exact
    discrete solution (beta = beta(z), phi independent of z): the GPU reproduces it."""
    n = (32, 16, 24)
    Ls = (1.0, 0.6, 0.6)
    lo, hi = [N_, D_, N_], [D_, N_, N_]
    dom = ((0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1))
    C = gmg.Context(dom, lo, hi, prob_hi=Ls, boxes=I.chop(*dom, 8), stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64)
    rng = np.random.default_rng(12)
    shape = (n[2], n[1], n[0])
    alpha = np.exp(rng.standard_normal(shape))
    beta = np.broadcast_to(np.exp(rng.standard_normal(n[2]))[:, None, None], shape).copy()
    C.set_scalars(1.0, 0.9)
    C.set_alpha(torch.from_numpy(alpha))
    C.set_beta(torch.from_numpy(beta))
    s, c0 = (1.5, -0.7, 0.0), 0.3
    x = [(np.arange(n[d]) + 0.5) * Ls[d] / n[d] for d in range(3)]
    exact = c0 + s[0] * x[0][None, None, :] + s[1] * x[1][None, :, None]
    vals = {}
    for f in range(6):
        d, side = f // 2, f % 2
        bc = (hi if side else lo)[d]
        t1, t2 = [e for e in range(3) if e != d]
        if bc == D_:
            xd = Ls[d] * side
            v = c0 + s[d] * xd + s[t1] * x[t1][None, :] + s[t2] * x[t2][:, None]
        else:
            v = np.full((n[t2], n[t1]), s[d] if side else -s[d])
        vals[f] = torch.from_numpy(np.ascontiguousarray(v))
    phi, info = C.solve(C.pack(torch.from_numpy(alpha * exact)), tol_rel=1e-13, max_iter=100, wall_values=vals)
    assert info.status == gmg.OK
    got = C.unpack(phi).cpu().numpy()
    assert np.abs(got - exact).max() <= 1e-11 * np.abs(exact).max()


def test_wall_values_refused():
    """A periodic face takes no values; multi-problem and two-level contexts take none."""
    cfg = CASES["mixed"]
    n = cfg["n"]
    dom = ((0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1))
    C = gmg.Context(dom, cfg["lo"], cfg["hi"], boxes=I.chop(*dom, 8), stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64)
    C.set_scalars(0.0, 1.0)
    C.set_beta(None)
    rhs = C.field(0)
    with pytest.raises(gmg.GmgError):
        C.wall_values_rhs(rhs, {2: torch.zeros(C.face_shape(2), dtype=torch.float64)})  # y is periodic
    with pytest.raises(ValueError):
        C.wall_values_rhs(rhs, {0: torch.zeros((3, 3), dtype=torch.float64)})  # wrong shape
    probs = [dict(domain=((0, 0, 0), (7, 7, 7)), boxes=I.chop((0, 0, 0), (7, 7, 7), 8), bc_lo=[D_] * 3,
                  bc_hi=[D_] * 3, prob_hi=(1, 1, 1)) for _ in range(2)]
    B = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    B.allocate(gmg.FP64)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.ones(8, 8, 8, dtype=torch.float64)] * 2)
    import ctypes as C_

    v = torch.zeros(64, dtype=torch.float64, device="cuda")
    arr = (C_.c_void_p * 6)()
    arr[0] = v.data_ptr()
    out = B.field(0)
    st = B.L.gmg_wall_values_rhs(B.h, C_.c_void_p(out.data_ptr()), C_.c_void_p(out.data_ptr()), arr)
    assert st == gmg.BAD_INPUT and b"single-problem" in B.L.gmg_last_error(B.h)
