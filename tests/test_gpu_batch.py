"""Batched form: many independent problems of uneven sizes in one context, solved by one
set of launches per V-cycle step, against independent oracle solves of each problem.

Each problem converges on its own schedule; converged problems are masked out of later
V-cycles, so every problem must take exactly the oracle's iteration count and reach its
iterate (1e-10 relative, the FP64 requirement)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_12009_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402

P_, D_ = I.PERIODIC, I.DIRICHLET

# uneven sizes: different depths and bottoms (8^3 aggregation, odd 5-cell bottoms, one
# problem that cannot coarsen at all), one singular periodic problem
SIZES = [(16, 24, 8), (32, 16, 16), (24, 8, 40), (8, 8, 8), (10, 20, 30), (16, 16, 16), (6, 18, 12), (40, 8, 8)]


def batch_problems(periodic_last=True, mgs=8):
    probs = []
    for i, sz in enumerate(SIZES):
        p = I.batch_problem(sz, i, seed=777, max_grid_size=mgs)
        if periodic_last and i == len(SIZES) - 1:
            p["bc_lo"] = [P_] * 3
            p["bc_hi"] = [P_] * 3
            p["rhs"] = p["rhs"] - p["rhs"].mean()
        probs.append(p)
    return probs


@pytest.fixture(scope="module")
def batch():
    probs = batch_problems()
    ctx = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    ctx.allocate(gmg.MIXED_FP32)
    ctx.set_scalars(0.0, 1.0)
    ctx.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    rhs = ctx.pack_all([torch.from_numpy(p["rhs"]) for p in probs])
    oracles = []
    for p in probs:
        P = O.Problem(p["domain"], p["boxes"], p["bc_lo"], p["bc_hi"], (0, 0, 0), p["prob_hi"])
        P.set_coeffs(0.0, 1.0, beta=p["beta"])
        oracles.append(P)
    return probs, ctx, rhs, oracles


def test_batch_hierarchy_is_union_of_problems(batch):
    probs, ctx, rhs, oracles = batch
    for m in range(ctx.nlevels):
        boxes, _ = ctx.level_boxes(m)
        want = []
        for P in oracles:
            if m < P.nlevels:
                want += P.level_boxes(m)
        assert boxes == want


@pytest.mark.parametrize("fused", [1, 0], ids=["fused_coarse", "per_level"])
@pytest.mark.parametrize("graph", [1, 0])
def test_batch_fixed_iterations(batch, graph, fused):
    probs, ctx, rhs, oracles = batch
    phi, infos = ctx.batch_solve(rhs, tol_rel=0.0, max_iter=4, use_graph=graph, fused_coarse=fused)
    for s, (p, P) in enumerate(zip(probs, oracles)):
        want, it, hist, st = P.solve(p["rhs"], tol_rel=0.0, maxit=4)
        got = ctx.unpack_solve(s, phi).cpu().numpy()
        assert infos[s].iterations == it == 4
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max(), s


def test_batch_to_tolerance_matches_independent_solves(batch):
    probs, ctx, rhs, oracles = batch
    phi, infos = ctx.batch_solve(rhs, tol_rel=1e-10, max_iter=200)
    iters = []
    for s, (p, P) in enumerate(zip(probs, oracles)):
        want, it, hist, st = P.solve(p["rhs"], tol_rel=1e-10, maxit=200)
        got = ctx.unpack_solve(s, phi).cpu().numpy()
        assert st == O.OK and infos[s].status == gmg.OK
        assert infos[s].iterations == it, (s, infos[s].iterations, it)
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max(), s
        iters.append(it)
    assert len(set(iters)) > 1  # the problems really converge on different schedules


@pytest.mark.parametrize("prec", [gmg.MIXED_FP32, gmg.MIXED_BF16])
def test_batch_mixed_precision(batch, prec):
    probs, ctx, rhs, oracles = batch
    phi, infos = ctx.batch_solve(rhs, tol_rel=1e-10, max_iter=200, precision=prec)
    for s, (p, P) in enumerate(zip(probs, oracles)):
        assert infos[s].status == gmg.OK
        got = ctx.unpack_solve(s, phi).cpu().numpy()
        r = (p["rhs"] - (p["rhs"].mean() if s == len(probs) - 1 else 0.0)) - P.apply(got)
        assert np.abs(r).max() <= 1.01e-10 * np.abs(p["rhs"]).max(), s


def test_batch_settled_residuals_change_only_rounding(batch):
    """The settled-colour residuals (the default) against computing every residual: every
    problem takes the same iterations to 1e-10 and reaches the same iterate to 1e-12."""
    probs, ctx, rhs, oracles = batch
    p1, i1 = ctx.batch_solve(rhs, tol_rel=1e-10, settled_zero=1)
    a1 = [ctx.unpack_solve(s, p1).cpu().numpy() for s in range(len(probs))]
    p0, i0 = ctx.batch_solve(rhs, tol_rel=1e-10, settled_zero=0)
    for s in range(len(probs)):
        a0 = ctx.unpack_solve(s, p0).cpu().numpy()
        assert i1[s].iterations == i0[s].iterations
        assert np.abs(a1[s] - a0).max() <= 1e-12 * np.abs(a0).max()
