"""Dataflow red-black sweeps (one launch per smoothing step, fused_sweep = 1) against one
launch per colour (fused_sweep = 0), bit for bit.

The flow kernel runs every colour phase of a smoothing step in one launch; an item waits
until the previous phase has finished on the slabs it reads, so each update sees the
operands of the two-pass sweep.  Every test here compares whole V-cycles and solves of the
two paths with torch.equal (same bits), on levels large enough to get flow tables (at least
2^17 smoothed cells): walls of every kind, periodic z (the slab dependencies wrap around),
several problems of uneven sizes with a per-problem active mask, the symmetric V-cycle,
more phases than one launch holds, and the three element types.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402
from paper_2009_12009_gb300 import inputs as I  # noqa: E402

DTS = [gmg.DT_F64, gmg.DT_F32, gmg.DT_BF16]
P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def _case(name):
    rng = np.random.default_rng({"dir64": 301, "per64": 302, "walls": 303, "tails": 304}[name])
    if name == "dir64":  # 64^3, 8 boxes of 32: the level-0 sweep of the abec recipe
        n, bc_lo, bc_hi, a, b, mgs = (64, 64, 64), [D_] * 3, [D_] * 3, 0.0, 1.0, 32
    elif name == "per64":  # singular, periodic in every direction: z-slab dependencies wrap
        n, bc_lo, bc_hi, a, b, mgs = (64, 64, 64), [P_] * 3, [P_] * 3, 0.0, 1.0, 32
    elif name == "walls":  # Neumann / Dirichlet per side, y periodic, a*alpha, boxes of 16
        n, bc_lo, bc_hi, a, b, mgs = (48, 64, 80), [N_, P_, D_], [D_, P_, N_], 0.7, 1.3, 16
    else:  # boxes of 32 with ragged tails (8- and 6-cell boxes on the high sides)
        n, bc_lo, bc_hi, a, b, mgs = (72, 70, 40), [D_] * 3, [D_] * 3, 0.0, 1.0, 32
    shape = (n[2], n[1], n[0])
    dom = ((0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1))
    beta = I.lognormal_beta(rng, shape, periodic=bc_lo[0] == P_ and bc_lo[1] == P_)
    alpha = np.exp(rng.standard_normal(shape)) if a else None
    rhs = rng.standard_normal(shape)
    if D_ not in bc_lo + bc_hi and a == 0.0:
        rhs -= rhs.mean()
    return dict(domain=dom, boxes=I.chop(*dom, mgs), bc_lo=bc_lo, bc_hi=bc_hi, a=a, b=b, alpha=alpha, beta=beta,
                rhs=rhs, prob_hi=(n[0] / 64, n[1] / 64, n[2] / 64))


def _ctx(cfg, krylov=False):
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], prob_hi=cfg["prob_hi"], boxes=cfg["boxes"],
                    stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.MIXED_FP32, krylov=krylov)
    C.set_scalars(cfg["a"], cfg["b"])
    if cfg["alpha"] is not None:
        C.set_alpha(torch.from_numpy(cfg["alpha"]))
    C.set_beta(torch.from_numpy(cfg["beta"]))
    return C


CASES = ["dir64", "per64", "walls", "tails"]


@pytest.fixture(scope="module", params=CASES)
def ctx(request):
    cfg = _case(request.param)
    return cfg, _ctx(cfg)


def test_flow_tables_exist(ctx):
    """Level 0 of every case is large enough to run the dataflow sweep: the profiled
    smoother launches of a flow solve cover several colour passes each."""
    cfg, C = ctx
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    _, i1 = C.solve(rhs, tol_rel=0.0, max_iter=2, fused_sweep=1, wave_sweep=0, profile=1, project_mean=1)
    _, i0 = C.solve(rhs, tol_rel=0.0, max_iter=2, fused_sweep=0, wave_sweep=0, profile=1, project_mean=1)
    assert i1.smooth0_passes == i0.smooth0_passes == i0.smooth0_launches
    assert i1.smooth0_launches < i1.smooth0_passes
    assert i1.kernel_launches < i0.kernel_launches


@pytest.mark.parametrize("dt", DTS)
def test_flow_vcycle_is_bitwise_two_pass(ctx, dt):
    cfg, C = ctx
    r = cfg["rhs"] - (cfg["rhs"].mean() if cfg["bc_lo"] == [P_] * 3 else 0.0)
    rb = C.pack(torch.from_numpy(r), 0, dt)
    e1 = C.unpack(C.vcycle(rb, dt, fused_sweep=1, wave_sweep=0), 0, dt)
    e0 = C.unpack(C.vcycle(rb, dt, fused_sweep=0, wave_sweep=0), 0, dt)
    assert torch.equal(e1, e0)


@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16])
@pytest.mark.parametrize("graph", [1, 0])
def test_flow_solve_is_bitwise_two_pass(ctx, prec, graph):
    """Whole solves (the outer residual's first red half-sweep, the fused correction update in
    the last phase, CUDA-graph replay or direct launches): the same iterates and histories."""
    cfg, C = ctx
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=3, precision=prec, use_graph=graph, fused_sweep=1, wave_sweep=0, project_mean=1)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=3, precision=prec, use_graph=graph, fused_sweep=0, wave_sweep=0, project_mean=1)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.history() == i0.history()


@pytest.mark.parametrize("nu", [(3, 3), (1, 4), (4, 0)], ids=["nu33", "nu14", "nu40"])
def test_flow_more_phases_than_one_launch(ctx, nu):
    """Smoothing steps of 5 to 8 colour passes run as two launches (at most 4 passes each)."""
    cfg, C = ctx
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    kw = dict(tol_rel=0.0, max_iter=2, nu1=nu[0], nu2=nu[1], project_mean=1)
    p1, _ = C.solve(rhs, fused_sweep=1, wave_sweep=0, **kw)
    a1 = C.unpack(p1).clone()
    p0, _ = C.solve(rhs, fused_sweep=0, wave_sweep=0, **kw)
    assert torch.equal(a1, C.unpack(p0))


def test_flow_symmetric_vcycle_and_cg():
    """Post-smoothing black before red (the symmetric V-cycle) and the conjugate-gradient top
    level that uses it."""
    cfg = _case("dir64")
    C = _ctx(cfg, krylov=True)
    rb = C.pack(torch.from_numpy(cfg["rhs"]))
    e1 = C.unpack(C.vcycle(rb, gmg.DT_F64, fused_sweep=1, wave_sweep=0, post_reverse=1))
    e0 = C.unpack(C.vcycle(rb, gmg.DT_F64, fused_sweep=0, wave_sweep=0, post_reverse=1))
    assert torch.equal(e1, e0)
    for kry in (1, 2):
        p1, i1 = C.solve(rb, tol_rel=0.0, max_iter=3, krylov=kry, fused_sweep=1, wave_sweep=0)
        a1 = C.unpack(p1).clone()
        p0, i0 = C.solve(rb, tol_rel=0.0, max_iter=3, krylov=kry, fused_sweep=0, wave_sweep=0)
        assert torch.equal(a1, C.unpack(p0)), kry
        assert i1.history() == i0.history()


SIZES = [(48, 40, 32), (64, 32, 48), (32, 32, 32), (40, 56, 24), (16, 64, 32), (48, 48, 48)]


def test_flow_batched_with_active_mask():
    """Six problems of uneven sizes in one batched context (level 0: 389,120 cells; the last
    one periodic and singular): each converges on its own schedule, converged problems are
    masked out of later V-cycles, and every problem's iterate and iteration count are those of
    the two-pass sweeps."""
    probs = []
    for i, sz in enumerate(SIZES):
        p = I.batch_problem(sz, i, seed=4242, max_grid_size=16)
        if i == len(SIZES) - 1:
            p["bc_lo"] = [P_] * 3
            p["bc_hi"] = [P_] * 3
            p["rhs"] = p["rhs"] - p["rhs"].mean()
        probs.append(p)
    B = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    B.allocate(gmg.MIXED_FP32)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    rhs = B.pack_all([torch.from_numpy(p["rhs"]) for p in probs])
    for prec in (gmg.FP64, gmg.MIXED_FP32):
        p1, i1 = B.batch_solve(rhs, tol_rel=1e-10, precision=prec, fused_sweep=1, wave_sweep=0)
        a1 = [B.unpack_solve(s, p1).clone() for s in range(len(probs))]
        p0, i0 = B.batch_solve(rhs, tol_rel=1e-10, precision=prec, fused_sweep=0, wave_sweep=0)
        its = []
        for s in range(len(probs)):
            assert i1[s].status == i0[s].status == gmg.OK
            assert i1[s].iterations == i0[s].iterations
            assert torch.equal(a1[s], B.unpack_solve(s, p0)), (prec, s)
            its.append(i0[s].iterations)
        assert len(set(its)) > 1  # the mask really changes between V-cycles
