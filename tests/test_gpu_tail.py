"""The shared-memory coarse end (tail_dense = 1) against the global-memory one (tail_dense = 0),
bit for bit.

With fused_coarse, one thread block per problem runs every V-cycle step of its coarse levels
(Sec. "Linear Solvers": smoothing, residual restriction, the Krylov bottom solve,
interpolation).  The dense form loads each of those levels once into shared memory as one
padded array over the problem's domain and runs the steps there; per cell it computes what
the global-memory form computes, in the same order, so V-cycles and whole solves must give
the same bits.  Covered: the shared parity layouts (ragged tails, aggregation, periodic and
Neumann singular problems, walls of every kind, anisotropic h, an a*alpha term), the abec
layouts whose coarse levels hold many 2^3 boxes, the three element types, CUDA graphs and
direct launches, sweep counts, the symmetric V-cycle and the conjugate-gradient bottom, the
Krylov top levels, batched problems of uneven sizes with a per-problem active mask, a tail
that is its 7^3 bottom alone (solved by the block-wide BiCGStab), and the abec256 workload at
full size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402
from paper_2009_12009_gb300 import inputs as I  # noqa: E402

from . import cases  # noqa: E402

P_, D_ = I.PERIODIC, I.DIRICHLET
DTS = [gmg.DT_F64, gmg.DT_F32, gmg.DT_BF16]


def _ctx(cfg, krylov=False):
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], prob_hi=cfg.get("prob_hi", (1.0, 1.0, 1.0)),
                    boxes=cfg["boxes"], stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.MIXED_FP32, krylov=krylov)
    C.set_scalars(cfg["a"], cfg["b"])
    if cfg.get("alpha") is not None:
        C.set_alpha(torch.from_numpy(cfg["alpha"]))
    C.set_beta(None if cfg["beta"] is None else torch.from_numpy(cfg["beta"]))
    return C


def _rhs(cfg):
    r = cfg["rhs"]
    singular = D_ not in list(cfg["bc_lo"]) + list(cfg["bc_hi"]) and cfg["a"] == 0.0
    return r - r.mean() if singular else r


def _make(name):
    if name == "abec64_8":  # 64^3 in 8 boxes of 32^3: the tail starts on 8^3 (one box per level)
        return I.abec(64, 32, 4601, name=name)
    if name == "abec128_64":  # 64 boxes of 32^3: the tail starts on 8^3 held in 64 boxes of 2^3
        return I.abec(128, 32, 4602, name=name)
    if name == "per128":  # singular periodic problem, 64 boxes
        return I.abec(128, 32, 4603, bc=P_, name=name)
    if name == "abec28":  # the tail is the 7^3 bottom alone (343 cells: the block-wide bottom solve)
        return I.abec(28, 16, 4604, name=name)
    return cases.make(name)


NAMES = [n for n in cases.NAMES if n != "oddlo"] + ["abec64_8", "abec128_64", "per128", "abec28"]


@pytest.fixture(scope="module", params=NAMES)
def ctx(request):
    cfg = _make(request.param)
    return cfg, _ctx(cfg)


def test_dense_plan_covers_the_layout(ctx):
    """Every tail of these layouts has its dense form (so the comparisons below compare two
    different kernels)."""
    cfg, C = ctx
    plans = [C.tail_plan(m, dt) for m in range(C.nlevels) for dt in DTS]
    assert any(n > 0 for n, _ in plans)
    assert all(b > 0 for n, b in plans if n > 0)


@pytest.mark.parametrize("dt", DTS)
def test_dense_vcycle_is_bitwise(ctx, dt):
    cfg, C = ctx
    rb = C.pack(torch.from_numpy(_rhs(cfg)), 0, dt)
    e1 = C.unpack(C.vcycle(rb, dt, fused_coarse=1, tail_dense=1), 0, dt).clone()
    e0 = C.unpack(C.vcycle(rb, dt, fused_coarse=1, tail_dense=0), 0, dt)
    assert torch.equal(e1, e0)


@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16])
@pytest.mark.parametrize("graph", [1, 0])
def test_dense_solve_is_bitwise(ctx, prec, graph):
    """Whole solves (graph replay or direct launches): the same iterates, residual histories
    and bottom iteration counts."""
    cfg, C = ctx
    rhs = C.pack(torch.from_numpy(_rhs(cfg)))
    kw = dict(tol_rel=0.0, max_iter=3, precision=prec, use_graph=graph, fused_coarse=1, project_mean=1)
    p1, i1 = C.solve(rhs, tail_dense=1, **kw)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, tail_dense=0, **kw)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.history() == i0.history()
    assert i1.bottom_iters == i0.bottom_iters


@pytest.mark.parametrize("kw", [dict(nu1=1, nu2=4), dict(nu1=3, nu2=0), dict(post_reverse=1),
                                dict(bottom_solver=1, post_reverse=1), dict(bottom_tol=1e-8)],
                         ids=["nu14", "nu30", "symmetric", "cg_bottom", "tight_bottom"])
def test_dense_cycle_variants(ctx, kw):
    cfg, C = ctx
    rhs = C.pack(torch.from_numpy(_rhs(cfg)))
    p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=2, fused_coarse=1, tail_dense=1, project_mean=1, **kw)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=2, fused_coarse=1, tail_dense=0, project_mean=1, **kw)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.history() == i0.history()


def test_dense_krylov_top_levels():
    cfg = _make("abec64_8")
    C = _ctx(cfg, krylov=True)
    rb = C.pack(torch.from_numpy(cfg["rhs"]))
    for kry in (1, 2):
        p1, i1 = C.solve(rb, tol_rel=0.0, max_iter=3, krylov=kry, fused_coarse=1, tail_dense=1)
        a1 = C.unpack(p1).clone()
        p0, i0 = C.solve(rb, tol_rel=0.0, max_iter=3, krylov=kry, fused_coarse=1, tail_dense=0)
        assert torch.equal(a1, C.unpack(p0)), kry
        assert i1.history() == i0.history()


SIZES = [(48, 40, 32), (64, 32, 48), (32, 32, 32), (40, 56, 24), (16, 64, 32), (48, 48, 64)]


def test_dense_batched_with_active_mask():
    """Six problems of uneven sizes in one batched context, the last periodic and singular:
    one block per problem, each with its own levels in shared memory; converged problems are
    masked out of later V-cycles, and every problem's iterate and iteration count are those of
    the global-memory coarse end."""
    probs = []
    for i, sz in enumerate(SIZES):
        p = I.batch_problem(sz, i, seed=5151, max_grid_size=16)
        if i == len(SIZES) - 1:
            p["bc_lo"] = [P_] * 3
            p["bc_hi"] = [P_] * 3
            p["rhs"] = p["rhs"] - p["rhs"].mean()
        probs.append(p)
    B = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    B.allocate(gmg.MIXED_FP32)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    plans = [B.tail_plan(m) for m in range(B.nlevels)]
    assert sum(n for n, _ in plans) == len(SIZES) and all(b > 0 for n, b in plans if n > 0)
    rhs = B.pack_all([torch.from_numpy(p["rhs"]) for p in probs])
    for prec in (gmg.FP64, gmg.MIXED_FP32):
        p1, i1 = B.batch_solve(rhs, tol_rel=1e-10, precision=prec, fused_coarse=1, tail_dense=1)
        a1 = [B.unpack_solve(s, p1).clone() for s in range(len(probs))]
        p0, i0 = B.batch_solve(rhs, tol_rel=1e-10, precision=prec, fused_coarse=1, tail_dense=0)
        its = []
        for s in range(len(probs)):
            assert i1[s].status == i0[s].status == gmg.OK
            assert i1[s].iterations == i0[s].iterations
            assert torch.equal(a1[s], B.unpack_solve(s, p0)), (prec, s)
            its.append(i0[s].iterations)
        assert len(set(its)) > 1  # the mask really changes between V-cycles


def test_dense_full_size_abec256():
    """The abec256 workload (256^3, 64 boxes of 64^3; the tail starts on 8^3 in 64 boxes of
    2^3): two FP64 and two mixed FP32 iterations, the same bits as the global-memory form."""
    cfg = I.abec256()
    C = _ctx(cfg)
    assert C.tail_plan(5) == (1, 69120)
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    for prec in (gmg.FP64, gmg.MIXED_FP32):
        p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=2, precision=prec, fused_coarse=1, tail_dense=1)
        a1 = C.unpack(p1).clone()
        p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=2, precision=prec, fused_coarse=1, tail_dense=0)
        assert torch.equal(a1, C.unpack(p0)), prec
        assert i1.history() == i0.history()
