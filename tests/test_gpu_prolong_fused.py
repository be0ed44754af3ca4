"""The interpolation of the coarse correction fused into the first post-smoothing red pass
(fuse_prolongation = 2: wherever it applies) against the separate interpolation launch (0).

In the V-cycle of Sec. "Linear Solvers" the coarse correction is interpolated (piecewise
constant, Sec. "Operations between levels") and added before post-smoothing; the first red
pass then reads each black neighbour as that addition leaves it -- its value plus its
parent's coarse value -- and the black cells, rewritten by the black pass without being read,
are not touched.  The iterates must be those of the separate passes bit for bit, in FP64 and
both mixed forms, with ghost push and with the exchange on the fine levels, with the scalar
and the vector smoothers on the other passes, with the coarse end fused or run level by
level, for single problems (walls of every linear kind, periodic images, aggregated coarse
boxes) and for batched problems with the active mask; the fused form launches fewer kernels.
Where the fine level's red pass cannot take the interpolation (the exchange on the fine level,
or an FP64 finest level whose pass is bound by the FP64 pipe), the coarse level's last
post-smoothing pass adds its final values to its children instead; those cases are covered
too (the exchange cases, and abec256 at full size).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402
from paper_2009_12009_gb300 import inputs as I  # noqa: E402

from . import cases  # noqa: E402

P_, D_ = I.PERIODIC, I.DIRICHLET


def _ctx(cfg):
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], prob_hi=cfg.get("prob_hi", (1.0, 1.0, 1.0)),
                    boxes=cfg["boxes"], stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.MIXED_FP32)
    C.set_scalars(cfg["a"], cfg["b"])
    if cfg.get("alpha") is not None:
        C.set_alpha(torch.from_numpy(cfg["alpha"]))
    C.set_beta(None if cfg["beta"] is None else torch.from_numpy(cfg["beta"]))
    return C


def _make(name):
    if name == "abec128_64":
        return I.abec(128, 32, 4712, name=name)
    if name == "per64":
        return I.abec(64, 16, 4713, bc=P_, name=name)
    return cases.make(name)


def _rhs(cfg):
    r = cfg["rhs"]
    singular = D_ not in list(cfg["bc_lo"]) + list(cfg["bc_hi"]) and cfg["a"] == 0.0
    return r - r.mean() if singular else r


NAMES = ["uneven", "periodic", "helmholtz", "poisson32", "neumann", "mixedwalls", "abec128_64", "per64"]


@pytest.fixture(scope="module", params=NAMES)
def ctx(request):
    cfg = _make(request.param)
    return cfg, _ctx(cfg)


@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16])
@pytest.mark.parametrize("push", [0, 1], ids=["exchange", "push"])
@pytest.mark.parametrize("fc", [1, 0], ids=["tail", "levels"])
def test_fused_prolongation_is_exact(ctx, prec, push, fc):
    cfg, C = ctx
    rhs = C.pack(torch.from_numpy(_rhs(cfg)))
    kw = dict(tol_rel=0.0, max_iter=3, precision=prec, ghost_push=push, fused_coarse=fc, project_mean=1)
    p1, i1 = C.solve(rhs, fuse_prolongation=2, **kw)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, fuse_prolongation=0, **kw)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.history() == i0.history()
    if C.nlevels > 2 and fc == 0 and push == 1:  # (the coarse level's ghosts must be pushed)
        assert i1.kernel_launches < i0.kernel_launches


@pytest.mark.parametrize("dt", [gmg.DT_F64, gmg.DT_F32, gmg.DT_BF16])
@pytest.mark.parametrize("vec", [0, 1], ids=["scalar", "vector"])
def test_fused_prolongation_vcycle(ctx, dt, vec):
    """One V-cycle from the API (gmg_vcycle), scalar or vector smoothers on every level."""
    cfg, C = ctx
    rb = C.pack(torch.from_numpy(_rhs(cfg)), 0, dt)
    e1 = C.unpack(C.vcycle(rb, dt, fuse_prolongation=2, vector_smooth=vec, fused_coarse=0), 0, dt).clone()
    e0 = C.unpack(C.vcycle(rb, dt, fuse_prolongation=0, vector_smooth=vec, fused_coarse=0), 0, dt)
    assert torch.equal(e1, e0)


@pytest.mark.parametrize("kw", [dict(nu1=1, nu2=2), dict(nu1=0, nu2=3), dict(post_reverse=1), dict(krylov=1),
                                dict(krylov=2)], ids=["nu12", "nu03", "symmetric", "bicgstab", "cg"])
def test_fused_prolongation_cycle_variants(kw):
    cfg = _make("abec128_64")
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"],
                    stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64, krylov=True)
    C.set_scalars(cfg["a"], cfg["b"])
    C.set_beta(torch.from_numpy(cfg["beta"]))
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=3, fuse_prolongation=2, fused_coarse=0, **kw)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=3, fuse_prolongation=0, fused_coarse=0, **kw)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.history() == i0.history()


SIZES = [(48, 40, 32), (64, 32, 48), (32, 32, 32), (40, 56, 24), (16, 64, 32), (48, 48, 64)]


@pytest.mark.parametrize("fc", [1, 0], ids=["tail", "levels"])
def test_fused_prolongation_batched(fc):
    """Batched problems of uneven sizes (their bottoms and tails on different levels) with the
    active mask: every problem's iterate and iteration count as with the separate passes."""
    probs = [I.batch_problem(sz, i, seed=6262, max_grid_size=16) for i, sz in enumerate(SIZES)]
    B = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    B.allocate(gmg.MIXED_FP32)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    rhs = B.pack_all([torch.from_numpy(p["rhs"]) for p in probs])
    for prec in (gmg.FP64, gmg.MIXED_FP32):
        p1, i1 = B.batch_solve(rhs, tol_rel=1e-10, precision=prec, fused_coarse=fc, fuse_prolongation=2)
        a1 = [B.unpack_solve(s, p1).clone() for s in range(len(probs))]
        p0, i0 = B.batch_solve(rhs, tol_rel=1e-10, precision=prec, fused_coarse=fc, fuse_prolongation=0)
        its = []
        for s in range(len(probs)):
            assert i1[s].status == i0[s].status == gmg.OK
            assert i1[s].iterations == i0[s].iterations
            assert torch.equal(a1[s], B.unpack_solve(s, p0)), (prec, s)
            its.append(i0[s].iterations)
        assert len(set(its)) > 1


def test_fused_prolongation_full_size_abec256():
    """abec256 at full size: the interpolation into the finest level done by level 1's last
    post-smoothing pass (every level-1 box has one exact child) -- FP64 with push
    (fuse_prolongation = 2: the default leaves that FP64-bound case out), float with the
    exchange on the finest level (the default) -- and the default's FP64 choice.  Two
    iterations, the same bits as no fusion."""
    cfg = I.abec256()
    C = _ctx(cfg)
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    for prec, push, fuse in ((gmg.FP64, 0, 2), (gmg.FP64, 1, 1), (gmg.MIXED_FP32, 0, 1), (gmg.MIXED_BF16, 2, 1)):
        kw = dict(tol_rel=0.0, max_iter=2, precision=prec, ghost_push=push)
        p1, i1 = C.solve(rhs, fuse_prolongation=fuse, **kw)
        a1 = C.unpack(p1).clone()
        p0, i0 = C.solve(rhs, fuse_prolongation=0, **kw)
        assert torch.equal(a1, C.unpack(p0)), prec
        assert i1.history() == i0.history()
        assert i1.kernel_launches < i0.kernel_launches
