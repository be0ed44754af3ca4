"""Wavefront red-black sweeps (one launch per Gauss-Seidel sweep, wave_sweep = 1) against one
launch per colour (wave_sweep = 0), bit for bit.

The wavefront kernel marches each tile (a band of rows of one box) through its planes, red
cells of a plane then black cells of the plane before, and waits for the tiles beside it to
report a plane's red cells before that plane's black cells; every value is computed from the
operands of the two-pass sweep in the same order.  The tests compare V-cycles and solves of
the two paths with torch.equal (same bits) on the shared parity layouts (ragged tails,
aggregation, periodic and Neumann singular problems, walls of every kind, anisotropic h, an
a*alpha term), on larger levels with several tiles per box, in the three element types,
with CUDA graphs and direct launches, several sweep counts, the symmetric V-cycle, the
per-level coarse end on and off, batched problems with a per-problem active mask, and at the
full 256^3 size of the abec256 workload.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402
from paper_2009_12009_gb300 import inputs as I  # noqa: E402

from . import cases  # noqa: E402

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN
DTS = [gmg.DT_F64, gmg.DT_F32, gmg.DT_BF16]


def _big(name):
    rng = np.random.default_rng({"dir64": 401, "per64": 402, "walls": 403, "tails": 404}[name])
    if name == "dir64":  # 8 boxes of 32^3: 8 rows per tile, 4 tiles per box
        n, bc_lo, bc_hi, a, b, mgs = (64, 64, 64), [D_] * 3, [D_] * 3, 0.0, 1.0, 32
    elif name == "per64":  # singular, periodic in every direction, boxes of 16 (4 around each axis)
        n, bc_lo, bc_hi, a, b, mgs = (64, 64, 64), [P_] * 3, [P_] * 3, 0.0, 1.0, 16
    elif name == "walls":  # Neumann / Dirichlet per side, y periodic, a*alpha, boxes of 16
        n, bc_lo, bc_hi, a, b, mgs = (48, 64, 80), [N_, P_, D_], [D_, P_, N_], 0.7, 1.3, 16
    else:  # boxes of 32 with ragged tails (8- and 6-cell boxes on the high sides), uneven z
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
    C.set_beta(None if cfg["beta"] is None else torch.from_numpy(cfg["beta"]))
    return C


CASES = [("small", n) for n in cases.NAMES] + [("big", n) for n in ("dir64", "per64", "walls", "tails")]


@pytest.fixture(scope="module", params=CASES, ids=[n for _, n in CASES])
def ctx(request):
    kind, name = request.param
    cfg = cases.make(name) if kind == "small" else _big(name)
    return cfg, _ctx(cfg)


def _rhs(cfg):
    r = cfg["rhs"]
    singular = D_ not in cfg["bc_lo"] + cfg["bc_hi"] and cfg["a"] == 0.0
    return r - r.mean() if singular else r


def test_wave_launches_cover_two_passes(ctx):
    """Where level 0 has wavefront tables, every profiled level-0 smoother launch of a solve
    covers a whole sweep (two colour passes) and the solve launches fewer kernels."""
    cfg, C = ctx
    ppt, T = C.wave_tiles(0)
    rhs = C.pack(torch.from_numpy(_rhs(cfg)))
    _, i1 = C.solve(rhs, tol_rel=0.0, max_iter=2, wave_sweep=1, profile=1, project_mean=1)
    _, i0 = C.solve(rhs, tol_rel=0.0, max_iter=2, wave_sweep=0, profile=1, project_mean=1)
    if len(T) == 0 or C.nlevels == 1:
        pytest.skip("no wavefront tables on level 0 (a bottom-only or unsupported layout)")
    assert ppt in (1, 2, 4)
    assert i1.smooth0_passes == 2 * i1.smooth0_launches
    assert i1.kernel_launches < i0.kernel_launches


@pytest.mark.parametrize("dt", DTS)
def test_wave_vcycle_is_bitwise_two_pass(ctx, dt):
    cfg, C = ctx
    rb = C.pack(torch.from_numpy(_rhs(cfg)), 0, dt)
    e1 = C.unpack(C.vcycle(rb, dt, wave_sweep=1), 0, dt)
    e0 = C.unpack(C.vcycle(rb, dt, wave_sweep=0), 0, dt)
    assert torch.equal(e1, e0)


@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16])
@pytest.mark.parametrize("graph", [1, 0])
def test_wave_solve_is_bitwise_two_pass(ctx, prec, graph):
    """Whole solves (the first pre-smoothing sweep from a zero correction in one launch, the
    correction update fused into the last post-smoothing sweep, CUDA-graph replay or direct
    launches): the same iterates and residual histories."""
    cfg, C = ctx
    rhs = C.pack(torch.from_numpy(_rhs(cfg)))
    p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=3, precision=prec, use_graph=graph, wave_sweep=1, project_mean=1)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=3, precision=prec, use_graph=graph, wave_sweep=0, project_mean=1)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.history() == i0.history()


@pytest.mark.parametrize("nu", [(3, 3), (1, 4), (4, 1), (2, 0)], ids=["nu33", "nu14", "nu41", "nu20"])
@pytest.mark.parametrize("fc", [1, 0], ids=["tail", "levels"])
def test_wave_sweep_counts_and_coarse_end(ctx, nu, fc):
    cfg, C = ctx
    rhs = C.pack(torch.from_numpy(_rhs(cfg)))
    kw = dict(tol_rel=0.0, max_iter=2, nu1=nu[0], nu2=nu[1], fused_coarse=fc, project_mean=1)
    p1, i1 = C.solve(rhs, wave_sweep=1, **kw)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, wave_sweep=0, **kw)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.history() == i0.history()


def test_wave_symmetric_vcycle_and_krylov():
    """The symmetric V-cycle (post-smoothing black first keeps one launch per colour, the
    pre-smoothing runs as wavefronts) and the Krylov top levels that use the V-cycle."""
    cfg = _big("dir64")
    C = _ctx(cfg, krylov=True)
    rb = C.pack(torch.from_numpy(cfg["rhs"]))
    e1 = C.unpack(C.vcycle(rb, gmg.DT_F64, wave_sweep=1, post_reverse=1))
    e0 = C.unpack(C.vcycle(rb, gmg.DT_F64, wave_sweep=0, post_reverse=1))
    assert torch.equal(e1, e0)
    for kry in (1, 2):
        p1, i1 = C.solve(rb, tol_rel=0.0, max_iter=3, krylov=kry, wave_sweep=1)
        a1 = C.unpack(p1).clone()
        p0, i0 = C.solve(rb, tol_rel=0.0, max_iter=3, krylov=kry, wave_sweep=0)
        assert torch.equal(a1, C.unpack(p0)), kry
        assert i1.history() == i0.history()


# (the periodic problem has an even number of boxes along z: marching directions alternate)
SIZES = [(48, 40, 32), (64, 32, 48), (32, 32, 32), (40, 56, 24), (16, 64, 32), (48, 48, 64)]


def test_wave_batched_with_active_mask():
    """Six problems of uneven sizes in one batched context, the last periodic and singular:
    each converges on its own schedule, converged problems are masked out of later V-cycles
    (their tiles are skipped), and every problem's iterate and iteration count are those of
    the two-pass sweeps."""
    probs = []
    for i, sz in enumerate(SIZES):
        p = I.batch_problem(sz, i, seed=4343, max_grid_size=16)
        if i == len(SIZES) - 1:
            p["bc_lo"] = [P_] * 3
            p["bc_hi"] = [P_] * 3
            p["rhs"] = p["rhs"] - p["rhs"].mean()
        probs.append(p)
    B = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    B.allocate(gmg.MIXED_FP32)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    _, T = B.wave_tiles(0)
    assert len(T) > 0
    rhs = B.pack_all([torch.from_numpy(p["rhs"]) for p in probs])
    for prec in (gmg.FP64, gmg.MIXED_FP32):
        p1, i1 = B.batch_solve(rhs, tol_rel=1e-10, precision=prec, wave_sweep=1)
        a1 = [B.unpack_solve(s, p1).clone() for s in range(len(probs))]
        p0, i0 = B.batch_solve(rhs, tol_rel=1e-10, precision=prec, wave_sweep=0)
        its = []
        for s in range(len(probs)):
            assert i1[s].status == i0[s].status == gmg.OK
            assert i1[s].iterations == i0[s].iterations
            assert torch.equal(a1[s], B.unpack_solve(s, p0)), (prec, s)
            its.append(i0[s].iterations)
        assert len(set(its)) > 1  # the mask really changes between V-cycles


def test_wave_full_size_abec256():
    """The abec256 workload (256^3, 64 boxes of 64^3, Dirichlet walls; level 0 in 1024 tiles of
    4 rows): two FP64 and two mixed FP32 iterations, the same bits as one launch per colour."""
    cfg = I.abec256()
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"],
                    stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.MIXED_FP32)
    C.set_scalars(cfg["a"], cfg["b"])
    C.set_beta(torch.from_numpy(cfg["beta"]))
    ppt, T = C.wave_tiles(0)
    assert len(T) == 1024 and ppt == 1
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    for prec in (gmg.FP64, gmg.MIXED_FP32):
        p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=2, precision=prec, wave_sweep=1)
        a1 = C.unpack(p1).clone()
        p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=2, precision=prec, wave_sweep=0)
        assert torch.equal(a1, C.unpack(p0)), prec
        assert i1.history() == i0.history()
