"""Bottom solves on a second stream in batched contexts (fork_bottoms = 1) against one stream
(fork_bottoms = 0).

In a batched context the problems reach their bottom levels (Sec. "Linear Solvers": the
Krylov bottom solve of the multigrid hierarchy) at different depths.  The bottom solves of
a level then run on the context's second stream while the other problems go on to coarser
levels, and are joined before the interpolation from that level reads them.  Each kernel
computes what it computes on one stream, on disjoint cells, so every problem's iterate,
residual history and iteration count must be the same bits; checked for the per-level and
the fused coarse end, FP64 and mixed FP32, CUDA graphs and direct launches, with the
per-problem active mask changing between V-cycles.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402
from paper_2009_12009_gb300 import inputs as I  # noqa: E402

SIZES = [(48, 40, 32), (64, 32, 48), (32, 32, 32), (40, 56, 24), (16, 64, 32), (48, 48, 64), (96, 80, 64)]


@pytest.fixture(scope="module")
def batch():
    probs = [I.batch_problem(sz, i, seed=7171, max_grid_size=16) for i, sz in enumerate(SIZES)]
    B = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    B.allocate(gmg.MIXED_FP32)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    return probs, B


@pytest.mark.parametrize("fc", [0, 1], ids=["levels", "tail"])
@pytest.mark.parametrize("graph", [1, 0])
@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32])
def test_forked_bottoms_same_bits(batch, fc, graph, prec):
    probs, B = batch
    rhs = B.pack_all([torch.from_numpy(p["rhs"]) for p in probs])
    kw = dict(tol_rel=1e-10, precision=prec, fused_coarse=fc, use_graph=graph)
    p1, i1 = B.batch_solve(rhs, fork_bottoms=1, **kw)
    a1 = [B.unpack_solve(s, p1).clone() for s in range(len(probs))]
    p0, i0 = B.batch_solve(rhs, fork_bottoms=0, **kw)
    its = []
    for s in range(len(probs)):
        assert i1[s].status == i0[s].status == gmg.OK
        assert i1[s].iterations == i0[s].iterations
        assert i1[s].history() == i0[s].history()
        assert torch.equal(a1[s], B.unpack_solve(s, p0)), s
        its.append(i0[s].iterations)
    assert len(set(its)) > 1

