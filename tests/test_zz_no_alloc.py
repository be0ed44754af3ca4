"""The allocation-free box solve against the workspace-based bottom solve and the oracle.

gmg_box_bicgstab_noalloc serves callers that cannot allocate device memory when they
solve (an operator handed only its input and output tensors, code running under CUDA
graph capture, hosts that forbid allocation after start-up): it takes dense device
arrays and keeps its scratch in a static device array of the library.  Here it must give
the answer of gmg_bottom_solve -- the same BiCGStab on the same box problem, with the
context's workspace as scratch -- within the bottom-solve tolerance of the parity tests
(1e-9 relative, same iteration count), and the oracle's BiCGStab (1e-9, iteration count
within one), on two calls in a row that follow a call on an unrelated box: the scratch
then holds another problem's values when the compared solves start.  A box of exactly
the limit, (nx+2)(ny+2)(nz+2) = 65536, uses the last entry of every scratch vector; its
solution is checked by the oracle's operator (the BiCGStab stopping test) and the two
calls must agree bit for bit.  The refusal of larger boxes is a CPU test (test_host.py):
it happens before any CUDA call.

Collected last (file name) so that a run stopping at the first failure has run
everything else first.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2009_12009_gb300 import gmg  # noqa: E402
from paper_2009_12009_gb300 import inputs as I  # noqa: E402

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN

# single boxes with an odd edge: nothing coarsens, so the whole box is the bottom level
CASES = [
    dict(n=(7, 5, 9), bc=[D_, D_, D_], a=0.0, seed=1),
    dict(n=(9, 7, 5), bc=[P_, P_, P_], a=0.0, seed=2),      # singular: zero-mean projection
    dict(n=(11, 9, 7), bc=[P_, D_, D_], a=1.0, seed=3),     # a*alpha term, mixed walls
    dict(n=(30, 31, 29), bc=[D_, D_, D_], a=0.0, seed=4),   # 32,736 ghosted elements
    dict(n=(9, 5, 7), bc=[N_, N_, N_], a=0.0, seed=5),      # singular: zero-flux walls
    dict(n=(7, 9, 5), bc=[N_, P_, D_], bc_hi=[D_, P_, N_], a=0.5, seed=6),  # Neumann/Dirichlet per side
]


def _dense_coeffs(ctx):
    wx, wy, wz, dg = ctx.coeffs(0)
    v = [ctx.box_views(t, 0)[0] for t in (wx, wy, wz, dg)]
    return (v[0][1:-1, 1:-1, 1:].contiguous(), v[1][1:-1, 1:, 1:-1].contiguous(),
            v[2][1:, 1:-1, 1:-1].contiguous(), v[3][1:-1, 1:-1, 1:-1].contiguous())


def _problem(n, bc, bc_hi, a, seed):
    """A one-box context, the oracle of the same box, and the problem's dense inputs."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    dom = ((0, 0, 0), (nx - 1, ny - 1, nz - 1))
    stream = torch.cuda.current_stream().cuda_stream
    ctx = gmg.Context(dom, bc, bc_hi, boxes=[dom], stream=stream)
    ctx.allocate(gmg.FP64)
    ctx.set_scalars(a, 1.0)
    alpha = np.exp(rng.standard_normal(shape)) if a else None
    if a:
        ctx.set_alpha(torch.from_numpy(alpha))
    beta = I.lognormal_beta(rng, shape, periodic=False)
    ctx.set_beta(torch.from_numpy(beta))
    P = O.Problem(dom, [dom], bc, bc_hi)
    P.set_coeffs(a, 1.0, alpha=alpha, beta=beta)
    rhs = rng.standard_normal(shape)
    singular = int(D_ not in list(bc) + list(bc_hi) and a == 0.0)
    return ctx, P, rhs, singular


def _noalloc(ctx, n, bc, bc_hi, singular, rhs, out=None):
    """One call of the entry point through the C ABI on the context's level-0 coefficients."""
    nx, ny, nz = n
    stream = torch.cuda.current_stream().cuda_stream
    wx, wy, wz, dg = _dense_coeffs(ctx)
    rhs_d = torch.from_numpy(rhs).cuda()
    x = torch.full(rhs.shape, float("nan"), dtype=torch.float64, device="cuda") if out is None else out
    iters = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = gmg.lib().gmg_box_bicgstab_noalloc(C.c_void_p(stream), nx, ny, nz, (C.c_int * 3)(*bc), (C.c_int * 3)(*bc_hi),
                                            singular, C.c_void_p(wx.data_ptr()), C.c_void_p(wy.data_ptr()),
                                            C.c_void_p(wz.data_ptr()), C.c_void_p(dg.data_ptr()),
                                            C.c_void_p(rhs_d.data_ptr()), C.c_void_p(x.data_ptr()), 200, 1e-4,
                                            C.c_void_p(iters.data_ptr()))
    assert st == gmg.OK, gmg.lib().gmg_last_error(None)
    return x.cpu().numpy(), int(iters.item())


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["n"])))
def test_noalloc_matches_workspace_bottom_and_oracle(case):
    n = case["n"]
    bc_hi = case.get("bc_hi", case["bc"])
    ctx, P, rhs, singular = _problem(n, case["bc"], bc_hi, case["a"], case["seed"])
    assert ctx.nlevels == 1 and P.nlevels == 1
    # existing entry point: the bottom solve with the context's workspace
    xref_b, it_ref = ctx.bottom_solve(ctx.pack(torch.from_numpy(rhs)))
    xref = ctx.unpack(xref_b).cpu().numpy()
    # the oracle's BiCGStab on the same box
    want_b, it_orc = P.bottom(P.to_boxed(0, rhs))
    want = P.to_dense(0, want_b)
    # an unrelated box first: the scratch holds its values when the compared calls start
    other = (13, 11, 9) if n != (13, 11, 9) else (9, 11, 13)
    octx, _, orhs, osing = _problem(other, [D_, D_, D_], [D_, D_, D_], 0.3, case["seed"] + 100)
    _noalloc(octx, other, [D_, D_, D_], [D_, D_, D_], osing, orhs)
    for call in range(2):
        got, it = _noalloc(ctx, n, case["bc"], bc_hi, singular, rhs)
        assert it == it_ref, (call, it, it_ref)
        assert np.abs(got - xref).max() <= 1e-9 * np.abs(xref).max(), (call, np.abs(got - xref).max())
        assert abs(it - it_orc) <= 1
        assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max() or abs(it - it_orc) == 1


def test_noalloc_box_at_the_limit():
    """(62+2)(30+2)(30+2) = 65536: every scratch vector used to its last entry.  The result
    meets the BiCGStab stopping test by the oracle's operator, and two calls agree bitwise."""
    n, bc = (62, 30, 30), [D_, D_, D_]
    # a large a*alpha term keeps the iteration count well inside max_iter on a box this size
    ctx, P, rhs, singular = _problem(n, bc, bc, 2000.0, 77)
    octx, _, orhs, osing = _problem((13, 11, 9), bc, bc, 0.3, 78)
    _noalloc(octx, (13, 11, 9), bc, bc, osing, orhs)
    x1, it1 = _noalloc(ctx, n, bc, bc, singular, rhs)
    x2, it2 = _noalloc(ctx, n, bc, bc, singular, rhs)
    assert it1 == it2 and np.array_equal(x1, x2)
    assert 0 < it1 < 200
    r = rhs - P.apply(x1)
    assert np.abs(r).max() <= 1.5e-4 * np.abs(rhs).max()
