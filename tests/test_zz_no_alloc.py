"""The allocation-free box solve against the workspace-based bottom solve.

gmg_box_bicgstab_noalloc serves callers that cannot allocate device memory when they
solve (an operator handed only its input and output tensors, code running under CUDA
graph capture, hosts that forbid allocation after start-up): it takes dense device
arrays and keeps its scratch in a static device array of the library.  Here it must give
the answer of gmg_bottom_solve -- the same BiCGStab on the same box problem, with the
context's workspace as scratch -- within the bottom-solve tolerance of the parity tests
(1e-9 relative, same iteration count), on two calls in a row: the second call starts
from the scratch contents the first one left behind.

Collected last (file name) so that a run stopping at the first failure has run
everything else first.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402
from paper_2009_12009_gb300 import inputs as I  # noqa: E402

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN

# single boxes with an odd edge: nothing coarsens, so the whole box is the bottom level
CASES = [
    dict(n=(7, 5, 9), bc=[D_, D_, D_], a=0.0, seed=1),
    dict(n=(9, 7, 5), bc=[P_, P_, P_], a=0.0, seed=2),      # singular: zero-mean projection
    dict(n=(11, 9, 7), bc=[P_, D_, D_], a=1.0, seed=3),     # a*alpha term, mixed walls
    dict(n=(30, 31, 29), bc=[D_, D_, D_], a=0.0, seed=4),   # near the static limit
    dict(n=(9, 5, 7), bc=[N_, N_, N_], a=0.0, seed=5),      # singular: zero-flux walls
    dict(n=(7, 9, 5), bc=[N_, P_, D_], bc_hi=[D_, P_, N_], a=0.5, seed=6),  # Neumann/Dirichlet per side
]


def _dense_coeffs(ctx):
    wx, wy, wz, dg = ctx.coeffs(0)
    v = [ctx.box_views(t, 0)[0] for t in (wx, wy, wz, dg)]
    return (v[0][1:-1, 1:-1, 1:].contiguous(), v[1][1:-1, 1:, 1:-1].contiguous(),
            v[2][1:, 1:-1, 1:-1].contiguous(), v[3][1:-1, 1:-1, 1:-1].contiguous())


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["n"])))
def test_noalloc_matches_workspace_bottom(case):
    nx, ny, nz = case["n"]
    rng = np.random.default_rng(case["seed"])
    shape = (nz, ny, nx)
    dom = ((0, 0, 0), (nx - 1, ny - 1, nz - 1))
    stream = torch.cuda.current_stream().cuda_stream
    bc_hi = case.get("bc_hi", case["bc"])
    ctx = gmg.Context(dom, case["bc"], bc_hi, boxes=[dom], stream=stream)
    assert ctx.nlevels == 1
    ctx.allocate(gmg.FP64)
    ctx.set_scalars(case["a"], 1.0)
    if case["a"]:
        ctx.set_alpha(torch.from_numpy(np.exp(rng.standard_normal(shape))))
    ctx.set_beta(torch.from_numpy(I.lognormal_beta(rng, shape, periodic=False)))
    rhs = rng.standard_normal(shape)
    singular = int(D_ not in case["bc"] + bc_hi and case["a"] == 0.0)
    # existing entry point: the bottom solve with the context's workspace
    xref_b, it_ref = ctx.bottom_solve(ctx.pack(torch.from_numpy(rhs)))
    xref = ctx.unpack(xref_b).cpu().numpy()
    wx, wy, wz, dg = _dense_coeffs(ctx)
    rhs_d = torch.from_numpy(rhs).cuda()
    bc = (C.c_int * 3)(*case["bc"])
    bch = (C.c_int * 3)(*bc_hi)
    iters = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = gmg.lib()
    for call in range(2):
        x = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
        st = L.gmg_box_bicgstab_noalloc(C.c_void_p(stream), nx, ny, nz, bc, bch, singular,
                                        C.c_void_p(wx.data_ptr()), C.c_void_p(wy.data_ptr()),
                                        C.c_void_p(wz.data_ptr()), C.c_void_p(dg.data_ptr()),
                                        C.c_void_p(rhs_d.data_ptr()), C.c_void_p(x.data_ptr()), 200, 1e-4,
                                        C.c_void_p(iters.data_ptr()))
        assert st == gmg.OK, L.gmg_last_error(None)
        got = x.cpu().numpy()
        assert int(iters.item()) == it_ref, (call, int(iters.item()), it_ref)
        assert np.abs(got - xref).max() <= 1e-9 * np.abs(xref).max(), (call, np.abs(got - xref).max())


def test_noalloc_rejects_oversize():
    L = gmg.lib()
    bc = (C.c_int * 3)(D_, D_, D_)
    # (62+2)^3 = 262144 > 65536: refused before anything is launched
    st = L.gmg_box_bicgstab_noalloc(None, 62, 62, 62, bc, bc, 0, C.c_void_p(8), C.c_void_p(8), C.c_void_p(8),
                                    C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), 200, 1e-4, None)
    assert st == gmg.BAD_INPUT
    assert b"static scratch limit" in L.gmg_last_error(None)
