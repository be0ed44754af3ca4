"""Edge cases of the solve on the GPU, against the oracle where there is a result to compare:
a zero right-hand side, boxes one cell wide (no coarsening: the bottom solve is the whole
solve), a single 2^3 box, a batch mixing a 2^3 problem, a singular periodic problem and
Dirichlet problems, the absolute tolerance, max_iter = 0, and a singular problem whose rhs
has a nonzero mean (refused unless projected)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_12009_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402

P_, D_ = I.PERIODIC, I.DIRICHLET


def problem(n, mgs, bc, seed, a=0.0):
    rng = np.random.default_rng(seed)
    dom = ((0, 0, 0), (n[0] - 1, n[1] - 1, n[2] - 1))
    shape = (n[2], n[1], n[0])
    rhs = rng.standard_normal(shape)
    if bc == P_ and a == 0.0:
        rhs -= rhs.mean()
    return dict(domain=dom, boxes=I.chop(*dom, mgs), bc_lo=[bc] * 3, bc_hi=[bc] * 3, a=a, b=1.0,
                beta=I.lognormal_beta(rng, shape, periodic=(bc == P_)), rhs=rhs,
                prob_hi=(n[0] / 8.0, n[1] / 8.0, n[2] / 8.0))


def pair(p, precision=gmg.MIXED_FP32):
    C = gmg.Context(p["domain"], p["bc_lo"], p["bc_hi"], prob_hi=p["prob_hi"], boxes=p["boxes"],
                    stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(precision)
    C.set_scalars(p["a"], p["b"])
    C.set_beta(torch.from_numpy(p["beta"]))
    P = O.Problem(p["domain"], p["boxes"], p["bc_lo"], p["bc_hi"], (0.0, 0.0, 0.0), p["prob_hi"])
    P.set_coeffs(p["a"], p["b"], beta=p["beta"])
    return C, P


@pytest.mark.parametrize("prec", [gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16])
def test_zero_rhs(prec):
    p = problem((16, 16, 16), 8, D_, 1)
    C, _ = pair(p)
    phi, info = C.solve(C.pack(torch.zeros(16, 16, 16, dtype=torch.float64)), tol_rel=1e-10, precision=prec)
    assert info.status == gmg.OK and info.iterations == 0
    assert float(C.unpack(phi).abs().max()) == 0.0


@pytest.mark.parametrize("n,mgs", [((9, 8, 8), 4), ((2, 2, 2), 2), ((6, 5, 4), 8)],
                         ids=["one_cell_wide_box", "single_2cube", "odd_single_box"])
def test_no_coarsening_bottom_is_the_solve(n, mgs):
    """Nothing coarsens (a 1-wide box, an odd or tiny domain): level 0 is the bottom and the
    solve is BiCGStab outer-iterated to 1e-10; same answer as the oracle to 1e-10."""
    p = problem(n, mgs, D_, 2)
    C, P = pair(p)
    assert C.nlevels == 1 == P.nlevels
    phi, info = C.solve(C.pack(torch.from_numpy(p["rhs"])), tol_rel=1e-12, max_iter=200)
    want, it, hist, st = P.solve(p["rhs"], tol_rel=1e-12, maxit=200)
    assert info.status == gmg.OK and st == O.OK
    got = C.unpack(phi).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_batch_of_mixed_kinds():
    """A 2^3 problem, a singular periodic one and Dirichlet ones of uneven sizes in one batch:
    each equals its independent oracle solve (same iteration count, 1e-10)."""
    probs = [problem((2, 2, 2), 2, D_, 3), problem((16, 8, 12), 8, P_, 4), problem((24, 16, 8), 8, D_, 5),
             problem((32, 32, 16), 16, D_, 6)]
    B = gmg.BatchContext(probs, stream=torch.cuda.current_stream().cuda_stream)
    B.allocate(gmg.MIXED_FP32)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.from_numpy(q["beta"]) for q in probs])
    rhs = B.pack_all([torch.from_numpy(q["rhs"]) for q in probs])
    phi, infos = B.batch_solve(rhs, tol_rel=1e-10, max_iter=100)
    for s, q in enumerate(probs):
        P = O.Problem(q["domain"], q["boxes"], q["bc_lo"], q["bc_hi"], (0.0, 0.0, 0.0), q["prob_hi"])
        P.set_coeffs(0.0, 1.0, beta=q["beta"])
        want, it, hist, st = P.solve(q["rhs"], tol_rel=1e-10, maxit=100)
        got = B.unpack_solve(s, phi).cpu().numpy()
        assert infos[s].status == gmg.OK and st == O.OK
        assert infos[s].iterations == it, (s, infos[s].iterations, it)
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max(), s


def test_absolute_tolerance_and_max_iter_zero():
    p = problem((32, 32, 32), 16, D_, 7)
    C, _ = pair(p)
    rhs = C.pack(torch.from_numpy(p["rhs"]))
    _, info = C.solve(rhs, tol_rel=0.0, tol_abs=1e-6)
    assert info.status == gmg.OK and info.final_resid <= 1e-6 < info.history()[-2]
    _, info0 = C.solve(rhs, tol_rel=1e-10, max_iter=0)
    assert info0.status == gmg.NOT_CONVERGED and info0.iterations == 0


def test_singular_rhs_with_nonzero_mean():
    p = problem((16, 16, 16), 8, P_, 8)
    C, P = pair(p)
    shifted = p["rhs"] + 0.25
    rhs = C.pack(torch.from_numpy(shifted))
    with pytest.raises(gmg.GmgError):
        C.solve(rhs, tol_rel=1e-10)
    phi, info = C.solve(rhs, tol_rel=1e-12, project_mean=1)
    assert info.status == gmg.OK
    got = C.unpack(phi).cpu().numpy()
    want, it, hist, st = P.solve(shifted, tol_rel=1e-12, project_mean=True)
    assert abs(got.mean()) <= 1e-12 * np.abs(got).max()
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
