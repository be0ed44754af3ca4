"""Conjugate-gradient bottom, symmetric V-cycle and multigrid-preconditioned Krylov solves
(Sec. "Linear Solvers": native CG and BiCG solvers next to multigrid) on the GPU against
the oracle.

Tolerances: FP64 V-cycles 1e-10 where the hierarchy coarsens to a small bottom; where the
V-cycle is itself the bottom solve of a 1000-cell level (oddlo: nothing coarsens), CG's ~30
steps carry the rounding of dot products summed in another order forward (measured up to
8e-8), so there the bottom, the V-cycle and the Krylov solves built on it are compared at
1e-6 (1e-4 for residual histories), with the same iteration count up to one and the bottom
stopping test checked by the oracle's operator; Krylov solves at a fixed
iteration count agree to 1e-9 relative with residual histories to 1e-7 (the Krylov scalars
are dot products summed in another order, and the recurrences carry that rounding forward);
solves to 1e-12 agree to 1e-10; mixed-precision preconditioners reach the FP64 tolerance,
checked with the oracle's operator.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402

NAMES = ["uneven", "helmholtz", "neumann", "mixedwalls", "periodic", "oddlo"]


class KPair:
    def __init__(self, name):
        self.cfg = c = cases.make(name)
        ph = c.get("prob_hi", (1.0, 1.0, 1.0))
        self.P = O.Problem(c["domain"], c["boxes"], c["bc_lo"], c["bc_hi"], (0, 0, 0), ph)
        self.P.set_coeffs(c["a"], c["b"], alpha=c["alpha"], beta=c["beta"])
        self.C = gmg.Context(c["domain"], c["bc_lo"], c["bc_hi"], prob_hi=ph, boxes=c["boxes"],
                             stream=torch.cuda.current_stream().cuda_stream)
        self.C.allocate(gmg.MIXED_FP32, krylov=True)
        self.C.set_scalars(c["a"], c["b"])
        if c["alpha"] is not None:
            self.C.set_alpha(torch.from_numpy(c["alpha"]))
        self.C.set_beta(torch.from_numpy(c["beta"]) if c["beta"] is not None else None)
        self.singular = gmg.DIRICHLET not in c["bc_lo"] + c["bc_hi"] and c["a"] == 0.0

    def rhs(self):
        r = self.cfg["rhs"]
        return r - r.mean() if self.singular else r


@pytest.fixture(scope="module", params=NAMES)
def kp(request):
    return KPair(request.param)


def test_cg_bottom(kp):
    P, C = kp.P, kp.C
    mb = P.nlevels - 1
    rng = np.random.default_rng(70)
    rhs = rng.standard_normal(P.level_shape(mb))
    x, it = C.bottom_solve(C.pack(torch.from_numpy(rhs), mb), bottom_solver=1)
    got = C.unpack(x, mb).cpu().numpy()
    P.set_cycle(bottom_cg=True)
    want_b, oit = P.bottom(P.to_boxed(mb, rhs))
    P.set_cycle()
    want = P.to_dense(mb, want_b)
    assert abs(it - oit) <= 1
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max() or abs(it - oit) == 1
    # the GPU's bottom solution meets the stopping test by the oracle's operator
    res = rhs - (rhs.mean() if kp.singular else 0.0) - P.to_dense(mb, P.apply_level(mb, P.to_boxed(mb, got)))
    r0 = np.abs(rhs - (rhs.mean() if kp.singular else 0.0)).max()
    assert np.abs(res - (res.mean() if kp.singular else 0.0)).max() <= 1.0001e-4 * r0


@pytest.mark.parametrize("fused", [1, 0], ids=["fused_coarse", "per_level"])
@pytest.mark.parametrize("push", [1, 0], ids=["push", "exchange"])
def test_symmetric_vcycle_matches_oracle(kp, fused, push):
    """Post-smoothing black before red and the CG bottom: one FP64 V-cycle equals the
    oracle's (in the fused coarse end and in per-level launches, with ghost push or
    exchange)."""
    rng = np.random.default_rng(71)
    r = rng.standard_normal(kp.P.level_shape(0))
    e = kp.C.vcycle(kp.C.pack(torch.from_numpy(r)), fused_coarse=fused, ghost_push=push, post_reverse=1,
                    bottom_solver=1)
    got = kp.C.unpack(e).cpu().numpy()
    kp.P.set_cycle(bottom_cg=True, post_reverse=True)
    want = kp.P.to_dense(0, kp.P.vcycle(0, kp.P.to_boxed(0, r)))
    kp.P.set_cycle()
    tol = 1e-10 if kp.P.nlevels > 1 else 1e-6
    assert np.abs(got - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("method", [1, 2], ids=["bicgstab", "cg"])
def test_krylov_fixed_iterations(kp, method):
    """Three Krylov iterations from phi = 0 on both sides (CG with the symmetric V-cycle and
    the CG bottom): the same recursive-residual history and iterate."""
    bs = 1 if method == 2 else 0
    phi, info = kp.C.solve(kp.C.pack(torch.from_numpy(kp.rhs())), tol_rel=0.0, max_iter=3, krylov=method,
                           bottom_solver=bs, project_mean=1)
    kp.P.set_cycle(bottom_cg=bool(bs), post_reverse=method == 2)
    want, it, hist, st = kp.P.solve_krylov(kp.rhs(), method, tol_rel=0.0, maxit=3, project_mean=True)
    kp.P.set_cycle()
    assert info.iterations == it
    deep = kp.P.nlevels > 1
    above = hist >= 1e-12 * hist[0]  # compared until the FP64 rounding floor
    np.testing.assert_allclose(np.asarray(info.history())[above], hist[above], rtol=1e-7 if deep else 1e-4)
    got = kp.C.unpack(phi).cpu().numpy()
    assert np.abs(got - want).max() <= (1e-9 if deep else 1e-6) * np.abs(want).max()


@pytest.mark.parametrize("method", [1, 2], ids=["bicgstab", "cg"])
def test_krylov_to_tolerance(kp, method):
    """To 1e-12 on both sides: solutions within 1e-10; the iteration counts differ by at
    most one."""
    phi, info = kp.C.solve(kp.C.pack(torch.from_numpy(kp.rhs())), tol_rel=1e-12, max_iter=100, krylov=method,
                           project_mean=1)
    assert info.status == gmg.OK
    kp.P.set_cycle(post_reverse=method == 2)
    want, it, hist, st = kp.P.solve_krylov(kp.rhs(), method, tol_rel=1e-12, maxit=100, project_mean=True)
    kp.P.set_cycle()
    assert st == O.OK and abs(info.iterations - it) <= 1
    got = kp.C.unpack(phi).cpu().numpy()
    assert np.abs(got - want).max() <= (1e-10 if kp.P.nlevels > 1 else 1e-8) * np.abs(want).max()


@pytest.mark.parametrize("prec", [gmg.MIXED_FP32, gmg.MIXED_BF16])
@pytest.mark.parametrize("method", [1, 2], ids=["bicgstab", "cg"])
def test_krylov_mixed_preconditioner_reaches_fp64(kp, method, prec):
    """A float or bfloat16 V-cycle as the preconditioner of FP64 Krylov vectors: the
    solution's residual by the oracle's operator is below 1e-10 of the rhs."""
    rhs = kp.rhs()
    phi, info = kp.C.solve(kp.C.pack(torch.from_numpy(rhs)), tol_rel=1e-10, max_iter=100, krylov=method,
                           precision=prec, project_mean=1)
    assert info.status == gmg.OK
    got = kp.C.unpack(phi).cpu().numpy()
    r = rhs - kp.P.apply(got)
    if kp.singular:
        r -= r.mean()
    assert np.abs(r).max() <= 1.5e-10 * np.abs(rhs).max()


def test_krylov_needs_its_workspace():
    c = cases.make("uneven")
    C = gmg.Context(c["domain"], c["bc_lo"], c["bc_hi"], boxes=c["boxes"], stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64)
    C.set_scalars(0.0, 1.0)
    C.set_beta(torch.from_numpy(c["beta"]))
    with pytest.raises(gmg.GmgError) as e:
        C.solve(C.pack(torch.from_numpy(c["rhs"])), krylov=1)
    assert e.value.status == gmg.NO_WORKSPACE
