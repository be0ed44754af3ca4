"""Pins of the oracle's conjugate-gradient bottom solve, its symmetric V-cycle and the
Krylov solvers preconditioned by multigrid (Sec. "Linear Solvers": native CG and BiCG
solvers next to geometric multigrid).

Facts that hold whatever the implementation: CG reaches the LAPACK solution of the bottom
system and, on n unknowns, needs at most about n iterations; a V-cycle whose post-smoothing
reverses the pre-smoothing colour order is a symmetric positive definite operator when A is
(the plain order is not symmetric); preconditioned CG minimises the A-norm error over the
Krylov space that contains the plain multigrid iterates with the same V-cycle, so its error
is never larger at any iteration; both Krylov solvers reach the LAPACK solution, also with
Neumann walls, wall values and singular problems.
"""
import numpy as np
import pytest

from paper_2009_12009_gb300 import inputs as I

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def dom3(nx, ny, nz):
    return ((0, 0, 0), (nx - 1, ny - 1, nz - 1))


def _assemble(P, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        A[:, j] = P.apply(e.reshape(shape)).reshape(-1)
    return A


def _problem(orc, n, bcs_lo, bcs_hi, a=0.0, seed=60, mgs=4, sigma=1.0):
    P = orc.Problem(dom3(*n), I.chop(*dom3(*n), mgs), bcs_lo, bcs_hi, (0, 0, 0), (1.0, 0.9, 1.1))
    rng = np.random.default_rng(seed)
    shape = n[::-1]
    P.set_coeffs(a, 1.0, alpha=np.exp(rng.standard_normal(shape)) if a else None,
                 beta=np.exp(sigma * rng.standard_normal(shape)))
    return P, rng, shape


@pytest.mark.parametrize("bc", [D_, N_])
def test_cg_bottom_vs_lapack(orc, bc):
    """Bottom level alone (nothing coarsens on a 5x6x7 box): CG to 1e-12 equals LAPACK's
    solution of the assembled bottom matrix (Neumann: singular, projected rhs, zero-mean
    result), within at most n + 10 iterations."""
    P, rng, shape = _problem(orc, (5, 6, 7), [bc] * 3, [bc] * 3, mgs=8)
    assert P.nlevels == 1
    P.set_cycle(bottom_cg=True)
    P.set_params(2, 2, 400, 1e-12)
    b = rng.standard_normal(shape) + 0.3
    x, it = P.bottom(P.to_boxed(0, b))
    got = P.to_dense(0, x)
    A = _assemble(P, shape)
    m = A.shape[0]
    if bc == N_:
        bp = b - b.mean()
        B = np.zeros((m + 1, m + 1))
        B[:m, :m] = A
        B[:m, m] = 1.0
        B[m, :m] = 1.0
        want = np.linalg.solve(B, np.concatenate([bp.reshape(-1), [0.0]]))[:m]
        assert abs(got.mean()) <= 1e-14 * np.abs(got).max()
    else:
        want = np.linalg.solve(A, b.reshape(-1))
    assert np.abs(got.reshape(-1) - want).max() <= 1e-10 * np.abs(want).max()
    assert 1 <= it <= m + 10


def test_cg_bottom_stops_at_tolerance(orc):
    """With the default 1e-4 the CG bottom stops at the first iterate whose residual is
    below 1e-4 of the initial one, reported as its iteration count."""
    P, rng, shape = _problem(orc, (5, 6, 7), [D_] * 3, [D_] * 3, mgs=8)
    P.set_cycle(bottom_cg=True)
    P.set_params(2, 2, 200, 1e-4)
    b = rng.standard_normal(shape)
    x, it = P.bottom(P.to_boxed(0, b))
    A = _assemble(P, shape)
    r = b.reshape(-1) - A @ P.to_dense(0, x).reshape(-1)
    assert np.abs(r).max() <= 1e-4 * np.abs(b).max()
    P.set_params(2, 2, it - 1, 1e-4)  # one iteration less does not reach it
    x1, it1 = P.bottom(P.to_boxed(0, b))
    r1 = b.reshape(-1) - A @ P.to_dense(0, x1).reshape(-1)
    assert it1 == it - 1 and np.abs(r1).max() > 1e-4 * np.abs(b).max()


def _vcycle_matrix(P, shape):
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        M[:, j] = P.to_dense(0, P.vcycle(0, P.to_boxed(0, e.reshape(shape)))).reshape(-1)
    return M


@pytest.mark.parametrize("bcs", [(D_, D_, D_), (N_, D_, P_)], ids=["DDD", "NDP"])
def test_symmetric_vcycle(orc, bcs):
    """With an exact bottom (CG to 1e-14) the V-cycle is a linear operator M.  Reversing the
    post-smoothing colour order makes M symmetric and positive definite; the plain order
    (red then black both times) does not give a symmetric M."""
    n = (8, 8, 8)
    P, rng, shape = _problem(orc, n, list(bcs), list(bcs), a=0.3)
    P.set_params(2, 2, 500, 1e-14)
    P.set_cycle(bottom_cg=True, post_reverse=True)
    M = _vcycle_matrix(P, shape)
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0.0
    P.set_cycle(bottom_cg=True, post_reverse=False)
    M0 = _vcycle_matrix(P, shape)
    assert np.abs(M0 - M0.T).max() > 1e-3 * np.abs(M0).max()


def test_pcg_error_never_above_multigrid(orc):
    """Preconditioned CG minimises ||x - x*||_A over x0 + K_k(M A, M r0), the space that holds
    the k-th plain multigrid iterate x_k = x_(k-1) + M (b - A x_(k-1)) with the same symmetric
    V-cycle M; so at every iteration its A-norm error is at most multigrid's."""
    n = (8, 8, 8)
    P, rng, shape = _problem(orc, n, [D_] * 3, [D_] * 3, seed=61, sigma=2.0)
    P.set_params(2, 2, 500, 1e-14)
    P.set_cycle(bottom_cg=True, post_reverse=True)
    A = _assemble(P, shape)
    b = rng.standard_normal(shape)
    xs = np.linalg.solve(A, b.reshape(-1))

    def anorm(x):
        e = x.reshape(-1) - xs
        return np.sqrt(e @ A @ e)

    for k in range(1, 6):
        x_mg, it_mg, _, _ = P.solve(b, tol_rel=0.0, maxit=k)
        x_cg, it_cg, _, _ = P.solve_krylov(b, 2, tol_rel=0.0, maxit=k)
        assert it_mg == it_cg == k
        assert anorm(x_cg) <= anorm(x_mg) * (1 + 1e-8) + 1e-13 * anorm(np.zeros_like(xs)), k


CASES = [
    dict(lo=[D_] * 3, hi=[D_] * 3, a=0.0, walls=False),
    dict(lo=[N_, D_, P_], hi=[D_, N_, P_], a=0.0, walls=True),
    dict(lo=[N_] * 3, hi=[N_] * 3, a=0.0, walls=True),   # singular
    dict(lo=[P_] * 3, hi=[P_] * 3, a=0.0, walls=False),  # singular
    dict(lo=[N_] * 3, hi=[N_] * 3, a=0.8, walls=True),
]


@pytest.mark.parametrize("method", [1, 2], ids=["bicgstab", "cg"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_krylov_reaches_lapack(orc, case, method):
    """8^3, variable beta (sigma 1.5), to 1e-12: the multigrid-preconditioned BiCGStab and CG
    equal LAPACK's solution (singular problems: bordered with the mean constraint), also
    with wall values (folded into the right-hand side)."""
    c = CASES[case]
    n = (8, 8, 8)
    P, rng, shape = _problem(orc, n, c["lo"], c["hi"], a=c["a"], seed=62 + case, sigma=1.5)
    if method == 2:
        P.set_cycle(bottom_cg=True, post_reverse=True)
    if c["walls"]:
        for f in range(6):
            if (c["hi"] if f % 2 else c["lo"])[f // 2] != P_:
                P.set_bc_values(f, rng.standard_normal(P.face_shape(f)))
    rhs = rng.standard_normal(shape)
    b = rhs - P.apply_bc(np.zeros(shape))
    A = _assemble(P, shape)
    m = A.shape[0]
    singular = c["a"] == 0.0 and D_ not in c["lo"] + c["hi"]
    if singular:
        rhs = rhs - b.mean()
        b = b - b.mean()
        B = np.zeros((m + 1, m + 1))
        B[:m, :m] = A
        B[:m, m] = 1.0
        B[m, :m] = 1.0
        want = np.linalg.solve(B, np.concatenate([b.reshape(-1), [0.0]]))[:m]
    else:
        want = np.linalg.solve(A, b.reshape(-1))
    got, it, hist, st = P.solve_krylov(rhs, method, tol_rel=1e-12, maxit=100)
    assert st == orc.OK, (st, hist)
    assert hist[0] == pytest.approx(np.abs(b).max(), rel=1e-14)
    assert hist[-1] <= 1e-12 * hist[0]
    assert np.abs(got.reshape(-1) - want).max() <= 1e-9 * np.abs(want).max()
    x_mg, it_mg, _, _ = P.solve(rhs, tol_rel=1e-12, maxit=100, project_mean=True)
    assert it <= it_mg


def test_krylov_singular_refuses_unbalanced_rhs(orc):
    P, rng, shape = _problem(orc, (8, 8, 8), [N_] * 3, [N_] * 3)
    _, it, _, st = P.solve_krylov(rng.standard_normal(shape) + 0.5, 1)
    assert st == orc.BAD_INPUT and it == 0
