"""Pins of the oracle's quadratic Dirichlet wall rule (boundary code DIRICHLET_QUAD; Sec.
"Linear Solvers": the operator equation with its boundary conditions, whose discretisation
at a wall the paper leaves open).

Reading pinned here: on a quadratic Dirichlet side the ghost of a box's wall cell phi_0 is
the value, half a cell outside the face, of the parabola through the wall value g (on the
face), phi_0 and the next cell inward phi_1: ghost = 8g/3 - 2 phi_0 + phi_1 / 3.  A box
with a single cell along the wall normal keeps the linear rule 2g - phi_0.  Gauss-Seidel
solves each cell's row exactly, so the ghost's own-cell term -2 phi_0 goes to the
denominator.  Facts that hold whatever the implementation:
  * the rule is exact for quadratics, so a quadratic phi with matching wall values (and
    matching Neumann values on the other walls) has zero discrete residual and is the
    discrete solution; the linear rule misses it by O(1) at the walls;
  * the scheme converges at second order to a smooth manufactured solution;
  * the assembled matrix differs from its transpose only in the entries that couple a
    quadratic wall cell and its inward neighbour, by -b beta_f / (3 h^2) (beta_f the wall
    face's beta, which is the wall cell's beta);
  * A^T from the matrix entries equals the transpose of the assembled A;
  * the multigrid iteration reaches the LAPACK solution;
  * after one colour pass every cell of that colour solves its row (zero residual), wall
    cells included;
  * the operator does not depend on the box layout (boxes of at least two cells);
  * the beta and wall-value gradients match central differences of full solves;
  * composite (multi-level AMR) problems refuse the rule.
"""
import numpy as np
import pytest

from paper_2009_12009_gb300 import inputs as I

P_, D_, N_, Q_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN, I.DIRICHLET_QUAD


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


def _face_points(P, face, ext):
    """(x, y, z) arrays of the face centres of wall face `face`, shaped like its value array"""
    d, side = face // 2, face % 2
    n = [P.domain[1][q] - P.domain[0][q] + 1 for q in range(3)]
    h = [ext[q] / n[q] for q in range(3)]
    t1, t2 = [q for q in range(3) if q != d]
    T2, T1 = np.meshgrid((np.arange(n[t2]) + 0.5) * h[t2], (np.arange(n[t1]) + 0.5) * h[t1], indexing="ij")
    pt = [None] * 3
    pt[d] = np.full_like(T1, ext[d] if side else 0.0)
    pt[t1], pt[t2] = T1, T2
    return pt


def _set_exact_walls(P, bc_lo, bc_hi, ext, f, grad):
    """wall values of the exact solution: f on Dirichlet faces, the outward normal
    derivative on Neumann faces"""
    for face in range(6):
        d, side = face // 2, face % 2
        bc = (bc_hi if side else bc_lo)[d]
        if bc == P_:
            continue
        pt = _face_points(P, face, ext)
        v = f(*pt) if bc in (D_, Q_) else (1.0 if side else -1.0) * grad[d](*pt)
        P.set_bc_values(face, np.asarray(v, dtype=np.float64) * np.ones_like(pt[(d + 1) % 3]))


QUADRATIC = (lambda x, y, z: 0.4 + 1.1 * x - 0.7 * y + 0.3 * z + 1.9 * x * x - 0.8 * y * y + 1.3 * z * z + 0.6 * x * y
             - 0.9 * y * z + 0.5 * x * z)
Q_GRAD = (lambda x, y, z: 1.1 + 3.8 * x + 0.6 * y + 0.5 * z,
          lambda x, y, z: -0.7 - 1.6 * y + 0.6 * x - 0.9 * z,
          lambda x, y, z: 0.3 + 2.6 * z - 0.9 * y + 0.5 * x)
Q_LAP = 2 * 1.9 - 2 * 0.8 + 2 * 1.3


@pytest.mark.parametrize("bc_lo,bc_hi", [([Q_] * 3, [Q_] * 3), ([Q_, N_, Q_], [N_, Q_, Q_])], ids=["QQQ", "QN"])
def test_quadratic_fields_have_zero_residual(orc, bc_lo, bc_hi):
    """Constant beta, a alpha phi term, anisotropic cells: A phi_exact (wall values in the
    ghosts) equals rhs at every cell to rounding; with the linear rule on the same walls
    the wall cells miss it by O(1)."""
    n, ext = (12, 10, 14), (1.2, 0.8, 1.1)
    shape = n[::-1]
    rng = np.random.default_rng(71)
    h = [ext[q] / n[q] for q in range(3)]
    Z, Y, X = np.meshgrid(*[(np.arange(n[q]) + 0.5) * h[q] for q in (2, 1, 0)], indexing="ij")
    alpha = np.exp(rng.standard_normal(shape))
    a, b, beta0 = 0.7, 1.3, 2.1
    phi = QUADRATIC(X, Y, Z)
    rhs = a * alpha * phi - b * beta0 * Q_LAP
    res = {}
    for rule in ("quad", "lin"):
        lo = bc_lo if rule == "quad" else [D_ if c == Q_ else c for c in bc_lo]
        hi = bc_hi if rule == "quad" else [D_ if c == Q_ else c for c in bc_hi]
        P = orc.Problem(dom3(*n), I.chop(*dom3(*n), 6), lo, hi, (0, 0, 0), ext)
        P.set_coeffs(a, b, alpha=alpha, beta=np.full(shape, beta0))
        _set_exact_walls(P, lo, hi, ext, QUADRATIC, Q_GRAD)
        res[rule] = np.abs(P.apply_bc(phi) - rhs).max() / np.abs(rhs).max()
        if rule == "quad":
            sol, it, hist, st = P.solve(rhs, tol_rel=1e-13, maxit=100)
            assert st == orc.OK
            assert np.abs(sol - phi).max() <= 1e-10 * np.abs(phi).max()
    assert res["quad"] <= 1e-12, res
    assert res["lin"] >= 1e-2, res


def test_second_order_convergence():
    """Smooth manufactured solution with variable beta (zero normal derivative on the walls)
    and quadratic Dirichlet walls with nonzero values: the error falls about 4x per
    refinement (16 -> 32 -> 64), and lies below the linear rule's on every grid."""
    sp = pytest.importorskip("sympy")
    from oracle import oracle as O

    x, y, z = sp.symbols("x y z")
    X = (x, y, z)
    phi_e = sp.exp(0.7 * x) * sp.sin(1.3 * y + 0.4) * sp.cos(0.9 * z + 0.2) + 0.5 * x * y
    beta_e = 1 + sp.Rational(1, 3) * sp.cos(sp.pi * x) * sp.cos(sp.pi * y) * sp.cos(sp.pi * z)
    rhs_e = -sum(sp.diff(beta_e * sp.diff(phi_e, v), v) for v in X)
    f_phi, f_beta, f_rhs = (sp.lambdify(X, e, "numpy") for e in (phi_e, beta_e, rhs_e))
    errs = {D_: [], Q_: []}
    for n in (16, 32, 64):
        c = (np.arange(n) + 0.5) / n
        Z, Y, Xg = np.meshgrid(c, c, c, indexing="ij")
        for rule in (D_, Q_):
            P = O.Problem(dom3(n, n, n), I.chop(*dom3(n, n, n), 16), [rule] * 3, [rule] * 3)
            P.set_coeffs(0.0, 1.0, beta=f_beta(Xg, Y, Z))
            _set_exact_walls(P, [rule] * 3, [rule] * 3, (1.0, 1.0, 1.0), f_phi, None)
            phi, it, hist, st = P.solve(f_rhs(Xg, Y, Z), tol_rel=1e-12, maxit=100)
            assert st == O.OK
            errs[rule].append(np.abs(phi - f_phi(Xg, Y, Z)).max())
    e = errs[Q_]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 3.3 < r1 < 4.8 and 3.5 < r2 < 4.5, (errs, r1, r2)
    assert all(q < l for q, l in zip(errs[Q_], errs[D_])), errs


def _case(orc, n, bc_lo, bc_hi, a, seed, mgs=4, ext=(0.9, 1.0, 0.7)):
    P = orc.Problem(dom3(*n), I.chop(*dom3(*n), mgs), bc_lo, bc_hi, (0, 0, 0), ext)
    rng = np.random.default_rng(seed)
    shape = n[::-1]
    beta = np.exp(0.5 * rng.standard_normal(shape))
    alpha = np.exp(rng.standard_normal(shape)) if a else None
    P.set_coeffs(a, 1.0, alpha=alpha, beta=beta)
    return P, rng, shape, beta, alpha


def test_asymmetry_is_the_wall_coupling_and_transpose_is_exact(orc):
    """(8, 6, 10) in boxes of 4 (the z boxes: 4, 4, 2), quadratic walls on four sides, a
    linear Dirichlet and a Neumann side, variable beta: A - A^T is nonzero exactly on the
    (wall cell, inward neighbour) pairs of the quadratic sides, where A[w][w+1] - A[w+1][w]
    = -b beta_w / (3 h^2); apply_transpose equals A^T y."""
    n = (8, 6, 10)
    bc_lo, bc_hi = [Q_, D_, Q_], [Q_, N_, Q_]
    P, rng, shape, beta, _ = _case(orc, n, bc_lo, bc_hi, 0.6, 72)
    A = _assemble(P, shape)
    h = [(0.9, 1.0, 0.7)[q] / n[q] for q in range(3)]
    want = np.zeros_like(A)
    strides = (1, n[0], n[0] * n[1])
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                c = (i, j, k)
                w = i + n[0] * (j + n[1] * k)
                for d in range(3):
                    for side in (0, 1):
                        if (bc_hi if side else bc_lo)[d] != Q_ or c[d] != (n[d] - 1 if side else 0):
                            continue
                        inner = w + (-strides[d] if side else strides[d])
                        want[w, inner] += -beta[k, j, i] / (3 * h[d] ** 2)
                        want[inner, w] -= -beta[k, j, i] / (3 * h[d] ** 2)
    got = A - A.T
    scale = np.abs(A).max()
    assert np.abs(got - want).max() <= 1e-13 * scale
    assert np.count_nonzero(np.abs(got) > 1e-9 * scale) == np.count_nonzero(want)
    for _ in range(3):
        y = rng.standard_normal(shape)
        assert np.abs(P.apply_transpose(y).reshape(-1) - A.T @ y.reshape(-1)).max() <= 1e-13 * scale * np.abs(y).max()


@pytest.mark.parametrize("bc_lo,bc_hi,a", [([Q_] * 3, [Q_] * 3, 0.0), ([Q_, N_, D_], [N_, Q_, Q_], 0.8)],
                         ids=["QQQ", "mixed_helmholtz"])
def test_multigrid_reaches_lapack(orc, bc_lo, bc_hi, a):
    """8^3, variable beta, random wall values: the multigrid solution equals LAPACK's solve of
    the assembled (non-symmetric) matrix with the wall term moved to the right-hand side."""
    P, rng, shape, beta, _ = _case(orc, (8, 8, 8), bc_lo, bc_hi, a, 73)
    for face in range(6):
        P.set_bc_values(face, rng.standard_normal(P.face_shape(face)))
    rhs = rng.standard_normal(shape)
    b = (rhs - P.apply_bc(np.zeros(shape))).reshape(-1)
    want = np.linalg.solve(_assemble(P, shape), b)
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-13, maxit=200)
    assert st == orc.OK
    assert np.abs(phi.reshape(-1) - want).max() <= 1e-10 * np.abs(want).max()
    phi_k, _, _, st = P.solve_krylov(rhs, 1, tol_rel=1e-13, maxit=200)  # BiCGStab around the V-cycle
    assert st == orc.OK
    assert np.abs(phi_k.reshape(-1) - want).max() <= 1e-10 * np.abs(want).max()


def test_colour_pass_solves_its_rows(orc):
    """One red pass, then one black pass, on level 0 with random phi and rhs: after each, the
    residual of every cell of that colour is zero to rounding, the cells next to the
    quadratic walls included.  (A linear Dirichlet or a Neumann wall cell reads its own old
    value through the ghost filled before the pass, so its residual stays nonzero.)"""
    n = (8, 12, 10)
    for rule in (Q_, D_):
        P, rng, shape, beta, _ = _case(orc, n, [rule, N_, rule], [rule, rule, N_], 0.5, 74)
        phi = P.to_boxed(0, rng.standard_normal(shape))
        rhs = P.to_boxed(0, rng.standard_normal(shape))
        kk, jj, ii = np.meshgrid(*[np.arange(m) for m in shape], indexing="ij")
        dwall = (ii == 0) | (ii == n[0] - 1) | (jj == n[1] - 1) | (kk == 0)
        nwall = (jj == 0) | (kk == n[2] - 1)
        for colour in (0, 1):
            P.smooth_colour(0, phi, rhs, colour)
            r = P.to_dense(0, P.residual(0, phi, rhs))
            mask = (ii + jj + kk) % 2 == colour
            scale = np.abs(P.to_dense(0, rhs)).max()
            assert np.abs(r[mask & ~dwall & ~nwall]).max() <= 1e-12 * scale
            assert np.abs(r[mask & nwall & ~dwall]).max() > 1e-3 * scale
            if rule == Q_:
                assert np.abs(r[mask & dwall & ~nwall]).max() <= 1e-12 * scale
            else:
                assert np.abs(r[mask & dwall & ~nwall]).max() > 1e-3 * scale


def test_thin_box_keeps_the_linear_rule(orc):
    """x extent 7 cut into boxes of 1 and 6 cells: the one-cell box's wall row couples only
    to the ghost of its own cell (symmetric entries there), the six-cell box's wall row takes
    the quadratic rule."""
    n = (7, 4, 4)
    boxes = [((0, 0, 0), (0, 3, 3)), ((1, 0, 0), (6, 3, 3))]
    P = orc.Problem(dom3(*n), boxes, [Q_, P_, P_], [Q_, P_, P_])
    P.set_coeffs(0.0, 1.0)
    A = _assemble(P, n[::-1])
    # cell (0, 0, 0) and its inward neighbour (1, 0, 0): linear rule, symmetric
    assert A[0, 1] == A[1, 0]
    # cell (6, 0, 0) next to the high wall and (5, 0, 0): quadratic rule, h = 1/7
    assert A[6, 5] - A[5, 6] == pytest.approx(-(7.0 ** 2) / 3, rel=1e-14)


def test_operator_does_not_depend_on_box_layout(orc):
    n = (16, 12, 8)
    rng = np.random.default_rng(75)
    shape = n[::-1]
    beta = np.exp(rng.standard_normal(shape))
    phi = rng.standard_normal(shape)
    vals = {f: rng.standard_normal(s) for f, s in ((0, (8, 12)), (3, (8, 16)), (5, (12, 16)))}
    out = []
    for mgs in (16, 8, 4, 2):
        P = orc.Problem(dom3(*n), I.chop(*dom3(*n), mgs), [Q_, N_, D_], [N_, Q_, Q_])
        P.set_coeffs(0.3, 1.0, alpha=np.ones(shape), beta=beta)
        for f, v in vals.items():
            P.set_bc_values(f, v)
        out.append(P.apply_bc(phi))
    assert all(np.array_equal(out[0], o) for o in out[1:])


def _loss(orc, P, a, alpha, beta, values, rhs, target):
    P.set_coeffs(a, 1.0, alpha=alpha, beta=beta)
    for f, v in values.items():
        P.set_bc_values(f, v)
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-14, tol_abs=1e-300, maxit=300)
    assert st == orc.OK
    return 0.5 * np.sum((phi - target) ** 2), phi


@pytest.mark.parametrize("bc_lo,bc_hi,a", [([Q_, N_, Q_], [N_, Q_, Q_], 0.0), ([Q_, P_, D_], [Q_, P_, Q_], 0.7)],
                         ids=["QN", "QPD_helmholtz"])
def test_gradients_finite_differences(orc, bc_lo, bc_hi, a):
    """dL/dbeta (cells) and dL/dg (every wall face) from phi and the adjoint lambda (LAPACK on
    the assembled transposed matrix) against central differences of L = 0.5 ||phi - phi_t||^2
    through full solves.  (6, 8, 5) in boxes of 4: the z boxes are 4 and 1 cells, so the high
    z wall mixes the quadratic rule (behind the 4-cell box) and the linear one."""
    n = (6, 8, 5)
    P, rng, shape, beta, alpha = _case(orc, n, bc_lo, bc_hi, a, 76)
    values = {f: rng.standard_normal(P.face_shape(f)) for f in range(6) if (bc_hi if f % 2 else bc_lo)[f // 2] != P_}
    rhs = rng.standard_normal(shape)
    target = rng.standard_normal(shape)
    L0, phi = _loss(orc, P, a, alpha, beta, values, rhs, target)
    A = _assemble(P, shape)
    lam = np.linalg.solve(A.T, (phi - target).reshape(-1)).reshape(shape)
    gb = P.grad_beta(phi, lam, beta)
    gw = {f: P.grad_wall_values(lam, f) for f in values}
    eps = 1e-4
    for trial in range(3):
        db = rng.standard_normal(shape) * beta * 0.1
        dv = {f: rng.standard_normal(v.shape) for f, v in values.items()}
        Lp = _loss(orc, P, a, alpha, beta + eps * db, {f: v + eps * dv[f] for f, v in values.items()}, rhs, target)[0]
        Lm = _loss(orc, P, a, alpha, beta - eps * db, {f: v - eps * dv[f] for f, v in values.items()}, rhs, target)[0]
        fd = (Lp - Lm) / (2 * eps)
        pred = np.sum(gb * db) + sum(np.sum(gw[f] * dv[f]) for f in values)
        assert abs(fd - pred) <= 1e-6 * abs(fd) + 1e-9, (trial, fd, pred)
    for f0 in sorted(values):  # each wall face on its own
        dv = rng.standard_normal(values[f0].shape)
        vp, vm = dict(values), dict(values)
        vp[f0] = values[f0] + eps * dv
        vm[f0] = values[f0] - eps * dv
        fd = (_loss(orc, P, a, alpha, beta, vp, rhs, target)[0] -
              _loss(orc, P, a, alpha, beta, vm, rhs, target)[0]) / (2 * eps)
        assert abs(fd - np.sum(gw[f0] * dv)) <= 1e-6 * abs(fd) + 1e-9, f0


def test_composite_problems_refuse_the_rule(orc):
    dom = dom3(8, 8, 8)
    with pytest.raises(ValueError):
        orc.AmrProblem(dom, I.chop(*dom, 8), [((4, 4, 4), (11, 11, 11))], [Q_] * 3, [D_] * 3)
