"""Pins of the oracle's Neumann walls and wall values (Sec. "Linear Solvers": the operator
equation with its boundary conditions; Sec. "Basic data structures": BCRec).

Readings pinned here: a homogeneous Neumann wall mirrors the adjacent interior value into
the ghost (zero flux through the wall); a Dirichlet wall value g sits on the face (ghost =
2g - interior, the line through both); a Neumann value g is the outward normal derivative
(ghost = interior + h g).  Facts that hold whatever the implementation: cosine modes are
exact discrete eigenvectors with mirrored ghosts; both ghost rules are exact for linear
functions, so a linear phi with matching wall values is the exact discrete solution; the
scheme converges at second order to a smooth manufactured solution; zero-flux walls keep
the operator conservative and symmetric with the constants in its null space; the wall
values enter the operator as a constant (A_g phi - A_g 0 = A_0 phi); the multigrid
iteration reaches the LAPACK solution of the assembled system.
"""
import numpy as np
import pytest

from paper_2009_12009_gb300 import inputs as I

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def dom3(nx, ny, nz):
    return ((0, 0, 0), (nx - 1, ny - 1, nz - 1))


def centres(n, L=1.0):
    return (np.arange(n) + 0.5) * (L / n)


def outer3(fx, fy, fz):
    return fz[:, None, None] * fy[None, :, None] * fx[None, None, :]


def mode(bc, m, x, L, h):
    """1-D eigenvector of the 3-point operator with this axis' boundary rule and its
    eigenvalue: periodic sin(2 pi m x / L), Dirichlet sin(m pi x / L), Neumann cos(m pi x / L)."""
    if bc == P_:
        return np.sin(2 * np.pi * m * x / L), 4 * np.sin(np.pi * m * h / L) ** 2 / h ** 2
    f = np.sin if bc == D_ else np.cos
    return f(m * np.pi * x / L), 4 * np.sin(m * np.pi * h / (2 * L)) ** 2 / h ** 2


AXES = [(N_, N_, N_), (N_, D_, P_), (D_, N_, N_), (N_, P_, D_)]


@pytest.mark.parametrize("bcs", AXES, ids=["NNN", "NDP", "DNN", "NPD"])
def test_operator_closed_form_with_neumann(orc, bcs):
    """Mirrored Neumann ghosts: cos(m pi x / L) is an exact eigenvector of the 3-point
    operator (the ghost at -h/2 and the first centre at +h/2 carry the same cosine), with
    eigenvalue 4 sin^2(m pi h / 2L) / h^2; anisotropic h, mixed with the other rules."""
    n = (16, 8, 12)
    Ls = (1.0, 2.0, 0.5)
    P = orc.Problem(dom3(*n), I.chop(*dom3(*n), 4), list(bcs), list(bcs), (0, 0, 0), Ls)
    h = [Ls[d] / n[d] for d in range(3)]
    fs, lam = [], 0.0
    for d, m in enumerate((1, 2, 3)):
        f, l = mode(bcs[d], m, centres(n[d], Ls[d]), Ls[d], h[d])
        fs.append(f)
        lam += l
    f = outer3(*fs)
    P.set_coeffs(a=2.0, b=0.5, alpha=np.full(f.shape, 3.0), beta=None)
    np.testing.assert_allclose(P.apply(f), (6.0 + 0.5 * lam) * f, rtol=0, atol=1e-12 * np.abs(lam * f).max())


@pytest.mark.parametrize("bcs", AXES, ids=["NNN", "NDP", "DNN", "NPD"])
def test_solve_closed_form_with_neumann(orc, bcs):
    """Poisson (a = 0) with a cosine/sine mode as rhs: the discrete solution is rhs / lambda.
    All-Neumann is singular; the mode has zero mean, so it is solvable and the solution
    (zero mean) is exactly rhs / lambda."""
    n = 16
    P = orc.Problem(dom3(n, n, n), I.chop(*dom3(n, n, n), 8), list(bcs), list(bcs))
    P.set_coeffs(0.0, 1.0)
    h = 1.0 / n
    fs, lam = [], 0.0
    for d, m in enumerate((1, 2, 1)):
        f, l = mode(bcs[d], m, centres(n), 1.0, h)
        fs.append(f)
        lam += l
    f = outer3(*fs)
    phi, it, hist, st = P.solve(f, tol_rel=1e-13, maxit=200)
    assert st == orc.OK
    np.testing.assert_allclose(phi, f / lam, rtol=0, atol=1e-12 * np.abs(f / lam).max())


def test_neumann_conservative_symmetric_nullspace(orc):
    """Zero-flux walls: with a = 0 the fluxes telescope to sum(A phi) = 0, constants give
    A c = 0, and one beta per face keeps A symmetric; a Neumann problem with a = 0 is
    singular and refuses a nonzero-mean rhs unless projected."""
    n = (10, 8, 6)
    P = orc.Problem(dom3(*n), I.chop(*dom3(*n), 4), [N_, N_, P_], [N_, N_, P_], (0, 0, 0), (1.0, 0.8, 0.6))
    rng = np.random.default_rng(40)
    shape = n[::-1]
    beta = np.exp(rng.standard_normal(shape))
    P.set_coeffs(0.0, 1.3, beta=beta)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    Ax = P.apply(x)
    assert abs(Ax.sum()) <= 1e-12 * np.abs(Ax).sum()
    assert np.abs(P.apply(np.full(shape, 1.75))).max() <= 1e-12
    assert abs(np.sum(Ax * y) - np.sum(x * P.apply(y))) <= 1e-12 * np.abs(Ax).max() * np.abs(y).sum()
    _, it, _, st = P.solve(rng.standard_normal(shape) + 0.2)
    assert st == orc.BAD_INPUT and it == 0


def _linear(shape_xyz, Ls, slopes, c0=0.3):
    n = shape_xyz
    x = [centres(n[d], Ls[d]) for d in range(3)]
    X = x[0][None, None, :]
    Y = x[1][None, :, None]
    Z = x[2][:, None, None]
    return c0 + slopes[0] * X + slopes[1] * Y + slopes[2] * Z


def _linear_wall_values(P, bcs, n, Ls, slopes, c0=0.3):
    """Face values that make c0 + s.x exact: phi on the face (Dirichlet) or the outward
    derivative, -s_d on the low face and +s_d on the high face (Neumann)."""
    for d in range(3):
        if bcs[d] == P_:
            continue
        t1, t2 = [e for e in range(3) if e != d]
        c1, c2 = centres(n[t1], Ls[t1]), centres(n[t2], Ls[t2])
        for side in (0, 1):
            if bcs[d] == D_:
                xd = 0.0 if side == 0 else Ls[d]
                v = c0 + slopes[d] * xd + slopes[t1] * c1[None, :] + slopes[t2] * c2[:, None]
            else:
                v = np.full((n[t2], n[t1]), -slopes[d] if side == 0 else slopes[d])
            P.set_bc_values(2 * d + side, v)


@pytest.mark.parametrize("bcs", [(D_, D_, D_), (N_, D_, D_), (N_, N_, D_), (N_, P_, D_), (N_, N_, N_)],
                         ids=["DDD", "NDD", "NND", "NPD", "NNN"])
def test_wall_values_linear_solution_is_exact(orc, bcs):
    """Both ghost rules reproduce a linear function exactly, so phi = c0 + s.x with its own
    wall values solves A phi = a alpha phi exactly for a beta that is constant along the
    directions phi varies in (here beta = beta(z) with s_z = 0, or beta constant).  The
    all-Neumann case with a = 0 is singular: rhs = 0 plus wall fluxes that balance, solution
    the linear function minus its mean."""
    n = (16, 8, 12)
    Ls = (1.0, 0.6, 0.6)  # h = 1/16, 3/40, 1/20: a rule that takes another axis' h fails
    P = orc.Problem(dom3(*n), I.chop(*dom3(*n), 4), list(bcs), list(bcs), (0, 0, 0), Ls)
    rng = np.random.default_rng(41)
    shape = n[::-1]
    slopes = [0.0 if bcs[d] == P_ else s for d, s in enumerate((1.5, -0.7, 0.9))]
    a = 0.0 if bcs == (N_, N_, N_) else 1.0
    if bcs[2] == D_:
        slopes[2] = 0.0
        beta = np.broadcast_to(np.exp(rng.standard_normal(n[2]))[:, None, None], shape).copy()
    else:
        beta = np.full(shape, 1.7)
    alpha = np.exp(rng.standard_normal(shape))
    P.set_coeffs(a, 0.9, alpha=alpha if a else None, beta=beta)
    exact = _linear(n, Ls, slopes)
    _linear_wall_values(P, bcs, n, Ls, slopes)
    # the affine operator reproduces a alpha phi at every cell
    np.testing.assert_allclose(P.apply_bc(exact), a * (alpha if a else 1.0) * exact, rtol=0, atol=1e-11)
    rhs = a * alpha * exact if a else np.zeros(shape)
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-13, maxit=200)
    assert st == orc.OK
    want = exact - exact.mean() if a == 0.0 else exact
    np.testing.assert_allclose(phi, want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_wall_values_enter_as_a_constant(orc):
    """A_g phi - A_g 0 = A_0 phi: the wall values add a phi-independent term, and it lives
    only in the cells next to a wall with a value."""
    n = (8, 6, 10)
    bcs_lo, bcs_hi = [D_, N_, D_], [N_, D_, N_]
    P = orc.Problem(dom3(*n), I.chop(*dom3(*n), 4), bcs_lo, bcs_hi, (0, 0, 0), (1.0, 0.6, 1.2))
    rng = np.random.default_rng(42)
    shape = n[::-1]
    P.set_coeffs(0.5, 1.1, alpha=np.exp(rng.standard_normal(shape)), beta=np.exp(rng.standard_normal(shape)))
    for face in range(6):
        P.set_bc_values(face, rng.standard_normal(P.face_shape(face)))
    x = rng.standard_normal(shape)
    c = P.apply_bc(np.zeros(shape))
    np.testing.assert_allclose(P.apply_bc(x) - c, P.apply(x), rtol=0, atol=1e-12 * np.abs(P.apply(x)).max())
    K, J, Ii = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    wall = (Ii == 0) | (Ii == n[0] - 1) | (J == 0) | (J == n[1] - 1) | (K == 0) | (K == n[2] - 1)
    assert np.all(c[~wall] == 0.0) and np.all(c[wall] != 0.0)
    for face in range(6):
        P.set_bc_values(face, None)
    assert np.all(P.apply_bc(np.zeros(shape)) == 0.0)
    with pytest.raises(ValueError):
        orc.Problem(dom3(*n), I.chop(*dom3(*n), 4), [P_] * 3, [P_] * 3).set_bc_values(0, np.zeros((10, 6)))


@pytest.mark.parametrize("bcs", [(N_, D_, N_), (D_, N_, D_)], ids=["NDN", "DND"])
def test_wall_values_second_order(orc, bcs):
    """Smooth manufactured solution with variable beta, a alpha phi term and nonzero wall
    values of both kinds: the error falls about 4x per refinement (16 -> 32 -> 64).  beta's
    normal derivative vanishes on every wall, so the wall face's one-sided beta is second
    order too."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    X = (x, y, z)
    phi_e = sp.exp(0.7 * x) * sp.sin(1.3 * y + 0.4) * sp.cos(0.9 * z + 0.2) + 0.5 * x * y
    beta_e = 1 + sp.Rational(1, 3) * sp.cos(sp.pi * x) * sp.cos(sp.pi * y) * sp.cos(sp.pi * z)
    alpha_e = 1 + x * x
    a, b = 0.8, 1.0
    rhs_e = a * alpha_e * phi_e - b * sum(sp.diff(beta_e * sp.diff(phi_e, v), v) for v in X)
    f_phi, f_beta, f_alpha, f_rhs = (sp.lambdify(X, e, "numpy") for e in (phi_e, beta_e, alpha_e, rhs_e))
    grads = [sp.lambdify(X, sp.diff(phi_e, v), "numpy") for v in X]
    errs = []
    for n in (16, 32, 64):
        P = orc.Problem(dom3(n, n, n), I.chop(*dom3(n, n, n), 16), list(bcs), list(bcs))
        c = centres(n)
        Z, Y, Xg = np.meshgrid(c, c, c, indexing="ij")
        P.set_coeffs(a, b, alpha=f_alpha(Xg, Y, Z), beta=f_beta(Xg, Y, Z))
        for d in range(3):
            t1, t2 = [e for e in range(3) if e != d]
            T2, T1 = np.meshgrid(c, c, indexing="ij")
            for side in (0, 1):
                pt = [None] * 3
                pt[d] = np.full_like(T1, float(side))
                pt[t1], pt[t2] = T1, T2
                if bcs[d] == D_:
                    v = f_phi(*pt)
                else:
                    v = (1.0 if side else -1.0) * grads[d](*pt)
                P.set_bc_values(2 * d + side, np.asarray(v, dtype=np.float64) * np.ones_like(T1))
        phi, it, hist, st = P.solve(f_rhs(Xg, Y, Z), tol_rel=1e-12, maxit=100)
        assert st == orc.OK
        errs.append(np.abs(phi - f_phi(Xg, Y, Z)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.5 < r2 < 4.5, (errs, r1, r2)


def _assemble(P, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        A[:, j] = P.apply(e.reshape(shape)).reshape(-1)
    return A


@pytest.mark.parametrize("bcs_lo,bcs_hi,a", [([N_, N_, N_], [N_, N_, N_], 0.0), ([N_, D_, P_], [D_, N_, P_], 0.0),
                                             ([N_, N_, N_], [N_, N_, N_], 1.0)], ids=["NNN0", "mixed", "NNN1"])
def test_multigrid_reaches_lapack_with_wall_values(orc, bcs_lo, bcs_hi, a):
    """8^3, variable beta, random wall values: the multigrid solution equals LAPACK's solve of
    the assembled (homogeneous) matrix with the wall term moved to the right-hand side,
    A_0 phi = rhs - A_g 0 (bordered with the mean constraint when singular)."""
    n = 8
    P = orc.Problem(dom3(n, n, n), I.chop(*dom3(n, n, n), 4), bcs_lo, bcs_hi)
    rng = np.random.default_rng(43)
    shape = (n, n, n)
    P.set_coeffs(a, 1.0, alpha=np.exp(rng.standard_normal(shape)) if a else None,
                 beta=np.exp(rng.standard_normal(shape)))
    for face in range(6):
        if (bcs_hi if face % 2 else bcs_lo)[face // 2] != P_:
            P.set_bc_values(face, rng.standard_normal(P.face_shape(face)))
    rhs = rng.standard_normal(shape)
    b = (rhs - P.apply_bc(np.zeros(shape))).reshape(-1)
    A = _assemble(P, shape)
    singular = a == 0.0 and D_ not in bcs_lo + bcs_hi
    if singular:
        b -= b.mean()
        rhs = rhs - (rhs - P.apply_bc(np.zeros(shape))).mean()
        m = A.shape[0]
        B = np.zeros((m + 1, m + 1))
        B[:m, :m] = A
        B[:m, m] = 1.0
        B[m, :m] = 1.0
        want = np.linalg.solve(B, np.concatenate([b, [0.0]]))[:m]
    else:
        want = np.linalg.solve(A, b)
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-13, maxit=200)
    assert st == orc.OK
    assert np.abs(phi.reshape(-1) - want).max() <= 1e-10 * np.abs(want).max()
    # the stopping test is relative to the initial residual rhs - A_g 0
    assert hist[0] == pytest.approx(np.abs(b).max(), rel=1e-14)


def _grad_case(orc, bcs_lo, bcs_hi, a, seed):
    n = (6, 8, 5)
    P = orc.Problem(dom3(*n), I.chop(*dom3(*n), 4), bcs_lo, bcs_hi, (0, 0, 0), (0.9, 1.0, 0.7))
    rng = np.random.default_rng(seed)
    shape = n[::-1]
    beta = np.exp(0.5 * rng.standard_normal(shape))
    alpha = np.exp(rng.standard_normal(shape)) if a else None
    values = {f: rng.standard_normal(P.face_shape(f)) for f in range(6)
              if (bcs_hi if f % 2 else bcs_lo)[f // 2] != P_}
    rhs = rng.standard_normal(shape)
    target = rng.standard_normal(shape)
    return P, rng, shape, beta, alpha, values, rhs, target


def _loss(P, a, alpha, beta, values, rhs, target):
    P.set_coeffs(a, 1.0, alpha=alpha, beta=beta)
    for f, v in values.items():
        P.set_bc_values(f, v)
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-14, tol_abs=1e-300, maxit=300)
    assert st == 0  # converged
    return 0.5 * np.sum((phi - target) ** 2), phi


@pytest.mark.parametrize("bcs_lo,bcs_hi,a", [([D_, N_, D_], [N_, D_, N_], 0.0), ([N_, P_, D_], [D_, P_, N_], 0.7)],
                         ids=["DN", "NPD_helmholtz"])
def test_gradients_with_wall_values_finite_differences(orc, bcs_lo, bcs_hi, a):
    """dL/dbeta (cells) and dL/dg (every wall face) from phi and the adjoint lambda
    (LAPACK on the assembled transposed matrix) against central differences of
    L = 0.5 ||phi - phi_t||^2 through full oracle solves, in random directions."""
    P, rng, shape, beta, alpha, values, rhs, target = _grad_case(orc, bcs_lo, bcs_hi, a, 44)
    L0, phi = _loss(P, a, alpha, beta, values, rhs, target)
    A = _assemble(P, shape)
    lam = np.linalg.solve(A.T, (phi - target).reshape(-1)).reshape(shape)
    gb = P.grad_beta(phi, lam, beta)
    gw = {f: P.grad_wall_values(lam, f) for f in values}
    for trial in range(3):
        db = rng.standard_normal(shape) * beta * 0.1
        dv = {f: rng.standard_normal(v.shape) for f, v in values.items()}
        eps = 1e-4
        Lp = _loss(P, a, alpha, beta + eps * db, {f: v + eps * dv[f] for f, v in values.items()}, rhs, target)[0]
        Lm = _loss(P, a, alpha, beta - eps * db, {f: v - eps * dv[f] for f, v in values.items()}, rhs, target)[0]
        fd = (Lp - Lm) / (2 * eps)
        pred = np.sum(gb * db) + sum(np.sum(gw[f] * dv[f]) for f in values)
        assert abs(fd - pred) <= 1e-6 * abs(fd) + 1e-9, (trial, fd, pred)
    # each part on its own: beta only, then the values only
    eps = 1e-4
    db = rng.standard_normal(shape) * beta * 0.1
    fd = (_loss(P, a, alpha, beta + eps * db, values, rhs, target)[0] -
          _loss(P, a, alpha, beta - eps * db, values, rhs, target)[0]) / (2 * eps)
    assert abs(fd - np.sum(gb * db)) <= 1e-6 * abs(fd) + 1e-9
    f0 = sorted(values)[0]
    dv = rng.standard_normal(values[f0].shape)
    vp, vm = dict(values), dict(values)
    vp[f0] = values[f0] + eps * dv
    vm[f0] = values[f0] - eps * dv
    fd = (_loss(P, a, alpha, beta, vp, rhs, target)[0] - _loss(P, a, alpha, beta, vm, rhs, target)[0]) / (2 * eps)
    assert abs(fd - np.sum(gw[f0] * dv)) <= 1e-6 * abs(fd) + 1e-9


def test_gradient_without_walls_is_the_face_formula(orc):
    """Periodic, homogeneous: the per-row derivative summed over both rows of a face equals
    -(b/h^2)(phi_R - phi_L)(lambda_R - lambda_L) through the harmonic mean; checked against
    a direct double loop over the faces of a small periodic grid."""
    n = (4, 3, 5)
    P = orc.Problem(dom3(*n), [dom3(*n)], [P_] * 3, [P_] * 3, (0, 0, 0), (1.0, 0.6, 1.5))
    rng = np.random.default_rng(45)
    shape = n[::-1]
    beta = np.exp(rng.standard_normal(shape))
    P.set_coeffs(0.0, 1.7, beta=beta)
    phi, lam = rng.standard_normal(shape), rng.standard_normal(shape)
    got = P.grad_beta(phi, lam, beta)
    h = (1.0 / 4, 0.6 / 3, 1.5 / 5)
    want = np.zeros(shape)
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                for d in range(3):  # the face on the high side of (i, j, k)
                    o = [i, j, k]
                    o[d] = (o[d] + 1) % n[d]
                    L_, R_ = (k, j, i), (o[2], o[1], o[0])
                    bl, br = beta[L_], beta[R_]
                    gf = -(1.7 / h[d] ** 2) * (phi[R_] - phi[L_]) * (lam[R_] - lam[L_])
                    want[L_] += gf * 2 * br * br / (bl + br) ** 2
                    want[R_] += gf * 2 * bl * bl / (bl + br) ** 2
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
