"""Pins of the FP64 CPU oracle against facts fixed by the mathematics, not by the oracle.

Each test names the passage of the paper (AMReX, arXiv 2009.12009) whose reading it pins.
The paper prints no worked numerical example for the solver (its solver figure is not
recoverable), so the pins are closed-form discrete eigen-solutions, second-order
convergence to a manufactured solution, dense direct solves with LAPACK, identities of
the operator and transfer operators, and box-layout invariance.
"""
import numpy as np
import pytest

from paper_2009_12009_gb300 import inputs as I

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def cube(n):
    return ((0, 0, 0), (n - 1, n - 1, n - 1))


def dom3(nx, ny, nz):
    return ((0, 0, 0), (nx - 1, ny - 1, nz - 1))


def centres(n, L=1.0):
    return (np.arange(n) + 0.5) * (L / n)


def outer3(fx, fy, fz):
    return fz[:, None, None] * fy[None, :, None] * fx[None, None, :]


# --------------------------------------------------------------------------------------
# Operator equation of Sec. "Linear Solvers": closed-form discrete eigenvectors


@pytest.mark.parametrize("bc", [P_, D_])
def test_operator_closed_form_anisotropic(orc, bc):
    """sin/cos modes are exact eigenvectors of the constant-coefficient 7-point operator
    with the periodic or reflected-ghost Dirichlet boundary; h differs per axis."""
    nx, ny, nz = 16, 8, 24
    P = orc.Problem(dom3(nx, ny, nz), I.chop(*dom3(nx, ny, nz), 8), [bc] * 3, [bc] * 3, (0, 0, 0), (1.0, 2.0, 0.5))
    h = (1.0 / nx, 2.0 / ny, 0.5 / nz)
    x, y, z = centres(nx, 1.0), centres(ny, 2.0), centres(nz, 0.5)
    if bc == P_:
        k = (1, 2, 3)  # wavenumbers per period
        fx, fy, fz = np.sin(2 * np.pi * k[0] * x / 1.0), np.cos(2 * np.pi * k[1] * y / 2.0), np.sin(2 * np.pi * k[2] * z / 0.5)
        lam = sum(4 * np.sin(np.pi * k[d] * h[d] / Ld) ** 2 / h[d] ** 2 for d, Ld in enumerate((1.0, 2.0, 0.5)))
    else:
        m = (1, 2, 3)  # half-wavelength modes sin(m pi x / L)
        fx, fy, fz = np.sin(m[0] * np.pi * x / 1.0), np.sin(m[1] * np.pi * y / 2.0), np.sin(m[2] * np.pi * z / 0.5)
        lam = sum(4 * np.sin(m[d] * np.pi * h[d] / (2 * Ld)) ** 2 / h[d] ** 2 for d, Ld in enumerate((1.0, 2.0, 0.5)))
    f = outer3(fx, fy, fz)
    # a*alpha*phi - b*lap(phi) with a = 2, alpha = 3, b = 0.5
    P.set_coeffs(a=2.0, b=0.5, alpha=np.full(f.shape, 3.0), beta=None)
    out = P.apply(f)
    np.testing.assert_allclose(out, (6.0 + 0.5 * lam) * f, rtol=0, atol=1e-12 * np.abs(lam * f).max())


def test_periodic_solve_closed_form(orc):
    """poisson32 workload: sin(2 pi x) sin(2 pi y) sin(2 pi z) is an eigenvector of the periodic
    discrete Laplacian with eigenvalue 3 * 4 sin^2(pi h) / h^2, so the discrete solution is
    known exactly."""
    cfg = I.poisson32()
    P = orc.Problem(cfg["domain"], cfg["boxes"], cfg["bc_lo"], cfg["bc_hi"])
    P.set_coeffs(0.0, 1.0)
    phi, it, hist, st = P.solve(cfg["rhs"], tol_rel=1e-13)
    h = 1.0 / 32
    lam = 3 * 4 * np.sin(np.pi * h) ** 2 / h ** 2
    exact = cfg["rhs"] / lam
    assert st == orc.OK
    assert np.abs(phi - exact).max() <= 1e-12 * np.abs(exact).max()
    # V(2,2) cycles with red-black Gauss-Seidel contract a smooth mode quickly
    assert it <= 12
    assert all(hist[i + 1] < 0.25 * hist[i] for i in range(len(hist) - 1))


@pytest.mark.parametrize("n,boxsz", [(16, 8), (24, 12)])
def test_dirichlet_solve_closed_form(orc, n, boxsz):
    """Homogeneous Dirichlet: prod_d sin(m_d pi x_d) satisfies the reflected ghost exactly,
    so it is a discrete eigenvector with eigenvalue sum_d 4 sin^2(m_d pi h / 2) / h^2."""
    P = orc.Problem(cube(n), I.chop(*cube(n), boxsz), [D_] * 3, [D_] * 3)
    P.set_coeffs(0.0, 1.0)
    h = 1.0 / n
    m = (1, 2, 3)
    x = centres(n)
    f = outer3(*(np.sin(mm * np.pi * x) for mm in m))
    lam = sum(4 * np.sin(mm * np.pi * h / 2) ** 2 / h ** 2 for mm in m)
    phi, it, hist, st = P.solve(f, tol_rel=1e-13)
    assert st == orc.OK
    np.testing.assert_allclose(phi, f / lam, rtol=0, atol=1e-12 * np.abs(f / lam).max())


# --------------------------------------------------------------------------------------
# Variable beta: second-order convergence to a manufactured solution


def _manufactured(n, bc):
    x = centres(n)
    X = x[None, None, :]
    Y = x[None, :, None]
    Z = x[:, None, None]
    tw = 2 * np.pi
    sb = [np.sin(tw * X + 0.3), np.sin(tw * Y + 0.7), np.sin(tw * Z + 1.1)]
    cb = [np.cos(tw * X + 0.3), np.cos(tw * Y + 0.7), np.cos(tw * Z + 1.1)]
    beta = 1.0 + 0.5 * sb[0] * sb[1] * sb[2]
    dbeta = [0.5 * tw * cb[0] * sb[1] * sb[2], 0.5 * tw * sb[0] * cb[1] * sb[2], 0.5 * tw * sb[0] * sb[1] * cb[2]]
    if bc == D_:
        k = (np.pi, 2 * np.pi, np.pi)
        s = [np.sin(k[0] * X), np.sin(k[1] * Y), np.sin(k[2] * Z)]
        c = [k[0] * np.cos(k[0] * X), k[1] * np.cos(k[1] * Y), k[2] * np.cos(k[2] * Z)]
    else:
        k = (2 * np.pi, 2 * np.pi, 4 * np.pi)
        s = [np.sin(k[0] * X), np.cos(k[1] * Y), np.sin(k[2] * Z)]
        c = [k[0] * np.cos(k[0] * X), -k[1] * np.sin(k[1] * Y), k[2] * np.cos(k[2] * Z)]
    phi = s[0] * s[1] * s[2]
    grad = [c[0] * s[1] * s[2], s[0] * c[1] * s[2], s[0] * s[1] * c[2]]
    lap = -(k[0] ** 2 + k[1] ** 2 + k[2] ** 2) * phi
    # -div(beta grad phi) = -(grad beta . grad phi) - beta lap phi
    f = -(dbeta[0] * grad[0] + dbeta[1] * grad[1] + dbeta[2] * grad[2]) - beta * lap
    return phi, beta, f


@pytest.mark.parametrize("bc", [D_, P_])
def test_second_order_convergence(orc, bc):
    """Finite-volume 7-point operator with harmonic face beta is second-order accurate:
    the max error falls by ~4 per halving of h.  A wrong face index or dropped term
    stalls the error at O(1) or O(h)."""
    errs = []
    for n in (16, 32, 64):
        phi_e, beta, f = _manufactured(n, bc)
        P = orc.Problem(cube(n), I.chop(*cube(n), 16), [bc] * 3, [bc] * 3)
        P.set_coeffs(0.0, 1.0, beta=beta)
        phi, it, hist, st = P.solve(f, tol_rel=1e-12, project_mean=True)
        assert st == orc.OK
        if bc == P_:
            phi_e = phi_e - phi_e.mean()
        errs.append(np.abs(phi - phi_e).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.6 < r2 < 4.4, (errs, r1, r2)


# --------------------------------------------------------------------------------------
# Dense direct solves (LAPACK) on 8^3: the multigrid iteration converges to A^-1 rhs


def _assemble(P, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        A[:, j] = P.apply(e.reshape(shape)).reshape(-1)
    return A


CASES = [
    dict(bc_lo=[P_] * 3, bc_hi=[P_] * 3, a=0.0, var=False, L=(1, 1, 1)),
    dict(bc_lo=[P_] * 3, bc_hi=[P_] * 3, a=0.0, var=True, L=(1, 1, 1)),
    dict(bc_lo=[D_] * 3, bc_hi=[D_] * 3, a=0.0, var=True, L=(1, 1, 1)),
    dict(bc_lo=[P_, D_, D_], bc_hi=[P_, P_, D_], a=0.0, var=True, L=(1, 1, 1)),
    dict(bc_lo=[P_, D_, D_], bc_hi=[P_, D_, D_], a=0.0, var=True, L=(1, 1, 1)),
    dict(bc_lo=[D_] * 3, bc_hi=[D_] * 3, a=1.0, var=True, L=(1.0, 2.0, 0.5)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("boxsz", [8, 4])
def test_dense_direct_8cubed(orc, case, boxsz):
    c = CASES[case]
    if c["bc_lo"][1] != c["bc_hi"][1] and (c["bc_lo"][1] == P_ or c["bc_hi"][1] == P_):
        # periodic must hold on both sides: the oracle refuses a half-periodic axis
        with pytest.raises(ValueError):
            orc.Problem(cube(8), I.chop(*cube(8), boxsz), c["bc_lo"], c["bc_hi"])
        return
    rng = np.random.default_rng(100 + case)
    P = orc.Problem(cube(8), I.chop(*cube(8), boxsz), c["bc_lo"], c["bc_hi"], (0, 0, 0), c["L"])
    shape = (8, 8, 8)
    beta = np.exp(rng.standard_normal(shape)) if c["var"] else None
    alpha = np.exp(rng.standard_normal(shape)) if c["a"] else None
    P.set_coeffs(c["a"], 1.0, alpha=alpha, beta=beta)
    A = _assemble(P, shape)
    rhs = rng.standard_normal(shape)
    singular = all(b == P_ for b in c["bc_lo"]) and c["a"] == 0.0
    if singular:
        rhs -= rhs.mean()
        n = A.shape[0]
        B = np.zeros((n + 1, n + 1))
        B[:n, :n] = A
        B[:n, n] = 1.0
        B[n, :n] = 1.0
        x = np.linalg.solve(B, np.concatenate([rhs.reshape(-1), [0.0]]))[:n]
    else:
        x = np.linalg.solve(A, rhs.reshape(-1))
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-13, maxit=200)
    assert st == orc.OK
    assert np.abs(phi.reshape(-1) - x).max() <= 1e-10 * np.abs(x).max()


# --------------------------------------------------------------------------------------
# Sec. "Operations on a level": ghost cells hold the owning box's values


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_fill_ghosts_matches_global_array(orc, bc):
    nx, ny, nz = 12, 10, 14
    boxes = I.chop(*dom3(nx, ny, nz), 5)
    P = orc.Problem(dom3(nx, ny, nz), boxes, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(7)
    g = rng.standard_normal((nz, ny, nx))
    f = P.to_boxed(0, g)
    P.fill_ghosts(0, f)
    n = (nx, ny, nz)
    checked = 0
    for b, (lo, hi) in enumerate(boxes):
        v = P.box_view(0, f, b)
        for d in range(3):
            for side in (0, 1):
                sl = [slice(1, -1)] * 3  # (z, y, x) interior
                ax = 2 - d
                sl[ax] = 0 if side == 0 else -1
                ghost = v[tuple(sl)]
                # global index of the ghost plane along d
                gd = lo[d] - 1 if side == 0 else hi[d] + 1
                idx = [np.arange(lo[q], hi[q] + 1) for q in range(3)]
                if 0 <= gd < n[d] or bc == P_:
                    idx[d] = np.array([gd % n[d]])
                    want = g[np.ix_(idx[2], idx[1], idx[0])]
                else:
                    idx[d] = np.array([lo[d] if side == 0 else hi[d]])
                    want = (1.0 if bc == N_ else -1.0) * g[np.ix_(idx[2], idx[1], idx[0])]
                np.testing.assert_array_equal(ghost, want.reshape(ghost.shape))
                checked += ghost.size
    assert checked > 0


# --------------------------------------------------------------------------------------
# Box-layout invariance (Sec. "Basic data structures": a level is the union of its boxes)


def test_box_layout_invariance(orc):
    n = 32
    rng = np.random.default_rng(11)
    beta = np.exp(rng.standard_normal((n, n, n)))
    rhs = rng.standard_normal((n, n, n))
    sols = {}
    for mgs in (32, 16, 8):
        P = orc.Problem(cube(n), I.chop(*cube(n), mgs), [D_] * 3, [D_] * 3)
        assert P.nlevels == 5
        P.set_coeffs(0.0, 1.0, beta=beta)
        phi, it, hist, st = P.solve(rhs, tol_rel=0.0, maxit=6)
        sols[mgs] = (phi, hist)
    ref = sols[32][0]
    for mgs in (16, 8):
        # same hierarchy, same colours, same order of operations per cell; only the order
        # of the bottom solver's dot products differs
        assert np.abs(sols[mgs][0] - ref).max() <= 1e-13 * np.abs(ref).max()
    # an uneven layout (12 + 12 + 8) gives a different hierarchy but the same solution
    P = orc.Problem(cube(n), I.chop(*cube(n), 12), [D_] * 3, [D_] * 3)
    P.set_coeffs(0.0, 1.0, beta=beta)
    phi12, it, hist, st = P.solve(rhs, tol_rel=1e-12, maxit=200)
    P1 = orc.Problem(cube(n), I.chop(*cube(n), 32), [D_] * 3, [D_] * 3)
    P1.set_coeffs(0.0, 1.0, beta=beta)
    phi1, it1, _, _ = P1.solve(rhs, tol_rel=1e-12, maxit=200)
    assert st == orc.OK
    assert np.abs(phi12 - phi1).max() <= 1e-9 * np.abs(phi1).max()


# --------------------------------------------------------------------------------------
# Operator identities


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_operator_symmetric(orc, bc):
    """Flux form with one beta per face and reflected Dirichlet ghosts gives a symmetric
    matrix: <Ax, y> = <x, Ay>.  A beta read from the wrong face breaks this."""
    nx, ny, nz = 12, 8, 10
    P = orc.Problem(dom3(nx, ny, nz), I.chop(*dom3(nx, ny, nz), 4), [bc] * 3, [bc] * 3, (0, 0, 0), (1.2, 0.8, 1.0))
    rng = np.random.default_rng(3)
    shape = (nz, ny, nx)
    P.set_coeffs(0.7, 1.3, alpha=np.exp(rng.standard_normal(shape)), beta=np.exp(rng.standard_normal(shape)))
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    lhs = np.sum(P.apply(x) * y)
    rhs = np.sum(x * P.apply(y))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(P.apply(x)).max())


def test_operator_conservative(orc):
    """Periodic, a = 0: fluxes telescope, sum(A phi) = 0; constant phi gives A phi = 0;
    with a != 0 a constant gives a * alpha * c."""
    n = 8
    P = orc.Problem(cube(n), I.chop(*cube(n), 4), [P_] * 3, [P_] * 3)
    rng = np.random.default_rng(5)
    beta = np.exp(rng.standard_normal((n, n, n)))
    P.set_coeffs(0.0, 1.0, beta=beta)
    phi = rng.standard_normal((n, n, n))
    out = P.apply(phi)
    assert abs(out.sum()) <= 1e-11 * np.abs(out).max()
    assert np.abs(P.apply(np.full((n, n, n), 2.5))).max() <= 1e-12
    alpha = np.exp(rng.standard_normal((n, n, n)))
    P.set_coeffs(0.5, 1.0, alpha=alpha, beta=beta)
    np.testing.assert_allclose(P.apply(np.full((n, n, n), 2.0)), 0.5 * alpha * 2.0, rtol=1e-12, atol=1e-11)


@pytest.mark.parametrize("src", [0, 5, 15])
def test_layered_medium_exact(orc, src):
    """1-D layered medium (beta piecewise constant per cell column along x, y and z
    periodic), unit point source on the plane through the centres of cells i = src,
    phi = 0 at x = 0 and x = 1.  The continuous solution is piecewise linear with flux
    jumping by 1 at the source; the cell-centred scheme with harmonic-mean faces and
    reflected wall ghosts is exact at cell centres for it (series conductance).  An
    arithmetic-mean face fails."""
    n = 16
    d = dom3(n, 4, 4)
    P = orc.Problem(d, I.chop(*d, 8), [D_, P_, P_], [D_, P_, P_])
    rng = np.random.default_rng(20 + src)
    bcell = np.exp(1.5 * rng.standard_normal(n))
    P.set_coeffs(0.0, 1.0, beta=np.broadcast_to(bcell[None, None, :], (4, 4, n)).copy())
    h = 1.0 / n
    rhs = np.zeros((4, 4, n))
    rhs[:, :, src] = 1.0 / h
    # exact: q = -beta phi' is q_L left of the source and q_L + 1 right of it;
    # phi(1) = 0 fixes q_L = -R_R / (R_L + R_R), R = integral of 1/beta
    xs = (src + 0.5) * h
    RL = np.sum(h / bcell[:src]) + 0.5 * h / bcell[src]
    RR = np.sum(h / bcell[src + 1:]) + 0.5 * h / bcell[src]
    qL = -RR / (RL + RR)
    exact = np.zeros(n)
    phi_face = 0.0  # phi at the left face of cell i
    for i in range(n):
        q_left = qL if i <= src else qL + 1.0
        exact[i] = phi_face - q_left * 0.5 * h / bcell[i]
        q_right = qL if i < src else qL + 1.0
        phi_face = exact[i] - q_right * 0.5 * h / bcell[i]
    assert abs(phi_face) <= 1e-12
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-13, maxit=300)
    assert st == orc.OK
    np.testing.assert_allclose(phi, np.broadcast_to(exact[None, None, :], phi.shape), rtol=0,
                               atol=1e-10 * np.abs(exact).max())


def test_positive_definite_dirichlet(orc):
    n = 8
    P = orc.Problem(cube(n), I.chop(*cube(n), 8), [D_] * 3, [D_] * 3)
    rng = np.random.default_rng(6)
    P.set_coeffs(0.0, 1.0, beta=np.exp(rng.standard_normal((n, n, n))))
    for _ in range(5):
        x = rng.standard_normal((n, n, n))
        assert np.sum(x * P.apply(x)) > 0


# --------------------------------------------------------------------------------------
# Red-black Gauss-Seidel


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_gauss_seidel_zeroes_colour_residual(orc, bc):
    """After one colour, every updated cell satisfies its own row of A phi = rhs (its
    neighbours have the other colour and did not move); the other colour is untouched."""
    nx, ny, nz = 10, 12, 6
    boxes = I.chop(*dom3(nx, ny, nz), 5)  # boxes with odd lo: colour is global parity
    P = orc.Problem(dom3(nx, ny, nz), boxes, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(8)
    shape = (nz, ny, nx)
    P.set_coeffs(0.3, 1.0, alpha=np.exp(rng.standard_normal(shape)), beta=np.exp(rng.standard_normal(shape)))
    phi0 = rng.standard_normal(shape)
    rhs = rng.standard_normal(shape)
    K, J, Ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    par = (Ii + J + K) % 2
    wall = (Ii == 0) | (Ii == nx - 1) | (J == 0) | (J == ny - 1) | (K == 0) | (K == nz - 1)
    for colour in (0, 1):
        f = P.to_boxed(0, phi0)
        P.smooth_colour(0, f, P.to_boxed(0, rhs), colour)
        new = P.to_dense(0, f)
        np.testing.assert_array_equal(new[par != colour], phi0[par != colour])
        r = rhs - P.apply(new)
        sel = (par == colour) if bc == P_ else (par == colour) & ~wall
        scale = np.abs(rhs).max() + 1e4 * np.abs(new).max()
        assert np.abs(r[sel]).max() <= 1e-13 * scale


# --------------------------------------------------------------------------------------
# Sec. "Operations between levels": restriction (average) and interpolation


def _hier(orc, n=16, mgs=8, bc=D_):
    return orc.Problem(cube(n), I.chop(*cube(n), mgs), [bc] * 3, [bc] * 3)


@pytest.mark.parametrize("n,mgs", [(16, 8), (32, 16)])
def test_restrict_linear_exact(orc, n, mgs):
    """The mean of 8 children of a linear function is its value at the coarse centre, on
    every level transition, the aggregated one included."""
    P = _hier(orc, n, mgs)
    for m in range(P.nlevels - 1):
        sh = P.level_shape(m)
        K, J, Ii = np.meshgrid(*(np.arange(s, dtype=float) for s in sh), indexing="ij")
        f = 1.0 + 0.25 * Ii - 0.5 * J + 2.0 * K
        c = P.to_dense(m + 1, P.restrict(m, P.to_boxed(m, f)))
        shc = P.level_shape(m + 1)
        Kc, Jc, Ic = np.meshgrid(*(np.arange(s, dtype=float) for s in shc), indexing="ij")
        want = 1.0 + 0.25 * (2 * Ic + 0.5) - 0.5 * (2 * Jc + 0.5) + 2.0 * (2 * Kc + 0.5)
        np.testing.assert_array_equal(c, want)
        assert abs(8 * c.sum() - f.sum()) <= 1e-12 * abs(f).sum()


def test_prolong_is_8x_restrict_transpose(orc):
    P = _hier(orc, 32, 16)
    rng = np.random.default_rng(9)
    for m in range(P.nlevels - 1):
        ec = rng.standard_normal(P.level_shape(m + 1))
        rf = rng.standard_normal(P.level_shape(m))
        fine = P.to_boxed(m, np.zeros(P.level_shape(m)))
        P.prolong_add(m, P.to_boxed(m + 1, ec), fine)
        Pe = P.to_dense(m, fine)
        Rr = P.to_dense(m + 1, P.restrict(m, P.to_boxed(m, rf)))
        assert abs(np.sum(Pe * rf) - 8 * np.sum(ec * Rr)) <= 1e-12 * np.abs(rf).sum()
        # piecewise constant: each fine cell holds its parent's value
        np.testing.assert_array_equal(Pe, np.repeat(np.repeat(np.repeat(ec, 2, 0), 2, 1), 2, 2))


def test_coarse_operator_closed_form(orc):
    """With beta = 1 every coarse level is the 7-point Laplacian at h_m = 2^m h: the periodic
    sin mode sampled at the coarse centres is again an exact eigenvector."""
    n = 32
    P = orc.Problem(cube(n), I.chop(*cube(n), 16), [P_] * 3, [P_] * 3)
    P.set_coeffs(0.0, 1.0)
    for m in range(P.nlevels):
        nm = n >> m
        if nm < 4:
            break
        h = 1.0 / nm
        f = outer3(*(np.sin(2 * np.pi * centres(nm)) for _ in range(3)))
        lam = 3 * 4 * np.sin(np.pi * h) ** 2 / h ** 2
        out = P.to_dense(m, P.apply_level(m, P.to_boxed(m, f)))
        np.testing.assert_allclose(out, lam * f, rtol=0, atol=1e-12 * lam)


def test_coefficient_coarsening_faces(orc):
    """beta that varies only along x: fine x-faces on a coarse face all carry the same value,
    so the coarse x-face equals it; coarse y- and z-faces are the mean over the two fine
    columns (x = 2I, 2I+1) of the cell value."""
    n = 16
    P = orc.Problem(cube(n), I.chop(*cube(n), 8), [D_] * 3, [D_] * 3)
    g = 1.0 + np.arange(n, dtype=float) / 4.0
    beta = np.broadcast_to(g[None, None, :], (n, n, n)).copy()
    P.set_coeffs(0.0, 1.0, beta=beta)
    _, bx0, by0, _ = P.coeffs(0)
    _, bx1, by1, bz1 = P.coeffs(1)
    # x-faces: coarse face I-1/2 <-> fine face 2I-1/2, in box 0 (lo = 0)
    v0 = P.box_view(0, bx0, 0)
    v1 = P.box_view(1, bx1, 0)
    for I_ in range(0, 5):
        np.testing.assert_allclose(v1[1:-1, 1:-1, I_ + 1], v0[1, 1, 2 * I_ + 1], rtol=1e-15)
    w1 = P.box_view(1, by1, 0)
    z1 = P.box_view(1, bz1, 0)
    for I_ in range(4):
        want = 0.5 * (g[2 * I_] + g[2 * I_ + 1])
        np.testing.assert_allclose(w1[1:-1, 1:-1, I_ + 1], want, rtol=1e-15)
        np.testing.assert_allclose(z1[1:-1, 1:-1, I_ + 1], want, rtol=1e-15)


def test_hierarchy_aggregation(orc):
    """Aggregation (Sec. "Linear Solvers"): boxes are coarsened one by one while they can
    be, then merged into one box to coarsen further."""
    P = orc.Problem(cube(32), I.chop(*cube(32), 16), [P_] * 3, [P_] * 3)
    assert [len(P.level_boxes(m)) for m in range(P.nlevels)] == [8, 8, 8, 8, 1]
    assert [P.level_shape(m)[0] for m in range(P.nlevels)] == [32, 16, 8, 4, 2]
    assert P.level_parents(3) == [0] * 8
    # 48 x 160 x 96 in boxes of at most 32: bottom is the 3 x 10 x 6 domain
    d = dom3(48, 160, 96)
    P = orc.Problem(d, I.chop(*d, 32), [D_] * 3, [D_] * 3)
    assert P.level_shape(P.nlevels - 1) == (6, 10, 3)
    assert len(P.level_boxes(P.nlevels - 1)) == 1
    # odd boxes (12 = 6 + 6 -> 3 + 3): no aggregation possible, multi-box bottom
    P = orc.Problem(cube(12), I.chop(*cube(12), 6), [D_] * 3, [D_] * 3)
    assert P.level_shape(P.nlevels - 1) == (6, 6, 6) and len(P.level_boxes(P.nlevels - 1)) == 8


# --------------------------------------------------------------------------------------
# Bottom solver (Sec. "Linear Solvers": Krylov bottom solve)


def test_bicgstab_bottom_vs_lapack(orc):
    P = orc.Problem(cube(12), I.chop(*cube(12), 6), [D_] * 3, [D_] * 3)
    rng = np.random.default_rng(10)
    P.set_coeffs(0.0, 1.0, beta=np.exp(rng.standard_normal((12, 12, 12))))
    mb = P.nlevels - 1
    sh = P.level_shape(mb)
    n = int(np.prod(sh))
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = P.to_dense(mb, P.apply_level(mb, P.to_boxed(mb, e.reshape(sh)))).reshape(-1)
    b = rng.standard_normal(n)
    P.set_params(bot_tol=1e-14, bot_maxit=500)
    x, it = P.bottom(P.to_boxed(mb, b.reshape(sh)))
    xd = P.to_dense(mb, x).reshape(-1)
    xe = np.linalg.solve(A, b)
    assert np.abs(xd - xe).max() <= 1e-10 * np.abs(xe).max()
    P.set_params(bot_tol=1e-4, bot_maxit=200)
    x, it = P.bottom(P.to_boxed(mb, b.reshape(sh)))
    xd = P.to_dense(mb, x).reshape(-1)
    assert np.abs(b - A @ xd).max() <= 1e-4 * np.abs(b).max()
    assert 1 <= it < 200


# --------------------------------------------------------------------------------------
# Solvability of the singular periodic problem


def test_periodic_solvability(orc):
    n = 16
    P = orc.Problem(cube(n), I.chop(*cube(n), 8), [P_] * 3, [P_] * 3)
    rng = np.random.default_rng(12)
    P.set_coeffs(0.0, 1.0, beta=np.exp(rng.standard_normal((n, n, n))))
    rhs = rng.standard_normal((n, n, n)) + 0.3
    _, it, _, st = P.solve(rhs)
    assert st == orc.BAD_INPUT and it == 0
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-11, project_mean=True)
    assert st == orc.OK
    assert abs(phi.mean()) <= 1e-14 * np.abs(phi).max()
    r = (rhs - rhs.mean()) - P.apply(phi)
    assert np.abs(r).max() <= 1e-11 * np.abs(rhs - rhs.mean()).max()
    assert abs(r.mean()) <= 1e-13 * np.abs(rhs).max()


def test_bicgstab_singular_bottom(orc):
    """Singular periodic bottom: the bottom right-hand side is projected onto zero mean
    (the range of A), the result carries zero mean, and the projected system is solved."""
    n = 8
    P = orc.Problem(cube(n), I.chop(*cube(n), 4), [P_] * 3, [P_] * 3)
    rng = np.random.default_rng(13)
    P.set_coeffs(0.0, 1.0, beta=np.exp(rng.standard_normal((n, n, n))))
    mb = P.nlevels - 1
    sh = P.level_shape(mb)
    b = rng.standard_normal(sh) + 0.7
    x, it = P.bottom(P.to_boxed(mb, b))
    xd = P.to_dense(mb, x)
    assert abs(xd.mean()) <= 1e-14 * np.abs(xd).max()
    bp = b - b.mean()
    r = bp - P.to_dense(mb, P.apply_level(mb, P.to_boxed(mb, xd)))
    assert np.abs(r).max() <= 1e-4 * np.abs(bp).max()


def test_threaded_oracle_is_bitwise_sequential():
    """OpenMP over boxes (colour sweeps, residuals, restriction, interpolation, ghost copies,
    max-norms) changes no operation of any cell: a threaded solve equals the sequential one
    bit for bit, iteration count and residual history included."""
    from oracle import oracle as O

    cfg = I.abec(32, 8, 5151, name="abec32")
    P = O.Problem(cfg["domain"], cfg["boxes"], cfg["bc_lo"], cfg["bc_hi"])
    P.set_coeffs(0.0, 1.0, beta=cfg["beta"])
    out = {}
    try:
        for th in (1, 3):
            O.set_threads(th)
            out[th] = P.solve(cfg["rhs"], tol_rel=1e-10, maxit=50)
    finally:
        O.set_threads(1)
    assert np.array_equal(out[1][0], out[3][0])
    assert out[1][1] == out[3][1] and list(out[1][2]) == list(out[3][2])
