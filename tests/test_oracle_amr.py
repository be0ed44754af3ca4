"""Pins of the oracle's two-level composite operator, solve and adjoint.

Sec. "Operations between levels" names interpolation to fine ghost cells, restriction
(average) and refluxing; Sec. "Linear Solvers" names multi-level geometric multigrid.  The
readings (quadratic coarse/fine interpolation, mean-of-fine-fluxes reflux) are pinned by
facts that hold whatever the implementation: exactness on quadratics, conservation,
constants in the null space, the transpose identity, LAPACK solves of the assembled
composite matrix, second-order convergence, and central finite differences of the
adjoint gradients.
"""
import numpy as np
import pytest

from paper_2009_12009_gb300 import inputs as I

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def two_level(orc, n=8, patch=(2, 6), bc=P_, nfb=1, L=1.0):
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    lo, hi = 2 * patch[0], 2 * patch[1] - 1
    fdom = ((lo, lo, lo), (hi, hi, hi))
    fb = I.chop(*fdom, (hi - lo + 1) // 2) if nfb == 8 else [fdom]  # 8 boxes: 2 per axis
    return orc.AmrProblem(dom, I.chop(*dom, n // 2), fb, [bc] * 3, [bc] * 3, (0, 0, 0), (L, L, L))


def average_down(P, xf):
    nz, ny, nx = P.coarse_shape
    return xf.reshape(nz, 2, ny, 2, nx, 2).mean(axis=(1, 3, 5))


def rand_coeffs(P, rng, a=0.0, sigma=1.0):
    """Log-normal beta smoothed by one 3x3x3 mean (the amr2 recipe) on both levels; coarse
    cells under the fine level carry the average of their fine children, so the coarse
    operator used for the coarse correction agrees with the fine one there."""
    per = P._keep[0][0] == P_
    bc = I.box_mean_filter(np.exp(sigma * rng.standard_normal(P.coarse_shape)), per)
    bf = I.box_mean_filter(np.exp(sigma * rng.standard_normal(P.fine_shape)), per)
    bc = np.where(P.covered, average_down(P, bf), bc)
    ac = np.exp(rng.standard_normal(P.coarse_shape)) if a else None
    af = np.exp(rng.standard_normal(P.fine_shape)) if a else None
    P.set_coeffs(a, 1.0, alpha_c=ac, beta_c=bc, alpha_f=af, beta_f=bf)
    return bc, bf


@pytest.mark.parametrize("nfb,bc", [(1, P_), (8, P_), (8, N_)])
def test_constants_and_conservation(orc, nfb, bc):
    """Periodic or zero-flux (Neumann) walls, a = 0: constants are in the null space
    (interpolation weights and the quadratic's weights 8/15 + 2/3 - 1/5 sum to 1) and the
    operator is conservative, sum of volume x (A x) = 0, which fixes the reflux weights and
    signs (and, with Neumann walls, the wall rows)."""
    P = two_level(orc, nfb=nfb, bc=bc)
    rng = np.random.default_rng(1)
    rand_coeffs(P, rng)
    yc, yf = P.apply(np.full(P.coarse_shape, 3.0), np.full(P.fine_shape, 3.0))
    assert max(np.abs(yc).max(), np.abs(yf).max()) <= 1e-10
    V = P.volumes()
    for _ in range(3):
        xc, xf = rng.standard_normal(P.coarse_shape), rng.standard_normal(P.fine_shape)
        y = P.pack(*P.apply(xc, xf))
        assert abs(V @ y) <= 1e-13 * (V @ np.abs(y))


def test_quadratic_exactness(orc):
    """With beta = 1 and no wall nearby, the composite operator applied to point samples of
    a quadratic without mixed terms returns -laplacian exactly on every composite unknown:
    the quadratic coarse/fine ghosts are exact, so are the fine fluxes whose mean the coarse
    side takes."""
    n = 12
    P = two_level(orc, n=n, patch=(4, 8), bc=D_)
    P.set_coeffs(0.0, 1.0)
    hc, hf = 1.0 / n, 0.5 / n

    def q(x, y, z):
        return 1.0 + 0.3 * x - 0.7 * y + 0.2 * z + x * x - 2.0 * y * y + 0.5 * z * z

    lap = 2.0 * (1.0 - 2.0 + 0.5)
    xc = (np.arange(n) + 0.5) * hc
    xf = (np.arange(2 * n) + 0.5) * hf
    Zc, Yc, Xc = np.meshgrid(xc, xc, xc, indexing="ij")
    Zf, Yf, Xf = np.meshgrid(xf, xf, xf, indexing="ij")
    yc, yf = P.apply(q(Xc, Yc, Zc), q(Xf, Yf, Zf))
    inner = np.zeros(P.coarse_shape, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True  # away from the walls (reflected ghosts are not quadratic)
    sel = inner & P.coarse_mask
    np.testing.assert_allclose(yc[sel], -lap, rtol=0, atol=1e-9)
    np.testing.assert_allclose(yf[P.fine_mask], -lap, rtol=0, atol=1e-9)
    # the check covers the coarse cells that reflux
    assert (sel & np.roll(P.covered, 1, 0)).any()


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_transpose(orc, bc):
    P = two_level(orc, bc=bc, nfb=8)
    rng = np.random.default_rng(2)
    rand_coeffs(P, rng, a=1.0 if bc == D_ else 0.0)
    for _ in range(3):
        x = rng.standard_normal(P.pack(np.zeros(P.coarse_shape), np.zeros(P.fine_shape)).size)
        y = rng.standard_normal(x.size)
        Ax = P.pack(*P.apply(*P.unpack(x)))
        ATy = P.pack(*P.apply(*P.unpack(y), transpose=True))
        assert abs(Ax @ y - x @ ATy) <= 1e-12 * np.abs(Ax).max() * np.abs(y).sum()


def lapack_solve(P, rhs, transpose=False):
    M = P.matrix()
    singular = np.abs(M.sum(axis=1)).max() <= 1e-9 * np.abs(M).max()  # A 1 = 0
    if transpose:
        M = M.T
    V = P.volumes()
    if not singular:
        return np.linalg.solve(M, rhs)
    n = M.shape[0]
    B = np.zeros((n + 1, n + 1))
    B[:n, :n] = M
    if transpose:  # A^T lam = g - V (sum g / sum V), sum lam = 0
        B[:n, n] = V
        B[n, :n] = 1.0
    else:  # A phi = rhs (V-orthogonal), V . phi = 0
        B[:n, n] = 1.0
        B[n, :n] = V
    return np.linalg.solve(B, np.concatenate([rhs, [0.0]]))[:n]


@pytest.mark.parametrize("bc,nfb", [(P_, 1), (P_, 8), (D_, 8), (N_, 8)])
def test_mlmg_matches_lapack(orc, bc, nfb):
    P = two_level(orc, bc=bc, nfb=nfb)
    rng = np.random.default_rng(3)
    rand_coeffs(P, rng)
    rc, rf = rng.standard_normal(P.coarse_shape), rng.standard_normal(P.fine_shape)
    rhs = P.pack(rc, rf)
    if bc != D_:
        V = P.volumes()
        rhs = rhs - (V @ rhs) / V.sum()
        rc, rf = P.unpack(rhs)
    pc, pf, it, hist, st = P.solve(rc, rf, tol_rel=1e-13, maxit=200)
    assert st == 0
    x = lapack_solve(P, rhs)
    got = P.pack(pc, pf)
    assert np.abs(got - x).max() <= 1e-10 * np.abs(x).max()
    # the iteration contracts steadily until the rounding floor
    h = hist[hist > 1e-11 * hist[0]]
    assert all(h[i + 1] < 0.5 * h[i] for i in range(len(h) - 1)), hist


def test_composite_second_order(orc):
    """Manufactured smooth solution on a Dirichlet domain with a refined patch in the middle:
    the max error over fine and uncovered coarse cells falls by about 4 per refinement."""
    errs = []
    for n in (8, 16, 32):
        P = two_level(orc, n=n, patch=(n // 4, 3 * n // 4), bc=D_)
        hc, hf = 1.0 / n, 0.5 / n

        def fields(h, m):
            x = (np.arange(m) + 0.5) * h
            Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
            beta = 1.0 + 0.5 * np.sin(2 * np.pi * X + 0.3) * np.sin(2 * np.pi * Y + 0.7) * np.sin(2 * np.pi * Z + 1.1)
            phi = np.sin(np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(np.pi * Z)
            tw = 2 * np.pi
            db = [0.5 * tw * np.cos(tw * X + 0.3) * np.sin(tw * Y + 0.7) * np.sin(tw * Z + 1.1),
                  0.5 * tw * np.sin(tw * X + 0.3) * np.cos(tw * Y + 0.7) * np.sin(tw * Z + 1.1),
                  0.5 * tw * np.sin(tw * X + 0.3) * np.sin(tw * Y + 0.7) * np.cos(tw * Z + 1.1)]
            g = [np.pi * np.cos(np.pi * X) * np.sin(tw * Y) * np.sin(np.pi * Z),
                 tw * np.sin(np.pi * X) * np.cos(tw * Y) * np.sin(np.pi * Z),
                 np.pi * np.sin(np.pi * X) * np.sin(tw * Y) * np.cos(np.pi * Z)]
            lap = -(np.pi ** 2 + tw ** 2 + np.pi ** 2) * phi
            f = -(db[0] * g[0] + db[1] * g[1] + db[2] * g[2]) - beta * lap
            return beta, phi, f

        bc_, pc_e, fc = fields(hc, n)
        bf_, pf_e, ff = fields(hf, 2 * n)
        P.set_coeffs(0.0, 1.0, beta_c=bc_, beta_f=bf_)
        pc, pf, it, hist, st = P.solve(fc, ff, tol_rel=1e-12, maxit=200)
        assert st == 0
        e = max(np.abs(pc - pc_e)[P.coarse_mask].max(), np.abs(pf - pf_e)[P.fine_mask].max())
        errs.append(e)
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r1 > 3.0 and r2 > 3.3, (errs, r1, r2)


# --------------------------------------------------------------------------- adjoint


def adjoint_case(orc, bc, seed=4):
    P = two_level(orc, bc=bc, nfb=8)
    rng = np.random.default_rng(seed)
    bc_, bf_ = rand_coeffs(P, rng, sigma=0.5)
    rhs = rng.standard_normal(P.pack(np.zeros(P.coarse_shape), np.zeros(P.fine_shape)).size)
    V = P.volumes()
    if bc != D_:
        rhs -= (V @ rhs) / V.sum()
    target = rng.standard_normal(rhs.size)
    return P, rng, bc_, bf_, rhs, target


def loss(P, rhs, target, tol=1e-13):
    pc, pf, it, hist, st = P.solve(*P.unpack(rhs), tol_rel=tol, maxit=300)
    assert st == 0
    phi = P.pack(pc, pf)
    return 0.5 * np.sum((phi - target) ** 2), phi


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_adjoint_rhs_gradient_finite_differences(orc, bc):
    """dL/d(rhs) = lambda with A^T lambda = (phi - phi_t) (projected for the periodic case):
    central differences of L = 0.5 ||phi - phi_t||^2 in random rhs directions."""
    P, rng, bc_, bf_, rhs, target = adjoint_case(orc, bc)
    L0, phi = loss(P, rhs, target)
    g = phi - target
    V = P.volumes()
    lam = lapack_solve(P, g, transpose=True)
    for _ in range(3):
        d = rng.standard_normal(rhs.size)
        if bc != D_:
            d -= (V @ d) / V.sum()
        eps = 1e-3
        Lp, _ = loss(P, rhs + eps * d, target)
        Lm, _ = loss(P, rhs - eps * d, target)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - lam @ d) <= 1e-6 * abs(fd) + 1e-10


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_adjoint_beta_gradient_finite_differences(orc, bc):
    """dL/dbeta at cells from the face gradient -(lambda^T dA/dbeta_face phi) through the
    harmonic face mean: central differences of L in random beta directions, coarse and
    fine; coarse cells under the fine level have zero gradient."""
    P, rng, bc_, bf_, rhs, target = adjoint_case(orc, bc, seed=5)
    L0, phi = loss(P, rhs, target)
    lam = lapack_solve(P, phi - target, transpose=True)
    pc, pf = P.unpack(phi)
    lc, lf = P.unpack(lam)
    gc, gf = P.grad_beta(pc, pf, lc, lf, bc_, bf_)
    assert np.abs(gc[P.covered]).max() == 0.0
    for trial in range(3):
        dc = rng.standard_normal(P.coarse_shape)
        df = rng.standard_normal(P.fine_shape) * P.fine_mask
        eps = 1e-4

        def L_at(s):
            P.set_coeffs(0.0, 1.0, beta_c=bc_ * (1 + s * dc * 0.1), beta_f=bf_ * (1 + s * df * 0.1))
            return loss(P, rhs, target)[0]

        fd = (L_at(eps) - L_at(-eps)) / (2 * eps)
        P.set_coeffs(0.0, 1.0, beta_c=bc_, beta_f=bf_)
        pred = np.sum(gc * bc_ * dc * 0.1) + np.sum(gf * bf_ * df * 0.1)
        assert abs(fd - pred) <= 1e-6 * abs(fd) + 1e-10, (trial, fd, pred)


@pytest.mark.parametrize("bc", [P_, D_])
def test_operator_ignores_coefficients_under_the_fine_level(orc, bc):
    """Covered coarse cells have no rows and refluxing replaces the coarse flux on the
    coarse/fine boundary, so the composite operator, its transpose and the solution read no
    level-0 coefficient under the fine level: changing beta and alpha there (and with them
    the coarse correction operator of the iteration) leaves A x, A^T y and phi unchanged."""
    P = two_level(orc, bc=bc, nfb=8)
    rng = np.random.default_rng(8)
    bc_, bf_ = rand_coeffs(P, rng, a=0.0 if bc == P_ else 1.0)
    xc, xf = rng.standard_normal(P.coarse_shape), rng.standard_normal(P.fine_shape)
    y0 = P.pack(*P.apply(xc, xf))
    yt0 = P.pack(*P.apply(xc, xf, transpose=True))
    rc, rf = P.unpack(rng.standard_normal(y0.size))
    if bc == P_:
        V = P.volumes()
        rc, rf = P.unpack(P.pack(rc, rf) - V * (V @ P.pack(rc, rf)) / V.sum())
    p0 = P.pack(*P.solve(rc, rf, tol_rel=1e-12, maxit=100)[:2])
    bc2 = np.where(P.covered, bc_ * np.exp(rng.standard_normal(P.coarse_shape)), bc_)
    P.set_coeffs(0.0, 1.0, beta_c=bc2, beta_f=bf_)
    if bc == D_:
        P.set_coeffs(1.0, 1.0, alpha_c=np.where(P.covered, 5.0, 1.0), beta_c=bc2, alpha_f=np.ones(P.fine_shape),
                     beta_f=bf_)
        P2 = two_level(orc, bc=bc, nfb=8)
        P2.set_coeffs(1.0, 1.0, alpha_c=np.ones(P.coarse_shape), beta_c=bc_, alpha_f=np.ones(P.fine_shape),
                      beta_f=bf_)
        y0 = P2.pack(*P2.apply(xc, xf))
        yt0 = P2.pack(*P2.apply(xc, xf, transpose=True))
        p0 = P2.pack(*P2.solve(rc, rf, tol_rel=1e-12, maxit=100)[:2])
    assert np.array_equal(P.pack(*P.apply(xc, xf)), y0)
    assert np.array_equal(P.pack(*P.apply(xc, xf, transpose=True)), yt0)
    p1 = P.pack(*P.solve(rc, rf, tol_rel=1e-12, maxit=100)[:2])
    assert np.abs(p1 - p0).max() <= 1e-9 * np.abs(p0).max()


@pytest.mark.parametrize("bc", [P_, D_])
def test_composite_iteration_contracts(orc, bc):
    """With the level-0 coefficients under the fine level restricted from the fine ones, the
    composite iteration contracts by at least 5x per iteration on average on the amr recipe
    (32^3 level 0, 32^3 fine cells, smoothed log-normal beta)."""
    a = I.amr2(n=32)
    P = orc.AmrProblem(a["domain"], a["coarse_boxes"], a["fine_boxes"], [bc] * 3, [bc] * 3)
    lo, hi = a["fine_slice"]
    sl = (slice(lo, hi + 1),) * 3
    bf = np.ones(P.fine_shape)
    bf[sl] = a["beta_f"]
    P.set_coeffs(0.0, 1.0, beta_c=a["beta_c"], beta_f=bf)
    rf = np.zeros(P.fine_shape)
    rf[sl] = a["rhs_f"]
    pc, pf, it, hist, st = P.solve(a["rhs_c"], rf, tol_rel=1e-10, maxit=100)
    assert st == 0 and it <= 14, (it, hist[1:] / hist[:-1])


# --------------------------------------------------------------- several fine patches


def two_patches(orc, bc=P_, shifted=False):
    """16^3 level 0 (boxes of 8^3) with two disjoint refined patches: coarse [2,6)^3 (one fine
    box) and coarse [10,14) x [2,6) x [8,12) (two fine boxes, split along x), or, shifted,
    the second patch moved so the two face each other across a two-cell coarse gap."""
    n = 16
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    fb = [((4, 4, 4), (11, 11, 11))]
    if shifted:
        fb += [((16, 4, 4), (19, 11, 11)), ((20, 4, 4), (23, 11, 11))]
    else:
        fb += [((20, 4, 16), (23, 11, 23)), ((24, 4, 16), (27, 11, 23))]
    return orc.AmrProblem(dom, I.chop(*dom, 8), fb, [bc] * 3, [bc] * 3)


@pytest.mark.parametrize("bc", [P_, N_])
@pytest.mark.parametrize("shifted", [False, True], ids=["apart", "facing"])
def test_patches_constants_and_conservation(orc, bc, shifted):
    """Two refined patches, a = 0 without Dirichlet walls: constants are in the null space
    and sum of volume x (A x) = 0 (refluxing on every patch's coarse/fine faces)."""
    P = two_patches(orc, bc, shifted)
    rng = np.random.default_rng(11)
    rand_coeffs(P, rng)
    yc, yf = P.apply(np.full(P.coarse_shape, 2.0), np.full(P.fine_shape, 2.0))
    assert max(np.abs(yc).max(), np.abs(yf).max()) <= 1e-10
    V = P.volumes()
    for _ in range(3):
        y = P.pack(*P.apply(rng.standard_normal(P.coarse_shape), rng.standard_normal(P.fine_shape)))
        assert abs(V @ y) <= 1e-13 * (V @ np.abs(y))


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_patches_transpose_and_lapack(orc, bc):
    """Two refined patches: <A x, y> = <x, A^T y>, and the composite multigrid iteration
    reaches LAPACK's solution of the assembled composite system."""
    P = two_patches(orc, bc)
    rng = np.random.default_rng(12)
    rand_coeffs(P, rng, a=1.0 if bc == D_ else 0.0)
    m = P.pack(np.zeros(P.coarse_shape), np.zeros(P.fine_shape)).size
    x, y = rng.standard_normal(m), rng.standard_normal(m)
    Ax = P.pack(*P.apply(*P.unpack(x)))
    ATy = P.pack(*P.apply(*P.unpack(y), transpose=True))
    assert abs(Ax @ y - x @ ATy) <= 1e-12 * np.abs(Ax).max() * np.abs(y).sum()
    rhs = rng.standard_normal(m)
    if bc != D_:
        V = P.volumes()
        rhs = rhs - (V @ rhs) / V.sum()
    pc, pf, it, hist, st = P.solve(*P.unpack(rhs), tol_rel=1e-13, maxit=200)
    assert st == 0
    want = lapack_solve(P, rhs)
    assert np.abs(P.pack(pc, pf) - want).max() <= 1e-10 * np.abs(want).max()
