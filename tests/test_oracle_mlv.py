"""Pins of the oracle's composite operator and multigrid solve over several AMR levels (Sec.
"Linear Solvers": multi-AMR-level geometric multigrid; Sec. "Operations between levels").

Facts that hold whatever the implementation: with two levels it is the (pinned) two-level
form, with one level the one-level solve; with three levels the constants are in the null
space and the operator is conservative (periodic or zero-flux walls, a = 0), the
quadratic coarse/fine ghosts and refluxed faces make it exact on quadratics at every
level, and the composite iteration converges to LAPACK's solution of the assembled
composite system, contracting steadily.
"""
import numpy as np
import pytest

from paper_2009_12009_gb300 import inputs as I

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def avg_down(x):
    nz, ny, nx = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))


def three_levels(n=16):
    """level 0: n^3 in boxes of n/2; level 1 over level-0 cells [n/4, 3n/4) (8 boxes); level 2
    over level-1 cells [3n/4, 5n/4) (8 boxes)"""
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    l1 = I.chop((n // 2,) * 3, (3 * n // 2 - 1,) * 3, n // 2)
    l2 = I.chop((3 * n // 2,) * 3, (5 * n // 2 - 1,) * 3, n // 2)
    return dom, [I.chop(*dom, n // 2), l1, l2]


def rand_coeffs(M, rng, per, a=0.0):
    """log-normal beta smoothed per level; cells of level l under level l + 1 take the average
    of their children (finest first), as in the amr recipe"""
    betas = [I.box_mean_filter(np.exp(rng.standard_normal(s)), per) for s in M.shapes]
    for l in range(M.L - 2, -1, -1):
        under = M.inside[l + 1].reshape(M.shapes[l][0], 2, M.shapes[l][1], 2, M.shapes[l][2], 2).all(axis=(1, 3, 5))
        betas[l] = np.where(under, avg_down(betas[l + 1]), betas[l])
    alphas = [np.exp(rng.standard_normal(s)) for s in M.shapes] if a else None
    M.set_coeffs(a, 1.0, alphas=alphas, betas=betas)
    return alphas, betas


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_two_levels_are_the_two_level_form(orc, bc):
    """L = 2: the same operator and the same iterates as the two-level oracle."""
    n = 8
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    fb = I.chop((4, 4, 4), (11, 11, 11), 4)
    M = orc.MultiLevelProblem(dom, [I.chop(*dom, 4), fb], [bc] * 3, [bc] * 3)
    A = orc.AmrProblem(dom, I.chop(*dom, 4), fb, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(30)
    alphas, betas = rand_coeffs(M, rng, bc == P_, a=0.0 if bc != D_ else 1.0)
    A.set_coeffs(0.0 if bc != D_ else 1.0, 1.0, alpha_c=None if alphas is None else alphas[0], beta_c=betas[0],
                 alpha_f=None if alphas is None else alphas[1], beta_f=betas[1])
    xs = [rng.standard_normal(s) for s in M.shapes]
    ym = M.apply(xs)
    yc, yf = A.apply(xs[0], xs[1])
    sc = max(np.abs(yc).max(), np.abs(yf).max())
    assert np.abs(ym[0] - yc).max() <= 1e-13 * sc and np.abs(ym[1] - yf).max() <= 1e-13 * sc
    r = [rng.standard_normal(s) * m for s, m in zip(M.shapes, M.masks)]
    if bc != D_:
        v = M.pack(r)
        V = M.volumes()
        r = M.unpack(v - (V @ v) / V.sum())
    pm, it, hist, st = M.solve(r, tol_rel=0.0, maxit=3)
    pc, pf, it2, hist2, st2 = A.solve(r[0], r[1], tol_rel=0.0, maxit=3)
    assert it == it2 == 3
    s2 = max(np.abs(pc).max(), np.abs(pf).max())
    assert np.abs(pm[0] - pc).max() <= 1e-12 * s2 and np.abs((pm[1] - pf) * M.inside[1]).max() <= 1e-12 * s2
    np.testing.assert_allclose(hist, hist2, rtol=1e-10)


def test_one_level_is_the_one_level_solve(orc):
    n = 16
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    M = orc.MultiLevelProblem(dom, [I.chop(*dom, 8)], [D_] * 3, [D_] * 3)
    P = orc.Problem(dom, I.chop(*dom, 8), [D_] * 3, [D_] * 3)
    rng = np.random.default_rng(31)
    beta = np.exp(rng.standard_normal((n, n, n)))
    M.set_coeffs(0.0, 1.0, betas=[beta])
    P.set_coeffs(0.0, 1.0, beta=beta)
    rhs = rng.standard_normal((n, n, n))
    pm, it, hist, st = M.solve([rhs], tol_rel=1e-12)
    pp, it2, hist2, st2 = P.solve(rhs, tol_rel=1e-12)
    assert st == st2 == 0 and it == it2
    assert np.abs(pm[0] - pp).max() <= 1e-13 * np.abs(pp).max()


@pytest.mark.parametrize("bc", [P_, N_])
def test_three_levels_constants_and_conservation(orc, bc):
    dom, lb = three_levels()
    M = orc.MultiLevelProblem(dom, lb, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(32)
    rand_coeffs(M, rng, bc == P_)
    ys = M.apply([np.full(s, 1.5) for s in M.shapes])
    assert max(np.abs(y).max() for y in ys) <= 1e-10
    V = M.volumes()
    for _ in range(3):
        y = M.pack(M.apply([rng.standard_normal(s) for s in M.shapes]))
        assert abs(V @ y) <= 1e-13 * (V @ np.abs(y))


def test_three_levels_quadratic_exactness(orc):
    """beta = 1, no wall nearby: -laplacian of a quadratic without mixed terms, exactly, on the
    composite cells of all three levels (the refluxing cells of levels 0 and 1 included)."""
    dom, lb = three_levels(16)
    M = orc.MultiLevelProblem(dom, lb, [D_] * 3, [D_] * 3)
    M.set_coeffs(0.0, 1.0)

    def q(x, y, z):
        return 1.0 + 0.3 * x - 0.7 * y + 0.2 * z + x * x - 2.0 * y * y + 0.5 * z * z

    lap = 2.0 * (1.0 - 2.0 + 0.5)
    xs = []
    for s in M.shapes:
        c = (np.arange(s[0]) + 0.5) / s[0]
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        xs.append(q(X, Y, Z))
    ys = M.apply(xs)
    inner = np.zeros(M.shapes[0], dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    np.testing.assert_allclose(ys[0][inner & M.masks[0]], -lap, rtol=0, atol=1e-8)
    for l in (1, 2):
        np.testing.assert_allclose(ys[l][M.masks[l]], -lap, rtol=0, atol=1e-8)


@pytest.mark.parametrize("bc", [D_, P_, N_])
def test_three_levels_reach_lapack(orc, bc):
    dom, lb = three_levels(8)
    M = orc.MultiLevelProblem(dom, lb, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(33)
    rand_coeffs(M, rng, bc == P_, a=1.0 if bc == D_ else 0.0)
    r = M.pack([rng.standard_normal(s) for s in M.shapes])
    A = M.matrix()
    if bc != D_:
        V = M.volumes()
        r = r - (V @ r) / V.sum()
        m = A.shape[0]
        B = np.zeros((m + 1, m + 1))
        B[:m, :m] = A
        B[:m, m] = 1.0
        B[m, :m] = V
        want = np.linalg.solve(B, np.concatenate([r, [0.0]]))[:m]
    else:
        want = np.linalg.solve(A, r)
    ps, it, hist, st = M.solve(M.unpack(r), tol_rel=1e-13, maxit=200)
    assert st == 0
    got = M.pack(ps)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    h = hist[hist > 1e-11 * hist[0]]
    assert all(h[i + 1] < 0.5 * h[i] for i in range(len(h) - 1)), hist


def test_coefficients_under_finer_levels_are_restricted(orc):
    """The correction operator of a level sees, under the next finer level, that level's
    coefficients restricted (mean of the 4 fine faces tiling a face), finest pair first: a
    level-0 face deep under level 2 is the mean of the 16 level-2 faces tiling it."""
    dom, lb = three_levels(16)
    M = orc.MultiLevelProblem(dom, lb, [D_] * 3, [D_] * 3)
    rng = np.random.default_rng(34)
    betas = [np.exp(rng.standard_normal(s)) for s in M.shapes]
    M.set_coeffs(0.0, 1.0, betas=betas)

    def face_x(l, g):  # beta of the x-face at the low side of global cell g of level l
        P = M.level(l)
        al, bx, by, bz = P.coeffs(0)
        for b, (lo, hi) in enumerate(M.level_boxes[l]):
            if all(lo[d] <= g[d] <= hi[d] for d in range(3)):
                v = P.box_view(0, bx, b)
                return v[g[2] - lo[2] + 1, g[1] - lo[1] + 1, g[0] - lo[0] + 1]
        raise KeyError(g)

    G = (7, 7, 8)  # a level-0 cell whose low x-face lies deep under level 2 ([6, 10) in level-0 units)
    want = np.mean([face_x(2, (4 * G[0], 4 * G[1] + u, 4 * G[2] + v)) for u in range(4) for v in range(4)])
    assert abs(face_x(0, G) - want) <= 1e-14 * want


def test_amr3_recipe_small(orc):
    """The three-level workload recipe at n = 16: covered cells of levels 0 and 1 carry the
    average of their children, the rhs has zero volume-weighted mean and vanishes under finer
    levels, and the oracle's composite solve reaches 1e-10 contracting steadily."""
    a = I.amr3(16)
    n = 16
    M = orc.MultiLevelProblem(a["domain"], a["level_boxes"], a["bc_lo"], a["bc_hi"])
    sl = [tuple(slice(lo[d], lo[d] + n) for d in (2, 1, 0)) for lo in a["level_lo"]]

    def embed(l, x, fill=0.0):
        out = np.full(M.shapes[l], fill)
        out[sl[l]] = x
        return out

    for l in (1, 2):  # every box, coarsened, inside one box of the level below
        for lo, hi in a["level_boxes"][l]:
            assert any(all(blo[d] <= lo[d] // 2 and hi[d] // 2 <= bhi[d] for d in range(3))
                       for blo, bhi in a["level_boxes"][l - 1])
    for l in (0, 1):
        cov = a["covered"][l]
        assert (embed(l, cov.astype(float)) > 0).sum() == cov.sum() == (n // 2) ** 3
        under = M.inside[l + 1].reshape(M.shapes[l][0], 2, M.shapes[l][1], 2, M.shapes[l][2], 2).all(axis=(1, 3, 5))
        assert np.array_equal(embed(l, cov.astype(float)) > 0, under)
        fine = embed(l + 1, a["betas"][l + 1], fill=np.nan)
        want = avg_down(fine)[under]
        assert np.allclose(embed(l, a["betas"][l])[under], want, rtol=1e-15, atol=0)
        assert not a["rhss"][l][cov].any()
    rs = [embed(l, r) for l, r in enumerate(a["rhss"])]
    assert abs(M.volumes() @ M.pack(rs)) <= 1e-13 * (M.volumes() @ np.abs(M.pack(rs)))
    M.set_coeffs(0.0, 1.0, betas=[embed(l, b, fill=1.0) for l, b in enumerate(a["betas"])])
    ps, it, hist, st = M.solve(rs, tol_rel=1e-10, maxit=100)
    assert st == 0 and hist[-1] <= 1e-10 * hist[0]
    assert all(hist[i + 1] < 0.5 * hist[i] for i in range(len(hist) - 1)), hist


# --------------------------------------------------------------- transpose and beta gradient

@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_term_walk_equals_the_rows(orc, bc):
    """The term-by-term walk that the transpose and the gradient scatter through sums to the
    rows evaluated directly (three levels, variable alpha and beta)."""
    dom, lb = three_levels(8)
    M = orc.MultiLevelProblem(dom, lb, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(35)
    rand_coeffs(M, rng, bc == P_, a=0.7)
    xs = [rng.standard_normal(s) for s in M.shapes]
    y0 = M.pack(M.apply(xs))
    y1 = M.pack(M.apply(xs, terms=True))
    assert np.abs(y1 - y0).max() <= 1e-13 * np.abs(y0).max()


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_two_level_transpose_and_gradient_are_the_two_level_form(orc, bc):
    """L = 2: A^T and dL/dbeta equal the two-level oracle's (separate code: row functions
    of the two-level form)."""
    n = 8
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    fb = I.chop((4, 4, 4), (11, 11, 11), 4)
    M = orc.MultiLevelProblem(dom, [I.chop(*dom, 4), fb], [bc] * 3, [bc] * 3)
    A = orc.AmrProblem(dom, I.chop(*dom, 4), fb, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(36)
    alphas, betas = rand_coeffs(M, rng, bc == P_, a=0.5)
    A.set_coeffs(0.5, 1.0, alpha_c=alphas[0], beta_c=betas[0], alpha_f=alphas[1], beta_f=betas[1])
    ys = [rng.standard_normal(s) * m for s, m in zip(M.shapes, M.masks)]
    xm = M.apply(ys, transpose=True)
    xc, xf = A.apply(ys[0], ys[1], transpose=True)
    sc = max(np.abs(xc).max(), np.abs(xf).max())
    assert np.abs(xm[0] - xc).max() <= 1e-13 * sc and np.abs(xm[1] - xf).max() <= 1e-13 * sc
    phis = [rng.standard_normal(s) for s in M.shapes]
    lams = [rng.standard_normal(s) * m for s, m in zip(M.shapes, M.masks)]
    gm = M.grad_beta(phis, lams, betas)
    gc, gf = A.grad_beta(phis[0], phis[1], lams[0], lams[1], betas[0], betas[1])
    gf = gf * M.masks[1]
    sc = max(np.abs(gc).max(), np.abs(gf).max())
    assert np.abs(gm[0] - gc).max() <= 1e-13 * sc and np.abs(gm[1] - gf).max() <= 1e-13 * sc


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_three_level_transpose_by_inner_products(orc, bc):
    """<A x, y> = <x, A^T y> over the composite unknowns: A x from the rows evaluated
    directly, A^T y scattered term by term."""
    dom, lb = three_levels(8)
    M = orc.MultiLevelProblem(dom, lb, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(37)
    rand_coeffs(M, rng, bc == P_, a=0.0 if bc != D_ else 1.0)
    for _ in range(3):
        xs = [rng.standard_normal(s) * m for s, m in zip(M.shapes, M.masks)]
        ys = [rng.standard_normal(s) * m for s, m in zip(M.shapes, M.masks)]
        ax = M.pack(M.apply(xs))
        aty = M.pack(M.apply(ys, transpose=True))
        lhs, rhs = ax @ M.pack(ys), M.pack(xs) @ aty
        assert abs(lhs - rhs) <= 1e-13 * (np.abs(ax) @ np.abs(M.pack(ys)))
    # and the assembled matrix's transpose, column by column, on one level-2 and one level-0 unknown
    A = M.matrix() if M.pack([np.zeros(s) for s in M.shapes]).size <= 2000 else None
    if A is not None:
        m = A.shape[0]
        for j in (0, m - 1):
            e = np.zeros(m)
            e[j] = 1.0
            assert np.abs(M.pack(M.apply(M.unpack(e), transpose=True)) - A[j]).max() <= 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("bc", [P_, D_, N_])
def test_three_level_gradient_by_central_differences(orc, bc):
    """dL/dbeta for L = lambda^T (rhs - A(beta) phi) against central differences of
    <lambda, A(beta (1 + eps v)) phi> in random relative directions v (all cells of every
    level, covered ones included: their beta shapes only the correction operator, so their
    gradient is 0), eps = 1e-5."""
    dom, lb = three_levels(8)
    M = orc.MultiLevelProblem(dom, lb, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(38)
    alphas, betas = rand_coeffs(M, rng, bc == P_, a=0.4)
    phis = [rng.standard_normal(s) for s in M.shapes]
    lams = [rng.standard_normal(s) * m for s, m in zip(M.shapes, M.masks)]
    g = M.grad_beta(phis, lams, betas)
    for l in range(M.L - 1):
        under = M.inside[l + 1].reshape(M.shapes[l][0], 2, M.shapes[l][1], 2, M.shapes[l][2], 2).all(axis=(1, 3, 5))
        assert not g[l][under].any()

    def F(bs):
        M.set_coeffs(0.4, 1.0, alphas=alphas, betas=bs)
        return M.pack(lams) @ M.pack(M.apply(phis))

    for _ in range(3):
        vs = [rng.standard_normal(s) * I_ for s, I_ in zip(M.shapes, M.inside)]
        eps = 1e-5
        fd = (F([b * (1 + eps * v) for b, v in zip(betas, vs)]) - F([b * (1 - eps * v) for b, v in zip(betas, vs)])) / (2 * eps)
        pred = -sum((gl * b * v).sum() for gl, b, v in zip(g, betas, vs))
        assert abs(fd - pred) <= 1e-7 * abs(fd), (fd, pred)
    M.set_coeffs(0.4, 1.0, alphas=alphas, betas=betas)


def test_transpose_refuses_nesting_closer_than_two_cells(orc):
    """Level 2 one level-1 cell inside level 1's low x boundary: the fine ghost interpolation
    of level 1 reads a covered cell, so A is not a matrix over the unknowns; the transpose
    and the gradient refuse, the forward operator runs."""
    n = 16
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    l1 = I.chop((8, 8, 8), (23, 23, 23), 8)
    l2 = [((18, 20, 20), (29, 27, 27))]
    M = orc.MultiLevelProblem(dom, [I.chop(*dom, 8), l1, l2], [D_] * 3, [D_] * 3)
    M.set_coeffs(0.0, 1.0)
    xs = [np.ones(s) for s in M.shapes]
    M.apply(xs)
    with pytest.raises(ValueError):
        M.apply(xs, transpose=True)
    with pytest.raises(ValueError):
        M.grad_beta(xs, xs)
    # two cells in: accepted
    M2 = orc.MultiLevelProblem(dom, [I.chop(*dom, 8), l1, [((20, 20, 20), (29, 27, 27))]], [D_] * 3, [D_] * 3)
    M2.set_coeffs(0.0, 1.0)
    M2.apply(xs, transpose=True)


def four_levels(n=8):
    """four levels: level 0 is n^3 in boxes of n/2; level l >= 1 is a cube of n of its own
    cells from n/2, 3n/2, 7n/2 (in boxes of n/2), i.e. two or more cells inside the level below
    it, each box coarsened inside one box of that level"""
    dom = ((0, 0, 0), (n - 1, n - 1, n - 1))
    h = n // 2
    los = [0, n // 2, 3 * n // 2, 7 * n // 2]  # low corner of level l in its own index space
    lbs = [I.chop(*dom, h)] + [I.chop((lo,) * 3, (lo + n - 1,) * 3, h) for lo in los[1:]]
    return dom, lbs


@pytest.mark.parametrize("bc", [P_, D_])
def test_four_levels_reach_lapack_and_transpose(orc, bc):
    """The maximum of four levels: the composite iteration reaches LAPACK's solution of the
    assembled system, and the transpose scatters the assembled matrix's rows."""
    dom, lb = four_levels(8)
    M = orc.MultiLevelProblem(dom, lb, [bc] * 3, [bc] * 3)
    rng = np.random.default_rng(39)
    rand_coeffs(M, rng, bc == P_, a=1.0 if bc == D_ else 0.0)
    A = M.matrix()
    m = A.shape[0]
    r = M.pack([rng.standard_normal(s) for s in M.shapes])
    if bc != D_:
        V = M.volumes()
        r = r - (V @ r) / V.sum()
        B = np.zeros((m + 1, m + 1))
        B[:m, :m] = A
        B[:m, m] = 1.0
        B[m, :m] = V
        want = np.linalg.solve(B, np.concatenate([r, [0.0]]))[:m]
    else:
        want = np.linalg.solve(A, r)
    ps, it, hist, st = M.solve(M.unpack(r), tol_rel=1e-13, maxit=200)
    assert st == 0
    assert np.abs(M.pack(ps) - want).max() <= 1e-10 * np.abs(want).max()
    y = rng.standard_normal(m)
    assert np.abs(M.pack(M.apply(M.unpack(y), transpose=True)) - A.T @ y).max() <= 1e-12 * np.abs(A).max() * np.abs(y).max() * 10
