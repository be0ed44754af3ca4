"""Pins of the oracle's trilinear interpolation of the coarse correction (the option next to
piecewise-constant interpolation; Sec. "Operations between levels" names interpolation
without fixing its order).

A fine cell's centre lies a quarter of a coarse cell from its parent's centre along each
axis, so trilinear interpolation takes weights 3/4 (parent's coordinate) and 1/4 (the
neighbour's) per axis.  Facts fixed by that, independent of the oracle's code:
  * a field linear in the coordinates is reproduced exactly wherever the eight coarse cells
    used lie in the domain;
  * constants are reproduced everywhere under periodic and Neumann walls (the homogeneous
    Neumann extension mirrors the value);
  * next to a Dirichlet wall the coarse field is extended by its negative mirror image, so a
    constant 1 interpolates to 3/4 - 1/4 = 1/2 in the fine cells touching one wall and to
    1/2 * 1/2 = 1/4 in the cells touching two;
  * the result does not depend on the box layout;
  * the multigrid iteration with it still converges to the discrete solution (LAPACK).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_12009_gb300 import inputs as I

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


def cube(n):
    return ((0, 0, 0), (n - 1, n - 1, n - 1))


def _prolong(P, coarse_dense):
    """fine = trilinear interpolation of a dense coarse field (level 1 -> level 0), dense."""
    P.set_prolong(trilinear=True)
    fine = np.zeros(P.level_size(0))
    P.prolong_add(0, P.to_boxed(1, coarse_dense), fine)
    return P.to_dense(0, fine)


def _centres(shape, h):
    nz, ny, nx = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * h[2], (np.arange(ny) + 0.5) * h[1], (np.arange(nx) + 0.5) * h[0],
                          indexing="ij")
    return x, y, z


@pytest.mark.parametrize("bc", [[P_] * 3, [D_] * 3, [N_, D_, P_]], ids=["periodic", "dirichlet", "mixed"])
def test_linear_fields_exact_in_the_interior(bc):
    n = 16
    P = O.Problem(cube(n), I.chop(*cube(n), 8), bc, bc)
    P.set_coeffs(0.0, 1.0)
    hc, hf = (2.0 / n,) * 3, (1.0 / n,) * 3
    xc, yc, zc = _centres((n // 2,) * 3, hc)
    lin = lambda x, y, z: 0.3 + 1.7 * x - 2.1 * y + 0.9 * z  # noqa: E731
    got = _prolong(P, lin(xc, yc, zc))
    xf, yf, zf = _centres((n,) * 3, hf)
    want = lin(xf, yf, zf)
    inner = (slice(1, -1),) * 3  # fine cells whose eight coarse cells are all in the domain
    assert np.abs(got[inner] - want[inner]).max() <= 1e-14 * np.abs(want).max()


@pytest.mark.parametrize("bc", [[P_] * 3, [N_] * 3, [N_, P_, N_]], ids=["periodic", "neumann", "neumann_periodic"])
def test_constants_reproduced_everywhere(bc):
    n = 16
    P = O.Problem(cube(n), I.chop(*cube(n), 8), bc, bc)
    P.set_coeffs(0.0, 1.0)
    got = _prolong(P, np.full((n // 2,) * 3, 3.7))
    assert np.abs(got - 3.7).max() <= 4e-16 * 3.7


def test_dirichlet_walls_halve_per_wall():
    n = 16
    bc = [D_, D_, P_]
    P = O.Problem(cube(n), I.chop(*cube(n), 8), bc, bc)
    P.set_coeffs(0.0, 1.0)
    got = _prolong(P, np.ones((n // 2,) * 3))  # (z, y, x)
    wx = np.ones(n)
    wx[0] = wx[-1] = 0.5
    want = np.broadcast_to(wx[None, :, None] * wx[None, None, :], got.shape)
    assert np.array_equal(got, want)


def test_box_layout_invariance():
    n = 16
    rng = np.random.default_rng(44)
    coarse = rng.standard_normal((n // 2,) * 3)
    out = []
    for mgs in (16, 8, 4):
        P = O.Problem(cube(n), I.chop(*cube(n), mgs), [D_, P_, N_], [N_, P_, D_])
        P.set_coeffs(0.0, 1.0)
        out.append(_prolong(P, coarse))
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_solve_with_trilinear_reaches_lapack():
    """The interpolation changes the V-cycle, not the fixed point: the iteration with
    trilinear interpolation converges to the LAPACK solution of the discrete system."""
    n = 8
    rng = np.random.default_rng(45)
    P = O.Problem(cube(n), I.chop(*cube(n), 4), [D_, N_, D_], [N_, D_, D_], (0, 0, 0), (1.0, 0.8, 1.2))
    beta = np.exp(rng.standard_normal((n,) * 3))
    P.set_coeffs(0.0, 1.0, beta=beta)
    N = n ** 3
    A = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N)
        e[c] = 1.0
        A[:, c] = P.apply(e.reshape((n,) * 3)).reshape(-1)
    rhs = rng.standard_normal((n,) * 3)
    x = np.linalg.solve(A, rhs.reshape(-1))
    P.set_prolong(trilinear=True)
    phi, it, hist, st = P.solve(rhs, tol_rel=1e-13, maxit=200)
    assert st == O.OK
    assert np.abs(phi.reshape(-1) - x).max() <= 1e-10 * np.abs(x).max()
