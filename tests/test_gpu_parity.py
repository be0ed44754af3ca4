"""CUDA path vs the FP64 CPU oracle, element by element, through the C ABI.

Every hot-path step (ghost exchange, one red-black colour, residual, restriction,
prolongation, coefficient coarsening, BiCGStab bottom, V-cycle, outer loop) is run on the
same seeded inputs by the library and by the oracle.  Tolerances:
  * copies (ghost exchange), restriction and prolongation in FP64: bit-exact (the same
    additions in the same order);
  * other FP64 steps: 1e-12 of the field's scale (a handful of rounding differences:
    the kernels multiply by a stored 1/D where the oracle divides, and fuse multiply-adds);
  * float steps: 1e-5 of scale (inputs rounded to float, float arithmetic);
  * bfloat16-stored steps: 2e-2 of scale (8-bit mantissa storage);
  * whole solves at a fixed iteration count: 1e-10 relative (the requirement for FP64).
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_12009_gb300 import gmg  # noqa: E402

DTS = [gmg.DT_F64, gmg.DT_F32, gmg.DT_BF16]
STEP_TOL = {gmg.DT_F64: 1e-12, gmg.DT_F32: 1e-5, gmg.DT_BF16: 2e-2}


def round_to(x, dt):
    t = torch.as_tensor(x, dtype=torch.float64)
    if dt == gmg.DT_F32:
        t = t.float().double()
    elif dt == gmg.DT_BF16:
        t = t.bfloat16().double()
    return t.numpy()


class Pair:
    """The same problem in the oracle (P) and in the library (C)."""

    def __init__(self, name, mixed=True):
        self.cfg = c = cases.make(name)
        ph = c.get("prob_hi", (1.0, 1.0, 1.0))
        self.P = O.Problem(c["domain"], c["boxes"], c["bc_lo"], c["bc_hi"], (0, 0, 0), ph)
        self.P.set_coeffs(c["a"], c["b"], alpha=c["alpha"], beta=c["beta"])
        self.C = gmg.Context(c["domain"], c["bc_lo"], c["bc_hi"], prob_hi=ph, boxes=c["boxes"],
                             stream=torch.cuda.current_stream().cuda_stream)
        self.C.allocate(gmg.MIXED_FP32 if mixed else gmg.FP64)
        self.C.set_scalars(c["a"], c["b"])
        if c["alpha"] is not None:
            self.C.set_alpha(torch.from_numpy(c["alpha"]))
        self.C.set_beta(torch.from_numpy(c["beta"]) if c["beta"] is not None else None)
        self.nlev = self.P.nlevels
        assert self.C.nlevels == self.nlev

    def gpu_boxes(self, buf, m):
        """GPU boxed buffer -> list of ghosted float64 numpy blocks."""
        return [v.double().cpu().numpy() for v in self.C.box_views(buf, m)]

    def orc_boxes(self, boxed, m):
        return [self.P.box_view(m, boxed, b) for b in range(len(self.P.level_boxes(m)))]


@pytest.fixture(scope="module", params=cases.NAMES)
def pair(request):
    return Pair(request.param)


def rand_level(pair, m, seed, dt):
    rng = np.random.default_rng(seed)
    return round_to(rng.standard_normal(pair.P.level_shape(m)), dt)


# ----------------------------------------------------------------------------- coefficients


def test_coefficients(pair):
    """Sec. "Linear Solvers" (beta on faces) and Sec. "Operations between levels" (averaged
    coarse coefficients): scaled weights w = b*beta/h^2 and diagonal on every level."""
    c = pair.cfg
    for m in range(pair.nlev):
        al, bx, by, bz = pair.P.coeffs(m)
        h = [c.get("prob_hi", (1, 1, 1))[d] / (c["domain"][1][d] + 1) * 2 ** m for d in range(3)]
        wx, wy, wz, D = pair.C.coeffs(m)
        want = [c["b"] * bx / h[0] ** 2, c["b"] * by / h[1] ** 2, c["b"] * bz / h[2] ** 2]
        for d, (g, w) in enumerate(zip((wx, wy, wz), want)):
            gb, ob = pair.gpu_boxes(g, m), pair.orc_boxes(w, m)
            for b, (gv, ov) in enumerate(zip(gb, ob)):
                # faces 0..n along d live in slots 1..n+1 of the ghosted block
                sl = [slice(1, -1)] * 3
                sl[2 - d] = slice(1, None)
                np.testing.assert_allclose(gv[tuple(sl)], ov[tuple(sl)], rtol=1e-14, atol=0)
        gb = pair.gpu_boxes(D, m)
        for b, gv in enumerate(gb):
            ob_al = pair.P.box_view(m, al, b)
            oxs = [pair.P.box_view(m, f, b) for f in (bx, by, bz)]
            want_d = c["a"] * ob_al[1:-1, 1:-1, 1:-1]
            want_d = want_d + c["b"] / h[0] ** 2 * (oxs[0][1:-1, 1:-1, 1:-1] + oxs[0][1:-1, 1:-1, 2:])
            want_d = want_d + c["b"] / h[1] ** 2 * (oxs[1][1:-1, 1:-1, 1:-1] + oxs[1][1:-1, 2:, 1:-1])
            want_d = want_d + c["b"] / h[2] ** 2 * (oxs[2][1:-1, 1:-1, 1:-1] + oxs[2][2:, 1:-1, 1:-1])
            np.testing.assert_allclose(gv[1:-1, 1:-1, 1:-1], want_d, rtol=1e-13, atol=0)


# ----------------------------------------------------------------------------- ghost exchange


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("colour", [-1, 0, 1])
def test_fill_boundary(pair, dt, colour):
    """Sec. "Operations on a level" / "Communication": every face ghost equals the owning
    box's cell (periodic images included) or minus the adjacent cell at a wall; a colour
    fill touches only ghosts of that global parity.  Exact copies."""
    for m in range(pair.nlev):
        x = rand_level(pair, m, 1000 + m, dt)
        f = pair.C.pack(torch.from_numpy(x), m, dt)
        before = pair.gpu_boxes(f, m)
        pair.C.fill_boundary(f, m, dt, colour)
        got = pair.gpu_boxes(f, m)
        ob = pair.P.to_boxed(m, x)
        pair.P.fill_ghosts(m, ob)
        want = pair.orc_boxes(ob, m)
        boxes = pair.P.level_boxes(m)
        for b, (g, w, g0) in enumerate(zip(got, want, before)):
            lo, hi = boxes[b]
            n = [hi[d] - lo[d] + 1 for d in range(3)]
            K, J, II = np.meshgrid(*(np.arange(-1, n[q] + 1) for q in (2, 1, 0)), indexing="ij")
            par = (II + J + K + lo[0] + lo[1] + lo[2]) % 2
            face = ((II < 0) | (II >= n[0])).astype(int) + ((J < 0) | (J >= n[1])) + ((K < 0) | (K >= n[2]))
            ghost = face == 1
            sel = ghost if colour < 0 else ghost & (par == colour)
            np.testing.assert_array_equal(g[sel], w[sel])
            np.testing.assert_array_equal(g[~sel], g0[~sel])


# ----------------------------------------------------------------------------- smoother


@pytest.mark.parametrize("dt", DTS)
def test_smooth_colour(pair, dt):
    """One red then one black half sweep (each preceded by its ghost fill) against the
    oracle's Gauss-Seidel colour update."""
    for m in range(pair.nlev):
        phi = rand_level(pair, m, 2000 + m, dt)
        rhs = rand_level(pair, m, 3000 + m, dt)
        g = pair.C.pack(torch.from_numpy(phi), m, dt)
        gr = pair.C.pack(torch.from_numpy(rhs), m, dt)
        o = pair.P.to_boxed(m, phi)
        orr = pair.P.to_boxed(m, rhs)
        for colour in (0, 1):
            pair.C.smooth(g, gr, m, dt, colour)
            pair.P.smooth_colour(m, o, orr, colour)
            got = pair.C.unpack(g, m, dt).cpu().numpy()
            want = pair.P.to_dense(m, o)
            scale = np.abs(want).max()
            assert np.abs(got - want).max() <= STEP_TOL[dt] * scale, (m, colour, np.abs(got - want).max(), scale)
            o = pair.P.to_boxed(m, round_to(want, dt))  # keep both sides on the same input


# ----------------------------------------------------------------------------- residual


@pytest.mark.parametrize("dt", DTS)
def test_residual(pair, dt):
    for m in range(pair.nlev):
        phi = rand_level(pair, m, 4000 + m, dt)
        rhs = rand_level(pair, m, 5000 + m, dt)
        g = pair.C.pack(torch.from_numpy(phi), m, dt)
        gr = pair.C.pack(torch.from_numpy(rhs), m, dt)
        r, nrm = pair.C.residual(g, gr, m, dt, dt, norm=True)
        got = pair.C.unpack(r, m, dt).cpu().numpy()
        want = pair.P.to_dense(m, pair.P.residual(m, pair.P.to_boxed(m, phi), pair.P.to_boxed(m, rhs)))
        D = pair.C.unpack(pair.C.coeffs(m)[3], m).cpu().numpy()
        scale = np.abs(rhs).max() + np.abs(D).max() * np.abs(phi).max()
        assert np.abs(got - want).max() <= STEP_TOL[dt] * scale
        # fused L-inf norm of what was computed in the kernel's own precision
        assert abs(nrm - np.abs(want).max()) <= STEP_TOL[dt] * scale


# ------------------------------------------------------------------- transfer operators


@pytest.mark.parametrize("dt", DTS)
def test_restrict_prolong(pair, dt):
    for m in range(pair.nlev - 1):
        fine = rand_level(pair, m, 6000 + m, dt)
        coarse = rand_level(pair, m + 1, 7000 + m, dt)
        gc = pair.C.restrict(pair.C.pack(torch.from_numpy(fine), m, dt), m, dt)
        got = pair.C.unpack(gc, m + 1, dt).cpu().numpy()
        want = pair.P.to_dense(m + 1, pair.P.restrict(m, pair.P.to_boxed(m, fine)))
        gf = pair.C.pack(torch.from_numpy(fine), m, dt)
        pair.C.prolong_add(pair.C.pack(torch.from_numpy(coarse), m + 1, dt), gf, m, dt)
        gotp = pair.C.unpack(gf, m, dt).cpu().numpy()
        of = pair.P.to_boxed(m, fine)
        pair.P.prolong_add(m, pair.P.to_boxed(m + 1, coarse), of)
        wantp = pair.P.to_dense(m, of)
        if dt == gmg.DT_F64:
            np.testing.assert_array_equal(got, want)
            np.testing.assert_array_equal(gotp, wantp)
        else:
            tol = STEP_TOL[dt]
            assert np.abs(got - want).max() <= tol * np.abs(want).max()
            assert np.abs(gotp - wantp).max() <= tol * np.abs(wantp).max()


# ------------------------------------------------------------------------- bottom solve


@pytest.mark.parametrize("dt", [gmg.DT_F64, gmg.DT_F32])
def test_bottom(pair, dt):
    mb = pair.nlev - 1
    rhs = rand_level(pair, mb, 8000, dt)
    x, it = pair.C.bottom_solve(pair.C.pack(torch.from_numpy(rhs), mb, dt), dt)
    got = pair.C.unpack(x, mb, dt).cpu().numpy()
    want_b, oit = pair.P.bottom(pair.P.to_boxed(mb, rhs))
    want = pair.P.to_dense(mb, want_b)
    tol = 1e-9 if dt == gmg.DT_F64 else 1e-5
    if dt == gmg.DT_F64:
        assert abs(it - oit) <= 1
    assert np.abs(got - want).max() <= tol * np.abs(want).max() or abs(it - oit) == 1


# ---------------------------------------------------------------------------- V-cycle


@pytest.mark.parametrize("fused", [1, 0], ids=["fused_coarse", "per_level"])
@pytest.mark.parametrize("dt", DTS)
def test_vcycle(pair, dt, fused):
    """One V-cycle, with the coarse end of the cycle run by one thread block (fused) or by
    a grid launch per step and level."""
    r = rand_level(pair, 0, 9000, dt)
    if pair.cfg["name"] == "periodic":
        r = round_to(r - r.mean(), dt)
    e = pair.C.vcycle(pair.C.pack(torch.from_numpy(r), 0, dt), dt, fused_coarse=fused)
    got = pair.C.unpack(e, 0, dt).cpu().numpy()
    want = pair.P.to_dense(0, pair.P.vcycle(0, pair.P.to_boxed(0, r)))
    tol = {gmg.DT_F64: 1e-10, gmg.DT_F32: 2e-4, gmg.DT_BF16: 6e-2}[dt]
    assert np.abs(got - want).max() <= tol * np.abs(want).max(), np.abs(got - want).max() / np.abs(want).max()


# ------------------------------------------------------------------------- whole solve


@pytest.mark.parametrize("fused", [1, 0], ids=["fused_coarse", "per_level"])
@pytest.mark.parametrize("graph", [1, 0])
def test_solve_fixed_iterations(pair, graph, fused):
    """Outer loop (Sec. "Linear Solvers"): the same number of V-cycles from phi = 0 gives the
    same iterate to 1e-10 relative, and the same residual history."""
    c = pair.cfg
    nit = 6
    rhs = pair.C.pack(torch.from_numpy(c["rhs"]))
    phi, info = pair.C.solve(rhs, tol_rel=0.0, max_iter=nit, use_graph=graph, fused_coarse=fused)
    got = pair.C.unpack(phi).cpu().numpy()
    want, it, hist, st = pair.P.solve(c["rhs"], tol_rel=0.0, maxit=nit)
    assert info.iterations == it == nit
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    gh = np.array(info.history())
    # residual histories agree until they reach the rounding floor of the FP64 residual
    np.testing.assert_allclose(gh, hist, rtol=1e-6, atol=1e-11 * hist[0])


def test_solve_to_tolerance(pair):
    """Both solvers stopped at 1e-12 agree to 1e-10 (the FP64 parity requirement)."""
    c = pair.cfg
    rhs = pair.C.pack(torch.from_numpy(c["rhs"]))
    phi, info = pair.C.solve(rhs, tol_rel=1e-12, max_iter=300)
    want, it, hist, st = pair.P.solve(c["rhs"], tol_rel=1e-12, maxit=300)
    assert info.status == gmg.OK and st == O.OK
    got = pair.C.unpack(phi).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    assert abs(info.iterations - it) <= 1


@pytest.mark.parametrize("prec", [gmg.MIXED_FP32, gmg.MIXED_BF16])
def test_mixed_precision_reaches_fp64_tolerance(pair, prec):
    """Iterative refinement with a float (or bfloat16-stored) V-cycle reaches the FP64
    relative residual 1e-10; its error against the FP64 oracle solution stays within ten
    times the FP64 solve's own error at that residual, or 1e-9 relative."""
    c = pair.cfg
    rhs = pair.C.pack(torch.from_numpy(c["rhs"]))
    phi, info = pair.C.solve(rhs, tol_rel=1e-10, max_iter=300, precision=prec)
    assert info.status == gmg.OK, info.status
    assert info.final_resid <= 1e-10 * info.rhs_norm
    # the FP64 residual of the returned solution, recomputed by the oracle
    got = pair.C.unpack(phi).cpu().numpy()
    rhs_eff = c["rhs"] - (c["rhs"].mean() if c["name"] == "periodic" else 0.0)
    r = rhs_eff - pair.P.apply(got)
    assert np.abs(r).max() <= 1.01e-10 * np.abs(c["rhs"]).max()
    want, it, hist, st = pair.P.solve(c["rhs"], tol_rel=1e-12, maxit=300)
    phi64, info64 = pair.C.solve(pair.C.pack(torch.from_numpy(c["rhs"])), tol_rel=1e-10, max_iter=300)
    e64 = np.abs(pair.C.unpack(phi64).cpu().numpy() - want).max()
    emx = np.abs(got - want).max()
    assert emx <= 10 * e64 + 1e-9 * np.abs(want).max(), (emx, e64)


def test_apply(pair):
    c = pair.cfg
    x = np.random.default_rng(11).standard_normal(pair.P.level_shape(0))
    out = pair.C.apply(pair.C.pack(torch.from_numpy(x)))
    got = pair.C.unpack(out).cpu().numpy()
    want = pair.P.apply(x)
    D = pair.C.unpack(pair.C.coeffs(0)[3]).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-12 * np.abs(D).max() * np.abs(x).max()


@pytest.mark.parametrize("graph", [1, 0])
def test_profiled_solve_times_kernels(graph):
    """profile = 1 records events around the finest-level smoother and outer residual
    launches (as timestamped graph nodes when the iteration is a captured graph)."""
    pair = Pair("uneven", mixed=False)
    rhs = pair.C.pack(torch.from_numpy(pair.cfg["rhs"]))
    for fuse, per_iter in ((0, 8), (1, 7)):  # fused: the first red half-sweep runs in the residual
        phi, info = pair.C.solve(rhs, tol_rel=0.0, max_iter=3, use_graph=graph, profile=1, fuse_residual_sweep=fuse,
                                 wave_sweep=0)
        assert info.status == gmg.NOT_CONVERGED  # tol 0 is never reached; 3 iterations run
        assert info.smooth0_launches == 3 * per_iter and info.resid0_launches == 3
        assert info.smooth0_ms > 0 and info.resid0_ms > 0
        assert info.kernel_launches > 3 * per_iter


def test_fused_coarse_launches_fewer_kernels():
    """abec-like 64^3 problem in 8 boxes: the fused coarse end replaces the per-level launches
    of the levels at or below 4096 cells by one launch per V-cycle, and gives the same
    iterates (the bottom's dot products add in another order: 1e-12)."""
    from paper_2009_12009_gb300 import inputs as I

    cfg = I.abec(64, 32, 4242, name="abec64")
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"],
                    stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64)
    C.set_scalars(cfg["a"], cfg["b"])
    C.set_beta(torch.from_numpy(cfg["beta"]))
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    out = {}
    for fused in (1, 0):
        phi, info = C.solve(rhs, tol_rel=0.0, max_iter=5, fused_coarse=fused)
        out[fused] = (C.unpack(phi).cpu().numpy(), info.kernel_launches)
    a, b = out[1][0], out[0][0]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert out[1][1] < out[0][1]


def _ctx_of(cfg, precision=gmg.MIXED_FP32):
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"],
                    prob_hi=cfg.get("prob_hi", (1.0, 1.0, 1.0)), stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(precision)
    C.set_scalars(cfg["a"], cfg["b"])
    C.set_beta(torch.from_numpy(cfg["beta"]))
    return C


def _sweep_cases():
    from paper_2009_12009_gb300 import inputs as I

    rng = np.random.default_rng(77)
    uneven_dom = ((0, 0, 0), (129, 99, 89))  # boxes 64/64/2 x 64/36 x 64/26: x-faces 2 cells apart
    shape = (90, 100, 130)
    uneven = dict(name="uneven_large", domain=uneven_dom, boxes=I.chop(*uneven_dom, 64), bc_lo=[I.DIRICHLET] * 3,
                  bc_hi=[I.DIRICHLET] * 3, a=0.0, b=1.0, beta=I.lognormal_beta(rng, shape, periodic=False),
                  rhs=rng.standard_normal(shape), prob_hi=(130 / 128, 100 / 128, 90 / 128))
    return [I.abec(128, 64, 4343, name="abec128"), I.abec(128, 32, 4344, bc=I.PERIODIC, name="per128"), uneven]


@pytest.mark.parametrize("case", [0, 1, 2], ids=["abec128", "periodic128_boxes32", "uneven_large"])
def test_fused_sweep_is_bitwise_two_half_sweeps(case):
    """Levels of >= 2^17 cells: the dataflow sweep (every colour pass of a smoothing step in
    one launch) gives bit for bit the V-cycle and the solve of one launch per colour, in
    FP64, FP32 and BF16, with fewer launches."""
    cfg = _sweep_cases()[case]
    C = _ctx_of(cfg)
    r = torch.from_numpy(cfg["rhs"] - (cfg["rhs"].mean() if cfg["bc_lo"][0] == gmg.PERIODIC else 0.0))
    for dt in DTS:
        rb = C.pack(r, 0, dt)
        e1 = C.vcycle(rb, dt, fused_sweep=1, wave_sweep=0)
        e0 = C.vcycle(rb, dt, fused_sweep=0, wave_sweep=0)
        assert torch.equal(C.unpack(e1, 0, dt), C.unpack(e0, 0, dt)), dt
    rhs = C.pack(r)
    p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=2, fused_sweep=1, project_mean=1, wave_sweep=0)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=2, fused_sweep=0, project_mean=1, wave_sweep=0)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.kernel_launches < i0.kernel_launches


@pytest.mark.parametrize("name", ["uneven", "periodic", "helmholtz", "poisson32", "neumann", "mixedwalls"])
def test_ghost_push_is_bitwise_ghost_exchange(name):
    """The smoother and interpolation writing their new values into the ghosts that copy
    them gives bit for bit the V-cycle and the solve of the ghost exchange before every
    colour, in FP64, FP32 and BF16 (walls, periodic images and uneven boxes)."""
    cfg = cases.make(name)
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], prob_hi=cfg.get("prob_hi", (1.0, 1.0, 1.0)),
                    boxes=cfg["boxes"], stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.MIXED_FP32)
    C.set_scalars(cfg["a"], cfg["b"])
    if cfg["alpha"] is not None:
        C.set_alpha(torch.from_numpy(cfg["alpha"]))
    C.set_beta(torch.from_numpy(cfg["beta"]) if cfg["beta"] is not None else None)
    r = cfg["rhs"] - (cfg["rhs"].mean() if name in ("periodic", "poisson32") else 0.0)
    for dt in DTS:
        rb = C.pack(torch.from_numpy(r), 0, dt)
        e1 = C.unpack(C.vcycle(rb, dt, ghost_push=1), 0, dt)
        e0 = C.unpack(C.vcycle(rb, dt, ghost_push=0), 0, dt)
        assert torch.equal(e1, e0), dt
    rhs = C.pack(torch.from_numpy(r))
    p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=3, ghost_push=1, project_mean=1)
    a1 = C.unpack(p1).clone()
    p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=3, ghost_push=0, project_mean=1)
    assert torch.equal(a1, C.unpack(p0))
    assert i1.kernel_launches < i0.kernel_launches


def test_autotune_keeps_results():
    """gmg_autotune measures push vs exchange per level and the fused coarse end, records a
    choice for every eligible level, and solves with the tuned defaults give the iterates of
    the untuned per-level path (the fused bottom adds its dot products in another order)."""
    from paper_2009_12009_gb300 import inputs as I

    cfg = I.abec(64, 16, 4545, name="abec64_16")
    C = _ctx_of(cfg, gmg.MIXED_FP32)
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    for prec in (gmg.FP64, gmg.MIXED_FP32):
        t = C.autotune(rhs, prec)
        assert t["fused_coarse"] in (0, 1) and min(t["vcycle_ms"]) > 0
        smoothed = [lv for lv in t["levels"] if lv[0] >= 0]
        assert smoothed and all(0 <= v <= 3 and a >= 0 and b > 0 for v, a, b in smoothed)
        p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=4, precision=prec)
        a1 = C.unpack(p1).cpu().numpy()
        p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=4, precision=prec, ghost_push=0, fused_coarse=0)
        a0 = C.unpack(p0).cpu().numpy()
        assert np.abs(a1 - a0).max() <= 1e-12 * np.abs(a0).max()


@pytest.mark.parametrize("case", ["abec64_boxes16", "helmholtz", "periodic"])
def test_vector_smooth_is_bitwise_pair_smooth(case):
    """One thread per 4 cells with vector loads (float and bfloat16), and one thread per pair
    with 128-bit pair loads (FP64), give bit for bit the V-cycle and the solve of one thread
    per cell pair with scalar loads."""
    from paper_2009_12009_gb300 import inputs as I

    cfg = I.abec(64, 16, 4646, name=case) if case == "abec64_boxes16" else cases.make(case)
    C = _ctx_of(cfg) if case == "abec64_boxes16" else None
    if C is None:
        C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], prob_hi=cfg.get("prob_hi", (1.0, 1.0, 1.0)),
                        boxes=cfg["boxes"], stream=torch.cuda.current_stream().cuda_stream)
        C.allocate(gmg.MIXED_FP32)
        C.set_scalars(cfg["a"], cfg["b"])
        if cfg["alpha"] is not None:
            C.set_alpha(torch.from_numpy(cfg["alpha"]))
        C.set_beta(torch.from_numpy(cfg["beta"]) if cfg["beta"] is not None else None)
    r = cfg["rhs"] - (cfg["rhs"].mean() if cfg["bc_lo"][0] == gmg.PERIODIC and cfg["a"] == 0 else 0.0)
    for dt in (gmg.DT_F64, gmg.DT_F32, gmg.DT_BF16):
        rb = C.pack(torch.from_numpy(r), 0, dt)
        for push in (0, 1):
            e1 = C.unpack(C.vcycle(rb, dt, vector_smooth=1, ghost_push=push), 0, dt)
            e0 = C.unpack(C.vcycle(rb, dt, vector_smooth=0, ghost_push=push), 0, dt)
            assert torch.equal(e1, e0), (dt, push)
    rhs = C.pack(torch.from_numpy(r))
    for prec in (gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16):
        p1, _ = C.solve(rhs, tol_rel=0.0, max_iter=3, precision=prec, vector_smooth=1, project_mean=1)
        a1 = C.unpack(p1).clone()
        p0, _ = C.solve(rhs, tol_rel=0.0, max_iter=3, precision=prec, vector_smooth=0, project_mean=1)
        assert torch.equal(a1, C.unpack(p0)), prec


@pytest.mark.parametrize("name", ["uneven", "periodic", "helmholtz", "poisson32", "neumann", "mixedwalls"])
def test_residual_fused_first_red_sweep_is_exact(name):
    """The outer residual also doing the first red half-sweep of the next V-cycle (e = r / D
    on red cells from e = 0) gives the iterates of the separate sweep (equal values; only
    the sign of exact zeros may differ), in FP64 and both mixed forms, with and without push."""
    cfg = cases.make(name)
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], prob_hi=cfg.get("prob_hi", (1.0, 1.0, 1.0)),
                    boxes=cfg["boxes"], stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.MIXED_FP32)
    C.set_scalars(cfg["a"], cfg["b"])
    if cfg["alpha"] is not None:
        C.set_alpha(torch.from_numpy(cfg["alpha"]))
    C.set_beta(torch.from_numpy(cfg["beta"]) if cfg["beta"] is not None else None)
    r = cfg["rhs"] - (cfg["rhs"].mean() if name in ("periodic", "poisson32") else 0.0)
    rhs = C.pack(torch.from_numpy(r))
    for prec in (gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16):
        for push in (0, 1):
            p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=4, precision=prec, ghost_push=push, fuse_residual_sweep=1,
                             project_mean=1, wave_sweep=0)
            a1 = C.unpack(p1).clone()
            p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=4, precision=prec, ghost_push=push, fuse_residual_sweep=0,
                             project_mean=1, wave_sweep=0)
            assert torch.equal(a1, C.unpack(p0)), (prec, push)
            assert i1.kernel_launches < i0.kernel_launches


@pytest.mark.parametrize("name", ["uneven", "periodic", "helmholtz", "poisson32", "neumann", "mixedwalls"])
def test_fused_correction_update_is_exact(name):
    """The last post-smoothing pass on the finest level also adding the correction to phi
    gives bit for bit the iterates of the separate update, in FP64 and both mixed forms,
    with ghost push and with exchange, and launches fewer kernels."""
    cfg = cases.make(name)
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], prob_hi=cfg.get("prob_hi", (1.0, 1.0, 1.0)),
                    boxes=cfg["boxes"], stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.MIXED_FP32)
    C.set_scalars(cfg["a"], cfg["b"])
    if cfg["alpha"] is not None:
        C.set_alpha(torch.from_numpy(cfg["alpha"]))
    C.set_beta(torch.from_numpy(cfg["beta"]) if cfg["beta"] is not None else None)
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    for prec in (gmg.FP64, gmg.MIXED_FP32, gmg.MIXED_BF16):
        for push in (0, 1):
            for graph in (1, 0):
                p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=4, precision=prec, ghost_push=push, fuse_correction=1,
                                 project_mean=1, use_graph=graph)
                a1 = C.unpack(p1).clone()
                p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=4, precision=prec, ghost_push=push, fuse_correction=0,
                                 project_mean=1, use_graph=graph)
                assert torch.equal(a1, C.unpack(p0)), (prec, push, graph)
                assert np.array_equal(i1.history(), i0.history())
                assert i1.kernel_launches < i0.kernel_launches


@pytest.mark.parametrize("name", ["uneven", "periodic", "helmholtz", "poisson32", "neumann", "mixedwalls", "oddlo"])
def test_settled_residuals_change_only_rounding(name):
    """Storing 0 for the residual of the colour smoothed last (away from walls) instead of
    computing it changes the iterates by rounding only: four FP64 iterations with and
    without agree to 1e-12 relative, residual histories to 1e-9, also with the symmetric
    V-cycle (last colour red) and without the ghost push.  A wall cell left out of the
    wall lists would keep a zero residual and fail this."""
    cfg = cases.make(name)
    C = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], prob_hi=cfg.get("prob_hi", (1.0, 1.0, 1.0)),
                    boxes=cfg["boxes"], stream=torch.cuda.current_stream().cuda_stream)
    C.allocate(gmg.FP64)
    C.set_scalars(cfg["a"], cfg["b"])
    if cfg["alpha"] is not None:
        C.set_alpha(torch.from_numpy(cfg["alpha"]))
    C.set_beta(torch.from_numpy(cfg["beta"]) if cfg["beta"] is not None else None)
    rhs = C.pack(torch.from_numpy(cfg["rhs"]))
    for rev in (0, 1):
        for push in (1, 0):
            p1, i1 = C.solve(rhs, tol_rel=0.0, max_iter=4, settled_zero=1, post_reverse=rev, ghost_push=push,
                             project_mean=1)
            a1 = C.unpack(p1).cpu().numpy()
            p0, i0 = C.solve(rhs, tol_rel=0.0, max_iter=4, settled_zero=0, post_reverse=rev, ghost_push=push,
                             project_mean=1)
            a0 = C.unpack(p0).cpu().numpy()
            assert np.abs(a1 - a0).max() <= 1e-12 * np.abs(a0).max(), (rev, push)
            np.testing.assert_allclose(i1.history(), i0.history(), rtol=1e-9)
            if rev == 0 and push == 1 and C.nlevels > 1:
                assert i1.kernel_launches >= i0.kernel_launches  # (the wall launches)


# ------------------------------------------------------------ trilinear interpolation option


@pytest.mark.parametrize("dt", DTS)
def test_prolong_trilinear(pair, dt):
    """Trilinear interpolation of a coarse field (its face, edge and corner ghosts filled by
    the homogeneous boundary rule) added to a fine one, on every pair of MG levels: FP64 bit
    for bit the oracle's (the same products and sums in the same order)."""
    pair.P.set_prolong(trilinear=True)
    try:
        import ctypes as C

        for m in range(pair.nlev - 1):
            coarse = rand_level(pair, m + 1, 9500 + m, dt)
            fine = rand_level(pair, m, 9600 + m, dt)
            fb = pair.C.pack(torch.from_numpy(fine), m, dt)
            cb = pair.C.pack(torch.from_numpy(coarse), m + 1, dt)
            st = gmg.lib().gmg_prolong_add_trilinear(pair.C.h, m, dt, C.c_void_p(cb.data_ptr()),
                                                     C.c_void_p(fb.data_ptr()))
            assert st == gmg.OK
            got = pair.C.unpack(fb, m, dt).cpu().numpy()
            wf = pair.P.to_boxed(m, fine)
            pair.P.prolong_add(m, pair.P.to_boxed(m + 1, coarse), wf)
            want = pair.P.to_dense(m, wf)
            if dt == gmg.DT_F64:
                assert np.array_equal(got, want), m
            else:
                want = round_to(want, dt)
                assert np.abs(got - want).max() <= STEP_TOL[dt] * np.abs(want).max(), m
    finally:
        pair.P.set_prolong(trilinear=False)


@pytest.mark.parametrize("dt", DTS)
def test_vcycle_trilinear(pair, dt):
    """One V-cycle with trilinear interpolation of the coarse corrections against the oracle's."""
    if pair.nlev < 2:
        pytest.skip("a single level: the V-cycle is the bottom solve, nothing is interpolated")
    r = rand_level(pair, 0, 9700, dt)
    if pair.cfg["name"] == "periodic":
        r = round_to(r - r.mean(), dt)
    e = pair.C.vcycle(pair.C.pack(torch.from_numpy(r), 0, dt), dt, prolongation=1)
    got = pair.C.unpack(e, 0, dt).cpu().numpy()
    pair.P.set_prolong(trilinear=True)
    try:
        want = pair.P.to_dense(0, pair.P.vcycle(0, pair.P.to_boxed(0, r)))
    finally:
        pair.P.set_prolong(trilinear=False)
    tol = {gmg.DT_F64: 1e-10, gmg.DT_F32: 2e-4, gmg.DT_BF16: 6e-2}[dt]
    assert np.abs(got - want).max() <= tol * np.abs(want).max(), np.abs(got - want).max() / np.abs(want).max()


def test_solve_trilinear(pair):
    """The multigrid iteration with trilinear interpolation: the same iterates and residual
    history as the oracle's for a fixed count, and to 1e-12 the same solution and count."""
    if pair.nlev < 2:
        pytest.skip("a single level: the V-cycle is the bottom solve, nothing is interpolated")
    c = pair.cfg
    rhs = pair.C.pack(torch.from_numpy(c["rhs"]))
    pair.P.set_prolong(trilinear=True)
    try:
        phi, info = pair.C.solve(rhs, tol_rel=0.0, max_iter=4, prolongation=1)
        got = pair.C.unpack(phi).cpu().numpy()
        want, it, hist, st = pair.P.solve(c["rhs"], tol_rel=0.0, maxit=4)
        assert info.iterations == it == 4
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
        np.testing.assert_allclose(np.array(info.history()), hist, rtol=1e-6, atol=1e-11 * hist[0])
        phi, info = pair.C.solve(rhs, tol_rel=1e-12, max_iter=300, prolongation=1)
        want, it, hist, st = pair.P.solve(c["rhs"], tol_rel=1e-12, maxit=300)
        assert info.status == gmg.OK and st == O.OK
        assert np.abs(pair.C.unpack(phi).cpu().numpy() - want).max() <= 1e-10 * np.abs(want).max()
        assert abs(info.iterations - it) <= 1
    finally:
        pair.P.set_prolong(trilinear=False)
