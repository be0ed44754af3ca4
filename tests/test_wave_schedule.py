"""The wavefront red-black sweep's tables and waiting rule, checked on the host (no GPU).

The wavefront kernel (one launch per Gauss-Seidel sweep of Sec. "Linear Solvers") lets each
thread block march through the planes of one tile -- a band of rows of one box -- a slab of
planes at a time: the red cells of the slab, a report, and then, once the tiles beside it
have reported those planes too, the black cells of every plane whose reds on both sides are
done.  These tests replay that schedule on the
host from the library's own tile tables (gmg_wave_tiles), cell by cell, in many random and
adversarial interleavings of the tiles' steps, and check what the two-pass sweep requires:
every red cell reads only black cells that are not yet updated, every black cell reads only
red cells that are (a wall's ghost is the cell's own image, read before its update), every
smoothed cell is updated exactly once, and no interleaving leaves every unfinished tile
waiting (no deadlock), also when fewer tiles than a batch holds can be resident at once.
Layouts whose boxes cannot be given marching directions (an odd number of boxes around a
periodic z, one box periodic in z) must have no tables.
"""
import numpy as np
import pytest

from paper_2009_12009_gb300 import gmg
from paper_2009_12009_gb300 import inputs as I

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN


class Prob:
    """one problem on one MG level: domain (bounding box of its boxes), walls, cell versions"""

    def __init__(self, lo, hi, bc_lo, bc_hi):
        self.lo = np.array(lo)
        self.n = np.array(hi) - self.lo + 1
        self.per = [bc_lo[d] == P_ for d in range(3)]
        self.V = np.zeros(tuple(self.n[::-1]), dtype=np.int8)  # (z, y, x)


def _nbr_versions(P, gi, gj, gk, d, sgn):
    """version of the neighbour across side sgn of axis d; a wall gives the cell's own image"""
    g = [gi - P.lo[0], gj - P.lo[1], gk - P.lo[2]]
    h = [a.copy() for a in g]
    h[d] = h[d] + sgn
    out = (h[d] < 0) | (h[d] >= P.n[d])
    if P.per[d]:
        h[d] = np.mod(h[d], P.n[d])
    else:
        h[d] = np.where(out, g[d], h[d])
    return P.V[h[2], h[1], h[0]]


class Replay:
    """tile t's program: steps of `slab` planes (marching order): red cells of planes
    [r0, r1), report r1, wait, black cells of planes [bdone, b1) with b1 = r1 - 1 (nz in the
    last step) -- the kernel's schedule, replayed cell by cell"""

    def __init__(self, C, m, probs_of_solve, slab):
        self.ppt, self.T = C.wave_tiles(m)
        boxes, _ = C.level_boxes(m)
        self.boxes = boxes
        self.probs = probs_of_solve
        self.slab = slab
        self.nt = len(self.T)
        self.r0 = np.zeros(self.nt, dtype=np.int64)     # next red plane (marching order)
        self.bdone = np.zeros(self.nt, dtype=np.int64)  # black planes done
        self.half = np.zeros(self.nt, dtype=np.int64)   # 0: red part of a step next, 1: black part
        self.count = np.zeros(self.nt, dtype=np.int64)  # red planes reported
        self.reds = 0
        self.blacks = 0

    def nz(self, t):
        lo, hi = self.boxes[self.T[t][0]]
        return hi[2] - lo[2] + 1

    def plane(self, t, q):
        return self.nz(t) - 1 - q if self.T[t][3] else q

    def done(self, t):
        return self.bdone[t] >= self.nz(t)

    def cells(self, t, k, colour):
        b, y0, y1 = self.T[t][0], self.T[t][1], self.T[t][2]
        lo, hi = self.boxes[b]
        ii, jj = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1] + y0, lo[1] + y1), indexing="xy")
        gk = np.full(ii.shape, lo[2] + k)
        sel = ((ii + jj + gk) & 1) == colour
        return ii[sel], jj[sel], gk[sel]

    def b1(self, t):
        r1 = self.count[t]
        return self.nz(t) if r1 == self.nz(t) else r1 - 1

    def waiting(self, t):
        """True if tile t's next action is a black part whose neighbours have not reported"""
        if self.half[t] == 0:
            return False
        b1, b0 = self.b1(t), self.bdone[t]
        if b1 <= b0:
            return False
        row = self.T[t]
        for u in range(4, 8):
            nb = row[u]
            if nb >= 0 and nb != t and self.count[nb] < b1:
                return True
        ks = [self.plane(t, q) for q in (b0, b1 - 1)]
        if min(ks) == 0 and row[8] >= 0 and self.count[row[8]] < row[10]:
            return True
        if max(ks) == self.nz(t) - 1 and row[9] >= 0 and self.count[row[9]] < row[11]:
            return True
        return False

    def act(self, t):
        P = self.probs[self.T[t][12]]
        nz = self.nz(t)
        if self.half[t] == 0:
            r0 = self.r0[t]
            r1 = min(nz, r0 + self.slab)
            for q in range(r0, r1):
                gi, gj, gk = self.cells(t, self.plane(t, q), 0)
                for d in range(3):
                    for sgn in (-1, 1):
                        v = _nbr_versions(P, gi, gj, gk, d, sgn)
                        assert not v.any(), f"red cell of tile {t} read an updated black cell"
                idx = (gk - P.lo[2], gj - P.lo[1], gi - P.lo[0])
                assert not P.V[idx].any(), "a red cell updated twice"
                P.V[idx] = 1
                self.reds += gi.size
            self.r0[t] = r1
            self.count[t] = r1
            self.half[t] = 1
            return
        for q in range(self.bdone[t], self.b1(t)):
            gi, gj, gk = self.cells(t, self.plane(t, q), 1)
            for d in range(3):
                for sgn in (-1, 1):
                    v = _nbr_versions(P, gi, gj, gk, d, sgn)
                    h = [gi - P.lo[0], gj - P.lo[1], gk - P.lo[2]][d] + sgn
                    wall = ((h < 0) | (h >= P.n[d])) & (not P.per[d])
                    assert np.all(v[~wall] == 1), f"black cell of tile {t} read a red cell not yet updated"
                    assert np.all(v[wall] == 0), "a black cell's wall image was updated before it"
            idx = (gk - P.lo[2], gj - P.lo[1], gi - P.lo[0])
            assert not P.V[idx].any(), "a black cell updated twice"
            P.V[idx] = 1
            self.blacks += gi.size
        self.bdone[t] = max(self.bdone[t], self.b1(t))
        self.half[t] = 0


def _run(C, m, probs, order, resident=None, rng=None, slab=1):
    """replay one sweep of level m; order: 'random', 'low', 'high' (which runnable tile acts next)"""
    R = Replay(C, m, probs, slab)
    slots = R.nt if resident is None else resident
    started = min(slots, R.nt)  # tiles get slots in ticket (table) order
    live = list(range(started))
    finished = 0
    while finished < R.nt:
        runnable = [t for t in live if not R.done(t) and not R.waiting(t)]
        assert runnable, f"level {m}: every resident unfinished tile waits (deadlock)"
        if order == "random":
            t = runnable[rng.integers(len(runnable))]
        elif order == "low":
            t = runnable[0]
        else:
            t = runnable[-1]
        R.act(t)
        if R.done(t):
            live.remove(t)
            finished += 1
            if started < R.nt:
                live.append(started)
                started += 1
    return R


def _single(domain, bc_lo, bc_hi, mgs):
    C = gmg.Context(domain, bc_lo, bc_hi, boxes=I.chop(*domain, mgs))
    return C


def _probs_single(C, m, bc_lo, bc_hi):
    _, dom = C.level_info(m)
    return [Prob(dom[0], dom[1], bc_lo, bc_hi)]


LAYOUTS = {
    "dir32_16": (((0, 0, 0), (31, 31, 31)), [D_] * 3, [D_] * 3, 16),
    "per32_8": (((0, 0, 0), (31, 31, 31)), [P_] * 3, [P_] * 3, 8),
    "walls": (((0, 0, 0), (23, 31, 39)), [N_, P_, D_], [D_, P_, N_], 8),
    "ragged": (((0, 0, 0), (35, 33, 19)), [D_] * 3, [D_] * 3, 16),
    "abec64_32": (((0, 0, 0), (63, 63, 63)), [D_] * 3, [D_] * 3, 32),
}


@pytest.mark.parametrize("name", list(LAYOUTS))
def test_wave_schedule_is_the_two_pass_sweep(name):
    domain, bc_lo, bc_hi, mgs = LAYOUTS[name]
    C = _single(domain, bc_lo, bc_hi, mgs)
    nl = C.nlevels
    seen = 0
    for m in range(nl):
        ppt, T = C.wave_tiles(m)
        if len(T) == 0:
            continue
        seen += 1
        assert ppt in (1, 2, 4)
        # tile rows fit the block: pairs per tile <= 128 * ppt
        boxes, _ = C.level_boxes(m)
        for row in T:
            lo, hi = boxes[row[0]]
            assert (hi[0] - lo[0] + 1) // 2 * (row[2] - row[1]) <= 128 * ppt
        rng = np.random.default_rng(7 + m)
        for order, slab in (("low", 1), ("high", 2), ("random", 1), ("random", 3), ("random", 4), ("low", 5)):
            probs = _probs_single(C, m, bc_lo, bc_hi)
            R = _run(C, m, probs, order, rng=rng, slab=slab)
            ncell = sum(int(np.prod(P.n)) for P in probs)
            assert R.reds + R.blacks == ncell
            assert all(P.V.all() for P in probs)
    assert seen >= 1


@pytest.mark.parametrize("domain,bc_lo,bc_hi,mgs", [
    (((0, 0, 0), (15, 15, 23)), [D_, D_, P_], [D_, D_, P_], 8),  # 3 boxes around a periodic z
    (((0, 0, 0), (15, 15, 15)), [P_] * 3, [P_] * 3, 16),  # one box, periodic in z
])
def test_wave_refuses_layouts_without_directions(domain, bc_lo, bc_hi, mgs):
    C = _single(domain, bc_lo, bc_hi, mgs)
    ppt, T = C.wave_tiles(0)
    assert len(T) == 0 and ppt == 0


def test_wave_batched_problems_with_few_resident_blocks():
    """Several problems of uneven sizes in one batch: tiles are handed out problem by
    problem, so a sweep finishes even when only as many tiles as the largest problem has
    can be resident at once (a problem's tiles wait only for tiles of the same problem)."""
    sizes = [(32, 48, 16), (16, 16, 32), (48, 32, 32), (32, 16, 48)]
    probs_cfg = [I.batch_problem(s, i, max_grid_size=16) for i, s in enumerate(sizes)]
    C = gmg.BatchContext(probs_cfg)
    rng = np.random.default_rng(11)
    checked = 0
    for m in range(C.nlevels):
        ppt, T = C.wave_tiles(m)
        if len(T) == 0:
            continue
        boxes, _ = C.level_boxes(m)
        per = np.bincount(T[:, 12], minlength=len(sizes))
        for order, slab in (("low", 1), ("random", 2), ("random", 3)):
            probs = []
            for s in range(len(sizes)):
                mine = [boxes[row[0]] for row in T if row[12] == s]
                if not mine:
                    probs.append(Prob((0, 0, 0), (0, 0, 0), [D_] * 3, [D_] * 3))
                    continue
                lo = np.min([b[0] for b in mine], axis=0)
                hi = np.max([b[1] for b in mine], axis=0)
                probs.append(Prob(lo, hi, [D_] * 3, [D_] * 3))
            R = _run(C, m, probs, order, resident=int(per.max()), rng=rng, slab=slab)
            for s, P in enumerate(probs):
                if per[s]:
                    assert P.V.all()
            assert R.reds + R.blacks == sum(int(np.prod(P.n)) for s, P in enumerate(probs) if per[s])
        checked += 1
    assert checked >= 1
