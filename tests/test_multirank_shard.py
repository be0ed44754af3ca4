"""Box sharding tables (gmg_partition, gmg_ghost_rects, gmg_exchange_plan) on CPU.

The solve is split by boxes in Sec. "Basic data structures" (a DistributionMapping along a
space-filling curve) and its ghost cells are exchanged between processes in Sec.
"Communication".  This library runs every solve on one GPU and builds only the tables for
a split; these tests show that the tables are right: ranks that own only their boxes, fill
the ghosts whose source they own locally and receive the others as packed face slabs in
the order the plan gives, hold exactly (bit for bit) the ghost cells and the stencil
iterates of a single rank that owns every box.  Data movement uses numpy on the host and
torch.distributed (gloo, world size 2); the arithmetic of the stencil is the test's own.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2009_12009_gb300 import gmg  # noqa: E402
from paper_2009_12009_gb300 import inputs as I  # noqa: E402

P_, D_, N_ = I.PERIODIC, I.DIRICHLET, I.NEUMANN
GX = 8
DOM = ((0, 0, 0), (47, 39, 31))  # boxes of 16: 3 x 3 (16, 16, 8) x 2
BC_LO, BC_HI = [P_, D_, N_], [P_, N_, D_]


def _ctx():
    return gmg.Context(DOM, BC_LO, BC_HI, boxes=I.chop(*DOM, 16))


class Level:
    """numpy views of one MG level's boxed layout"""

    def __init__(self, C, m):
        self.boxes, _ = C.level_boxes(m)
        self.nelem, self.offs, self.sx = C.layout(m)
        self.rects = C.ghost_rects(m)

    def view(self, a, b):
        (lo, hi), off, sx = self.boxes[b], self.offs[b], self.sx[b]
        n = [hi[d] - lo[d] + 1 for d in range(3)]
        return a[off:off + sx * (n[1] + 2) * (n[2] + 2)].reshape(n[2] + 2, n[1] + 2, sx), n

    def cells(self, r, which):
        """element (k, j, i) index tuples of rectangle r's ghost cells (which='dst') or their
        sources ('src'), u fastest"""
        g = self.rects[r]
        base = g[which]
        out = []
        for v in range(g["n2"]):
            for u in range(g["n1"]):
                c = list(base)
                c[g["d1"]] += u
                c[g["d2"]] += v
                out.append((c[2] + 1, c[1] + 1, GX + c[0]))
        return out

    def pack(self, a, r):
        vw, _ = self.view(a, self.rects[r]["src_box"])
        return np.array([vw[c] for c in self.cells(r, "src")])

    def unpack(self, a, r, vals):
        vw, _ = self.view(a, self.rects[r]["dst_box"])
        s = self.rects[r]["sign"]
        for c, x in zip(self.cells(r, "dst"), vals):
            vw[c] = -x if s < 0 else x

    def fill_local(self, a, owner=None, rank=0):
        for r, g in enumerate(self.rects):
            if owner is not None and (owner[g["dst_box"]] != rank or (g["kind"] == 0 and owner[g["src_box"]] != rank)):
                continue
            self.unpack(a, r, self.pack(a, r))

    def jacobi(self, a, boxes):
        """a <- a + 0.1 (sum of the 6 neighbours - 6 a) on the valid cells of `boxes`"""
        new = a.copy()
        for b in boxes:
            vw, n = self.view(a, b)
            nv, _ = self.view(new, b)
            c = vw[1:-1, 1:-1, GX:GX + n[0]]
            s = (vw[1:-1, 1:-1, GX - 1:GX - 1 + n[0]] + vw[1:-1, 1:-1, GX + 1:GX + 1 + n[0]] +
                 vw[1:-1, :-2, GX:GX + n[0]] + vw[1:-1, 2:, GX:GX + n[0]] +
                 vw[:-2, 1:-1, GX:GX + n[0]] + vw[2:, 1:-1, GX:GX + n[0]])
            nv[1:-1, 1:-1, GX:GX + n[0]] = c + 0.1 * (s - 6.0 * c)
        a[:] = new


def _field(lev, seed=5):
    a = np.zeros(lev.nelem)
    rng = np.random.default_rng(seed)
    for b in range(len(lev.boxes)):
        vw, n = lev.view(a, b)
        vw[1:-1, 1:-1, GX:GX + n[0]] = rng.standard_normal((n[2], n[1], n[0]))
    return a


def _reference(lev, steps):
    a = _field(lev)
    lev.fill_local(a)
    ghosts0 = a.copy()
    for _ in range(steps):
        lev.jacobi(a, range(len(lev.boxes)))
        lev.fill_local(a)
    return ghosts0, a


def _sharded(lev, owner, rank, steps, exchange):
    """rank's array after the ghost fill and `steps` stencil steps, exchange(send, recv) moving
    the packed slabs: send = {peer: values}, returns {peer: values}"""
    C = _ctx()
    a = _field(lev)
    mine = [b for b in range(len(lev.boxes)) if owner[b] == rank]
    plan_s, plan_r = C.exchange_plan(0, owner, rank)

    def fill():
        lev.fill_local(a, owner, rank)
        out = {}
        for peer, r in plan_s:
            out.setdefault(peer, []).append(lev.pack(a, r))
        got = exchange({p: np.concatenate(v) for p, v in out.items()}, sorted({p for p, _ in plan_r}))
        pos = {p: 0 for p in got}
        for peer, r in plan_r:
            k = lev.rects[r]["n1"] * lev.rects[r]["n2"]
            lev.unpack(a, r, got[peer][pos[peer]:pos[peer] + k])
            pos[peer] += k
        assert all(pos[p] == len(got[p]) for p in got)

    fill()
    ghosts0 = a.copy()
    for _ in range(steps):
        lev.jacobi(a, mine)
        fill()
    return mine, ghosts0, a


def _same_boxes(lev, x, y, boxes):
    for b in boxes:
        vx, _ = lev.view(x, b)
        vy, _ = lev.view(y, b)
        if not np.array_equal(vx, vy):
            return False
    return True


def test_partition_is_balanced_and_consolidates():
    C = _ctx()
    lev = Level(C, 0)
    vol = [np.prod([h - l + 1 for l, h in zip(*b)]) for b in lev.boxes]
    for n in (2, 3, 5):
        own = C.partition(0, n)
        load = [sum(v for v, o in zip(vol, own) if o == r) for r in range(n)]
        assert set(own) == set(range(n))
        assert max(load) - min(load) <= 2 * max(vol)
        assert own == C.partition(0, n)  # deterministic
    # a level of fewer than nranks * min_cells cells lives on rank 0: no exchange at all
    own = C.partition(1, 4, 10 ** 6)
    assert set(own) == {0}
    assert C.exchange_plan(1, own, 0) == ([], [])


@pytest.mark.parametrize("nranks", [1, 2, 3, 5])
def test_sharded_ghosts_and_iterates_in_one_process(nranks):
    """All ranks simulated in one process: the slabs each rank sends reach their receiver
    through an in-memory mailbox."""
    C = _ctx()
    lev = Level(C, 0)
    owner = C.partition(0, nranks)
    ref0, ref = _reference(lev, 4)
    from collections import defaultdict, deque

    queues = defaultdict(deque)  # (sender, receiver) -> slabs in posting order

    def make_exchange(rank):
        def exchange(send, peers):
            for p, v in send.items():
                queues[(rank, p)].append(v)
            got = {}
            for p in peers:
                while not queues[(p, rank)]:
                    yield  # the peer has not posted this round yet
                got[p] = queues[(p, rank)].popleft()
            return got
        return exchange

    results = {}

    def run(rank):
        results[rank] = yield from _sharded_gen(lev, owner, rank, 4, make_exchange(rank))

    live = {r: run(r) for r in range(nranks)}
    while live:
        for r in list(live):
            try:
                next(live[r])
            except StopIteration:
                del live[r]
    for r in range(nranks):
        mine, g0, a = results[r]
        assert _same_boxes(lev, g0, ref0, mine), r
        assert _same_boxes(lev, a, ref, mine), r


def _sharded_gen(lev, owner, rank, steps, exchange):
    """generator form of _sharded for the in-process simulation (yields between the posting
    and the reading of each exchange round)"""
    C = _ctx()
    a = _field(lev)
    mine = [b for b in range(len(lev.boxes)) if owner[b] == rank]
    plan_s, plan_r = C.exchange_plan(0, owner, rank)

    def fill():
        lev.fill_local(a, owner, rank)
        out = {}
        for peer, r in plan_s:
            out.setdefault(peer, []).append(lev.pack(a, r))
        got = yield from exchange({p: np.concatenate(v) for p, v in out.items()}, sorted({p for p, _ in plan_r}))
        pos = {p: 0 for p in got}
        for peer, r in plan_r:
            k = lev.rects[r]["n1"] * lev.rects[r]["n2"]
            lev.unpack(a, r, got[peer][pos[peer]:pos[peer] + k])
            pos[peer] += k

    yield from fill()
    ghosts0 = a.copy()
    for _ in range(steps):
        lev.jacobi(a, mine)
        yield from fill()
    return mine, ghosts0, a


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        C = _ctx()
        lev = Level(C, 0)
        owner = C.partition(0, world)

        def exchange(send, peers):
            sizes = {}
            reqs = []
            for p, v in send.items():  # sizes first, then the slabs (one message per peer)
                reqs.append(dist.isend(torch.tensor([len(v)], dtype=torch.int64), p, tag=1))
            for p in peers:
                t = torch.zeros(1, dtype=torch.int64)
                dist.recv(t, p, tag=1)
                sizes[p] = int(t.item())
            for r_ in reqs:
                r_.wait()
            reqs = [dist.isend(torch.from_numpy(v), p, tag=2) for p, v in send.items()]
            got = {}
            for p in peers:
                t = torch.zeros(sizes[p], dtype=torch.float64)
                dist.recv(t, p, tag=2)
                got[p] = t.numpy()
            for r_ in reqs:
                r_.wait()
            return got

        mine, g0, a = _sharded(lev, owner, rank, 4, exchange)
        ref0, ref = _reference(lev, 4)
        q.put((rank, len(mine), _same_boxes(lev, g0, ref0, mine), _same_boxes(lev, a, ref, mine)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_sharded_ghosts_and_iterates_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    assert sum(g[1] for g in got) == len(I.chop(*DOM, 16))
    assert all(g[2] and g[3] for g in got), got
