"""Host-side checks of the CUDA library that need no GPU: the C ABI loads and exports
every symbol of include/gmg.h, the multigrid hierarchy and its box metadata match the
oracle's, the boxed layout keeps every row's first valid cell 16-byte aligned, and bad
input is refused with an error code.  No compute call is made here."""
import ctypes as C
import os
import re

import pytest

from paper_2009_12009_gb300 import gmg
from paper_2009_12009_gb300 import inputs as I
from tests import cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_exports_match_header():
    src = open(os.path.join(ROOT, "include", "gmg.h")).read()
    declared = sorted(set(re.findall(r"\b(gmg_[a-z0-9_]+)\s*\(", src)))
    L = gmg.lib()
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing, missing
    assert len(set(gmg.EXPORTS)) == len(gmg.EXPORTS)
    assert set(declared) == set(gmg.EXPORTS)


HIER_CASES = [
    ("poisson32", None),
    ("uneven", None),
    ("periodic", None),
    ("helmholtz", None),
    ("oddlo", None),
    ("batch", ((0, 0, 0), (47, 159, 95))),
    ("odd12", ((0, 0, 0), (11, 11, 11))),
]


@pytest.mark.parametrize("name,dom", HIER_CASES)
def test_hierarchy_matches_oracle(orc, name, dom):
    """Per-box coarsening, then aggregation into one box (Sec. "Linear Solvers"): the
    library builds the same levels, boxes and parent links as the oracle."""
    if dom is None:
        c = cases.make(name)
        dom, boxes, bl, bh = c["domain"], c["boxes"], c["bc_lo"], c["bc_hi"]
    else:
        boxes = I.chop(*dom, 32 if name == "batch" else 6)
        bl = bh = [I.DIRICHLET] * 3
    P = orc.Problem(dom, boxes, bl, bh)
    Cx = gmg.Context(dom, bl, bh, boxes=boxes)
    assert Cx.nlevels == P.nlevels
    for m in range(P.nlevels):
        cb, par = Cx.level_boxes(m)
        assert cb == P.level_boxes(m)
        assert Cx.level_info(m)[1] == P.level_domain(m)
        assert par == P.level_parents(m)


def test_chop_matches_inputs():
    dom = ((0, 0, 0), (47, 159, 95))
    Cx = gmg.Context(dom, [1] * 3, [1] * 3, max_grid_size=32)
    assert Cx.level_boxes(0)[0] == I.chop(*dom, 32)


@pytest.mark.parametrize("name", ["uneven", "poisson32", "oddlo"])
def test_layout_alignment(name):
    c = cases.make(name)
    Cx = gmg.Context(c["domain"], c["bc_lo"], c["bc_hi"], boxes=c["boxes"])
    for m in range(Cx.nlevels):
        boxes, _ = Cx.level_boxes(m)
        for dt, es in ((gmg.DT_F64, 8), (gmg.DT_F32, 4), (gmg.DT_BF16, 2)):
            ne, offs, sxs = Cx.layout(m, dt)
            prev_end = 0
            for (lo, hi), off, sx in zip(boxes, offs, sxs):
                n = [hi[d] - lo[d] + 1 for d in range(3)]
                assert off >= prev_end and (off * es) % 16 == 0
                assert ((off + gmg.GX) * es) % 16 == 0 and (sx * es) % 16 == 0
                assert sx >= gmg.GX + n[0] + 1
                prev_end = off + sx * (n[1] + 2) * (n[2] + 2)
            assert prev_end <= ne


def test_bad_input_refused():
    dom = ((0, 0, 0), (7, 7, 7))
    with pytest.raises(gmg.GmgError) as e:
        gmg.Context(dom, [0, 1, 1], [1, 1, 1], max_grid_size=4)  # half-periodic axis
    assert e.value.status == gmg.BAD_INPUT
    with pytest.raises(gmg.GmgError) as e:
        gmg.Context(dom, [1] * 3, [1] * 3, boxes=[((0, 0, 0), (7, 7, 7)), ((4, 4, 4), (7, 7, 7))])  # overlap
    assert e.value.status == gmg.BAD_INPUT
    with pytest.raises(gmg.GmgError) as e:
        gmg.Context(dom, [1] * 3, [1] * 3, boxes=[((0, 0, 0), (3, 7, 7))])  # does not cover
    assert e.value.status == gmg.BAD_INPUT
    with pytest.raises(gmg.GmgError) as e:
        gmg.Context(dom, [1] * 3, [1] * 3, boxes=[((0, 0, 0), (8, 7, 7))])  # outside
    assert e.value.status == gmg.BAD_INPUT
    Cx = gmg.Context(dom, [1] * 3, [1] * 3, max_grid_size=4)
    st = Cx.L.gmg_fill_boundary(Cx.h, 0, gmg.DT_F64, None, -1)
    assert st == gmg.NO_WORKSPACE
    st = Cx.L.gmg_set_workspace(Cx.h, C.c_void_p(256), C.c_size_t(16))
    assert st == gmg.NO_WORKSPACE
    st = Cx.L.gmg_set_workspace(Cx.h, C.c_void_p(257), C.c_size_t(1 << 40))
    assert st == gmg.BAD_INPUT
    assert Cx.L.gmg_set_scalars(Cx.h, 0.0, 0.0) == gmg.BAD_INPUT


def test_covered_masks_match_oracle(orc):
    """The host's per-level covered masks (bounding-box arrays) are the oracle's cells inside a
    level and not among its unknowns, for the three-level recipe at n = 16."""
    import numpy as np

    a = I.amr3(16)
    M = orc.MultiLevelProblem(a["domain"], a["level_boxes"], a["bc_lo"], a["bc_hi"])
    n = 16
    shapes = [(n, n, n)] * 3
    got = gmg.covered_masks(a["level_boxes"], a["level_lo"], shapes)
    for lev in range(3):
        sl = tuple(slice(a["level_lo"][lev][d], a["level_lo"][lev][d] + n) for d in (2, 1, 0))
        assert np.array_equal(got[lev], (M.inside[lev] & ~M.masks[lev])[sl])
        assert np.array_equal(got[lev], a["covered"][lev])


def _header_struct(name):
    """(type, field) pairs of `typedef struct { ... } name;` in include/gmg.h, in order"""
    src = open(os.path.join(ROOT, "include", "gmg.h")).read()
    end = src.index("} " + name + ";")
    start = src.rindex("typedef struct {", 0, end)
    body = re.sub(r"/\*.*?\*/", "", src[start:end], flags=re.S)
    return re.findall(r"\b(long long|int|double|int64_t)\s+([a-z_0-9]+)(?:\[[0-9A-Z_]+\])?\s*;", body)


def test_params_struct_matches_header():
    """The Python mirror of gmg_params has the header's fields, in order and of the same C
    types (the struct crosses the ABI by pointer)."""
    want = _header_struct("gmg_params")
    ct = {"int": C.c_int, "double": C.c_double, "int64_t": C.c_int64, "long long": C.c_longlong}
    got = [(n, t) for n, t in gmg.Params._fields_]
    assert [n for n, _ in got] == [n for _, n in want]
    assert all(t == ct[w] for (_, t), (w, _) in zip(got, want))
    p = gmg.default_params()
    assert p.settled_zero == 1 and p.use_graph == 1 and p.nu1 == 2 and p.nu2 == 2


def test_solve_info_struct_matches_header():
    want = [n for _, n in _header_struct("gmg_solve_info")]
    assert [n for n, _ in gmg.SolveInfo._fields_] == want
    assert C.sizeof(gmg.SolveInfo) >= 8 * 256


def test_every_declaration_cites_a_passage():
    """Every entry point of include/gmg.h (or the group of declarations its comment covers)
    names the paper's section that defines it, or says that the paper has no counterpart."""
    import re

    text = open(os.path.join(ROOT, "include", "gmg.h")).read()
    body = text[text.index("/* ---------------------------------------------------------------- context */"):]
    missing = []
    for m in re.finditer(r"\n(?:gmg_status|const char\*) (gmg_\w+)\(", body):
        pre = body[:m.start()]
        # walk back over declarations that share the comment above them
        while True:
            cend, semi = pre.rfind("*/"), pre.rfind(";")
            if semi > cend:
                pre = pre[:pre.rfind("\n", 0, semi)]
                continue
            break
        com = pre[pre.rfind("/*", 0, cend):cend]
        if not re.search(r'Sec\.\s+"', com) and "no counterpart" not in com:
            missing.append(m.group(1))
    assert not missing, missing


def test_noalloc_refuses_large_boxes_before_any_cuda_call():
    """gmg_box_bicgstab_noalloc checks its size limit, (nx+2)(ny+2)(nz+2) <= 65536, on the host
    before it touches CUDA: edges near INT_MAX (whose +2 would overflow 32 bits), a cube of
    64^3 ghosted elements and a box one row over the limit all return GMG_ERR_BAD_INPUT
    with the limit named, whatever the (never used) pointers."""
    from paper_2009_12009_gb300 import gmg

    L = gmg.lib()
    bc = (C.c_int * 3)(1, 1, 1)
    big = 2 ** 31 - 2
    for n in [(big, 1, 1), (1, big, 1), (1, 1, big), (big, big, big), (62, 62, 62), (63, 30, 30), (62, 31, 30)]:
        st = L.gmg_box_bicgstab_noalloc(None, n[0], n[1], n[2], bc, bc, 0, C.c_void_p(8), C.c_void_p(8),
                                        C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), C.c_void_p(8), 200, 1e-4, None)
        assert st == gmg.BAD_INPUT, n
        assert b"static scratch limit" in L.gmg_last_error(None), n


def test_tail_plan_dense_bytes():
    """The coarse end's dense form (fused_coarse, tail_dense): abec256 (256^3 in 64 boxes of
    64^3) starts its tail on level 5, 8^3 cells in 64 boxes of 2^3, then 4^3 and the 2^3 bottom.
    One padded array per level: 10^3, 6^3 and 4^3 elements; e and r in the element type, and
    five coefficient arrays (wx, wy, wz, 1/D, D: double for FP64, float otherwise) on the two
    smoothed levels, each array rounded up to 16 bytes."""
    cfg = I.abec256()
    ctx = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"])
    al = lambda b: (b + 15) // 16 * 16  # noqa: E731
    for dt, es, cs in ((gmg.DT_F64, 8, 8), (gmg.DT_F32, 4, 4), (gmg.DT_BF16, 2, 4)):
        want = sum(2 * al(ne * es) + (5 * al(ne * cs) if sm else 0)
                   for ne, sm in ((1000, True), (216, True), (64, False)))
        assert ctx.tail_plan(5, dt) == (1, want)
        assert all(ctx.tail_plan(m, dt) == (0, 0) for m in range(ctx.nlevels) if m != 5)
    # 28^3 in boxes of 16: the tail is the 7^3 bottom alone (9^3 elements, e and r only)
    c28 = I.abec(28, 16, 1)
    ctx28 = gmg.Context(c28["domain"], c28["bc_lo"], c28["bc_hi"], boxes=c28["boxes"])
    assert ctx28.tail_plan(ctx28.nlevels - 1) == (1, 2 * al(729 * 8))
    # batched: one block per problem, grouped by the level its tail starts on
    sizes = [(32, 48, 16), (16, 16, 32), (48, 32, 32), (32, 16, 48), (64, 64, 64)]
    B = gmg.BatchContext([I.batch_problem(s, i, max_grid_size=16) for i, s in enumerate(sizes)])
    plans = [B.tail_plan(m) for m in range(B.nlevels)]
    assert sum(n for n, _ in plans) == len(sizes)
    assert all(b > 0 for n, b in plans if n > 0)


def test_new_launch_options_refused_out_of_range():
    """The coarse-end and fusion options take only their documented values; a call with any
    other value is refused (BAD_INPUT) before it touches the device, while the defaults get as
    far as the missing workspace."""
    Cx = gmg.Context(((0, 0, 0), (15, 15, 15)), [1] * 3, [1] * 3, max_grid_size=8)
    for name, bad in (("tail_dense", 2), ("fuse_restriction_sweep", -1), ("fuse_prolongation", 3),
                      ("fork_bottoms", 2)):
        p = gmg.default_params(**{name: bad})
        assert Cx.L.gmg_autotune(Cx.h, gmg.FP64, None, C.byref(p)) == gmg.BAD_INPUT, name
    p = gmg.default_params()
    assert (p.tail_dense, p.fuse_restriction_sweep, p.fuse_prolongation, p.fork_bottoms) == (1, 1, 1, 1)
    assert Cx.L.gmg_autotune(Cx.h, gmg.FP64, None, C.byref(p)) == gmg.NO_WORKSPACE
