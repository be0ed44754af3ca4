#!/usr/bin/env python
"""Benchmark: FP64 multigrid solve to 1e-10 relative residual on the abec256 workload.

Workload (shaped like the solver study of Sec. "Linear Solvers", which runs 256^3 cells on
each node with variable coefficients): 256^3 cells, Dirichlet walls, 64 boxes of 64^3, a = 0, b = 1, beta =
exp(N(0,1)) smoothed by one 3x3x3 mean filter (harmonic faces), rhs N(0,1), seed 12011.

A step is one whole solve from phi = 0 to ||r||_inf <= 1e-10 ||rhs||_inf: every V-cycle
step of the hot path (ghost exchange, red-black Gauss-Seidel, residual, average-down,
prolongation, BiCGStab bottom) and the outer FP64 residual loop.

  value  = Mcell-updates/s = sum over smoothed levels of cells x (nu1 + nu2) x V-cycles
           / time to tolerance, device-timed (CUDA events) with inputs resident in HBM;
  e2e    = the same metric through the public API with host buffers: pinned rhs copied
           in, packed, solved, unpacked and copied back inside the timed region;
  mixed  = the same solve with the float and bfloat16-storage V-cycles inside FP64
           iterative refinement (time, Mcell-updates/s, error against the FP64 solve);
  roofline: the finest-level smoother kernel (dominant), its algorithmic bytes per launch
           (28 B per cell per colour pass: 56 B per cell per red+black sweep) over its average
           launch time, CUDA events recorded around each of its launches in the last timed
           solve (inside the timed region; the other solves run without the events); beside
           it, the same launches' FP64-pipe rate (7 operations per updated cell) over the FP64
           ceiling measured in this run (fp64_peak: the library's DFMA probe);
  cpu_baseline: the FP64 CPU oracle solving the same workload to 1e-10 on the host cores
           (OpenMP over boxes), plus one V-cycle on one thread; rel_err_vs_oracle: every
           precision's solution against the oracle's;
  summary: the headline figures of every workload, last in the line.

--impl reference times the oracle itself (each step: one V-cycle iteration of the
workload, OpenMP over boxes on the host cores).  Multi-GPU: independent replicas (the solve does not shard
in this version), weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson solve time to 1e-10 rel. residual & Mcell-updates/s; mixed vs FP64"
UNIT = "Mcell-updates/s"
WORKLOAD = ("abec256: 256^3 ABecLaplacian a=0 b=1, Dirichlet walls, 64 boxes of 64^3, beta log-normal "
            "(3x3x3 mean filter, harmonic faces), rhs N(0,1) seed 12011; V(2,2) red-black GS, "
            "BiCGStab bottom at 2^3, FP64, tol 1e-10")
# algorithmic bytes of the red-black smoother: 56 B per cell per full sweep (phi, rhs, 3 face
# weights, 1/D read and phi written once, 8 B each), so 28 B per cell per colour pass
SWEEP_BYTES_PER_CELL = 56
PASS_BYTES_PER_CELL = SWEEP_BYTES_PER_CELL // 2
# FP64-pipe operations of one Gauss-Seidel update: 6 fused multiply-adds and 1 multiply
UPDATE_FP64_OPS = 7
TOL = 1e-10


def mcell_updates_per_vcycle(ctx, nu):
    """sum over smoothed levels (all but the bottom) of cells x smoothing sweeps"""
    tot = 0
    for m in range(ctx.nlevels - 1):
        nz, ny, nx = ctx.level_shape(m)
        tot += nx * ny * nz * nu
    return tot


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def source_text(names):
    """Bytes of the listed csrc sources; "file#text" stands for the definition in that file
    that starts at the first occurrence of `text` and ends at the next closing brace in
    column 0 (a function, or a struct with its ";")."""
    out = b""
    for name in names:
        fname, _, sym = name.partition("#")
        with open(os.path.join(ROOT, "paper_2009_12009_gb300", "csrc", fname), "rb") as f:
            text = f.read()
        if sym:
            start = text.index(sym.encode())
            text = text[start:text.index(b"\n}", start) + 3]
        out += text
    return out


def kernel_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if the sources it
    was measured on (the kernel and the workspace placement) are the current ones (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    try:
        h = hashlib.sha256(source_text(rec.get("sources", [])))
    except (OSError, ValueError):  # a hashed definition moved or is gone: the record is stale
        return None
    if not rec.get("sources") or h.hexdigest()[:16] != rec.get("sources_sha256_16"):
        return None
    return rec.get("dram_bytes_per_launch_full_size")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def cpu_baseline(cfg):
    """The FP64 oracle on the host cores: the whole abec256 solve to 1e-10 with OpenMP over
    boxes on every core this process may use (its solution is the reference of the error
    figures), and one V-cycle iteration on one thread.  Returns (record, oracle solution)."""
    from oracle import oracle as O

    P = O.Problem(cfg["domain"], cfg["boxes"], cfg["bc_lo"], cfg["bc_hi"])
    P.set_coeffs(cfg["a"], cfg["b"], alpha=cfg["alpha"], beta=cfg["beta"])
    cells = 0
    for m in range(P.nlevels - 1):
        nz, ny, nx = P.level_shape(m)
        cells += nx * ny * nz * 4
    ncores = len(os.sched_getaffinity(0))
    O.set_threads(1)
    t0 = time.perf_counter()
    _, it1, _, _ = P.solve(cfg["rhs"], tol_rel=0.0, maxit=1)
    dt1 = time.perf_counter() - t0
    O.set_threads(ncores)
    t0 = time.perf_counter()
    sol, it, _, st = P.solve(cfg["rhs"], tol_rel=TOL, maxit=100)
    dt = time.perf_counter() - t0
    O.set_threads(1)
    rec = {"value": cells * it / dt / 1e6, "unit": UNIT, "cores": ncores, "kind": "oracle",
           "time_to_tol_ms": 1e3 * dt, "iterations": it, "status": st,
           "sample": f"the whole abec256 solve to 1e-10 ({it} V-cycles, FP64 oracle, OpenMP over boxes on "
                     f"{ncores} threads), {dt:.1f} s",
           "single_thread": {"value": cells * it1 / dt1 / 1e6, "unit": UNIT, "cores": 1,
                             "sample": f"{it1} V-cycle iteration of the same solve, {dt1:.1f} s"}}
    return rec, sol


def fp64_peak(stream, clocks_index):
    """FP64 ceiling of this GPU: the library's DFMA probe (independent FMA chains) timed with
    CUDA events on the bench stream, best over 4, 8 and 16 blocks of 256 threads per SM."""
    import torch

    from paper_2009_12009_gb300 import gmg

    clk = ClockSampler(clocks_index)
    clk.start()
    time.sleep(0.2)
    best = (0.0, 0)
    for bps in (4, 8, 16):
        gmg.dfma_probe(stream.cuda_stream, bps, 1 << 12)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = sum(gmg.dfma_probe(stream.cuda_stream, bps, 1 << 15) for _ in range(3))
        e1.record(stream)
        torch.cuda.synchronize()
        tf = fl / (e0.elapsed_time(e1) * 1e-3) / 1e12
        if tf > best[0]:
            best = (tf, bps)
    c = clk.stop()
    return {"tflops": best[0], "fma_per_s": best[0] * 1e12 / 2, "blocks_per_sm": best[1],
            "how": "gmg_dfma_probe: 16 independent FP64 FMA chains per thread, 256-thread blocks, CUDA events",
            "sm_mhz": c.get("sm_mhz"), "reasons": c.get("reasons")}


def whole_job(ms_local, updates_local, world, device):
    """Whole-job throughput of N replicas: the timed region is the slowest rank's (max over
    ranks), the work is every rank's (sum over ranks).  Returns (ms, updates, Mcell-upd/s)."""
    import torch

    ms, updates = float(ms_local), float(updates_local)
    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([updates], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, updates = float(t.item()), float(u.item())
    return ms, updates, updates / (ms * 1e-3) / 1e6


def summarize_tuning(t):
    """sweep variant chosen per MG level (bit 0: ghost push, bit 1: one thread per 4 cells;
    -1: no smoothing there) and the fused coarse end (1 on), as gmg_autotune measured them"""
    return {"sweep_variant_per_level": [lv[0] for lv in t["levels"]], "fused_coarse": t["fused_coarse"],
            "vcycle_ms_fused_vs_levels": [round(x, 4) for x in t["vcycle_ms"]]}


def _timed(fn, steps, warmup, stream, barrier):
    """device time (ms) per call of fn over `steps` calls after `warmup`; returns (ms, last)"""
    import torch

    last = None
    for _ in range(warmup):
        last = fn()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        last = fn()
    e1.record(stream)
    barrier()
    return e0.elapsed_time(e1) / steps, last


def _updates_per_vcycle_problem(ctx, s):
    """cells x 4 sweeps over the smoothed levels of problem s of a batched context"""
    tot, levels = 0, []
    for m in range(ctx.nlevels):
        boxes, _ = ctx.level_boxes(m)
        import ctypes as C

        first, count = C.c_int(), C.c_int()
        ctx.L.gmg_solve_boxes(ctx.h, m, s, C.byref(first), C.byref(count))
        if count.value == 0:
            break
        cells = sum((b[1][0] - b[0][0] + 1) * (b[1][1] - b[0][1] + 1) * (b[1][2] - b[0][2] + 1)
                    for b in boxes[first.value:first.value + count.value])
        levels.append(cells)
    return 4 * sum(levels[:-1])


def measure_forms(stream, barrier, dev, only=None):
    """The other workloads, each at full size: abec512 in FP64 and both mixed forms, batch64
    (64 uneven problems, batched form), amr2 (two-level composite forward + adjoint +
    beta gradient), amr3 (the same over three levels), walls256, krylov.  Device time to
    1e-10 per solve."""
    forms = {}
    if only in (None, "abec512"):
        forms["abec512"] = _form_abec512(stream, barrier)
    if only in (None, "batch64"):
        forms["batch64"] = _form_batch64(stream, barrier)
    if only in (None, "amr2"):
        forms["amr2"] = _form_amr2(stream, barrier, dev)
    if only in (None, "amr3"):
        forms["amr3"] = _form_amr3(stream, barrier)
    if only in (None, "walls256"):
        forms["walls256"] = _form_walls256(stream, barrier)
    if only in (None, "krylov"):
        forms["krylov"] = _form_krylov(stream, barrier)
    return forms


def _form_abec512(stream, barrier):
    import torch

    from paper_2009_12009_gb300 import gmg
    from paper_2009_12009_gb300 import inputs as I

    cfg = I.abec512()
    ctx = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"], stream=stream.cuda_stream)
    ctx.allocate(gmg.MIXED_FP32)
    ctx.set_scalars(0.0, 1.0)
    ctx.set_beta(torch.from_numpy(cfg["beta"]))
    rhs = ctx.pack(torch.from_numpy(cfg["rhs"]))
    del cfg
    phi = ctx.field(0)
    upd = mcell_updates_per_vcycle(ctx, 4)
    res = {"workload": "abec512: 512^3 Dirichlet, 64 boxes of 128^3, abec recipe seed 12012, tol 1e-10",
           "autotuned": {name: summarize_tuning(ctx.autotune(rhs, prec))
                         for name, prec in (("fp64", gmg.FP64), ("fp32", gmg.MIXED_FP32), ("bf16", gmg.MIXED_BF16))}}
    ref = None
    for name, prec in (("fp64", gmg.FP64), ("fp32", gmg.MIXED_FP32), ("bf16", gmg.MIXED_BF16)):
        ms, info = _timed(lambda: ctx.solve(rhs, phi, tol_rel=TOL, precision=prec)[1], 3, 1, stream, barrier)
        sol = ctx.unpack(phi)
        if ref is None:
            ref = sol.clone()
        res[name] = {"time_to_tol_ms": ms, "iterations": info.iterations, "status": info.status,
                     "value": upd * info.iterations / (ms * 1e-3) / 1e6, "unit": UNIT,
                     "final_rel_resid": info.final_resid / info.rhs_norm,
                     "rel_err_vs_fp64": float((sol - ref).abs().max() / ref.abs().max())}
    res["mixed_speedup_fp32"] = res["fp64"]["time_to_tol_ms"] / res["fp32"]["time_to_tol_ms"]
    res["mixed_speedup_bf16"] = res["fp64"]["time_to_tol_ms"] / res["bf16"]["time_to_tol_ms"]
    del ctx, rhs, phi, ref, sol
    torch.cuda.empty_cache()
    return res


def _form_walls256(stream, barrier):
    import torch

    from paper_2009_12009_gb300 import gmg
    from paper_2009_12009_gb300 import inputs as I

    cfg = I.walls256()
    ctx = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"], stream=stream.cuda_stream)
    ctx.allocate(gmg.MIXED_FP32)
    ctx.set_scalars(0.0, 1.0)
    ctx.set_beta(torch.from_numpy(cfg["beta"]))
    rhs = ctx.pack(torch.from_numpy(cfg["rhs"]))
    vals = {f: torch.from_numpy(v).cuda() for f, v in cfg["wall_values"].items()}
    del cfg
    phi = ctx.field(0)
    folded = ctx.field(0)
    upd = mcell_updates_per_vcycle(ctx, 4)
    ms_fold, _ = _timed(lambda: ctx.wall_values_rhs(rhs, vals, out=folded), 5, 2, stream, barrier)
    res = {"workload": "walls256: the abec256 recipe (seed 12015) with Neumann x-, y+, z- and Dirichlet x+, y-, "
                       "z+ walls, N(0,1) values on every wall face; tol 1e-10 of the initial residual",
           "wall_values_rhs_ms": ms_fold,
           "autotuned": {name: summarize_tuning(ctx.autotune(folded, prec))
                         for name, prec in (("fp64", gmg.FP64), ("fp32", gmg.MIXED_FP32), ("bf16", gmg.MIXED_BF16))}}
    for name, prec in (("fp64", gmg.FP64), ("fp32", gmg.MIXED_FP32), ("bf16", gmg.MIXED_BF16)):
        ms, info = _timed(lambda: ctx.solve(rhs, phi, tol_rel=TOL, precision=prec, wall_values=vals)[1], 3, 1,
                          stream, barrier)
        res[name] = {"time_to_tol_ms": ms, "iterations": info.iterations, "status": info.status,
                     "value": upd * info.iterations / (ms * 1e-3) / 1e6, "unit": UNIT,
                     "final_rel_resid": info.final_resid / info.rhs_norm}
    del ctx, rhs, phi, folded
    torch.cuda.empty_cache()
    return res


def _form_krylov(stream, barrier):
    """Multigrid iteration vs multigrid-preconditioned BiCGStab and CG (symmetric V-cycle)
    on abec256 and on the high-contrast contrast256, to 1e-10."""
    import torch

    from paper_2009_12009_gb300 import gmg
    from paper_2009_12009_gb300 import inputs as I

    res = {}
    for cfg_fn in (I.abec256, I.contrast256):
        cfg = cfg_fn()
        ctx = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"], stream=stream.cuda_stream)
        ctx.allocate(gmg.MIXED_FP32, krylov=True)
        ctx.set_scalars(0.0, 1.0)
        ctx.set_beta(torch.from_numpy(cfg["beta"]))
        rhs = ctx.pack(torch.from_numpy(cfg["rhs"]))
        name = cfg["name"]
        del cfg
        phi = ctx.field(0)
        ctx.autotune(rhs, gmg.FP64)
        ctx.autotune(rhs, gmg.MIXED_FP32)
        out = {}
        for label, kw in (("mg_fp64", dict(krylov=0)), ("bicgstab_fp64", dict(krylov=1)),
                          ("cg_fp64", dict(krylov=2)), ("mg_fp32", dict(krylov=0, precision=gmg.MIXED_FP32)),
                          ("bicgstab_fp32", dict(krylov=1, precision=gmg.MIXED_FP32))):
            ms, info = _timed(lambda: ctx.solve(rhs, phi, tol_rel=TOL, max_iter=300, **kw)[1], 3, 1, stream, barrier)
            vc = info.iterations * (2 if kw["krylov"] == 1 else 1)
            out[label] = {"time_to_tol_ms": ms, "iterations": info.iterations, "vcycles": vc, "status": info.status,
                          "final_rel_resid": info.final_resid / info.rhs_norm}
        res[name] = out
        del ctx, rhs, phi
        torch.cuda.empty_cache()
    res["workload"] = ("abec256 and contrast256 (256^3, 64 boxes; beta = exp(3 N(0,1)) filtered, seed 12016), tol "
                       "1e-10: multigrid iteration, multigrid-preconditioned BiCGStab (2 V-cycles per iteration) "
                       "and CG (symmetric V-cycle)")
    return res


def _form_batch64(stream, barrier):
    import numpy as np
    import torch

    from paper_2009_12009_gb300 import gmg
    from paper_2009_12009_gb300 import inputs as I

    probs = I.batch64()
    bctx = gmg.BatchContext(probs, stream=stream.cuda_stream)
    bctx.allocate(gmg.MIXED_FP32)
    bctx.set_scalars(0.0, 1.0)
    bctx.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    brhs = bctx.pack_all([torch.from_numpy(p["rhs"]) for p in probs])
    cells = sum(int(np.prod(p["rhs"].shape)) for p in probs)
    upd_s = [_updates_per_vcycle_problem(bctx, s) for s in range(len(probs))]
    bphi = bctx.field(0)
    tuned = {name: summarize_tuning(bctx.autotune(brhs, prec)) for name, prec in (("fp64", gmg.FP64),
                                                                                 ("fp32", gmg.MIXED_FP32))}
    res = {"autotuned": tuned, "workload": f"batch64: 64 problems, edges from {{32,...,160}}, boxes <= 32^3, {cells} cells, "
                       f"{bctx.level_info(0)[0]} boxes, abec recipe seeds 12014+i (i = 0..63), tol 1e-10 each"}
    for name, prec in (("fp64", gmg.FP64), ("fp32", gmg.MIXED_FP32)):
        ms, infos = _timed(lambda: bctx.batch_solve(brhs, bphi, tol_rel=TOL, precision=prec)[1], 3, 1, stream, barrier)
        its = [i.iterations for i in infos]
        res[name] = {"time_to_tol_ms": ms, "iterations_min": min(its), "iterations_max": max(its),
                     "all_converged": all(i.status == gmg.OK for i in infos),
                     "value": sum(u * k for u, k in zip(upd_s, its)) / (ms * 1e-3) / 1e6, "unit": UNIT}
    del bctx, brhs, bphi
    torch.cuda.empty_cache()
    # the same 64 problems solved one after another, each in its own context (FP64)
    ctxs = []
    for p in probs:
        c1 = gmg.Context(p["domain"], p["bc_lo"], p["bc_hi"], prob_hi=p["prob_hi"], boxes=p["boxes"],
                         stream=stream.cuda_stream)
        c1.allocate(gmg.FP64)
        c1.set_scalars(0.0, 1.0)
        c1.set_beta(torch.from_numpy(p["beta"]))
        ctxs.append((c1, c1.pack(torch.from_numpy(p["rhs"])), c1.field(0)))

    def one_by_one():
        return [c1.solve(r1, f1, tol_rel=TOL)[1] for c1, r1, f1 in ctxs]

    ms_seq, infos_seq = _timed(one_by_one, 2, 1, stream, barrier)
    res["sequential_fp64"] = {"time_to_tol_ms": ms_seq,
                              "all_converged": all(i.status == gmg.OK for i in infos_seq),
                              "batched_speedup": ms_seq / res["fp64"]["time_to_tol_ms"]}
    del ctxs
    torch.cuda.empty_cache()
    return res


def _form_amr2(stream, barrier, dev):
    import torch

    from paper_2009_12009_gb300 import gmg
    from paper_2009_12009_gb300 import inputs as I

    a = I.amr2()
    actx = gmg.AmrContext(a["domain"], a["coarse_boxes"], a["fine_boxes"], a["bc_lo"], a["bc_hi"],
                          stream=stream.cuda_stream)
    actx.allocate(gmg.FP64)
    actx.set_coeffs(0.0, 1.0, beta_c=torch.from_numpy(a["beta_c"]), beta_f=torch.from_numpy(a["beta_f"]))
    rc, rf = actx.pack_level(0, torch.from_numpy(a["rhs_c"])), actx.pack_level(1, torch.from_numpy(a["rhs_f"]))
    tuned = summarize_tuning(actx.autotune(rc, gmg.FP64))
    ms_f, (pc, pf, info_f) = _timed(lambda: actx.solve2(rc, rf, tol_rel=TOL), 3, 1, stream, barrier)
    # dL/dphi of L = 0.5 |phi - phi_target|^2 over the composite cells
    keep = torch.as_tensor(~a["covered"], device=dev, dtype=torch.float64)
    gc = actx.pack_level(0, (actx.unpack_level(0, pc) - torch.from_numpy(a["target_c"]).to(dev)) * keep)
    gf = actx.pack_level(1, actx.unpack_level(1, pf) - torch.from_numpy(a["target_f"]).to(dev))
    ms_a, (lc, lf, info_a) = _timed(lambda: actx.solve_adjoint2(gc, gf, tol_rel=TOL), 3, 1, stream, barrier)
    ms_g, _ = _timed(lambda: actx.beta_grad2(pc, pf, lc, lf), 5, 1, stream, barrier)
    return {"workload": "amr2: 128^3 periodic level 0 (8 boxes) + ratio-2 level 1 over the central 64^3 "
                        "coarse cells (128^3 fine cells, 8 boxes), seed 12014, tol 1e-10",
            "forward": {"time_to_tol_ms": ms_f, "iterations": info_f.iterations, "status": info_f.status},
            "adjoint": {"time_to_tol_ms": ms_a, "iterations": info_a.iterations, "status": info_a.status},
            "beta_grad_ms": ms_g, "autotuned_level0_hierarchy": tuned}


def _form_amr3(stream, barrier):
    import torch

    from paper_2009_12009_gb300 import gmg
    from paper_2009_12009_gb300 import inputs as I

    a = I.amr3()
    ctx = gmg.MultiLevelContext(a["domain"], a["level_boxes"], a["bc_lo"], a["bc_hi"], stream=stream.cuda_stream)
    ctx.allocate(gmg.FP64)
    ctx.set_coeffs(0.0, 1.0, betas=[torch.from_numpy(b) for b in a["betas"]])
    rs = [ctx.pack_level(lev, torch.from_numpy(r)) for lev, r in enumerate(a["rhss"])]
    tuned = summarize_tuning(ctx.autotune(rs[0], gmg.FP64))
    ms, (phis, info) = _timed(lambda: ctx.solve_levels(rs, tol_rel=TOL), 3, 1, stream, barrier)
    # adjoint of L = 0.5 |phi|^2 over the composite cells: g = phi (zero volume-weighted mean),
    # projected by the solver onto the range of A^T
    ms_a, (lams, info_a) = _timed(lambda: ctx.solve_adjoint_levels(phis, tol_rel=TOL), 3, 1, stream, barrier)
    ms_g, _ = _timed(lambda: ctx.beta_grad_levels(phis, lams), 5, 1, stream, barrier)
    cells = sum(int((~c).sum()) for c in a["covered"])
    res = {"workload": "amr3: 128^3 periodic level 0 (8 boxes) + ratio-2 level 1 over the central 64^3 "
                       "level-0 cells + ratio-2 level 2 over 64^3 level-1 cells off its centre (128^3 cells "
                       "per level; 8, 8 and 64 boxes), seed 12017, tol 1e-10",
           "composite_cells": cells,
           "forward": {"time_to_tol_ms": ms, "iterations": info.iterations, "status": info.status},
           "adjoint": {"time_to_tol_ms": ms_a, "iterations": info_a.iterations, "status": info_a.status},
           "beta_grad_ms": ms_g, "autotuned_level0_hierarchy": tuned}
    del ctx, rs, phis, lams
    torch.cuda.empty_cache()
    return res


def oracle_table(stream, barrier, dev):
    """GPU time to 1e-10 next to the oracle's (all host cores) and the largest relative
    difference of the GPU result from the oracle's, for the small periodic case, the 512^3
    mixed forms, the 64 batched solves and the two-level adjoint (the 256^3 case is the main
    line).  Prints one JSON record; used to fill the GPU table of the baseline notes."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2009_12009_gb300 import gmg
    from paper_2009_12009_gb300 import inputs as I

    ncores = len(os.sched_getaffinity(0))
    O.set_threads(ncores)

    def ms_of(fn):
        t0 = time.perf_counter()
        out = fn()
        return (time.perf_counter() - t0) * 1e3, out

    def rel(a, b):
        return float(np.abs(a - b).max() / np.abs(b).max())

    res = {"oracle_cores": ncores}
    # poisson32: periodic, singular (projected), FP64
    c = I.poisson32()
    ctx = gmg.Context(c["domain"], c["bc_lo"], c["bc_hi"], boxes=c["boxes"], stream=stream.cuda_stream)
    ctx.allocate(gmg.FP64)
    ctx.set_scalars(0.0, 1.0)
    ctx.set_beta(None)
    rhs = ctx.pack(torch.from_numpy(c["rhs"]))
    ms, (phi, info) = _timed(lambda: ctx.solve(rhs, tol_rel=TOL, project_mean=1), 5, 2, stream, barrier)
    P = O.Problem(c["domain"], c["boxes"], c["bc_lo"], c["bc_hi"])
    P.set_coeffs(0.0, 1.0)
    oms, (want, it, hist, st) = ms_of(lambda: P.solve(c["rhs"], tol_rel=TOL, project_mean=True))
    res["poisson32"] = {"gpu_ms": ms, "iterations": info.iterations, "value": mcell_updates_per_vcycle(ctx, 4) *
                        info.iterations / (ms * 1e-3) / 1e6, "oracle_ms": oms, "oracle_iterations": it,
                        "rel_err_vs_oracle": rel(ctx.unpack(phi).cpu().numpy(), want)}
    del ctx
    # abec512: FP64 oracle solve; the GPU's FP32 and BF16 forms
    c = I.abec512()
    P = O.Problem(c["domain"], c["boxes"], c["bc_lo"], c["bc_hi"])
    P.set_coeffs(c["a"], c["b"], alpha=c["alpha"], beta=c["beta"])
    oms, (want, it, hist, st) = ms_of(lambda: P.solve(c["rhs"], tol_rel=TOL))
    del P
    ctx = gmg.Context(c["domain"], c["bc_lo"], c["bc_hi"], boxes=c["boxes"], stream=stream.cuda_stream)
    ctx.allocate(gmg.MIXED_FP32)
    ctx.set_scalars(c["a"], c["b"])
    ctx.set_beta(torch.from_numpy(c["beta"]))
    rhs = ctx.pack(torch.from_numpy(c["rhs"]))
    ctx.autotune(rhs, gmg.MIXED_FP32)
    ctx.autotune(rhs, gmg.MIXED_BF16)
    r = {"oracle_ms": oms, "oracle_iterations": it}
    for name, prec in (("fp32", gmg.MIXED_FP32), ("bf16", gmg.MIXED_BF16)):
        ms, (phi, info) = _timed(lambda: ctx.solve(rhs, tol_rel=TOL, precision=prec), 2, 1, stream, barrier)
        r[name] = {"gpu_ms": ms, "iterations": info.iterations, "value": mcell_updates_per_vcycle(ctx, 4) *
                   info.iterations / (ms * 1e-3) / 1e6, "rel_err_vs_oracle": rel(ctx.unpack(phi).cpu().numpy(), want)}
    res["abec512_mixed"] = r
    del ctx, rhs, want
    torch.cuda.empty_cache()
    # batch64: every problem on the oracle, one after another
    probs = I.batch64()
    wants, oms = [], 0.0
    for p in probs:
        P = O.Problem(p["domain"], p["boxes"], p["bc_lo"], p["bc_hi"], (0, 0, 0), p["prob_hi"])
        P.set_coeffs(0.0, 1.0, beta=p["beta"])
        t, (w, it, hist, st) = ms_of(lambda: P.solve(p["rhs"], tol_rel=TOL))
        oms += t
        wants.append(w)
    B = gmg.BatchContext(probs, stream=stream.cuda_stream)
    B.allocate(gmg.FP64)
    B.set_scalars(0.0, 1.0)
    B.set_beta_all([torch.from_numpy(p["beta"]) for p in probs])
    brhs = B.pack_all([torch.from_numpy(p["rhs"]) for p in probs])
    B.autotune(brhs, gmg.FP64)
    ms, (phi, infos) = _timed(lambda: B.batch_solve(brhs, tol_rel=TOL), 3, 1, stream, barrier)
    upd = sum(_updates_per_vcycle_problem(B, s) * i.iterations for s, i in enumerate(infos))
    res["batch64"] = {"gpu_ms": ms, "value": upd / (ms * 1e-3) / 1e6, "oracle_ms": oms,
                      "rel_err_vs_oracle": max(rel(B.unpack_solve(s, phi).cpu().numpy(), w)
                                               for s, w in enumerate(wants))}
    del B, brhs, phi
    torch.cuda.empty_cache()
    # amr2: the oracle's composite forward solve; the GPU's forward and adjoint solves
    a = I.amr2()
    P = O.AmrProblem(a["domain"], a["coarse_boxes"], a["fine_boxes"], a["bc_lo"], a["bc_hi"])
    lo, hi = a["fine_slice"]
    sl = (slice(lo, hi + 1),) * 3

    def full_fine(x):
        out = np.zeros(P.fine_shape)
        out[sl] = x
        return out

    bf = np.ones(P.fine_shape)
    bf[sl] = a["beta_f"]
    P.set_coeffs(0.0, 1.0, beta_c=a["beta_c"], beta_f=bf)
    oms, (oc, of, it, hist, st) = ms_of(lambda: P.solve(a["rhs_c"], full_fine(a["rhs_f"]), tol_rel=TOL))
    actx = gmg.AmrContext(a["domain"], a["coarse_boxes"], a["fine_boxes"], a["bc_lo"], a["bc_hi"],
                          stream=stream.cuda_stream)
    actx.allocate(gmg.FP64)
    actx.set_coeffs(0.0, 1.0, beta_c=torch.from_numpy(a["beta_c"]), beta_f=torch.from_numpy(a["beta_f"]))
    rc, rf = actx.pack_level(0, torch.from_numpy(a["rhs_c"])), actx.pack_level(1, torch.from_numpy(a["rhs_f"]))
    actx.autotune(rc, gmg.FP64)
    ms_f, (pc, pf, info_f) = _timed(lambda: actx.solve2(rc, rf, tol_rel=TOL), 3, 1, stream, barrier)
    phi_c = actx.unpack_level(0, pc).cpu().numpy() * P.coarse_mask
    phi_f = full_fine(actx.unpack_level(1, pf).cpu().numpy())
    gcn = (phi_c - a["target_c"]) * P.coarse_mask
    gfn = phi_f[sl] - a["target_f"]
    gc, gf = actx.pack_level(0, torch.from_numpy(gcn)), actx.pack_level(1, torch.from_numpy(gfn))
    ms_a, (lc, lf, info_a) = _timed(lambda: actx.solve_adjoint2(gc, gf, tol_rel=TOL), 3, 1, stream, barrier)
    lam = (actx.unpack_level(0, lc).cpu().numpy() * P.coarse_mask, full_fine(actx.unpack_level(1, lf).cpu().numpy()))
    g = P.pack(gcn, full_fine(gfn))
    V = P.volumes()
    g = g - V * g.sum() / V.sum()
    res["amr2_adjoint"] = {"gpu_forward_ms": ms_f, "gpu_adjoint_ms": ms_a, "forward_iterations": info_f.iterations,
                           "adjoint_iterations": info_a.iterations, "oracle_forward_ms": oms,
                           "oracle_forward_iterations": it,
                           "forward_rel_err_vs_oracle": rel(P.pack(phi_c, phi_f), P.pack(oc, of)),
                           "adjoint_rel_resid_by_oracle_transpose":
                               float(np.abs(g - P.pack(*P.apply(*lam, transpose=True))).max() / np.abs(g).max())}
    O.set_threads(1)
    return res


def summary(out):
    """The headline figures in one small record, printed last in the JSON line."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return round(d, 4) if isinstance(d, float) else d

    f = out.get("forms", {})
    return {
        "abec256_ms": {"fp64": g(out, "time_to_tol_ms"), "fp32": g(out, "mixed", "fp32", "time_to_tol_ms"),
                       "bf16": g(out, "mixed", "bf16", "time_to_tol_ms")},
        "abec256_mixed_speedup": {"fp32": g(out, "mixed", "fp32", "speedup_vs_fp64"),
                                  "bf16": g(out, "mixed", "bf16", "speedup_vs_fp64")},
        "abec256_rel_err_vs_oracle": out.get("rel_err_vs_oracle"),
        "abec512_ms": {k: g(f, "abec512", k, "time_to_tol_ms") for k in ("fp64", "fp32", "bf16")},
        "abec512_mixed_speedup": {"fp32": g(f, "abec512", "mixed_speedup_fp32"),
                                  "bf16": g(f, "abec512", "mixed_speedup_bf16")},
        "batch64_ms": {"fp64": g(f, "batch64", "fp64", "time_to_tol_ms"),
                       "fp32": g(f, "batch64", "fp32", "time_to_tol_ms"),
                       "fp64_one_by_one": g(f, "batch64", "sequential_fp64", "time_to_tol_ms")},
        "amr2_ms": {"forward": g(f, "amr2", "forward", "time_to_tol_ms"),
                    "adjoint": g(f, "amr2", "adjoint", "time_to_tol_ms"), "beta_grad": g(f, "amr2", "beta_grad_ms")},
        "amr3_ms": {"forward": g(f, "amr3", "forward", "time_to_tol_ms"),
                    "adjoint": g(f, "amr3", "adjoint", "time_to_tol_ms")},
        "smoother_frac": {"hbm_algorithmic": g(out, "roofline", "frac"),
                          "fp64_pipe": g(out, "roofline", "fp64_pipe", "frac")},
        "fp64_peak_tflops": g(out, "fp64_peak", "tflops"),
        "oracle_ms": g(out, "cpu_baseline", "time_to_tol_ms"), "oracle_cores": g(out, "cpu_baseline", "cores"),
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2009_12009_gb300 import inputs as I
    from oracle import oracle as O

    cfg = I.abec256()
    P = O.Problem(cfg["domain"], cfg["boxes"], cfg["bc_lo"], cfg["bc_hi"])
    P.set_coeffs(cfg["a"], cfg["b"], alpha=cfg["alpha"], beta=cfg["beta"])
    cells = sum(P.level_shape(m)[0] * P.level_shape(m)[1] * P.level_shape(m)[2] * 4 for m in range(P.nlevels - 1))
    ncores = len(os.sched_getaffinity(0))
    O.set_threads(ncores)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        P.solve(cfg["rhs"], tol_rel=0.0, maxit=1)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = cells * len(times) / tot / 1e6
    sample = f"each step: 1 V-cycle iteration of the abec256 solve (FP64 oracle, OpenMP over boxes, {ncores} threads)"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
                      "cpu_baseline": {"value": val, "unit": UNIT, "cores": ncores, "kind": "oracle", "sample": sample},
                      "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the 512^3, batched and two-level workloads")
    ap.add_argument("--oracle-table", action="store_true",
                    help="print only GPU and oracle times and differences for the other workloads")
    ap.add_argument("--only", choices=["abec512", "batch64", "amr2", "amr3", "walls256", "krylov"], default=None,
                    help="run and print only this one of the other workloads (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2009_12009_gb300 import gmg
    from paper_2009_12009_gb300 import inputs as I

    stream = torch.cuda.current_stream()
    if args.oracle_table:
        print(json.dumps({"oracle_table": oracle_table(stream, torch.cuda.synchronize, dev)}))
        return
    if args.only:
        def sync():
            torch.cuda.synchronize()
        print(json.dumps({"forms": measure_forms(stream, sync, dev, only=args.only)}))
        return
    cfg = I.abec256()
    ctx = gmg.Context(cfg["domain"], cfg["bc_lo"], cfg["bc_hi"], boxes=cfg["boxes"], stream=stream.cuda_stream)
    ctx.allocate(gmg.FP64 if args.no_mixed else gmg.MIXED_FP32)
    ctx.set_scalars(cfg["a"], cfg["b"])
    ctx.set_beta(torch.from_numpy(cfg["beta"]))
    rhs = ctx.pack(torch.from_numpy(cfg["rhs"]))
    phi = ctx.field(0)
    ncells = int(np.prod(ctx.level_shape(0)))
    nu = 4
    tuned = {"fp64": ctx.autotune(rhs, gmg.FP64)}
    if not args.no_mixed:
        tuned["fp32"] = ctx.autotune(rhs, gmg.MIXED_FP32)
        tuned["bf16"] = ctx.autotune(rhs, gmg.MIXED_BF16)
    upd_per_vc = mcell_updates_per_vcycle(ctx, nu)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed_solves(precision, steps, warmup, profile=0):
        """profile: the last timed solve records CUDA events around its finest-level smoother
        and outer residual launches (its captured graph, built in the warm-up, holds them);
        the other solves replay the plain graph"""
        for _ in range(warmup):
            ctx.solve(rhs, phi, tol_rel=TOL, precision=precision)
        if profile:
            ctx.solve(rhs, phi, tol_rel=TOL, precision=precision, profile=profile)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for k in range(steps):
            _, info = ctx.solve(rhs, phi, tol_rel=TOL, precision=precision,
                                profile=profile if k == steps - 1 else 0)
            infos.append(info)
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1), infos

    fp64pk = fp64_peak(stream, local)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, infos = timed_solves(gmg.FP64, args.steps, args.warmup, profile=1)
    clk = clocks.stop()
    its = [i.iterations for i in infos]
    assert all(i.status == gmg.OK for i in infos), [i.status for i in infos]
    ms, updates, value = whole_job(ms, sum(upd_per_vc * k for k in its), world, dev)
    phi64 = ctx.unpack(phi).clone()

    # roofline of the dominant kernel: the finest-level red-black smoother.  Wavefront
    # launches cover a whole sweep (two colour passes): 56 B/cell, except the first
    # pre-smoothing sweep of each V-cycle, which starts from a zero correction and does not
    # read it (48 B/cell); the two-pass form covers one colour pass per launch (28 B/cell).
    sm_ms = sum(i.smooth0_ms for i in infos)
    sm_n = sum(i.smooth0_launches for i in infos)
    sm_passes = sum(i.smooth0_passes for i in infos)
    launch_s = sm_ms * 1e-3 / max(sm_n, 1)
    wave = sm_n > 0 and sm_passes == 2 * sm_n
    sweeps = nu  # level-0 sweeps per V-cycle (nu1 + nu2)
    if wave:
        alg_bytes = ncells * (SWEEP_BYTES_PER_CELL * sweeps - 8) / sweeps
        # 7 FP64-pipe operations per updated cell; the zero-start sweep's red cells take 2
        fp64_ops = ncells * (UPDATE_FP64_OPS * sweeps - 2.5) / sweeps
    else:
        alg_bytes = PASS_BYTES_PER_CELL * ncells * sm_passes / max(sm_n, 1)
        fp64_ops = UPDATE_FP64_OPS * (ncells / 2) * sm_passes / max(sm_n, 1)
    achieved = alg_bytes / launch_s / 1e9
    peak, peak_kind = peaks()
    fp64_rate = fp64_ops / launch_s
    rs_ms = sum(i.resid0_ms for i in infos)
    rs_n = sum(i.resid0_launches for i in infos)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "time_to_tol_ms": ms / args.steps,
           "iterations": its[0], "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "cells": ncells, "mg_levels": ctx.nlevels,
                      "cell_updates_per_vcycle": upd_per_vc, "parallelism": f"replicas x{world}",
                      "l2": "inputs larger than L2 (finest-level working set ~1.2 GB of fields and coefficients)",
                      "autotuned": {k: summarize_tuning(v) for k, v in tuned.items()}},
           "gpu_launches": int(sum(i.kernel_launches for i in infos)),
           "roofline": {"bound": "hbm",
                        "kernel": ("k_wave<double> (finest level, one red+black sweep per launch)" if wave
                                   else "k_smooth<double> (finest level, one colour pass)"),
                        "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "peak_kind": peak_kind,
                        "traffic": kernel_traffic("k_wave_f64" if wave else "k_smooth_f64"),
                        "algorithmic_bytes_per_launch": alg_bytes,
                        "bytes_rule": ("56 B/cell per red+black sweep (48 for the sweep from a zero "
                                       "correction, once per V-cycle), averaged over the launches" if wave
                                       else "56 B/cell per red+black sweep = 28 B/cell per colour pass"),
                        "avg_launch_us": launch_s * 1e6, "launches_timed": sm_n, "passes_timed": sm_passes,
                        "fp64_pipe": {"ops_per_launch": fp64_ops, "achieved_gops": fp64_rate / 1e9,
                                      "peak_gops": fp64pk["fma_per_s"] / 1e9,
                                      "frac": fp64_rate / fp64pk["fma_per_s"],
                                      "peak_kind": "measured in this run (gmg_dfma_probe)"}},
           "outer_residual": {"kernel": "k_residual<double> (finest level, FP64)", "avg_launch_us":
                              1e3 * rs_ms / max(rs_n, 1), "launches_timed": rs_n},
           # per V-cycle iteration, and the finest level's share of the cell updates
           "ms_per_iteration": ms / args.steps / max(its[0], 1),
           "finest_level_value": ncells * nu * sum(its) * world / (ms * 1e-3) / 1e6,
           "clocks": clk}

    sols = {"fp64": phi64.cpu().numpy()}
    if not args.no_mixed:
        mixed = {}
        for name, prec in (("fp32", gmg.MIXED_FP32), ("bf16", gmg.MIXED_BF16)):
            ms_m, inf_m = timed_solves(prec, max(3, args.steps // 2), 2)
            itm = inf_m[0].iterations
            ms_m, _, val_m = whole_job(ms_m, sum(upd_per_vc * i.iterations for i in inf_m), world, dev)
            sol_m = ctx.unpack(phi)
            err = float((sol_m - phi64).abs().max() / phi64.abs().max())
            sols[name] = sol_m.cpu().numpy()
            mixed[name] = {"time_to_tol_ms": ms_m / len(inf_m), "value": val_m, "unit": UNIT,
                           "iterations": itm, "final_rel_resid": inf_m[-1].final_resid / inf_m[-1].rhs_norm,
                           "rel_err_vs_fp64_solve": err,
                           "speedup_vs_fp64": (ms / args.steps) / (ms_m / len(inf_m))}
        out["mixed"] = mixed

    if not args.no_e2e:
        host_rhs = torch.from_numpy(cfg["rhs"]).pin_memory()
        host_out = torch.empty(ctx.level_shape(0), dtype=torch.float64).pin_memory()
        dense = torch.empty(ctx.level_shape(0), dtype=torch.float64, device=dev)
        nsteps = max(3, args.steps // 2)
        barrier()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tot_upd = 0
        for _ in range(nsteps):
            dense.copy_(host_rhs, non_blocking=True)
            r = ctx.pack(dense, out=rhs)
            _, info = ctx.solve(r, phi, tol_rel=TOL)
            host_out.copy_(ctx.unpack(phi), non_blocking=True)
            tot_upd += upd_per_vc * info.iterations
        e1.record(stream)
        barrier()
        ms_e, _, val_e = whole_job(e0.elapsed_time(e1), tot_upd, world, dev)
        out["e2e"] = {"value": val_e, "unit": UNIT,
                      "h2d_bytes_per_step": 8 * ncells, "d2h_bytes_per_step": 8 * ncells,
                      "wall_ms_per_step": 1e3 * (time.perf_counter() - t0) / nsteps}

    if not args.no_forms:
        del ctx, rhs, phi
        torch.cuda.empty_cache()
        out["forms"] = measure_forms(stream, barrier, dev)

    if not args.no_cpu and rank == 0 and world == 1:
        out["cpu_baseline"], ref = cpu_baseline(cfg)
        den = float(np.abs(ref).max())
        out["rel_err_vs_oracle"] = {k: float(np.abs(v - ref).max() / den) for k, v in sols.items()}
    out["fp64_peak"] = fp64pk
    if rank == 0:
        out["summary"] = summary(out)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
