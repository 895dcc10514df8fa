#!/usr/bin/env python3
"""FLD radiation substep benchmark (one JSON line on rank 0).

Workload: the 3D stratified box of 256^3 cells (x, y periodic, z Dirichlet,
Kramers-like opacity, dt = 10x the explicit limit), the radiative-magnetoconvection
shaped case whose metric compares mixed precision with FP64. One step is one whole
substep on the resident fields: limiter -> backward-Euler multigrid solve to a
relative residual of 1e-10 -> exchange quartic, through the C ABI (fld_step).

value    cell-updates/s = cells x steps x ranks / max-over-ranks device time
e2e      the same through the C ABI with pinned HOST buffers: every step copies
         rho, T, E (and the Dirichlet faces) to the device and T, E back
roofline the dominant kernel's algorithmic bytes per launch / its event-timed
         launch duration, against the measured copy bandwidth
cpu_baseline  the CPU oracle on a bounded sample of the same workload (rank 0)

--impl reference times that CPU oracle alone (the comparison arm).
Multi-GPU: each rank solves its own independent replica (no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FLD cell-updates/s (limiter + multigrid solve to 1e-10 + exchange)"
UNIT = "cell-updates/s"

# algorithmic bytes per cell of each kernel family (FP64 = 8 B, FP32 = 4 B),
# counting each array once per launch: reads + writes
BYTES_PER_CELL = {
    "limiter": 32.0,          # E, rho, T read; D written (power-law opacity)
    "prep": 36.0,             # D, E read; K64, K32, b written
    "split_df": 16.0,         # E read; its FP32 (hi, lo) pair written
    "df_setup": 48.0,         # E, b, K read; their FP32 (hi, lo) pairs written
    "df_finish": 16.0,        # x (hi, lo) read; E written
    "sumsq": 8.0,             # b read
    "resid64": 28.0,          # x, b, K read; r32 written (mixed) / 24 (fp64)
    "resid_df": 40.0,         # x (hi, lo), e32, b (hi, lo), K (hi, lo) read; x (hi, lo), r32 written
    "rbhalf32": 10.0,         # one colour: the other colour's x and every K read (faces),
    "rbhalf64": 20.0,         #   this colour's b read and x written
    "rbsweep32": 16.0,        # x, K, b read; x written (both colours in one pass)
    "rbsweep64": 32.0,
    "add_correction": 20.0,   # x, e32 read; x written
    "smooth32": 16.0,         # xin, b, K read; xout written
    "smooth64": 32.0,
    "resid_restrict32": 12.0,
    "resid_restrict64": 24.0,
    "prolong32": 8.0,
    "prolong64": 16.0,
    "exchange": 40.0,         # rho, T, E read; T, E written (kappa evaluated from rho, T)
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# FP64 ALU peak of the GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA lanes
# per SM per clock (the rate a dependent-FMA probe sustains) x 2 flop x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def ncu_traffic(kernel, cells_per_launch):
    """DRAM bytes per launch from the committed ncu capture (profiles/dram_traffic.json),
    scaled by cells per launch; None when the kernel's source changed since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    k = d.get("kernels", {}).get(kernel)
    if not k:
        return None
    src = os.path.join(ROOT, k["source"])
    if not os.path.exists(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != k["sha256_16"]:
        return None
    return k["dram_bytes"] * cells_per_launch / d["cells"]


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
                except ValueError:
                    pass
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows)}


def cpu_sample_step(n=40, steps=1):
    """The oracle on a bounded sample of the workload: the same recipe at n^3."""
    from oracle import fld as O
    from paper_2503_02764_gb300 import inputs as I
    P = I.stratified_3d(n)
    T, E = P.T.copy(), P.E.copy()
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(steps):
        T, E, _ = O.step(P.rho, T, E, P.h, P.bc, P.E_bc, P.dt, P.c, P.a_r, P.gamma, P.R_gas,
                         P.opacity, P.limiter, method="pcg")
    dt = time.perf_counter() - t0
    cores = max(1, round((time.process_time() - c0) / dt))
    return P.ncells * steps / dt, dt, P.ncells, cores


def cpu_baseline(n=64):
    """The oracle timed on the host cores; cores = CPU time / wall time of the sample."""
    v, secs, cells, cores = cpu_sample_step(n, 1)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one oracle substep (numpy/scipy FP64, PCG solve, long-double exchange) "
                      "of the stratified recipe at %d^3 = %d cells, %.1f s" % (n, cells, secs)}


def aggregate(ms_local, units_local, steps, dist=None, device="cpu"):
    """Whole-job throughput over ranks: the slowest rank's time (MAX) and all ranks' units
    (SUM). Returns (ms_max, units_total, value_per_second)."""
    ms_max, units = float(ms_local), float(units_local)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        u = torch.tensor([units_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms_max, units = float(t.item()), float(u.item())
    return ms_max, units, units * steps / (ms_max * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def next_rows(hd, P, prec, gkw, consts, op, rho, T, E, ebc, peak_hbm):
    """Per-call timings of the widening rows on the bench workload (CUDA events, after
    warm-up, averaged over a few calls): the explicit coupling terms (with a velocity
    field), the three limiters, a tabulated opacity against the power law it extends (the
    table built around the recipe's Kramers coefficient), and the 1D radiation-MHD wave
    step of the strongly radiative fast wave (280 cells)."""
    import torch
    from paper_2503_02764_gb300 import fld, inputs as I
    stream = torch.cuda.current_stream()
    n = P.ncells

    def timed(fn, reps=5, warm=2):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def hbm(ms, bpc):
        gbs = bpc * n / (ms * 1e-3) / 1e9
        return {"ms": ms, "bytes_per_cell": bpc, "achieved_GBs": gbs, "frac": gbs / peak_hbm}

    out = {"cells": n}
    z = lambda m: torch.empty(m, dtype=torch.float64, device="cuda")
    hd.set_opts(precision=prec, tol=1e-10, max_cycles=50, limiter=fld.LIMITER_LP, **gkw)
    v = z(3 * n).uniform_(-1.0, 1.0)
    Fo, fro, fe, vfr, pt = z(3 * n), z(3 * n), z(n), z(n), z(n)
    # reads E, rho, T, v (6 words), writes F, f_r (3 each), f, v.f_r, P:grad v
    out["coupling"] = hbm(timed(lambda: hd.coupling(consts, op, E, rho, T, ebc, v, Fo, fro, fe,
                                                    vfr, pt)), 120.0)
    del v, Fo, fro, fe, vfr, pt
    D = z(n)
    lim = {}
    for name, mode in (("levermore_pomraning", fld.LIMITER_LP),
                       ("diffusion_1_3", fld.LIMITER_DIFFUSION),
                       ("minerbo", fld.LIMITER_MINERBO)):
        hd.set_opts(precision=prec, tol=1e-10, max_cycles=50, limiter=mode, **gkw)
        # the split of E into FP32 pairs (16 B) and the limiter proper (32 B) in MIXED_DF
        lim[name] = hbm(timed(lambda: hd.limiter(consts, op, E, rho, T, ebc, D)),
                        48.0 if prec == fld.PREC_MIXED_DF else 32.0)
    out["limiter"] = lim
    hd.set_opts(precision=prec, tol=1e-10, max_cycles=50, limiter=fld.LIMITER_LP, **gkw)
    table, grid = I.opacity_table(P.opacity[1])
    tdev = torch.from_numpy(table).cuda()
    top = fld.make_opacity((I.OPACITY_TABLE, 1.0, table, grid), tdev)
    tab = {"table_shape": list(table.shape)}
    for name, o in (("power_law", op), ("table", top)):
        Tc, Ec = T.clone(), E.clone()
        tab[name] = {
            "limiter": hbm(timed(lambda: hd.limiter(consts, o, E, rho, T, ebc, D)),
                           48.0 if prec == fld.PREC_MIXED_DF else 32.0),
            "exchange": hbm(timed(lambda: hd.exchange(consts, o, P.dt, rho, Tc, Ec)), 40.0),
            "step_ms": timed(lambda: hd.step(consts, o, P.dt, rho, Tc, Ec, ebc,
                                             raise_on_error=False), reps=3, warm=1),
        }
        del Tc, Ec
    out["tabulated_opacity"] = tab
    wp = I.wave1d(I.WAVE_BACKGROUNDS["strong"], 280, 7, "fast")
    wv = fld.Wave1D(wp, precision=fld.PREC_FP64, tol=1e-13, max_cycles=200)
    W = np.repeat(np.asarray(wp.W0, dtype=float)[:, None], wp.n, axis=1)
    U = np.stack([W[0], W[0] * W[1], W[0] * W[2], W[0] * W[3], W[4], W[5],
                  W[6] / (wp.gamma - 1.0) + 0.5 * (wp.Bx ** 2 + W[4] ** 2 + W[5] ** 2), W[7]])
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    state = {"t": 0.0}

    def wave_step():
        dt = wv.max_dt(Ud, 0.8)
        wv.step(Ud, state["t"], dt)
        state["t"] += dt

    ms = timed(wave_step, reps=50, warm=5)
    out["wave1d"] = {"cells": wp.n, "ms_per_step": ms, "cell_updates_per_s": wp.n / (ms * 1e-3),
                     "note": "launch- and synchronisation-bound on 280 cells: three Runge-Kutta "
                             "stages of four launches, the substep's FP64 multigrid cycles and "
                             "several host synchronisations per step"}
    wv.close()
    return out


def workload_name(n):
    return ("stratified3d_%d^3 (x,y periodic, z Dirichlet, Kramers opacity, "
            "dt = 10x explicit limit)" % n)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = 32
    for _ in range(args.warmup):
        cpu_sample_step(n, 1)
    t0 = time.perf_counter()
    total, cores = 0, 1
    for _ in range(args.steps):
        _, _, cells, c = cpu_sample_step(n, 1)
        total += cells
        cores = max(cores, c)
    secs = time.perf_counter() - t0
    v = total / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.n), "cells": args.n ** 3,
                       "precision": "f64 (oracle)", "tol": 1e-10,
                       "sample": "each step one oracle substep of the same recipe at %d^3" % n},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d oracle substeps of the stratified recipe at %d^3" %
                                       (args.steps, n)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def tuned_opts(kind, problems):
    """Autotuner cache entry for this GPU and workload, or None."""
    try:
        from paper_2503_02764_gb300 import autotune
        c = autotune.cached(kind, autotune.signature(kind, problems))
        return c["best"] if c else None
    except Exception:
        return None


def run_batch(args):
    """The batched workload: 512 independent 2D problems (sides U{32..512}) advanced in
    one persistent launch per step (fld_step_batched), replayed from a CUDA graph."""
    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2503_02764_gb300 import build, fld
    from paper_2503_02764_gb300 import inputs as I
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    # each rank advances its own independent batch (weak scaling, no collective)
    ps = I.batch(args.nprob, seed_base=I.SEED_BASE + 4 + 100000 * rank)
    tuned = tuned_opts("batch", ps)
    kw = dict(block=args.block, cluster=args.cluster, nu1=2, nu2=2)
    if tuned and not (args.block or args.cluster):
        kw = {k: tuned[k] for k in ("block", "cluster", "nu1", "nu2")}
        kw["inner"] = tuned.get("inner", 1)
    b = fld.Batch([(p.shape, p.h, p.bc) for p in ps], tol=1e-10, max_cycles=50, graph=1, **kw)
    cat = lambda xs: torch.from_numpy(np.concatenate([x.ravel() for x in xs])).cuda()
    rho, T, E = cat([p.rho for p in ps]), cat([p.T for p in ps]), cat([p.E for p in ps])
    consts = fld.make_consts(1.0, 1.0, 5.0 / 3.0, 1.0)
    ops = [fld.make_opacity(p.opacity) for p in ps]
    dts = [p.dt for p in ps]
    for _ in range(args.warmup):
        b.step(consts, ops, dts, rho, T, E)
    n0 = fld.fld_launch_count()
    stream = torch.cuda.current_stream()
    clk = Clocks(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    cyc = []
    for _ in range(args.steps):
        rc, st = b.step(consts, ops, dts, rho, T, E)
        cyc.append(max(x["cycles"] for x in st))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = clk.stop()
    ms_local = ev0.elapsed_time(ev1)
    ms, cells_all, value = aggregate(ms_local, b.cells, args.steps, dist, "cuda")
    cells = b.cells
    line = {"metric": METRIC + " [batched]", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 V-cycles + double-f32 refinement + f64 limiter/exchange",
            "data": "synthetic",
            "config": {"workload": "batch of %d 2D problems, sides U{32..512}, one persistent "
                                   "launch per step, CUDA graph" % args.nprob,
                       "cells": cells, "block": kw["block"] or 512,
                       "cluster": kw["cluster"] or "auto", "nu1": kw["nu1"], "nu2": kw["nu2"],
                       "inner": kw.get("inner", 1),
                       "autotuned": bool(tuned and not (args.block or args.cluster))},
            "max_cycles_per_step": cyc, "clocks": clocks,
            "gpu_launches": args.steps}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed_df", choices=["mixed_df", "mixed", "fp64"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the timings of the widening rows (coupling, limiters, tabulated "
                         "opacity, 1D wave step)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--smoother", type=int, default=-1,
                    help="-1 the tuned choice (else 0); 0 in-place half sweeps, 1 out-of-place "
                         "half sweeps, 2 single-pass z-marching sweep")
    ap.add_argument("--nu1", type=int, default=-1, help="pre-smoothing sweeps (-1: tuned)")
    ap.add_argument("--nu2", type=int, default=-1, help="post-smoothing sweeps (-1: tuned)")
    ap.add_argument("--inner", type=int, default=-1,
                    help="FP32 V-cycles per refinement step (-1: tuned)")
    ap.add_argument("--no-ttt", action="store_true", help="skip the mixed-vs-FP64 solve timing")
    ap.add_argument("--workload", default="stratified", choices=["stratified", "batch"],
                    help="stratified: one 3D box (default); batch: 512 uneven 2D problems")
    ap.add_argument("--nprob", type=int, default=512)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--cluster", type=int, default=0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)

    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2503_02764_gb300 import build, fld
    from paper_2503_02764_gb300 import inputs as I
    if rank == 0:
        build.build()
    barrier()

    P = I.stratified_3d(args.n)
    prec = {"mixed_df": fld.PREC_MIXED_DF, "mixed": fld.PREC_MIXED, "fp64": fld.PREC_FP64}[
        args.precision]
    tuned = tuned_opts("grid", [P])
    gkw = dict(nu1=2, nu2=2, smoother=0, inner=1)
    if tuned:
        gkw = {k: tuned[k] for k in ("nu1", "nu2", "smoother")}
        gkw["inner"] = tuned.get("inner", 1)
    for k in ("smoother", "nu1", "nu2", "inner"):     # explicit choices override the tuner
        if getattr(args, k) >= 0:
            gkw[k] = getattr(args, k)
            tuned = None
    hd = fld.Handle(P.shape, P.h, P.bc, precision=prec, tol=1e-10, max_cycles=50, **gkw)
    consts = fld.make_consts(P.c, P.a_r, P.gamma, P.R_gas)
    op = fld.make_opacity(P.opacity)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rho, T, E = dev(P.rho), dev(P.T), dev(P.E)
    ebc = dev(I.pack_dirichlet(P.shape, P.bc, P.E_bc))
    stream = torch.cuda.current_stream()

    stats = None
    for _ in range(args.warmup):
        stats = hd.step(consts, op, P.dt, rho, T, E, ebc)

    # ---------------- timed region (device-resident inputs, graphs on, no profiling)
    n0 = fld.fld_launch_count()
    clk = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    cycles = []
    for _ in range(args.steps):
        st = hd.step(consts, op, P.dt, rho, T, E, ebc)
        cycles.append(st["cycles"])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    launches = fld.fld_launch_count() - n0
    ms = ev0.elapsed_time(ev1)
    ms_max, _, value = aggregate(ms, P.ncells, args.steps, dist, "cuda")

    # ---------------- the same steps again with every launch bracketed by events: the
    # per-kernel durations for the roofline and the breakdown (graphs are off while
    # profiling, so this pass is slightly slower than the one above)
    hd.prof_enable(True, 65536)
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        hd.step(consts, op, P.dt, rho, T, E, ebc)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_prof = e2.elapsed_time(e3)
    prof = hd.prof_read()
    hd.prof_enable(False)

    # ---------------- roofline of the dominant level-0 kernel
    peak_hbm, peak_kind = load_peaks()
    lvl0 = [e for e in prof if e["level"] == 0 and e["name"] in BYTES_PER_CELL]
    dom = max(lvl0, key=lambda e: e["ms"]) if lvl0 else None
    roof = None
    if dom:
        bpc = BYTES_PER_CELL[dom["name"]]
        if dom["name"] == "resid64" and prec == fld.PREC_FP64:
            bpc = 24.0
        achieved = bpc * dom["cells"] / (dom["ms"] * 1e-3) / 1e9
        roof = {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": peak_hbm,
                "unit": "GB/s", "frac": achieved / peak_hbm,
                "traffic": ncu_traffic(dom["name"], dom["cells"] / dom["launches"]),
                "peak_source": peak_kind, "launches": dom["launches"],
                "avg_launch_us": 1e3 * dom["ms"] / dom["launches"],
                "bytes_per_cell": bpc}
    total_prof = sum(e["ms"] for e in prof)
    breakdown = sorted(({"kernel": e["name"], "level": e["level"], "launches": e["launches"],
                         "ms": round(e["ms"], 4), "share": round(e["ms"] / total_prof, 4)}
                        for e in prof), key=lambda d: -d["ms"])[:12]

    # ---------------- end to end through the C ABI with host buffers. Every step copies its
    # inputs (rho, T, E, the Dirichlet face values) from pinned host memory and reads its
    # results (T, E) back. The inputs are the state the device-resident steps above reached,
    # so that these steps do the same solve work as those (steps from the initial fields
    # take longer). Serial: copy in, step, copy out, on one stream.
    # Pipelined (the reported value): three device buffer sets; while step k computes, step
    # k+1's inputs go up on one copy stream and step k-1's results come down on another (the
    # two directions overlap each other too), each transfer ordered by events.
    e2e = None
    if not args.no_e2e:
        h_in = tuple(x.detach().cpu().pin_memory() for x in (rho, T, E, ebc))
        e2e_cycles = []
        NSET = 3
        h_out = [tuple(torch.empty_like(h_in[i]).pin_memory() for i in (1, 2))
                 for _ in range(NSET)]
        d_in = [tuple(torch.empty_like(x, device="cuda") for x in h_in) for _ in range(NSET)]

        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            for d, h in zip(d_in[0], h_in):
                d.copy_(h, non_blocking=True)
            hd.step(consts, op, P.dt, *d_in[0][:3], d_in[0][3])
            for o, d in zip(h_out[0], d_in[0][1:3]):
                o.copy_(d, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_serial = ev0.elapsed_time(ev1)
        E_serial = h_out[0][1].clone()

        up, down = torch.cuda.Stream(), torch.cuda.Stream()
        ev = lambda: torch.cuda.Event()
        ready, stepped, freed = ([ev() for _ in range(NSET)] for _ in range(3))
        used = [False] * NSET

        def upload(k):
            b = k % NSET
            with torch.cuda.stream(up):
                if used[b]:
                    up.wait_event(freed[b])       # the results of step k-3 are back on the host
                for d, h in zip(d_in[b], h_in):
                    d.copy_(h, non_blocking=True)
                ready[b].record(up)

        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(stream)
        up.wait_event(ev0)
        upload(0)
        for k in range(args.steps):
            b = k % NSET
            if k + 1 < args.steps:
                upload(k + 1)
            stream.wait_event(ready[b])
            e2e_cycles.append(hd.step(consts, op, P.dt, *d_in[b][:3], d_in[b][3])["cycles"])
            stepped[b].record(stream)
            with torch.cuda.stream(down):
                down.wait_event(stepped[b])
                for o, d in zip(h_out[b], d_in[b][1:3]):
                    o.copy_(d, non_blocking=True)
                freed[b].record(down)
            used[b] = True
        for b in range(NSET):
            if used[b]:
                stream.wait_event(freed[b])
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms_e2e = ev0.elapsed_time(ev1)
        barrier()
        # every step starts from the same inputs: the pipelined result must match the serial one
        diff = float(((h_out[(args.steps - 1) % NSET][1] - E_serial).abs()
                      / E_serial.abs().clamp_min(1e-300)).max())
        if diff > 1e-9:
            raise RuntimeError(f"pipelined end-to-end result differs from the serial one: {diff}")
        h2d = sum(x.numel() * x.element_size() for x in h_in)
        d2h = sum(x.numel() * x.element_size() for x in h_out[0])
        _, _, e2e_value = aggregate(ms_e2e, P.ncells, args.steps, dist, "cuda")
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": ms_e2e / args.steps, "wall_ms_per_step": 1e3 * wall / args.steps,
               "pipelined": True, "serial_ms_per_step": ms_serial / args.steps,
               "max_rel_diff_pipelined_vs_serial": diff,
               "cycles_per_step_mean": float(np.mean(e2e_cycles))}

    # ---------------- mixed vs FP64 time to 1e-10 on the same GPU (diffusion solve alone)
    ttt = {}
    if rank == 0 and not args.no_ttt:
        D = torch.empty_like(E)
        hd.limiter(consts, op, E, rho, T, ebc, D)
        for name, pr in (("mixed_df", fld.PREC_MIXED_DF), ("mixed", fld.PREC_MIXED),
                         ("fp64", fld.PREC_FP64)):
            hd.set_opts(precision=pr, tol=1e-10, max_cycles=50, **gkw)
            times, cyc = [], 0
            for rep in range(4):
                X = E.clone()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st = hd.diffuse(P.dt, D, ebc, X)
                b.record(stream)
                torch.cuda.synchronize()
                if rep:
                    times.append(a.elapsed_time(b))
                cyc = st["cycles"]
            ttt[name] = {"ms": float(np.median(times)), "cycles": cyc}

    # ---------------- the widening rows, timed on the same workload (rank 0)
    rows = None
    if rank == 0 and not args.no_next:
        try:
            rows = next_rows(hd, P, prec, gkw, consts, op, rho, T, E, ebc, load_peaks()[0])
        except Exception as exc:                 # reported, never fatal to the headline
            rows = {"error": "%s: %s" % (type(exc).__name__, exc)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {fld.PREC_MIXED_DF: "f32 V-cycles + double-f32 (48-bit) refinement residual/"
                                         "correction + f64 limiter/exchange/coarse solve",
                      fld.PREC_MIXED: "f32 V-cycles + f64 refinement residual/correction/"
                                      "limiter/exchange/coarse solve",
                      fld.PREC_FP64: "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": workload_name(args.n),
                       "cells": P.ncells, "precision": args.precision, "tol": 1e-10,
                       "nu1": gkw["nu1"], "nu2": gkw["nu2"], "smoother": gkw["smoother"],
                       "inner": gkw.get("inner", 1),
                       "autotuned": bool(tuned),
                       "l2": "inputs larger than L2 (fields %.0f MB + workspace)" %
                             (3 * P.ncells * 8 / 1e6),
                       "parallelism": "replicas x%d" % world},
            "gpu_launches": launches, "cycles_per_step": cycles,
            "profiled_pass_ms_per_step": ms_prof / args.steps,
            "roofline": roof, "kernel_breakdown": breakdown,
            "time_to_1e-10_ms": ttt, "clocks": clocks, "e2e": e2e}
    if rows is not None:
        line["next_rows"] = rows
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
