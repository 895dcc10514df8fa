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
    "limiter": 40.0,          # E, rho, T read; D and kappa rho written (power-law opacity)
    "prep": 36.0,             # D, E read; K64, K32, b written
    "split_df": 16.0,         # E read; its FP32 (hi, lo) pair written
    "df_setup": 48.0,         # E, b, K read; their FP32 (hi, lo) pairs written
    "df_finish": 16.0,        # x (hi, lo) read; E written
    "sumsq": 8.0,             # b read
    "resid64": 28.0,          # x, b, K read; r32 written (mixed) / 24 (fp64)
    "resid64x": 40.0,         # x, e32, b, K read; x + e, r32 written
    "resid32": 24.0,          # x, b (FP64), K32 read; r32 written (FP32 arithmetic)
    "resid_upd": 32.0,        # x, e32, K32, r32 read; x + e, r32 written (r - A e in FP32)
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
    "exchange": 48.0,         # rho, T, E, kappa rho read; T, E written
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# FP64 operations per cell of the FP64-bound level-0 kernels, counted in their source for
# an interior cell of the 3D workload (add, multiply = 1 flop, FMA = 2; the FP32 seeds and
# the integer format conversions are not counted): the FP64 limiter with the Kramers
# opacity (15 for kappa, 23 for the gradient, 29 for D from one square root and one
# division), the FP64 exchange given kappa rho (FP32 Newton seed, one FP64 Newton step,
# E'), the FP64 refinement residual with each face flux evaluated once (3D levels), and
# the same with the correction x + e added in it.
FP64_FLOPS_PER_CELL = {
    "limiter": 67.0,
    "exchange": 29.0,
    "resid64": 21.0,
    "resid64x": 22.0,
}


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


def host_cores():
    """CPU cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample_step(n=40, steps=1):
    """The Python oracle on a bounded sample of the workload: the same recipe at n^3."""
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


def cpu_oracle_step(P, threads, method="vcycle", steps=1):
    """The C oracle's substep (oracle/cfld.c: limiter, V-cycle or Jacobi-PCG solve to
    1e-10, exchange; FP64) on the problem P with `threads` OpenMP threads, `steps` times
    from the same fields. Returns (cell-updates/s, seconds, iterations of the last)."""
    from oracle import cfld as CF
    CF.threads(threads)
    it = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        _, _, _, it = CF.step(P.rho, P.T, P.E, P.h, P.bc, P.E_bc, P.dt, P.c, P.a_r, P.gamma,
                              P.R_gas, P.opacity, method=method, tol=1e-10)
    secs = time.perf_counter() - t0
    return P.ncells * steps / secs, secs, it


def cpu_baseline(n=256):
    """The oracle timed on the host cores: the C substep on the benchmark's own workload
    (n^3) with every core, and beside it the same at (n/2)^3 single-threaded, Jacobi-PCG in
    place of the V-cycle, and the Python oracle (numpy/scipy) at 64^3."""
    from paper_2503_02764_gb300 import inputs as I
    cores = host_cores()
    P = I.stratified_3d(n)
    v, secs, it = cpu_oracle_step(P, cores)
    Ph = I.stratified_3d(n // 2)
    v1, s1, it1 = cpu_oracle_step(Ph, 1)
    vp, sp, itp = cpu_oracle_step(Ph, cores, "pcg")
    vpy, spy, cells_py, _ = cpu_sample_step(64, 1)
    # the other configurations: the 1D pulse and the 2D log-normal field on all cores and
    # on one, and a 256^3 sample of the 512^3 linear mode on all cores
    configs = {}
    for name, Pc, single in (("pulse1d_256", I.make_config(1), True),
                             ("lognormal2d_1024", I.make_config(2), True),
                             ("linmode3d_512_sample_256", I.linear_mode_3d(256, 1.0, steps=1),
                              False)):
        va, sa, ia = cpu_oracle_step(Pc, cores, steps=20 if Pc.ncells < 4096 else 1)
        configs[name] = {"all_cores": va, "seconds": sa, "cycles": ia, "cells": Pc.ncells}
        if single:
            configs[name]["single_thread"] = cpu_oracle_step(
                Pc, 1, steps=20 if Pc.ncells < 4096 else 1)[0]
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one C-oracle substep (oracle/cfld.c, FP64: limiter, V(2,2) multigrid "
                      "to 1e-10 in %d cycles, exchange) of the stratified recipe at %d^3 = %d "
                      "cells from its initial fields, %d OpenMP threads, %.2f s"
                      % (it, n, P.ncells, cores, secs),
            "single_thread": {"value": v1, "cells": Ph.ncells, "seconds": s1, "cycles": it1,
                              "sample": "the same at %d^3, 1 thread" % (n // 2)},
            "pcg_all_cores": {"value": vp, "cells": Ph.ncells, "seconds": sp, "iterations": itp,
                              "sample": "Jacobi-PCG to 1e-10 in place of the V-cycle, %d^3, "
                                        "%d threads" % (n // 2, cores)},
            "python_oracle": {"value": vpy, "cells": cells_py, "seconds": spy,
                              "sample": "oracle/fld.py (numpy/scipy, PCG, long-double "
                                        "exchange) at 64^3, one core"},
            "configs": configs}


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
    waves = {}
    for n_cells, nw in ((280, 7), (3200, 40)):
        wp = I.wave1d(I.WAVE_BACKGROUNDS["strong"], n_cells, nw, "fast")
        W = np.repeat(np.asarray(wp.W0, dtype=float)[:, None], wp.n, axis=1)
        U = np.stack([W[0], W[0] * W[1], W[0] * W[2], W[0] * W[3], W[4], W[5],
                      W[6] / (wp.gamma - 1.0) + 0.5 * (wp.Bx ** 2 + W[4] ** 2 + W[5] ** 2),
                      W[7]])
        for scheme, sname in ((1, "ars3"), (0, "split")):
            wv = fld.Wave1D(wp, scheme=scheme, precision=fld.PREC_FP64, tol=1e-13,
                            max_cycles=200)
            Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
            state = {"t": 0.0}

            def wave_step():
                dt = wv.max_dt(Ud, 0.8)
                wv.step(Ud, state["t"], dt)
                state["t"] += dt

            ms = timed(wave_step, reps=50, warm=5)
            waves["%s_%d" % (sname, n_cells)] = {"cells": wp.n, "ms_per_step": ms,
                                                 "cell_updates_per_s": wp.n / (ms * 1e-3)}
            wv.close()
    waves["note"] = ("launch- and synchronisation-bound: per step three explicit evaluations "
                     "of a few launches each and one (split) or two (ARS3) substeps with the "
                     "direct 1D solve and their read-backs")
    out["wave1d"] = waves
    return out


def workload_name(n):
    return ("stratified3d_%d^3 (x,y periodic, z Dirichlet, Kramers opacity, "
            "dt = 10x explicit limit)" % n)


def run_reference(args):
    """The comparison arm: the C oracle's substep on all host cores, each step a bounded
    sample of the workload (the same recipe at 128^3, from its initial fields)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2503_02764_gb300 import inputs as I
    n = 128
    cores = host_cores()
    P = I.stratified_3d(n)
    cpu_oracle_step(P, cores, steps=args.warmup)
    v, secs, it = cpu_oracle_step(P, cores, steps=args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.n), "cells": args.n ** 3,
                       "precision": "f64 (oracle)", "tol": 1e-10,
                       "sample": "each step one C-oracle substep of the same recipe at %d^3"
                                 % n},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d C-oracle substeps (oracle/cfld.c: limiter, V(2,2) "
                                       "multigrid to 1e-10 in %d cycles, exchange) of the "
                                       "stratified recipe at %d^3, %d OpenMP threads"
                                       % (args.steps, it, n, cores)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


DTYPE = {
    "mixed": "f32 V-cycles (smoothing, restriction, prolongation) inside f64 iterative "
             "refinement (f64 corrections x + e; the first correction from the f32 residual "
             "of E^n, the residual after it in f64, later ones updated as r - A e in f32 with "
             "a rigorous rounding bound added to the reported residual); f64 coarsest "
             "solve; f64 limiter; f64 exchange (f32 Newton seed, f64 Newton polish)",
    "mixed_fp64res": "as mixed, with every refinement residual after the first correction "
                     "formed in f64 (b - A x)",
    "mixed_df": "f32 V-cycles inside double-f32 (48-bit) iterative refinement; f64 coarsest "
                "solve; double-f32 limiter and exchange polish (f64 for cells outside the f32 "
                "exponent window)",
    "fp64": "f64 V-cycles; f64 coarsest solve; f64 limiter; f64 exchange (f32 Newton seed, "
            "f64 Newton polish)",
    "mixed_dflim": "as mixed (f32 V-cycles inside f64 iterative refinement, f64 coarsest solve, "
                   "f64 exchange), with the double-f32 (48-bit) limiter: gradient from f32 "
                   "pairs of E, R, lambda, D",
}
BATCH_DTYPE = {
    "mixed": "f32 V-cycles inside f64 iterative refinement (f64 residuals and corrections); "
             "f64 coarsest solve; f64 limiter; f64 exchange (f32 Newton seed, f64 Newton polish)",
    "mixed_df": "f32 V-cycles inside double-f32 (48-bit) iterative refinement; f64 coarsest "
                "solve; double-f32 limiter and exchange polish (f64 for cells outside the f32 "
                "exponent window)",
}
PREC = {"mixed_df": 2, "mixed": 1, "fp64": 0}

# FP64 peak of the GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA per SM per
# clock x 2 flop x the maximum SM clock (1.26 TFLOP/s at 2070 MHz)
def fp64_peak_tflops():
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return 152 * 2 * 2 * mhz * 1e6 / 1e12


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
    seed = I.SEED_BASE + 4 + 100000 * rank
    res = batch_workload(fld, I, torch, args.nprob, seed, args.steps, args.warmup, args.block,
                         args.cluster, dist=dist, local=local,
                         precision=args.precision if args.precision != "fp64" else "mixed")
    ms, cells_all, value = aggregate(res["ms_per_step"] * args.steps, res["cells"], args.steps,
                                     dist, "cuda")
    line = {"metric": METRIC + " [batched]", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": res["dtype"], "data": "synthetic",
            "config": {"workload": res["workload"], "cells": res["cells"],
                       "precision": res["precision"],
                       "block": res["options"]["block"], "cluster": res["options"]["cluster"],
                       "nu1": res["options"]["nu1"], "nu2": res["options"]["nu2"],
                       "inner": res["options"]["inner"], "autotuned": res["autotuned"]},
            "max_cycles_per_step": res["max_cycles_per_step"], "clocks": res["clocks"],
            "gpu_launches": res["gpu_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def batch_workload(fld, I, torch, nprob, seed, steps, warmup, block=0, cluster=0, dist=None,
                   local=0, precision="mixed"):
    """Time `steps` batched substeps (after `warmup`) of the nprob-member batch in the given
    precision mode (mixed: FP64 refinement, limiter and exchange; mixed_df: double-FP32)."""
    ps = I.batch(nprob, seed_base=seed)
    from paper_2503_02764_gb300 import autotune
    tuned = autotune.batch_options(ps, PREC[precision])
    kw = dict(block=block, cluster=cluster, nu1=2, nu2=2, inner=1)
    if tuned and not (block or cluster):
        kw = tuned
    b = fld.Batch([(p.shape, p.h, p.bc) for p in ps], tol=1e-10, max_cycles=50, graph=1,
                  precision=PREC[precision], **kw)
    cat = lambda xs: torch.from_numpy(np.concatenate([x.ravel() for x in xs])).cuda()
    rho, T, E = cat([p.rho for p in ps]), cat([p.T for p in ps]), cat([p.E for p in ps])
    consts = fld.make_consts(1.0, 1.0, 5.0 / 3.0, 1.0)
    ops = [fld.make_opacity(p.opacity) for p in ps]
    dts = [p.dt for p in ps]
    for _ in range(warmup):
        b.step(consts, ops, dts, rho, T, E)
    stream = torch.cuda.current_stream()
    n0 = fld.fld_launch_count()
    clk = Clocks(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    cyc = []
    for _ in range(steps):
        rc, st = b.step(consts, ops, dts, rho, T, E)
        cyc.append(max(x["cycles"] for x in st))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    cells = b.cells
    b.close()
    return {"workload": "batch of %d 2D problems, sides U{32..512}, one persistent launch per "
                        "step, CUDA graph" % nprob,
            "cells": cells, "ms_per_step": ms / steps, "cell_updates_per_s": cells * steps / (ms * 1e-3),
            "options": {"block": kw["block"] or 512, "cluster": kw["cluster"] or "auto",
                        "nu1": kw["nu1"], "nu2": kw["nu2"], "inner": kw.get("inner", 1)},
            "autotuned": bool(tuned and not (block or cluster)),
            "max_cycles_per_step": cyc, "clocks": clocks, "precision": precision,
            "dtype": BATCH_DTYPE[precision], "gpu_launches": fld.fld_launch_count() - n0}


def step_series(hd, consts, op, P, rho, T, E, ebc, steps, warmup, torch):
    """Event-timed `steps` substeps after `warmup` ones on the caller's stream (the fields
    evolve in place); returns (ms per step, cycles per step, last status)."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        hd.step(consts, op, P.dt, rho, T, E, ebc, raise_on_error=False)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    cyc, st = [], None
    for _ in range(steps):
        st = hd.step(consts, op, P.dt, rho, T, E, ebc, raise_on_error=False)
        cyc.append(st["cycles"])
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps, cyc, st


def profile_steps(hd, consts, op, P, rho, T, E, ebc, steps, torch, peak_hbm, prec):
    """The same steps with every launch bracketed by events: per-kernel breakdown, the
    whole step's algorithmic bytes, the dominant level-0 kernel's roofline."""
    hd.prof_enable(True, 65536)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(steps):
        hd.step(consts, op, P.dt, rho, T, E, ebc, raise_on_error=False)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_prof = e2.elapsed_time(e3)
    prof = hd.prof_read()
    hd.prof_enable(False)

    def bpc(e):
        b = BYTES_PER_CELL.get(e["name"])
        if e["name"] == "resid64" and prec == 0:
            b = 24.0
        return b

    total_ms = sum(e["ms"] for e in prof)
    alg_bytes = sum(bpc(e) * e["cells"] for e in prof if bpc(e) is not None)
    lvl0 = [e for e in prof if e["level"] == 0 and bpc(e) is not None]
    dom = max(lvl0, key=lambda e: e["ms"]) if lvl0 else None
    kernels = []
    for e in sorted(prof, key=lambda e: -e["ms"])[:14]:
        k = {"kernel": e["name"], "level": e["level"], "launches": e["launches"],
             "ms": round(e["ms"], 4), "share": round(e["ms"] / total_ms, 4),
             "avg_launch_us": round(1e3 * e["ms"] / e["launches"], 2)}
        if bpc(e) is not None:
            gbs = bpc(e) * e["cells"] / (e["ms"] * 1e-3) / 1e9
            k.update(bytes_per_cell=bpc(e), achieved_GBs=round(gbs, 1),
                     frac_hbm=round(gbs / peak_hbm, 4))
        kernels.append(k)
    def hbm_roof(e):
        b = bpc(e)
        achieved = b * e["cells"] / (e["ms"] * 1e-3) / 1e9
        return {"kernel": e["name"], "bound": "hbm", "achieved": achieved, "peak": peak_hbm,
                "unit": "GB/s", "frac": achieved / peak_hbm,
                "traffic": ncu_traffic(e["name"], e["cells"] / e["launches"]),
                "peak_source": "measured", "launches": e["launches"],
                "avg_launch_us": 1e3 * e["ms"] / e["launches"], "bytes_per_cell": b}

    fp64_bound = lambda e: (e["name"] in FP64_FLOPS_PER_CELL and
                            not (prec == 2 and e["name"] in ("limiter", "exchange")))
    roof = None
    if dom and fp64_bound(dom):
        # an FP64-bound kernel: its FP64 flops against the FP64 peak
        f = FP64_FLOPS_PER_CELL[dom["name"]]
        pk = fp64_peak_tflops()
        achieved = f * dom["cells"] / (dom["ms"] * 1e-3) / 1e12
        roof = {"kernel": dom["name"], "bound": "alu", "achieved": achieved, "peak": pk,
                "unit": "TFLOP/s", "frac": achieved / pk,
                "traffic": ncu_traffic(dom["name"], dom["cells"] / dom["launches"]),
                "peak_source": "FP64 unit counts and clock: 152 SMs x 2 FMA/clk x 2 flop x "
                               "max SM clock", "launches": dom["launches"],
                "avg_launch_us": 1e3 * dom["ms"] / dom["launches"],
                "fp64_flops_per_cell": f}
    elif dom:
        roof = hbm_roof(dom)
    hb = [e for e in lvl0 if not fp64_bound(e)]
    roof_hbm = hbm_roof(max(hb, key=lambda e: e["ms"])) if hb else None
    whole = {"algorithmic_bytes_per_cell": alg_bytes / steps / P.ncells,
             "achieved_GBs": alg_bytes / (ms_prof * 1e-3) / 1e9,
             "frac_hbm": alg_bytes / (ms_prof * 1e-3) / 1e9 / peak_hbm}
    return prof, ms_prof / steps, kernels, roof, whole, roof_hbm


def fp64_kernels(prof, peak_tflops, prec):
    """The FP64-bound level-0 kernels against the FP64 peak: their FP64 operations per
    cell (FMA = 2 flops) counted from the kernels' source, times the cells, over the
    event-timed duration. In MIXED_DF mode the limiter and exchange are double-FP32
    kernels and are not listed."""
    out = {}
    for e in prof:
        f = FP64_FLOPS_PER_CELL.get(e["name"])
        if f is None or e["level"] != 0:
            continue
        if prec == 2 and e["name"] in ("limiter", "exchange"):
            continue
        tf = f * e["cells"] / (e["ms"] * 1e-3) / 1e12
        out[e["name"]] = {"fp64_flops_per_cell": f, "achieved_TFLOPs": round(tf, 4),
                          "peak_TFLOPs": round(peak_tflops, 4), "frac": round(tf / peak_tflops, 4),
                          "avg_launch_us": round(1e3 * e["ms"] / e["launches"], 2)}
    return out


def config_workloads(fld, I, torch, peak_hbm, nprob=512, big=512):
    """The other workloads of the metric, each with its own precision, bounded in time:
    the 1D pulse (FP64, tol 1e-12), the 2D log-normal field at 1024^2 (FP64, 10 steps, tol
    1e-10), the 512-member batch (one launch per step) and the linear mode at big^3 (mixed,
    100 steps) for both radiation-to-gas pressure ratios, with its decay against the exact
    per-step amplification and the roofline of its dominant kernel at that size."""
    out = {}
    consts_of = lambda P: fld.make_consts(P.c, P.a_r, P.gamma, P.R_gas)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    # 1: pulse1d, FP64 plain method, one step + exchange, tol 1e-12: the direct 1D solve
    # (parallel cyclic reduction) and FP64 V-cycles
    P = I.gaussian_pulse_1d(256)
    res = {"cells": P.ncells, "precision": "fp64", "tol": 1e-12,
           "note": "256 cells: latency-bound (launches and read-backs), no HBM roofline"}
    for name, direct in (("direct", 1), ("vcycles", 0)):
        hd = fld.Handle(P.shape, P.h, P.bc, precision=fld.PREC_FP64, tol=1e-12, max_cycles=50,
                        direct1d=direct)
        first = hd.step(consts_of(P), fld.make_opacity(P.opacity), P.dt, dev(P.rho), dev(P.T),
                        dev(P.E), None, raise_on_error=False)
        rho, T, E = dev(P.rho), dev(P.T), dev(P.E)
        ms, cyc, st = step_series(hd, consts_of(P), fld.make_opacity(P.opacity), P, rho, T, E,
                                  None, 20, 3, torch)
        res[name] = {"first_step_cycles": first["cycles"], "ms_per_step": ms,
                     "cycles_per_step": cyc[-1], "rel_resid_last": st["rel_resid"],
                     "cell_updates_per_s": P.ncells / (ms * 1e-3)}
        hd.close()
    out["pulse1d_256"] = res
    # 2: lognormal2d 1024^2, FP64 plain GMG, 10 implicit steps, tol 1e-10
    P = I.lognormal_2d(1024)
    for name, prec in (("fp64", fld.PREC_FP64), ("mixed", fld.PREC_MIXED)):
        hd = fld.Handle(P.shape, P.h, P.bc, precision=prec, tol=1e-10, max_cycles=50)
        rho, T, E = dev(P.rho), dev(P.T), dev(P.E)
        hd.step(consts_of(P), fld.make_opacity(P.opacity), P.dt, dev(P.rho), dev(P.T),
                dev(P.E), None, raise_on_error=False)          # warm-up on a copy
        ms, cyc, st = step_series(hd, consts_of(P), fld.make_opacity(P.opacity), P, rho, T, E,
                                  None, 10, 0, torch)
        _, msp, _, _, whole, _ = profile_steps(hd, consts_of(P), fld.make_opacity(P.opacity), P,
                                               dev(P.rho), dev(P.T), dev(P.E), None, 2, torch,
                                               peak_hbm, prec)
        out.setdefault("lognormal2d_1024", {"cells": P.ncells, "steps": 10, "tol": 1e-10,
                                            "note": "8 MB per field: L2-resident, so the "
                                                    "whole-step fraction is of HBM peak but "
                                                    "the traffic is largely L2"})
        out["lognormal2d_1024"][name] = {"ms_per_step": ms, "cycles_per_step": cyc,
                                         "cell_updates_per_s": P.ncells / (ms * 1e-3),
                                         "whole_step": whole}
        hd.close()
    # 4: the 512-member batch, one launch per step
    out["batch_%d" % nprob] = batch_workload(fld, I, torch, nprob, I.SEED_BASE + 4, 5, 2)
    out["batch_%d" % nprob]["mixed_df"] = {
        k: v for k, v in batch_workload(fld, I, torch, nprob, I.SEED_BASE + 4, 5, 2,
                                        precision="mixed_df").items()
        if k in ("ms_per_step", "cell_updates_per_s", "max_cycles_per_step", "dtype")}
    # 5: linear mode at big^3, mixed, 100 steps, for both pressure ratios, seeded with the
    # fast magnetosonic eigenmode (B at 45 degrees to k); the complex amplitudes of the
    # k = 2 pi mode before and after are reported (the GPU tests compare them with the
    # exact per-step amplification and the dispersion relation)
    res = {}
    for ratio in (0.1, 1.0):
        P = I.linear_mode_3d(big, ratio=ratio, amp=1e-4, steps=100)
        opts = dict(nu1=2, nu2=2, smoother=2, inner=2)
        hd = fld.Handle(P.shape, P.h, P.bc, precision=fld.PREC_MIXED, tol=1e-12, max_cycles=60,
                        **opts)
        rho, T, E = dev(P.rho), dev(P.T), dev(P.E)
        ph = np.exp(-2j * np.pi * (np.arange(big) + 0.5) / big)

        def modes(Tf, Ef):
            e = (P.R_gas * Tf / (P.gamma - 1)).reshape(P.shape).mean(axis=(0, 1))
            Em = Ef.reshape(P.shape).mean(axis=(0, 1))
            return np.array([2.0 / big * np.sum(e * ph), 2.0 / big * np.sum(Em * ph)])

        v0 = modes(P.T, P.E)
        ms, cyc, st = step_series(hd, consts_of(P), fld.make_opacity(P.opacity), P, rho, T, E,
                                  None, 100, 0, torch)
        got = modes(T.cpu().numpy(), E.cpu().numpy())
        r = {"cells": P.ncells, "steps": 100, "precision": "mixed", "tol": 1e-12,
             "seed": "fast magnetosonic eigenmode, amplitude 1e-4", "options": opts,
             "ms_per_step": ms, "cycles_last_step": cyc[-1],
             "cell_updates_per_s": P.ncells / (ms * 1e-3),
             "E1_before": [v0[1].real, v0[1].imag], "E1_after_100": [got[1].real, got[1].imag],
             "e1_before": [v0[0].real, v0[0].imag], "e1_after_100": [got[0].real, got[0].imag],
             "E1_decay_per_step": float((abs(got[1]) / abs(v0[1])) ** 0.01)}
        if ratio == 1.0:
            _, msp, kern, roof, whole, roof_h = profile_steps(
                hd, consts_of(P), fld.make_opacity(P.opacity), P, rho, T, E, None, 2, torch,
                peak_hbm, fld.PREC_MIXED)
            r["roofline"] = roof
            r["roofline_hbm_kernel"] = roof_h
            r["whole_step"] = whole
            r["kernels"] = kern[:6]
        res["Pr/Pg=%g" % ratio] = r
        hd.close()
        del rho, T, E
        torch.cuda.empty_cache()
    out["linmode3d_%d" % big] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_df", "fp64"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the timings of the widening rows (coupling, limiters, tabulated "
                         "opacity, 1D wave step)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the substep in the other two precision modes")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads (1D pulse, 2D log-normal, batch, 512^3 mode)")
    ap.add_argument("--smoother", type=int, default=-1,
                    help="-1 the tuned choice (else 0); 0 in-place half sweeps, 1 out-of-place "
                         "half sweeps, 2 single-pass z-marching sweep")
    ap.add_argument("--nu1", type=int, default=-1, help="pre-smoothing sweeps (-1: tuned)")
    ap.add_argument("--nu2", type=int, default=-1, help="post-smoothing sweeps (-1: tuned)")
    ap.add_argument("--prolong", type=int, default=-1,
                    help="prolongation: -1 the tuned choice (else linear); 0 linear, 1 constant")
    ap.add_argument("--truncate", type=int, default=-1,
                    help="V-cycle depth from the operator: 1 on (the default), 0 full depth")
    ap.add_argument("--inner", type=int, default=-1,
                    help="FP32 V-cycles per refinement step (-1: tuned)")
    ap.add_argument("--no-ttt", action="store_true", help="skip the mixed-vs-FP64 solve timing")
    ap.add_argument("--workload", default="stratified", choices=["stratified", "batch"],
                    help="stratified: one 3D box (default); batch: 512 uneven 2D problems")
    ap.add_argument("--nprob", type=int, default=512)
    ap.add_argument("--big", type=int, default=512, help="side of the linear-mode workload")
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

    from paper_2503_02764_gb300 import autotune, build, fld
    from paper_2503_02764_gb300 import inputs as I
    if rank == 0:
        build.build()
    barrier()

    P = I.stratified_3d(args.n)
    prec = PREC[args.precision]

    def options(pr):
        o, t = autotune.grid_options(P, pr)
        for k in ("smoother", "nu1", "nu2", "inner", "prolong", "truncate"):   # explicit choices override the tuner
            if getattr(args, k) >= 0:
                o[k] = getattr(args, k)
                t = False
        return o, t

    gkw, tuned = options(prec)
    hd = fld.Handle(P.shape, P.h, P.bc, precision=prec, tol=1e-10, max_cycles=50, **gkw)
    consts = fld.make_consts(P.c, P.a_r, P.gamma, P.R_gas)
    op = fld.make_opacity(P.opacity)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rho, T, E = dev(P.rho), dev(P.T), dev(P.E)
    ebc = dev(I.pack_dirichlet(P.shape, P.bc, P.E_bc))
    stream = torch.cuda.current_stream()

    # the first substep from the recipe's fields (graphs captured on a copy beforehand)
    hd.step(consts, op, P.dt, rho.clone(), T.clone(), E.clone(), ebc)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    st_first = hd.step(consts, op, P.dt, rho, T, E, ebc)
    f1.record(stream)
    torch.cuda.synchronize()
    first = {"ms": f0.elapsed_time(f1), "cycles": st_first["cycles"],
             "rel_resid": st_first["rel_resid"]}
    for _ in range(max(args.warmup - 1, 0)):
        hd.step(consts, op, P.dt, rho, T, E, ebc)
    T_start, E_start = T.clone(), E.clone()          # the state the timed steps start from

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
    peak_hbm, peak_kind = load_peaks()
    Tp, Ep = T_start.clone(), E_start.clone()
    prof, ms_prof, kernels, roof, whole, roof_hbm = profile_steps(
        hd, consts, op, P, rho, Tp, Ep, ebc, args.steps, torch, peak_hbm, prec)
    for r in (roof, roof_hbm):
        if r and r["bound"] == "hbm":
            r["peak_source"] = peak_kind
    del Tp, Ep
    fp64 = fp64_kernels(prof, fp64_peak_tflops(), prec)

    # ---------------- end to end through the C ABI with host buffers. Every step copies its
    # inputs (rho, T, E, the Dirichlet face values) from pinned host memory and reads its
    # results (T, E) back. The inputs are the state the device-resident steps started
    # from, so that these steps do the same solve work as those. Serial: copy in, step,
    # copy out, on one stream.
    # Pipelined (the reported value): three device buffer sets; while step k computes, step
    # k+1's inputs go up on one copy stream and step k-1's results come down on another (the
    # two directions overlap each other too), each transfer ordered by events.
    e2e = None
    if not args.no_e2e:
        h_in = tuple(x.detach().cpu().pin_memory() for x in (rho, T_start, E_start, ebc))
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
        del d_in, h_out, h_in

    # ---------------- the whole substep in the other two precision modes, each with its own
    # tuned options, from the same state (rank 0)
    variants = {}
    if rank == 0 and not args.no_variants:
        for name in ("mixed_df", "fp64", "mixed", "mixed_dflim", "mixed_fp64res"):
            if name == args.precision:
                continue
            base = "mixed" if name in ("mixed_dflim", "mixed_fp64res") else name
            o, t = options(PREC[base])
            o = dict(o, limiter_df=1) if name == "mixed_dflim" else o
            o = dict(o, resid_update=0) if name == "mixed_fp64res" else o
            hv = fld.Handle(P.shape, P.h, P.bc, precision=PREC[base], tol=1e-10, max_cycles=50, **o)
            Tv, Ev = T_start.clone(), E_start.clone()
            nst = max(5, args.steps // 4) if name == "fp64" else args.steps
            msv, cyc, stv = step_series(hv, consts, op, P, rho, Tv, Ev, ebc, nst, 2, torch)
            variants[name] = {"ms_per_step": msv, "cell_updates_per_s": P.ncells / (msv * 1e-3),
                              "steps": nst, "cycles_per_step": cyc[-1], "options": o,
                              "autotuned": t, "dtype": DTYPE[name],
                              "rel_resid_last": stv["rel_resid"]}
            hv.close()
            del Tv, Ev

    # ---------------- mixed vs FP64 time to 1e-10 on the same GPU (diffusion solve alone)
    ttt = {}
    if rank == 0 and not args.no_ttt:
        D = torch.empty_like(E)
        hd.limiter(consts, op, E_start, rho, T_start, ebc, D)
        for name, pr, extra in (("mixed_df", fld.PREC_MIXED_DF, {}), ("mixed", fld.PREC_MIXED, {}),
                                ("mixed_fp64res", fld.PREC_MIXED, {"resid_update": 0}),
                                ("fp64", fld.PREC_FP64, {})):
            o, _ = options(pr)
            o = dict(o, **extra)
            hd.set_opts(precision=pr, tol=1e-10, max_cycles=50, **o)
            times, cyc = [], 0
            for rep in range(4):
                X = E_start.clone()
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                st = hd.diffuse(P.dt, D, ebc, X)
                b.record(stream)
                torch.cuda.synchronize()
                if rep:
                    times.append(a.elapsed_time(b))
                cyc = st["cycles"]
            ttt[name] = {"ms": float(np.median(times)), "cycles": cyc, "options": o}
        hd.set_opts(precision=prec, tol=1e-10, max_cycles=50, **gkw)
        del D, X

    # ---------------- the widening rows, timed on the same workload (rank 0)
    rows = None
    if rank == 0 and not args.no_next:
        try:
            rows = next_rows(hd, P, prec, gkw, consts, op, rho, T, E, ebc, peak_hbm)
        except Exception as exc:                 # reported, never fatal to the headline
            rows = {"error": "%s: %s" % (type(exc).__name__, exc)}
    hd.close()
    del rho, T, E, T_start, E_start
    torch.cuda.empty_cache()

    # ---------------- the metric's other workloads (rank 0), each bounded in time
    configs = None
    if rank == 0 and world == 1 and not args.no_configs:
        try:
            configs = config_workloads(fld, I, torch, peak_hbm, args.nprob, args.big)
        except Exception as exc:                 # reported, never fatal to the headline
            configs = {"error": "%s: %s" % (type(exc).__name__, exc)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
            "data": "synthetic",
            "config": {"workload": workload_name(args.n),
                       "cells": P.ncells, "precision": args.precision, "tol": 1e-10,
                       "nu1": gkw["nu1"], "nu2": gkw["nu2"], "smoother": gkw["smoother"],
                       "inner": gkw.get("inner", 1), "prolong": gkw.get("prolong", 0), "graph": 1,
                       "autotuned": bool(tuned),
                       "l2": "inputs larger than L2 (fields %.0f MB + workspace)" %
                             (3 * P.ncells * 8 / 1e6),
                       "parallelism": "replicas x%d" % world},
            "gpu_launches": launches, "cycles_per_step": cycles,
            "first_step_from_recipe": first,
            "profiled_pass_ms_per_step": ms_prof,
            "roofline": roof, "roofline_hbm_kernel": roof_hbm, "whole_step": whole,
            "fp64_kernels": fp64,
            "kernel_breakdown": kernels,
            "precision_variants": variants,
            "time_to_1e-10_ms": ttt, "clocks": clocks, "e2e": e2e}
    if configs is not None:
        line["workloads"] = configs
    if rows is not None:
        line["next_rows"] = rows
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
