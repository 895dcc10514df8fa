"""Autotuner for the launch shapes and smoother sweep counts of the FLD solver.

For the batched substep it times (threads per block, blocks per problem cluster,
pre/post smoothing sweeps, FP32 V-cycles per refinement step); for a single grid
(pre/post sweeps, smoother kind, V-cycles per refinement step). Each
candidate runs the real substep on a copy of the caller's fields; a candidate counts
only if every problem reaches the tolerance. The fastest is cached in a JSON file keyed
by the GPU name and a signature of the workload (shapes, boundary kinds), so later runs
on the same GPU and workload pick it up without tuning.

Usage from Python::

    best = autotune.tune_batch(batch_problems)          # list of inputs.Problem
    best = autotune.tune_grid(problem)
    opts = autotune.cached("batch", signature, gpu)     # or None

The cache lives next to this file (tuned.json) unless FLD_TUNE_CACHE names another path.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "tuned.json")


def cache_path():
    return os.environ.get("FLD_TUNE_CACHE", DEFAULT_CACHE)


def gpu_name():
    import torch
    return torch.cuda.get_device_name(0)


PRECISION_NAMES = {0: "fp64", 1: "mixed", 2: "mixed_df"}

# options of a single grid when nothing is cached: V(2,2), in-place half sweeps, one FP32
# V-cycle per refinement step
DEFAULT_GRID = {"nu1": 2, "nu2": 2, "smoother": 0, "inner": 1}


def signature(kind, problems, precision=None):
    """Workload key: kind (with the precision mode when given) plus a hash of the shapes
    and boundary kinds."""
    h = hashlib.sha256()
    for p in problems:
        h.update(repr((p.shape, p.bc)).encode())
    key = kind if precision is None else "%s-%s" % (kind, PRECISION_NAMES[int(precision)])
    return "%s:%d:%s" % (key, len(problems), h.hexdigest()[:16])


def grid_options(problem, precision, gpu=None):
    """Options a single grid runs with in the benchmark: the cached best for this GPU,
    workload and precision mode (else the entry cached without a precision), else the
    defaults. Returns (options, tuned)."""
    try:
        c = (cached("grid", signature("grid", [problem], precision), gpu)
             or cached("grid", signature("grid", [problem]), gpu))
    except Exception:
        c = None
    if not c:
        return dict(DEFAULT_GRID), False
    b = c["best"]
    return {"nu1": b["nu1"], "nu2": b["nu2"], "smoother": b["smoother"],
            "inner": b.get("inner", 1), "prolong": b.get("prolong", 0)}, True


def batch_options(problems, precision=None, gpu=None):
    """Options of the batched substep in the benchmark: the cached best for this GPU, batch
    and precision mode (else the entry cached without a precision) as (block, cluster,
    nu1, nu2, inner), else None."""
    try:
        c = ((precision is not None and cached("batch", signature("batch", problems, precision),
                                                gpu))
             or cached("batch", signature("batch", problems), gpu))
    except Exception:
        c = None
    if not c:
        return None
    b = c["best"]
    return {"block": b["block"], "cluster": b["cluster"], "nu1": b["nu1"], "nu2": b["nu2"],
            "inner": b.get("inner", 1)}


def _load():
    p = cache_path()
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except (OSError, ValueError):
            return {}
    return {}


def cached(kind, sig, gpu=None):
    d = _load()
    return d.get(gpu or gpu_name(), {}).get(sig)


def _store(sig, entry, gpu):
    d = _load()
    d.setdefault(gpu, {})[sig] = entry
    with open(cache_path(), "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)


def _time_batch(fld, torch, problems, opts, reps=3):
    import numpy as np
    b = fld.Batch([(p.shape, p.h, p.bc) for p in problems], **opts)
    cat = lambda xs: torch.from_numpy(np.concatenate([x.ravel() for x in xs])).cuda()
    rho = cat([p.rho for p in problems])
    T0, E0 = cat([p.T for p in problems]), cat([p.E for p in problems])
    consts = fld.make_consts(problems[0].c, problems[0].a_r, problems[0].gamma, problems[0].R_gas)
    ops = [fld.make_opacity(p.opacity) for p in problems]
    dts = [p.dt for p in problems]
    best = float("inf")
    ok = True
    for _ in range(reps + 1):
        T, E = T0.clone(), E0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = b.step(consts, ops, dts, rho, T, E, raise_on_error=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ok = ok and rc == 0
        best = min(best, dt)
    b.close()
    return best, ok


def tune_batch(problems, blocks=(256, 512, 1024), clusters=(1, 2, 4, 8),
               sweeps=((2, 2), (1, 1), (2, 1), (3, 3)), inners=(1, 2), tol=1e-10, store=True,
               precision=None):
    """Time every (block, cluster, nu1, nu2, inner) candidate on the batch in the given
    precision mode (the library's default when None); return the best."""
    import torch
    from . import fld
    results = []
    for nb in blocks:
        for cl in clusters:
            for nu1, nu2 in sweeps:
                for inner in inners:
                    opts = dict(tol=tol, max_cycles=60, block=nb, cluster=cl, nu1=nu1, nu2=nu2,
                                inner=inner, graph=0)
                    if precision is not None:
                        opts["precision"] = int(precision)
                    try:
                        t, ok = _time_batch(fld, torch, problems, opts)
                    except fld.FldError:
                        continue
                    results.append({"block": nb, "cluster": cl, "nu1": nu1, "nu2": nu2,
                                    "inner": inner, "seconds": t, "converged": ok})
    good = [r for r in results if r["converged"]]
    best = min(good, key=lambda r: r["seconds"]) if good else None
    if store and best:
        gpu = gpu_name()
        _store(signature("batch", problems, precision), {"best": best, "candidates": results,
                                              "when": time.strftime("%Y-%m-%dT%H:%M:%SZ",
                                                                    time.gmtime())}, gpu)
    return best, results


def tune_grid(problem, precision=2, sweeps=((2, 2), (1, 1), (2, 1), (1, 2), (3, 3)),
              smoothers=(0, 2), inners=(1, 2, 3), tol=1e-10, store=True, reps=3, presteps=3):
    """Time (nu1, nu2, smoother, inner) for one grid's full substep; return the best.

    The fields are first advanced `presteps` substeps with the default options, so the
    candidates are timed on the state a running simulation meets after its first steps
    (the very first substep of the synthetic initial state needs more cycles)."""
    import numpy as np
    import torch
    from . import fld
    from . import inputs as I
    P = problem
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rho, T0, E0 = dev(P.rho), dev(P.T), dev(P.E)
    packed = I.pack_dirichlet(P.shape, P.bc, P.E_bc)
    ebc = dev(packed) if packed.size else None
    consts = fld.make_consts(P.c, P.a_r, P.gamma, P.R_gas)
    op = fld.make_opacity(P.opacity)
    results = []
    hd = fld.Handle(P.shape, P.h, P.bc, precision=precision, tol=tol)
    for _ in range(presteps):
        hd.step(consts, op, P.dt, rho, T0, E0, ebc)
    candidates = [(sm, inner, nu) for sm in smoothers for inner in inners for nu in sweeps]
    for sm, inner, (nu1, nu2) in candidates:
        hd.set_opts(precision=precision, tol=tol, max_cycles=60, nu1=nu1, nu2=nu2, smoother=sm,
                    inner=inner)
        best, ok = float("inf"), True
        for _ in range(reps + 1):
            T, E = T0.clone(), E0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = hd.step(consts, op, P.dt, rho, T, E, ebc, raise_on_error=False)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
            ok = ok and st["status"] == 0
        results.append({"nu1": nu1, "nu2": nu2, "smoother": sm, "inner": inner,
                        "seconds": best, "converged": ok, "cycles": st["cycles"]})
    hd.close()
    good = [r for r in results if r["converged"]]
    best = min(good, key=lambda r: r["seconds"]) if good else None
    if store and best:
        _store(signature("grid", [P], precision), {"best": best, "candidates": results,
                                        "when": time.strftime("%Y-%m-%dT%H:%M:%SZ",
                                                              time.gmtime())}, gpu_name())
    return best, results


if __name__ == "__main__":
    import sys
    from . import inputs as I
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("batch", "all"):
        best, _ = tune_batch(I.batch(512))
        print("batch", best)
    if what in ("grid", "all"):
        for prec in (1, 2, 0):
            best, _ = tune_grid(I.stratified_3d(256), precision=prec)
            print("grid", PRECISION_NAMES[prec], best)
