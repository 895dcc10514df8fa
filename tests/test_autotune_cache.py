"""The autotuner's cache on the host: workload signatures, storing and reading entries
per GPU name, and a damaged cache file read as empty (no GPU needed)."""
import json
import os

from paper_2503_02764_gb300 import autotune as A
from paper_2503_02764_gb300 import build
from paper_2503_02764_gb300 import inputs as I


def _cache(monkeypatch, name):
    os.makedirs(build.BUILD, exist_ok=True)
    path = os.path.join(build.BUILD, name)
    if os.path.exists(path):
        os.remove(path)
    monkeypatch.setenv("FLD_TUNE_CACHE", path)
    return path


def test_signature_depends_on_shapes_and_boundaries_only():
    a = I.lognormal_2d(32, seed=1, ny=24, steps=1)
    b = I.lognormal_2d(32, seed=2, ny=24, steps=1)         # other values, same shape
    c = I.lognormal_2d(32, seed=1, ny=26, steps=1)         # other shape
    assert A.signature("grid", [a]) == A.signature("grid", [b])
    assert A.signature("grid", [a]) != A.signature("grid", [c])
    assert A.signature("grid", [a]) != A.signature("batch", [a])
    assert A.signature("batch", [a, c]) != A.signature("batch", [c, a])
    assert A.signature("batch", [a, c]).startswith("batch:2:")


def test_store_and_read_back_per_gpu(monkeypatch):
    path = _cache(monkeypatch, "tune_cache_test.json")
    assert A.cached("grid", "grid:1:abc", gpu="GPU-A") is None
    A._store("grid:1:abc", {"best": {"nu1": 1}}, "GPU-A")
    A._store("grid:1:abc", {"best": {"nu1": 2}}, "GPU-B")
    A._store("batch:3:def", {"best": {"block": 512}}, "GPU-A")
    assert A.cached("grid", "grid:1:abc", gpu="GPU-A")["best"]["nu1"] == 1
    assert A.cached("grid", "grid:1:abc", gpu="GPU-B")["best"]["nu1"] == 2
    assert A.cached("batch", "batch:3:def", gpu="GPU-A")["best"]["block"] == 512
    assert A.cached("batch", "batch:3:def", gpu="GPU-B") is None
    d = json.load(open(path))
    assert set(d) == {"GPU-A", "GPU-B"}
    os.remove(path)


def test_damaged_cache_reads_as_empty(monkeypatch):
    path = _cache(monkeypatch, "tune_cache_damaged.json")
    with open(path, "w") as f:
        f.write("{not json")
    assert A.cached("grid", "grid:1:abc", gpu="GPU-A") is None
    A._store("grid:1:abc", {"best": {"nu1": 3}}, "GPU-A")     # rewritten whole
    assert A.cached("grid", "grid:1:abc", gpu="GPU-A")["best"]["nu1"] == 3
    os.remove(path)


def test_committed_cache_entries_are_well_formed():
    d = json.load(open(A.DEFAULT_CACHE))
    for gpu, entries in d.items():
        for sig, e in entries.items():
            kind = sig.split(":")[0].split("-")[0]
            assert kind in ("grid", "batch"), sig
            if "-" in sig.split(":")[0]:
                assert sig.split(":")[0].split("-")[1] in A.PRECISION_NAMES.values(), sig
            best = e["best"]
            assert best["converged"] is True
            assert best["nu1"] + best["nu2"] >= 1
            if kind == "batch":
                assert best["block"] in (256, 512, 1024) and best["cluster"] in (1, 2, 4, 8)
            else:
                assert best["smoother"] in (0, 1, 2) and best["inner"] >= 1


def test_grid_options_prefer_the_precision_entry(monkeypatch):
    # the benchmark and the parity tests of the timed configuration read the options
    # through grid_options: the entry tuned for the precision mode wins, the entry cached
    # without a precision is the fallback, the defaults come last
    _cache(monkeypatch, "tune_cache_prec.json")
    P = I.stratified_3d(16, nz=12, ny=10)
    assert A.signature("grid", [P], 1) != A.signature("grid", [P], 2)
    assert A.signature("grid", [P], 1).startswith("grid-mixed:1:")
    assert A.grid_options(P, 1, gpu="GPU-A") == (A.DEFAULT_GRID, False)
    A._store(A.signature("grid", [P]), {"best": {"nu1": 1, "nu2": 1, "smoother": 2,
                                                 "inner": 3}}, "GPU-A")
    opts, tuned = A.grid_options(P, 1, gpu="GPU-A")
    assert tuned and opts == {"nu1": 1, "nu2": 1, "smoother": 2, "inner": 3, "prolong": 0}
    A._store(A.signature("grid", [P], 1), {"best": {"nu1": 2, "nu2": 1, "smoother": 0,
                                                    "inner": 2, "prolong": 1}}, "GPU-A")
    assert A.grid_options(P, 1, gpu="GPU-A")[0] == {"nu1": 2, "nu2": 1, "smoother": 0,
                                                   "inner": 2, "prolong": 1}
    assert A.grid_options(P, 2, gpu="GPU-A")[0]["inner"] == 3
    assert A.batch_options([P], gpu="GPU-A") is None
