"""Helpers shared by the GPU parity tests: move a seeded Problem to the device, run
the C-ABI path, and compare with the oracle."""
import numpy as np
import pytest

from paper_2503_02764_gb300 import inputs as I


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def library():
    from paper_2503_02764_gb300 import build, fld
    build.build()
    fld.lib()
    return fld


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def handle_for(fld, P, **opts):
    return fld.Handle(P.shape, P.h, P.bc, **opts)


def consts_of(fld, P):
    return fld.make_consts(P.c, P.a_r, P.gamma, P.R_gas)


def ebc_dev(torch, P):
    packed = I.pack_dirichlet(P.shape, P.bc, P.E_bc)
    return dev(torch, packed) if packed.size else None


def maxrel(a, b):
    """max-norm relative difference ||a - b||_inf / ||b||_inf"""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def pertrel(a, b):
    """perturbation-relative difference ||a - b||_inf / ||b - mean(b)||_inf"""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b - b.mean())), 1e-300))


def bench_grid_options(precision):
    """The options bench.py reads for its 256^3 stratified workload in this precision mode
    (only the shape and the boundary kinds enter the autotuner's cache key)."""
    from types import SimpleNamespace
    from paper_2503_02764_gb300 import autotune
    key = SimpleNamespace(shape=(256, 256, 256), bc=I.stratified_3d(16, nz=8, ny=8).bc)
    return autotune.grid_options(key, precision)[0]
