"""MIXED refinement with the recursive residual (r - A e in FP32 after the first FP64
residual) against the same solve with every refinement residual in FP64, and its reported
relative residual against the true one, b - A x formed by the oracle in FP64."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host

pytestmark = pytest.mark.gpu

# 3D shapes (z, y, x) whose level 0 the z-marching residual kernels cover: one tile and a
# ragged tile in x, every boundary kind on every axis, and a stiff case (dt D / h^2 up to
# ~1e3, so the face-flux term of the rounding bound dominates)
CASES = [
    ((24, 20, 32), (1 / 32, 1 / 20, 1 / 24), ((0, 0), (0, 0), (2, 2)), 2e-4, 1.0),
    ((40, 36, 128), (1.0, 1.0, 1.0), ((0, 0), (1, 2), (2, 1)), 0.8, 1.0),
    ((18, 17, 68), (1.0, 0.9, 1.1), ((2, 2), (1, 1), (0, 0)), 1.5, 1.2),
    ((33, 45, 70), (1.0, 1.0, 1.0), ((1, 1), (2, 2), (0, 0)), 40.0, 1.5),
]


def _problem(shape, bc, sigma, seed):
    rng = np.random.default_rng(seed)
    D = I.lognormal(rng, shape, sigma, 4.0)
    E = 1.0 + rng.uniform(0, 1, shape)
    Eb = {}
    nd = len(shape)
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1.0 + rng.uniform(0, 1, fs)
    return D, E, Eb


def _solve(fld, torch, shape, h, bc, dt, D, E, Eb, tol, update, prof=False):
    hd = fld.Handle(shape, h, bc, precision=fld.PREC_MIXED, tol=tol, max_cycles=40,
                    smoother=2, resid_update=update)
    Ed = dev(torch, E)
    packed = I.pack_dirichlet(shape, bc, Eb)
    if prof:
        hd.prof_enable(True, 4096)
    st = hd.diffuse(dt, dev(torch, D), dev(torch, packed) if packed.size else None, Ed,
                    raise_on_error=False)
    names = {e["name"] for e in hd.prof_read()} if prof else set()
    return host(Ed).reshape(shape), st, names


@pytest.mark.parametrize("tol", [1e-8, 1e-10, 1e-12])
@pytest.mark.parametrize("shape,h,bc,dt,sigma", CASES)
def test_recursive_residual_bounds_the_true_residual(shape, h, bc, dt, sigma, tol):
    torch = torch_cuda()
    fld = library()
    D, E, Eb = _problem(shape, bc, sigma, 5 + shape[2])
    A, g = O.assemble(D, h, bc, Eb, dt)
    bn = np.linalg.norm(E.ravel() + g)
    out = {}
    for update in (1, 0):
        x, st, names = _solve(fld, torch, shape, h, bc, dt, D, E, Eb, tol, update,
                              prof=update == 1)
        assert st["status"] in (0, 3), st
        true = O.relative_residual(x, E, D, h, bc, Eb, dt)
        # the reported residual bounds the true one (up to the rounding of an FP64
        # residual, below 1e-14 here) and passes tol when the status says so
        assert true <= st["rel_resid"] * (1 + 1e-6) + 1e-14, (update, true, st["rel_resid"])
        if st["status"] == 0:
            assert st["rel_resid"] <= tol
        if update == 1 and st["cycles"] >= 2:
            assert "resid_upd" in names, names       # the update path ran
        out[update] = (x, st)
    (x1, s1), (x0, s0) = out[1], out[0]
    if s1["cycles"] == s0["cycles"] <= 2:
        # x + e is the same FP64 sum in both kernels, and the first two corrections see
        # the same right-hand sides (the FP32 residual of E^n, then an FP64 residual): the
        # same iterate. From the third on, the update's right-hand side is the recursive
        # residual.
        assert np.array_equal(x1, x0)
    # both iterates solve A x = b to their residuals: ||x1 - x0|| <= (r1 + r0) ||b||
    # (||A^-1||_2 <= 1)
    dx = np.linalg.norm((x1 - x0).ravel())
    assert dx <= (s1["rel_resid"] + s0["rel_resid"]) * bn * (1 + 1e-6) + 2e-14 * bn


def test_recursive_residual_with_tolerance_below_the_fp64_floor():
    # at tol 1e-18 no FP64 residual passes (the rounding of x itself moves A x by more),
    # and the bound of the x + e rounding alone passes tol/2 after one update: the loop
    # falls back to FP64 residuals and ends at the cycle limit with the reported residual
    # still bounding the true one
    torch = torch_cuda()
    fld = library()
    shape, h, bc, dt, sigma = CASES[1]
    D, E, Eb = _problem(shape, bc, sigma, 77)
    x, st, _ = _solve(fld, torch, shape, h, bc, dt, D, E, Eb, 1e-18, 1)
    assert st["status"] == fld.FLD_ERR_NOT_CONVERGED and st["cycles"] == 40, st
    true = O.relative_residual(x, E, D, h, bc, Eb, dt)
    assert true <= st["rel_resid"] * (1 + 1e-6) + 1e-14
    assert np.all(np.isfinite(x))
