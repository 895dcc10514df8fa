"""GPU multigrid diffusion solve (fld_diffuse) against the oracle's direct solve."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, maxrel

pytestmark = pytest.mark.gpu

# (shape, h, bc, dt, sigma)
CASES = [
    ((256,), (1 / 256,), ((0, 0),), 0.002, 1.0),
    ((2,), (0.5,), ((1, 2),), 0.3, 0.5),
    ((31,), (0.1,), ((2, 2),), 0.5, 1.0),
    ((5, 3), (0.2, 0.3), ((0, 0), (1, 2)), 0.1, 1.0),
    ((29, 37), (1.0, 1.0), ((0, 0), (0, 0)), 2.0, 1.5),
    ((80, 96), (1.0, 1.0), ((0, 0), (0, 0)), 5.0, 1.0),
    ((9, 11, 13), (0.1, 0.1, 0.1), ((1, 2), (0, 0), (2, 1)), 0.004, 1.0),
    ((24, 20, 32), (1 / 32, 1 / 20, 1 / 24), ((0, 0), (0, 0), (2, 2)), 2e-4, 1.0),
    ((11, 13, 17), (1.0, 1.0, 1.0), ((0, 0), (0, 0), (0, 0)), 1.5, 1.0),
    ((2, 40), (0.5, 0.5), ((1, 2), (0, 0)), 0.2, 1.0),
    ((70, 9, 131), (1.0, 1.0, 1.0), ((1, 1), (0, 0), (2, 1)), 0.8, 0.7),
]


def _problem(shape, bc, sigma, seed, ell=4.0):
    # D log-normal with a correlation length of a few cells, like the workloads'
    # D = c lambda / (kappa rho) with a correlated log-normal rho
    rng = np.random.default_rng(seed)
    D = I.lognormal(rng, shape, sigma, ell) if min(shape) > 2 else np.exp(
        sigma * rng.standard_normal(shape))
    E = 1.0 + rng.uniform(0, 1, shape)
    Eb = {}
    nd = len(shape)
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1.0 + rng.uniform(0, 1, fs)
    return D, E, Eb


def _solve_gpu(fld, torch, shape, h, bc, dt, D, E, Eb, precision, tol=1e-14, smoother=0):
    hd = fld.Handle(shape, h, bc, precision=precision, tol=tol, max_cycles=100, smoother=smoother)
    Ed = dev(torch, E)
    packed = I.pack_dirichlet(shape, bc, Eb)
    st = hd.diffuse(dt, dev(torch, D), dev(torch, packed) if packed.size else None, Ed,
                    raise_on_error=False)
    assert st["status"] in (0, 3), st
    # tol, or the residual floor: ~1e-13 for an FP64 residual; for the double-FP32
    # residual (48-bit) the floor is cond(A) x 2^-48, ~1e-11 on the stiffest case here
    floor = 1e-13 if precision != 2 else 1e-10
    assert st["rel_resid"] < max(tol, floor), st
    return host(Ed).reshape(shape), st


@pytest.mark.parametrize("smoother", [0, 1, 2])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-10), (2, 1e-10)])
@pytest.mark.parametrize("shape,h,bc,dt,sigma", CASES)
def test_diffuse_matches_direct_solve(shape, h, bc, dt, sigma, precision, tol, smoother):
    # smoother 0: in-place half sweeps, 1: out-of-place half sweeps, 2: z-marching sweep
    torch = torch_cuda()
    fld = library()
    D, E, Eb = _problem(shape, bc, sigma, 17 + len(shape) + shape[0])
    x, st = _solve_gpu(fld, torch, shape, h, bc, dt, D, E, Eb, precision, smoother=smoother)
    xo = O.diffuse(E, D, h, bc, Eb, dt, method="lu" if E.size <= 4096 else "splu")
    assert maxrel(x, xo) < tol, (maxrel(x, xo), st)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_convergence_rate_and_determinism(precision):
    torch = torch_cuda()
    fld = library()
    P = I.make_config(2, small=True)
    D, _, _ = O.limiter(P.E, P.rho, P.T, P.h, P.bc, P.E_bc, P.c, P.opacity)
    x1, st = _solve_gpu(fld, torch, P.shape, P.h, P.bc, P.dt, D, P.E, {}, precision, tol=1e-10)
    x2, _ = _solve_gpu(fld, torch, P.shape, P.h, P.bc, P.dt, D, P.E, {}, precision, tol=1e-10)
    assert np.array_equal(x1, x2)                 # bitwise reproducible (fixed reductions)
    hist = st["resid_hist"]
    rates = [hist[i + 1] / hist[i] for i in range(len(hist) - 1)]
    assert max(rates) < 0.5, hist                 # each V-cycle removes most of the residual


def test_not_converged_status_keeps_iterate():
    torch = torch_cuda()
    fld = library()
    D, E, _ = _problem((64, 64), ((0, 0), (0, 0)), 1.0, 3)
    hd = fld.Handle((64, 64), (1, 1), ((0, 0), (0, 0)), tol=1e-14, max_cycles=1)
    Ed = dev(torch, E)
    st = hd.diffuse(5.0, dev(torch, D), None, Ed, raise_on_error=False)
    assert st["status"] == fld.FLD_ERR_NOT_CONVERGED and st["cycles"] == 1
    assert st["rel_resid"] < st["resid_hist"][0]
    assert np.all(np.isfinite(host(Ed)))


def test_conservation_periodic():
    torch = torch_cuda()
    fld = library()
    for precision in (0, 1, 2):
        D, E, _ = _problem((33, 47), ((0, 0), (0, 0)), 1.5, 8)
        x, _ = _solve_gpu(fld, torch, (33, 47), (1, 1), ((0, 0), (0, 0)), 3.0, D, E, {}, precision)
        assert abs(x.sum() - E.sum()) / E.sum() < 1e-13


# 3D shapes (z, y, x) whose level 0 (and some coarser levels) the single-pass z-marching
# sweep covers: x extents a multiple of 4 (one full tile, two tiles, a ragged 64 + 4),
# every boundary kind on every axis, an odd non-periodic extent.
FUSED_CASES = [
    ((24, 20, 32), (1 / 32, 1 / 20, 1 / 24), ((0, 0), (0, 0), (2, 2)), 2e-4, 1.0),
    ((40, 36, 128), (1.0, 1.0, 1.0), ((0, 0), (1, 2), (2, 1)), 0.8, 1.0),
    ((18, 17, 68), (1.0, 0.9, 1.1), ((2, 2), (1, 1), (0, 0)), 1.5, 1.2),
    ((16, 16, 16), (1.0, 1.0, 1.0), ((1, 1), (2, 2), (0, 0)), 1.0, 1.0),
]


_FUSED_ORACLE = {}


@pytest.mark.parametrize("nu", [(1, 1), (2, 2), (1, 2), (2, 1)])
@pytest.mark.parametrize("shape,h,bc,dt,sigma", FUSED_CASES)
def test_fused_sweep_matches_half_sweeps_and_oracle(shape, h, bc, dt, sigma, nu):
    # the fused sweep performs the same arithmetic as two in-place half sweeps, so both
    # smoothers take the same number of cycles to the same iterate; both match the oracle
    torch = torch_cuda()
    fld = library()
    D, E, Eb = _problem(shape, bc, sigma, 91 + shape[2])
    packed = I.pack_dirichlet(shape, bc, Eb)
    key = (shape, bc)
    if key not in _FUSED_ORACLE:
        # sparse LU fills in badly on 3D grids: the oracle's PCG (to 1e-14) above ~20k cells
        _FUSED_ORACLE[key] = O.diffuse(E, D, h, bc, Eb, dt,
                                       method="splu" if E.size <= 20000 else "pcg")
    xo = _FUSED_ORACLE[key]
    for precision in (1, 2):
        res = {}
        for smoother in (0, 2):
            # tol at the residual floor (~1e-13 FP64, ~1e-11 double-FP32): the error
            # against the oracle is then well inside 1e-10
            hd = fld.Handle(shape, h, bc, precision=precision, tol=1e-12, max_cycles=30,
                            smoother=smoother, nu1=nu[0], nu2=nu[1], graph=smoother == 2)
            Ed = dev(torch, E)
            st = hd.diffuse(dt, dev(torch, D), dev(torch, packed) if packed.size else None, Ed,
                            raise_on_error=False)
            assert st["status"] in (0, 3) and st["rel_resid"] < 1e-10, st
            res[smoother] = (host(Ed).reshape(shape), st["cycles"])
            hd.close()
        assert res[0][1] == res[2][1], (res[0][1], res[2][1])
        assert maxrel(res[2][0], res[0][0]) < 1e-13
        assert maxrel(res[2][0], xo) < 1e-10
