"""The harmonic face mean (fld_opts.face_mean = FLD_FACE_HARM) on the GPU: the diffusion
solve and the whole substep against the oracle's with face_mean="harm", in FP64 and MIXED,
on 1D (direct and V-cycle), 2D and 3D grids with strongly varying log-normal D, and the
layered-medium closed form (resistances in series) as a fixed point."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, handle_for, consts_of, ebc_dev, maxrel

pytestmark = pytest.mark.gpu

# (shape (z, y, x), h, bc, dt, sigma): 1D, 2D, and 3D boxes spanning several 32 x 8 tiles
# with ragged edges (the oracle's sparse direct solve keeps them to ~2e4 cells)
CASES = [
    ((200,), (0.01,), ((2, 1),), 0.05, 2.0),
    ((48, 37), (1.0, 1.0), ((0, 0), (2, 2)), 3.0, 2.0),
    ((20, 21, 36), (1.0, 0.8, 1.2), ((2, 2), (0, 0), (1, 1)), 2.0, 1.5),
    ((24, 16, 48), (1.0, 1.0, 1.0), ((0, 0), (0, 0), (0, 0)), 4.0, 2.0),
]
_REF = {}


def _oracle(case, seed, face_mean):
    key = (case, seed, face_mean)
    if key not in _REF:
        shape, h, bc, dt, sigma = CASES[case]
        D, E, Eb = _problem(shape, bc, sigma, seed)
        _REF[key] = O.diffuse(E, D, h, bc, Eb, dt, method="splu", face_mean=face_mean)
    return _REF[key]


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


@pytest.mark.parametrize("direct1d", [1, 0])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-10)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_diffuse_harmonic_matches_oracle(case, precision, tol, direct1d):
    shape, h, bc, dt, sigma = CASES[case]
    if direct1d == 0 and len(shape) > 1:
        pytest.skip("the direct solve is 1D only")
    torch = torch_cuda()
    fld = library()
    D, E, Eb = _problem(shape, bc, sigma, 17)
    hd = fld.Handle(shape, h, bc, precision=precision, tol=1e-13, max_cycles=200,
                    face_mean=fld.FACE_HARM, direct1d=direct1d, smoother=2)
    Ed = dev(torch, E)
    packed = I.pack_dirichlet(shape, bc, Eb)
    st = hd.diffuse(dt, dev(torch, D), dev(torch, packed) if packed.size else None, Ed,
                    raise_on_error=False)
    assert st["status"] == 0 and st["rel_resid"] < 1e-12, st
    ref = _oracle(case, 17, "harm")
    assert maxrel(host(Ed).reshape(shape), ref) < tol
    # the arithmetic answer differs from it by far more than the tolerance (the option
    # reaches the operator)
    assert maxrel(_oracle(case, 17, "arith"), ref) > 100 * tol


@pytest.mark.parametrize("precision", [0, 1])
def test_layered_profile_is_a_fixed_point_on_the_gpu(precision):
    nx, ny, nz = 64, 16, 16
    rng = np.random.default_rng(3)
    Dx = np.exp(2.0 * rng.standard_normal(nx))
    h = (0.5, 0.8, 1.3)
    R = h[0] / Dx
    q = (2.0 - 5.0) / R.sum()
    Ex = 2.0 - q * (np.concatenate(([0.0], np.cumsum(R)[:-1])) + 0.5 * R)
    D = np.broadcast_to(Dx, (nz, ny, nx)).copy()
    E = np.broadcast_to(Ex, (nz, ny, nx)).copy()
    bc = ((2, 2), (0, 0), (0, 0))
    Eb = {(0, 0): np.full((nz, ny), 2.0), (0, 1): np.full((nz, ny), 5.0)}
    torch = torch_cuda()
    fld = library()
    hd = fld.Handle((nz, ny, nx), h, bc, precision=precision, tol=1e-14, max_cycles=100,
                    face_mean=fld.FACE_HARM)
    Ed = dev(torch, E)
    st = hd.diffuse(0.5, dev(torch, D), dev(torch, I.pack_dirichlet(E.shape, bc, Eb)), Ed,
                    raise_on_error=False)
    assert st["status"] == 0, st
    # ||A^-1||_2 <= 1, so the error is below the residual norm, 1e-14 ||b||_2 (about 1e-9
    # here, b carrying the walls' 2 dt D E_b / h^2)
    assert np.max(np.abs(host(Ed).reshape(E.shape) - E)) < 5e-9


@pytest.mark.parametrize("cfg", [2, 3])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-10)])
def test_step_harmonic_matches_oracle(cfg, precision, tol):
    torch = torch_cuda()
    fld = library()
    P = I.make_config(cfg, small=True)
    hd = handle_for(fld, P, precision=precision, tol=1e-14, max_cycles=200,
                    face_mean=fld.FACE_HARM)
    Td, Ed, rd = dev(torch, P.T), dev(torch, P.E), dev(torch, P.rho)
    st = hd.step(consts_of(fld, P), fld.make_opacity(P.opacity), P.dt, rd, Td, Ed,
                 ebc_dev(torch, P), raise_on_error=False)
    assert st["status"] in (0, 3) and st["rel_resid"] < 1e-13, st
    T, E, _ = O.step(P.rho, P.T, P.E, P.h, P.bc, P.E_bc, P.dt, P.c, P.a_r, P.gamma, P.R_gas,
                     P.opacity, P.limiter, method="splu", face_mean="harm")
    assert maxrel(host(Ed).reshape(P.shape), E) < tol
    assert maxrel(host(Td).reshape(P.shape), T) < tol


def test_switching_the_face_mean_on_a_handle():
    # fld_set_opts to HARM and back: each solve matches its oracle (the captured FP32
    # V-cycle graph is rebuilt with the new levels)
    torch = torch_cuda()
    fld = library()
    shape, h, bc, dt, sigma = CASES[3]
    D, E, Eb = _problem(shape, bc, sigma, 5)
    hd = fld.Handle(shape, h, bc, precision=1, tol=1e-12, max_cycles=100, smoother=2, graph=1)
    for fm, name in ((fld.FACE_ARITH, "arith"), (fld.FACE_HARM, "harm"),
                     (fld.FACE_ARITH, "arith")):
        hd.set_opts(precision=1, tol=1e-12, max_cycles=100, smoother=2, graph=1, face_mean=fm)
        Ed = dev(torch, E)
        st = hd.diffuse(dt, dev(torch, D), None, Ed, raise_on_error=False)
        assert st["status"] == 0, st
        assert maxrel(host(Ed).reshape(shape), _oracle(3, 5, name)) < 1e-10, name


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", range(1, len(CASES)))
def test_constant_prolongation_reaches_the_same_solution(case, precision):
    # the prolongation kind changes the convergence path, never the answer: both kinds
    # converge to the oracle's solution (arithmetic mean), along different iterates (on
    # these strongly varying D the constant one often takes fewer cycles)
    shape, h, bc, dt, sigma = CASES[case]
    torch = torch_cuda()
    fld = library()
    D, E, Eb = _problem(shape, bc, sigma, 23)
    packed = I.pack_dirichlet(shape, bc, Eb)
    ref = _oracle(case, 23, "arith")
    cycles, first = {}, {}
    for pk in (fld.PROLONG_LINEAR, fld.PROLONG_CONSTANT):
        hd = fld.Handle(shape, h, bc, precision=precision, tol=1e-12, max_cycles=200,
                        prolong=pk, smoother=2)
        Ed = dev(torch, E)
        st = hd.diffuse(dt, dev(torch, D), dev(torch, packed) if packed.size else None, Ed,
                        raise_on_error=False)
        assert st["status"] == 0, (pk, st)
        assert maxrel(host(Ed).reshape(shape), ref) < (1e-11 if precision == 0 else 1e-10)
        cycles[pk] = st["cycles"]
        first[pk] = st["resid_hist"][1]
    # the option reaches the V-cycle: the first cycle leaves a different residual
    assert first[fld.PROLONG_CONSTANT] != first[fld.PROLONG_LINEAR], (first, cycles)
