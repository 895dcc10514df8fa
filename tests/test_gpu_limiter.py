"""GPU limiter kernel (fld_limiter) against the oracle, element by element."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, handle_for, consts_of, ebc_dev

pytestmark = pytest.mark.gpu

CASES = [
    ((300,), (0.01,), ((0, 0),)),
    ((7,), (0.3,), ((2, 1),)),
    ((2, 3), (0.5, 0.25), ((1, 1), (0, 0))),
    ((37, 70), (0.1, 0.2), ((0, 0), (2, 1))),
    ((13, 19, 70), (0.1, 0.2, 0.3), ((1, 2), (0, 0), (2, 2))),
    ((9, 33, 40), (0.05, 0.05, 0.05), ((0, 0), (1, 1), (0, 0))),
]


def _fields(shape, bc, seed):
    rng = np.random.default_rng(seed)
    E = 1 + 0.5 * rng.uniform(0, 1, shape) + np.linspace(0, 1, shape[-1])
    rho = 10 ** rng.uniform(-1, 1, shape)
    T = 10 ** rng.uniform(-0.3, 0.3, shape)
    Eb = {}
    nd = len(shape)
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1 + rng.uniform(0, 1, fs)
    return E, rho, T, Eb


@pytest.mark.parametrize("precision,limiter_df", [(0, 0), (2, 0), (1, 1)])
@pytest.mark.parametrize("shape,h,bc", CASES)
@pytest.mark.parametrize("op", [(0, 2.0, 0.0, 0.0), (1, 5.0, 1.0, -3.5)])
def test_limiter_matches_oracle(shape, h, bc, op, precision, limiter_df):
    # precision 2 (MIXED_DF) and the limiter_df option run the double-FP32 limiter, the
    # others the FP64 one
    torch = torch_cuda()
    fld = library()
    E, rho, T, Eb = _fields(shape, bc, len(shape) * 100 + shape[-1])
    for mode in (0, 1, 2):
        hd = fld.Handle(shape, h, bc, limiter=mode, precision=precision, limiter_df=limiter_df)
        D = torch.empty(E.size, dtype=torch.float64, device="cuda")
        lam = torch.empty_like(D)
        packed = I.pack_dirichlet(shape, bc, Eb)
        hd.limiter(fld.make_consts(3.0, 1.0, 5 / 3, 1.0), fld.make_opacity(op), dev(torch, E),
                   dev(torch, rho), dev(torch, T), dev(torch, packed) if packed.size else None, D, lam)
        assert hd.status() == 0
        Do, lo, _ = O.limiter(E, rho, T, h, bc, Eb, 3.0, op, mode)
        # FP64: rounding-level; double-FP32 (48-bit): a few units of 2^-48
        tol = 1e-13 if precision == 0 and not limiter_df else 1e-12
        assert np.max(np.abs(host(D).reshape(shape) / Do - 1)) < tol
        assert np.max(np.abs(host(lam).reshape(shape) / lo - 1)) < tol


@pytest.mark.parametrize("precision", [0, 2])
def test_limiter_workload_fields(precision):
    torch = torch_cuda()
    fld = library()
    for P in (I.make_config(1), I.make_config(2, small=True), I.make_config(3, small=True)):
        hd = handle_for(fld, P, precision=precision)
        D = torch.empty(P.ncells, dtype=torch.float64, device="cuda")
        hd.limiter(consts_of(fld, P), fld.make_opacity(P.opacity), dev(torch, P.E), dev(torch, P.rho),
                   dev(torch, P.T), ebc_dev(torch, P), D)
        Do, _, _ = O.limiter(P.E, P.rho, P.T, P.h, P.bc, P.E_bc, P.c, P.opacity)
        assert np.max(np.abs(host(D).reshape(P.shape) / Do - 1)) < (1e-13 if precision == 0 else 1e-12)


def test_limiter_rejects_nonpositive_E():
    torch = torch_cuda()
    fld = library()
    E = np.ones((4, 6))
    E[2, 3] = 0.0
    hd = fld.Handle((4, 6), (1, 1), ((0, 0), (0, 0)))
    D = torch.zeros(24, dtype=torch.float64, device="cuda")
    hd.limiter(fld.make_consts(1, 1, 5 / 3, 1), fld.make_opacity((0, 1, 0, 0)), dev(torch, E),
               dev(torch, np.ones((4, 6))), None, None, D)
    assert hd.status() == fld.FLD_ERR_DOMAIN
