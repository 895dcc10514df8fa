"""GPU exchange kernel (fld_exchange) against the oracle, element by element."""
import json
import os

import numpy as np
import pytest

from oracle import fld as O
from oracle import dispersion as Disp
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _run(fld, torch, rho, T, E, dt, consts, op, precision=0):
    # precision 2 (MIXED_DF) runs the double-FP32 exchange, the others the FP64 one
    n = rho.size
    h = fld.Handle((n,), (1.0,), ((0, 0),), precision=precision)
    Td, Ed = dev(torch, T), dev(torch, E)
    h.exchange(fld.make_consts(*consts), fld.make_opacity(op), dt, dev(torch, rho), Td, Ed)
    assert h.status() == 0
    return host(Td), host(Ed)


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("n", [1000, 65536 + 77])
def test_exchange_random_cells_constant_kappa(n, precision):
    torch = torch_cuda()
    fld = library()
    rho, T, E, kap = I.random_cells(n, seed=5)
    for dt in (1e-6, 0.37, 1e4):
        op = (0, 3.7, 0.0, 0.0)
        Tg, Eg = _run(fld, torch, rho, T, E, dt, (1.0, 1.0, 5 / 3, 1.0), op, precision)
        To, Eo = O.exchange(rho, T, E, dt, 1.0, 1.0, 5 / 3, 1.0, op)
        assert np.max(np.abs(Tg / To - 1)) < 1e-12
        assert np.max(np.abs(Eg / Eo - 1)) < 1e-12


@pytest.mark.parametrize("precision", [0, 2])
def test_exchange_kramers_opacity_and_cgs_units(precision):
    torch = torch_cuda()
    fld = library()
    rng = np.random.default_rng(9)
    n = 20000
    rho = 10 ** rng.uniform(-10, -2, n)
    T = 10 ** rng.uniform(3, 7, n)
    E = Disp.A_RAD * T ** 4 * 10 ** rng.uniform(-2, 2, n)
    R_gas = Disp.K_B / (0.6 * Disp.M_P)
    op = (1, 4e25, 1.0, -3.5)
    consts = (Disp.C_LIGHT, Disp.A_RAD, 5 / 3, R_gas)
    Tg, Eg = _run(fld, torch, rho, T, E, 1e-3, consts, op, precision)
    To, Eo = O.exchange(rho, T, E, 1e-3, *consts, op)
    assert np.max(np.abs(Tg / To - 1)) < 1e-12
    assert np.max(np.abs(Eg / Eo - 1)) < 1e-12


@pytest.mark.parametrize("precision", [0, 2])
def test_exchange_fixed_point_table1(precision):
    torch = torch_cuda()
    fld = library()
    st = GOLD["table1_states"]
    R_gas = Disp.K_B / (st["mu"] * Disp.M_P)
    for s in st["states"]:
        rho, T = np.array([s["rho"]] * 3), np.array([s["T"]] * 3)
        E = Disp.A_RAD * T ** 4
        Tg, Eg = _run(fld, torch, rho, T, E, 10.0, (Disp.C_LIGHT, Disp.A_RAD, s["gamma"], R_gas),
                      (0, 0.4, 0, 0), precision)
        # one FP64 Newton step from an FP32 seed leaves ~1e-15 relative in T (4x in T^4);
        # the double-FP32 path (48-bit significand) a few units of 2^-48 ~ 1e-14
        tt = 1e-14 if precision == 0 else 5e-14
        assert np.max(np.abs(Tg / T - 1)) < tt and np.max(np.abs(Eg / E - 1)) < 4 * tt


@pytest.mark.parametrize("precision", [0, 2])
def test_exchange_domain_error_leaves_cell(precision):
    torch = torch_cuda()
    fld = library()
    rho = np.ones(64)
    T = np.ones(64)
    E = np.full(64, 2.0)
    T[7] = -1.0
    h = fld.Handle((64,), (1.0,), ((0, 0),), precision=precision)
    Td, Ed = dev(torch, T), dev(torch, E)
    h.exchange(fld.make_consts(1, 1, 5 / 3, 1), fld.make_opacity((0, 1.0, 0, 0)), 0.1,
               dev(torch, rho), Td, Ed)
    assert h.status() == fld.FLD_ERR_DOMAIN
    assert host(Td)[7] == -1.0 and host(Ed)[7] == 2.0
    assert h.status() == 0          # the flag is cleared once read
