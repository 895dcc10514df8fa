"""Whole FLD substep (fld_step) on the seeded workloads at reduced size, against the
oracle's substep."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, handle_for, consts_of, ebc_dev, maxrel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [1, 2, 3, 5])
@pytest.mark.parametrize("precision,tol,limiter_df", [(0, 1e-12, 0), (1, 1e-10, 0), (2, 1e-10, 0),
                                                      (1, 1e-10, 1)])
def test_step_matches_oracle(cfg, precision, tol, limiter_df):
    torch = torch_cuda()
    fld = library()
    P = I.make_config(cfg, small=True)
    hd = handle_for(fld, P, precision=precision, tol=1e-14, max_cycles=100,
                    limiter_df=limiter_df)
    Td, Ed, rd = dev(torch, P.T), dev(torch, P.E), dev(torch, P.rho)
    ebc = ebc_dev(torch, P)
    T, E = P.T.copy(), P.E.copy()
    for _ in range(2):
        st = hd.step(consts_of(fld, P), fld.make_opacity(P.opacity), P.dt, rd, Td, Ed, ebc,
                     raise_on_error=False)
        assert st["status"] in (0, 3) and st["rel_resid"] < 1e-13, st
        T, E, _ = O.step(P.rho, T, E, P.h, P.bc, P.E_bc, P.dt, P.c, P.a_r, P.gamma, P.R_gas,
                         P.opacity, P.limiter, method="lu" if P.ncells <= 4096 else "splu")
    assert maxrel(host(Ed).reshape(P.shape), E) < tol
    assert maxrel(host(Td).reshape(P.shape), T) < tol


def test_total_energy_conserved_on_periodic_step():
    torch = torch_cuda()
    fld = library()
    P = I.make_config(2, small=True)
    hd = handle_for(fld, P, precision=1, tol=1e-12)
    Td, Ed, rd = dev(torch, P.T), dev(torch, P.E), dev(torch, P.rho)
    e0 = (O.internal_energy(P.rho, P.T, P.gamma, P.R_gas) + P.E).sum()
    hd.step(consts_of(fld, P), fld.make_opacity(P.opacity), P.dt, rd, Td, Ed, None)
    e1 = (O.internal_energy(P.rho, host(Td).reshape(P.shape), P.gamma, P.R_gas)
          + host(Ed).reshape(P.shape)).sum()
    assert abs(e1 - e0) / e0 < 1e-12


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-10)])
def test_ars3_stage_is_the_substep_over_gamma_dt(precision, tol):
    # fld_ars3_stage: the substep over gamma dt from the predictor, and the implicit
    # increments (stage - predictor)/(gamma dt) of E and of the gas energy rho c_v T
    torch = torch_cuda()
    fld = library()
    P = I.make_config(3, small=True)
    hd = handle_for(fld, P, precision=precision, tol=1e-14, max_cycles=100)
    g = (3 + np.sqrt(3)) / 6
    Td, Ed, rd = dev(torch, P.T), dev(torch, P.E), dev(torch, P.rho)
    FE, Fe = torch.empty_like(Ed), torch.empty_like(Ed)
    st = fld.fld_ars3_stage(hd.h, consts_of(fld, P), fld.make_opacity(P.opacity), P.dt, 1, rd, Td,
                            Ed, ebc_dev(torch, P), FE, Fe, raise_on_error=False)
    assert st["status"] in (0, 3) and st["rel_resid"] < 1e-13, st
    To, Eo, _ = O.step(P.rho, P.T, P.E, P.h, P.bc, P.E_bc, g * P.dt, P.c, P.a_r, P.gamma,
                       P.R_gas, P.opacity, P.limiter, method="splu")
    assert maxrel(host(Ed).reshape(P.shape), Eo) < tol
    assert maxrel(host(Td).reshape(P.shape), To) < tol
    cv = P.R_gas / (P.gamma - 1)
    assert maxrel(host(FE).reshape(P.shape), (Eo - P.E) / (g * P.dt)) < 1e3 * tol
    assert maxrel(host(Fe).reshape(P.shape), P.rho * cv * (To - P.T) / (g * P.dt)) < 1e3 * tol


@pytest.mark.parametrize("cfg", [2, 3])
def test_step_diagnostics_energy_and_phase_times(cfg):
    # diag = energy | times: the energy sums are those of the fields before and after the
    # step (rho c_v T + E times the cell volume, summed in numpy), equal to each other on the
    # periodic config 2; Dirichlet walls (config 3) let energy through. Phase times are
    # positive and the whole call covers the three phases
    torch = torch_cuda()
    fld = library()
    P = I.make_config(cfg, small=True)
    hd = handle_for(fld, P, precision=1, tol=1e-12, diag=fld.DIAG_ENERGY | fld.DIAG_TIMES)
    Td, Ed, rd = dev(torch, P.T), dev(torch, P.E), dev(torch, P.rho)
    vol = float(np.prod(P.h))

    def total(T, E):
        return float((O.internal_energy(P.rho, T, P.gamma, P.R_gas) + E).sum()) * vol

    e0 = total(P.T, P.E)
    st = hd.step(consts_of(fld, P), fld.make_opacity(P.opacity), P.dt, rd, Td, Ed,
                 ebc_dev(torch, P))
    e1 = total(host(Td).reshape(P.shape), host(Ed).reshape(P.shape))
    assert st["energy_before"] == pytest.approx(e0, rel=1e-13)
    assert st["energy_after"] == pytest.approx(e1, rel=1e-13)
    if cfg == 2:
        assert abs(st["energy_after"] - st["energy_before"]) <= 1e-12 * e0
    t = st["t_ms"]
    assert all(x > 0 for x in t), t
    assert t[3] >= 0.99 * (t[0] + t[1] + t[2]), t
    # the solve alone through fld_diffuse: E summed before and after
    Dd = torch.empty_like(Ed)
    hd.limiter(consts_of(fld, P), fld.make_opacity(P.opacity), Ed, rd, Td, ebc_dev(torch, P), Dd)
    E0 = host(Ed).reshape(P.shape)
    st = hd.diffuse(P.dt, Dd, ebc_dev(torch, P), Ed)
    assert st["energy_before"] == pytest.approx(float(E0.sum()) * vol, rel=1e-13)
    assert st["energy_after"] == pytest.approx(float(host(Ed).sum()) * vol, rel=1e-13)
    assert st["t_ms"][1] > 0 and st["t_ms"][0] == 0 and st["t_ms"][2] == 0
    # without diag the fields stay zero
    hd.set_opts(precision=1, tol=1e-12)
    st = hd.step(consts_of(fld, P), fld.make_opacity(P.opacity), P.dt, rd, Td, Ed,
                 ebc_dev(torch, P))
    assert st["energy_before"] == 0 and st["t_ms"] == [0.0] * 4
