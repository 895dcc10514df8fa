"""The 1D radiation-MHD wave step on the GPU (fld_wave1d_step: WENO3 + HLL + SSP-RK3
kernels around fld_coupling and fld_step) against the oracle's step (oracle/rmhd1d.py):
element by element over a dozen steps, then the measured damping of the strongly
radiative fast wave over a whole run."""
import json
import os

import numpy as np
import pytest

from oracle import rmhd1d as R
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
OPTS = dict(precision=0, tol=1e-13, max_cycles=200)


def _problem(n=280, nw=7, kind="fast", case="table3_strong"):
    return I.wave1d(GOLD[case]["background"], n, nw, kind)


@pytest.mark.parametrize("kind", ["fast", "slow", "alfven"])
def test_wave_steps_match_oracle(kind):
    torch = torch_cuda()
    fld = library()
    P = _problem(kind=kind)
    orc = R.Wave(P, cfl=0.8)
    gpu = fld.Wave1D(P, **OPTS)
    U = orc.initial()
    Ud = dev(torch, U)
    t = 0.0
    for _ in range(12):
        dt = orc.dt_max(U)
        assert gpu.max_dt(Ud, 0.8) == pytest.approx(dt, rel=1e-12)
        U = orc.step(U, t, dt)
        st = gpu.step(Ud, t, dt)
        assert st["status"] in (0, 3)
        t += dt
    G = host(Ud).reshape(8, -1)
    # every variable against its physical scale (rho_0, rho_0 c_f for the momenta, |B|,
    # e_0, E_0): the radiation solve's tolerance (1e-13) bounds the agreement
    W0 = P.W0[:, None]
    cf = float(R.fast_speed(W0, P.Bx, P.gamma)[0])
    e0 = float(R.conserved(W0, P.Bx, P.gamma)[R.PG][0])
    Bmag = float(np.sqrt(P.Bx ** 2 + P.W0[4] ** 2 + P.W0[5] ** 2))
    scales = [P.W0[0], P.W0[0] * cf, P.W0[0] * cf, P.W0[0] * cf, Bmag, Bmag, e0, P.E0]
    for v in range(8):
        assert np.max(np.abs(G[v] - U[v])) <= 1e-11 * scales[v], v
    # the driven perturbations themselves to 1e-7 of their size
    for v in ((R.BY,) if kind == "alfven" else (R.RHO, R.BZ)):
        d = U[v] - P.W0[v]
        assert np.max(np.abs(G[v] - U[v])) <= 1e-7 * np.max(np.abs(d)), v
    gpu.close()


@pytest.mark.parametrize("kind", ["fast", "slow", "alfven"])
def test_ars3_steps_match_oracle(kind):
    # the ARS3 IMEX step (explicit hyperbolic and coupling terms, the FLD substep as its two
    # implicit stages over gamma dt) against the oracle's, as for the split step
    torch = torch_cuda()
    fld = library()
    P = _problem(kind=kind)
    orc = R.Wave(P, cfl=0.8, scheme="ars3")
    gpu = fld.Wave1D(P, scheme=1, **OPTS)
    U = orc.initial()
    Ud = dev(torch, U)
    t = 0.0
    for _ in range(12):
        dt = orc.dt_max(U)
        U = orc.step(U, t, dt)
        st = gpu.step(Ud, t, dt)
        assert st["status"] in (0, 3)
        t += dt
    G = host(Ud).reshape(8, -1)
    W0 = P.W0[:, None]
    cf = float(R.fast_speed(W0, P.Bx, P.gamma)[0])
    e0 = float(R.conserved(W0, P.Bx, P.gamma)[R.PG][0])
    Bmag = float(np.sqrt(P.Bx ** 2 + P.W0[4] ** 2 + P.W0[5] ** 2))
    scales = [P.W0[0], P.W0[0] * cf, P.W0[0] * cf, P.W0[0] * cf, Bmag, Bmag, e0, P.E0]
    for v in range(8):
        assert np.max(np.abs(G[v] - U[v])) <= 1e-11 * scales[v], v
    gpu.close()


@pytest.mark.parametrize("scheme", [0, 1])
def test_ideal_mhd_steps_match_oracle(scheme):
    # without radiation (no coupling terms, no substep): the hyperbolic scheme alone, the
    # reference for the scheme's own damping
    torch = torch_cuda()
    fld = library()
    P = I.wave1d(GOLD["table2_weak"]["background"], 280, 7, "fast", radiation=False)
    orc = R.Wave(P, cfl=0.8, scheme="ars3" if scheme else "split")
    gpu = fld.Wave1D(P, scheme=scheme, **OPTS)
    U = orc.initial()
    Ud = dev(torch, U)
    t = 0.0
    for _ in range(12):
        dt = orc.dt_max(U)
        U = orc.step(U, t, dt)
        gpu.step(Ud, t, dt)
        t += dt
    G = host(Ud).reshape(8, -1)
    assert np.max(np.abs(G - U) / np.maximum(np.abs(U).max(axis=1, keepdims=True), 1e-300)) < 1e-12
    gpu.close()


def test_radiative_fast_wave_damping_matches_oracle():
    # the strongly radiative fast wave of Table 3 over 5.5 wavelengths of travel at CFL 0.2:
    # the GPU run's measured spatial damping equals the oracle run's
    torch = torch_cuda()
    fld = library()
    P = _problem()
    orc = R.Wave(P, cfl=0.2)
    t_end = 5.5 * P.lam / P.phase_speed
    U, t_or, steps = orc.run(t_end)
    gpu = fld.Wave1D(P, **OPTS)
    Ud = dev(torch, orc.initial())
    t, n = 0.0, 0
    while t < t_end * (1.0 - 1e-12):
        dt = min(gpu.max_dt(Ud, 0.2), t_end - t)
        assert gpu.step(Ud, t, dt)["status"] in (0, 3)
        t += dt
        n += 1
    assert n == steps
    G = host(Ud).reshape(8, -1)
    k_or = orc.damping(U, 1, 5)
    k_gpu = orc.damping(G, 1, 5)
    assert k_gpu == pytest.approx(k_or, rel=1e-6)
    d_or, d_gpu = U[R.RHO] - P.W0[0], G[R.RHO] - P.W0[0]
    assert np.max(np.abs(d_gpu - d_or)) <= 1e-6 * np.max(np.abs(d_or))
    gpu.close()


def test_wave_argument_errors():
    torch = torch_cuda()
    fld = library()
    P = _problem()
    gpu = fld.Wave1D(P, **OPTS)
    with pytest.raises(ValueError):
        gpu.step(torch.zeros(8 * P.n - 1, dtype=torch.float64, device="cuda"), 0.0, 1.0)
    Ud = dev(torch, R.Wave(P).initial())
    with pytest.raises(fld.FldError):
        gpu.step(Ud, 0.0, -1.0)
    # a state with a NaN density, or with a negative gas energy (negative pressure), in one
    # cell: the signal-speed maximum is +inf and the time-step call reports a domain error
    for var, cell, value in ((0, 100, np.nan), (6, 50, -1.0)):
        U = np.array(R.Wave(P).initial(), dtype=np.float64).reshape(8, -1)
        U[var, cell] = value
        with pytest.raises(fld.FldError) as ei:
            gpu.max_dt(dev(torch, U), 0.8)
        assert ei.value.code == fld.FLD_ERR_DOMAIN
    gpu.close()
    bad = fld.make_wave1d_params(P, **OPTS)
    bad.n_driven = bad.n
    with pytest.raises(fld.FldError):
        fld.fld_wave1d_create(bad)
