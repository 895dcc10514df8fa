"""Pins of the oracle's 1D radiation-MHD travelling-wave step (Sect. 3 scheme, Sect. 4.3
tests): the WENO3 reconstruction and HLL flux against their defining properties, the
banded diffusion solve against the general assembly, the spatial damping from the
Appendix-B matrix against the damping per length the paper prints, an ideal-MHD fast
wave travelling at its analytic speed, radiation leaving the Alfven wave alone, and the
damping of the strongly radiative fast wave converging in dt to the dispersion relation."""
import json
import os

import numpy as np
import pytest

from oracle import dispersion as Disp
from oracle import fld as F
from oracle import rmhd1d as R
from paper_2503_02764_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _bg(case):
    b = GOLD[case]["background"]
    return Disp.background(b["rho0"], b["p0"], b["B0_gauss"], b["gamma"], b["mu"], b["kappa"],
                           tau=b["tau"])


def _wave(case, n, nw, kind="fast", radiation=True, cfl=0.8):
    return R.Wave(I.wave1d(GOLD[case]["background"], n, nw, kind, radiation=radiation), cfl=cfl)


def test_recipe_backgrounds_are_the_printed_ones():
    for key, case in (("weak", "table2_weak"), ("strong", "table3_strong")):
        g = GOLD[case]["background"]
        b = I.WAVE_BACKGROUNDS[key]
        for name in ("rho0", "p0", "gamma", "mu", "kappa", "tau"):
            assert b[name] == pytest.approx(g[name], rel=1e-15), (key, name)
        assert list(b["B0_gauss"]) == list(g["B0_gauss"])


@pytest.mark.parametrize("case", ["table2_weak", "table3_strong"])
def test_recipe_matches_the_dispersion_background(case):
    bg = _bg(case)
    P = I.wave1d(GOLD[case]["background"], 40, 1)
    assert P.E0 == pytest.approx(bg["E0"], rel=1e-14)
    assert P.k == pytest.approx(bg["k"], rel=1e-14)
    assert P.Bx == pytest.approx(bg["B"][0], rel=1e-14)
    assert P.phase_speed == pytest.approx(Disp.magnetosonic_speed(bg, fast=True), rel=1e-14)
    assert P.E0 == pytest.approx(GOLD[case]["E0"], rel=1e-5)           # printed E_0
    S = I.wave1d(GOLD[case]["background"], 40, 1, "slow", radiation=False)
    assert S.phase_speed == pytest.approx(
        Disp.magnetosonic_speed(bg, fast=False, isothermal=False), rel=1e-14)


def test_weno3_exact_on_lines_third_order_and_bounded_at_a_step():
    x = np.arange(12, dtype=float)
    qL, qR = R.weno3((3.0 + 0.5 * x)[None, :])
    faces = 3.0 + 0.5 * (np.arange(1, 10) + 0.5)        # interfaces m + 1/2, m = 1 .. 9
    np.testing.assert_allclose(qL[0], faces, rtol=1e-14)
    np.testing.assert_allclose(qR[0], faces, rtol=1e-14)
    # third order on smooth monotone data (cell averages of exp(x); at critical points
    # the Jiang-Shu weights leave the linear ones and the max-norm order drops to two)
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        xc = (np.arange(-2, n + 2) + 0.5) * h
        cell = (np.exp(xc + h / 2) - np.exp(xc - h / 2)) / h
        qL, qR = R.weno3(cell[None, :])
        xf = (np.arange(1, n + 2) - 1.0) * h
        errs.append(max(np.max(np.abs(qL[0] - np.exp(xf))), np.max(np.abs(qR[0] - np.exp(xf)))))
    assert errs[0] / errs[1] > 7.0 and errs[1] / errs[2] > 7.0
    step = np.where(np.arange(20) < 10, 1.0, 2.0)[None, :]
    qL, qR = R.weno3(step)
    assert np.all((qL >= 1.0 - 1e-3) & (qL <= 2.0 + 1e-3))
    assert np.all((qR >= 1.0 - 1e-3) & (qR <= 2.0 + 1e-3))


def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([1.0 + 0.3 * rng.random(n), rng.standard_normal(n), rng.standard_normal(n),
                     rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(n),
                     1.0 + 0.3 * rng.random(n), 1.0 + 0.3 * rng.random(n)])


def test_hll_consistent_and_flux_form_conservative():
    W = _random_state(50, 1)
    np.testing.assert_allclose(R.hll(W, W, 0.7, 5 / 3), R.flux(W, 0.7, 5 / 3), rtol=1e-13,
                               atol=1e-13)
    # conservative <-> primitive round trip
    np.testing.assert_allclose(R.primitive(R.conserved(W, 0.7, 5 / 3), 0.7, 5 / 3), W, rtol=1e-12,
                               atol=1e-13)
    # periodic ghosts: the first and last interfaces see the same four cells, so their
    # fluxes are identical and the flux differences sum to zero (totals conserved)
    Wg = np.concatenate([W[:, -2:], W, W[:, :2]], axis=1)
    qL, qR = R.weno3(Wg)
    Fi = R.hll(qL, qR, 0.7, 5 / 3)
    assert np.array_equal(Fi[:, 0], Fi[:, -1])
    dU = -(Fi[:, 1:] - Fi[:, :-1])
    assert np.all(np.abs(dU.sum(axis=1)) <= 1e-12 * np.max(np.abs(Fi), axis=1))


@pytest.mark.parametrize("bc", [((1, 1),), ((1, 2),), ((2, 2),)])
def test_banded_diffusion_equals_general_assembly(bc):
    rng = np.random.default_rng(3)
    n = 60
    E = 1.0 + rng.random(n)
    D = 0.1 + rng.random(n)
    E_bc = {(0, 0): np.array(0.7), (0, 1): np.array(1.9)}
    want = F.diffuse(E, D, (0.05,), bc, E_bc, 0.01, method="lu")
    np.testing.assert_allclose(R.diffuse_1d(E, D, 0.05, bc, E_bc, 0.01), want, rtol=1e-13)


@pytest.mark.parametrize("case", ["table2_weak", "table3_strong"])
@pytest.mark.parametrize("kind", ["fast", "slow"])
def test_spatial_damping_matches_printed_damping_per_length(case, kind):
    # the wave driven at omega = k c_ms (isothermal magnetosonic speed) decays as
    # exp(-Im k x); the paper prints omega_Im / (omega_Re / k) for the same modes
    bg = _bg(case)
    wv = _wave(case, 40, 1, kind)
    k = R.spatial_damping(bg, wv.omega, bg["k"])
    assert k.imag == pytest.approx(GOLD[case]["damping_per_length_" + kind], rel=3e-3)
    assert k.real == pytest.approx(bg["k"], rel=3e-3)


def test_ideal_mhd_fast_wave_travels_at_its_speed():
    # radiation off, adiabatic eigenmode: after 5.5 wavelengths of travel the profile
    # behind the front is the analytic wave, up to the scheme's small numerical damping
    bg = _bg("table3_strong")
    wv = _wave("table3_strong", 280, 7, "fast", radiation=False)
    U, t, _ = wv.run(5.5 * wv.lam / wv.phase_speed)
    assert wv.damping(U, 1, 5) * wv.lam < 0.05
    W = R.primitive(U, wv.Bx, wv.gamma)
    d = W[R.RHO] - bg["rho0"]
    for j in range(1, 5):                      # phase of each wavelength against the wave
        s = slice(40 * j, 40 * (j + 1))
        arg = wv.k * wv.x[s] - wv.omega * t
        phase = np.arctan2(np.sum(d[s] * np.cos(arg)), np.sum(d[s] * np.sin(arg)))
        assert abs(phase) < 0.1, (j, phase)


def test_radiation_leaves_the_alfven_wave_alone():
    # the Alfven pair decouples from the radiative terms (Appendix B): with and without
    # radiation the transverse velocity profiles agree, and rho, p, E stay unperturbed
    bg = _bg("table3_strong")
    out = []
    for rad in (True, False):
        wv = _wave("table3_strong", 200, 5, "alfven", radiation=rad)
        U, _, _ = wv.run(3.5 * wv.lam / wv.phase_speed)
        out.append(R.primitive(U, wv.Bx, wv.gamma))
    np.testing.assert_allclose(out[0][R.VY], out[1][R.VY], rtol=0, atol=1e-3 * wv.hat[R.VY])
    assert np.max(np.abs(out[0][R.ER] / bg["E0"] - 1.0)) < 1e-5
    assert np.max(np.abs(out[0][R.RHO] / bg["rho0"] - 1.0)) < 1e-4


def test_radiative_fast_wave_damping_converges_to_the_dispersion_relation():
    # strongly radiative fast wave (Table 3): the measured spatial damping approaches Im k
    # of the Appendix-B matrix at first order in dt (the backward-Euler FLD substep lags
    # the diffusion's response by O(D k^2 dt)); the Richardson value from CFL 0.2 and 0.1
    # lands within the hyperbolic scheme's own numerical damping at 40 cells per wavelength
    bg = _bg("table3_strong")
    rates = []
    for cfl in (0.2, 0.1):
        wv = _wave("table3_strong", 280, 7, "fast", cfl=cfl)
        U, _, _ = wv.run(5.5 * wv.lam / wv.phase_speed)
        rates.append(wv.damping(U, 1, 5))
    exact = R.spatial_damping(bg, wv.omega, bg["k"]).imag
    e0, e1 = rates[0] - exact, rates[1] - exact
    assert e0 > e1 > 0
    assert 1.5 < e0 / e1 < 2.5
    assert (2.0 * rates[1] - rates[0]) / exact == pytest.approx(1.0, abs=0.06)


def test_ars3_scheme_damping_converges_and_beats_the_split():
    # the same wave with the ARS3 IMEX scheme of Sect. 3 (hyperbolic and coupling terms
    # explicit, the FLD substep as its implicit stages): once the hyperbolic scheme's own
    # damping (the same grid without radiation) is taken off, the error against Im k is
    # ~9 % at CFL 0.8 and ~3 % at CFL 0.4 on 40 cells per wavelength, where the first-order
    # split misses by ~90 % and ~40 %: halving dt cuts the ARS3 error at least twofold
    bg = _bg("table3_strong")
    P = I.wave1d(GOLD["table3_strong"]["background"], 280, 7, "fast")
    t_end = 5.5 * P.lam / P.phase_speed
    exact = R.spatial_damping(bg, P.omega, bg["k"]).imag
    Pi = I.wave1d(GOLD["table3_strong"]["background"], 280, 7, "fast", radiation=False)
    oi = R.Wave(Pi, cfl=0.8, scheme="ars3")
    Ui, _, _ = oi.run(t_end)
    k_num = oi.damping(Ui, 1, 5)
    errs = {}
    for scheme in ("ars3", "split"):
        for cfl in (0.8, 0.4):
            wv = R.Wave(P, cfl=cfl, scheme=scheme)
            U, _, _ = wv.run(t_end)
            errs[scheme, cfl] = abs((wv.damping(U, 1, 5) - k_num) / exact - 1.0)
    assert errs["ars3", 0.4] < 0.5 * errs["ars3", 0.8] < 0.06
    assert errs["ars3", 0.8] < 0.2 * errs["split", 0.8]
    assert errs["ars3", 0.4] < 0.2 * errs["split", 0.4]
