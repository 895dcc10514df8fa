"""Pins of the oracle's linear-mode tool against the numbers printed in Sect. 4.3
(Tables 2 and 3, damping lengths) and the octic of Appendix B."""
import json
import os

import numpy as np
import pytest

from oracle import dispersion as Disp

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _bg(case):
    b = GOLD[case]["background"]
    return Disp.background(b["rho0"], b["p0"], b["B0_gauss"], b["gamma"], b["mu"], b["kappa"],
                           tau=b["tau"])


def _pick(w, re, im):
    """Eigenvalue closest to re + i im (positive-real branch of each pair)."""
    return w[np.argmin(np.abs(w - complex(re, im)))]


@pytest.mark.parametrize("case,tol_slow_fast,tol_rad", [("table2_weak", 2e-5, 5e-4),
                                                        ("table3_strong", 5e-4, 5e-4)])
def test_tables_2_and_3(case, tol_slow_fast, tol_rad):
    g = GOLD[case]
    w = Disp.eigenfrequencies(_bg(case))
    for mode in ("fast", "slow"):
        re, im = g[mode]
        got = _pick(w, re, im)
        assert got.real == pytest.approx(re, rel=2e-5)
        assert got.imag == pytest.approx(im, rel=tol_slow_fast)
    got = _pick(w, *g["alfven"])
    assert got.real == pytest.approx(g["alfven"][0], rel=2e-5) and abs(got.imag) < 1e-15
    got = _pick(w, *g["thermal"])
    assert got.imag == pytest.approx(g["thermal"][1], rel=2e-5)
    got = _pick(w, *g["radiative_diffusion"])
    assert got.imag == pytest.approx(g["radiative_diffusion"][1], rel=tol_rad)
    # every mode decays or is neutral
    assert np.all(w.imag < 1e-15)


def test_background_numbers():
    bg = _bg("table2_weak")
    g = GOLD["table2_weak"]
    assert bg["E0"] == pytest.approx(g["E0"], rel=1e-5)
    assert 2 * np.pi / bg["k"] == pytest.approx(g["lambda_w"], rel=1e-5)
    assert bg["k"] == pytest.approx(g["k"], rel=1e-5)
    assert _bg("table3_strong")["E0"] == pytest.approx(GOLD["table3_strong"]["E0"], rel=1e-5)


@pytest.mark.parametrize("case,tol", [("table2_weak", 2e-5), ("table3_strong", 5e-4)])
def test_damping_lengths(case, tol):
    # omega_Im / (isothermal ideal-MHD fast/slow speed), Sect. 4.3
    g = GOLD[case]
    bg = _bg(case)
    w = Disp.eigenfrequencies(bg)
    for mode, key, fast in (("fast", "damping_per_length_fast", True),
                            ("slow", "damping_per_length_slow", False)):
        wi = -_pick(w, *g[mode]).imag
        assert wi / Disp.magnetosonic_speed(bg, fast) == pytest.approx(g[key], rel=tol)


def test_alfven_pair_is_kvax():
    bg = _bg("table2_weak")
    w = Disp.eigenfrequencies(bg)
    vax = np.sqrt(Disp.char_speeds(bg)[3])
    for s in (1, -1):
        assert _pick(w, s * bg["k"] * vax, 0).real == pytest.approx(s * bg["k"] * vax, rel=1e-12)


@pytest.mark.parametrize("case", ["table2_weak", "table3_strong"])
def test_octic_roots_equal_matrix_eigenvalues(case):
    # The printed octic (with q_Tr in the omega^1 bracket) and the 8x8 system agree.
    bg = _bg(case)
    w = np.sort_complex(Disp.eigenfrequencies(bg))
    r = np.sort_complex(np.roots(Disp.octic(bg)))
    scale = np.abs(w)
    for wi in w:
        j = np.argmin(np.abs(r - wi))
        assert abs(r[j] - wi) <= 1e-6 * max(abs(wi), 1e-6 * scale.max())


def test_hydro_frozen_block_close_to_full_modes():
    for case in ("table2_weak", "table3_strong"):
        bg = _bg(case)
        fr = Disp.hydro_frozen(bg)
        g = GOLD[case]
        rad = fr[np.argmin(fr.imag)]
        assert rad.imag == pytest.approx(g["radiative_diffusion"][1], rel=5e-4)


@pytest.mark.parametrize("ratio", [0.1, 1.0])
def test_substep_generator_is_hydro_frozen_block(ratio):
    # The continuum generator behind the substep's amplification matrix,
    # c kappa rho [[-beta, 1], [beta, -1]] - diag(0, D k^2), has the eigenvalues of the
    # (p, E) block of the Appendix-B system (rho_1 = v_1 = B_1 = 0): the gas energy and
    # pressure differ by the constant factor gamma - 1. Code units of the linear-mode
    # workload: rho = T0 = R_gas = 1, c = kappa = 1e4, a_r = 3 x ratio.
    a_r, c, kap, gam = 3.0 * ratio, 1e4, 1e4, 5.0 / 3.0
    bg = dict(rho0=1.0, p0=1.0, B=np.zeros(3), gamma=gam, mu=1.0, kappa=kap, T0=1.0,
              E0=a_r, k=2 * np.pi, c=c, a_r=a_r)
    frozen = np.sort(Disp.hydro_frozen(bg).imag)
    beta = 4 * a_r / (1.0 / (gam - 1))
    D = c / (3 * kap)
    J = c * kap * np.array([[-beta, 1.0], [beta, -1.0]]) - np.diag([0, D * (2 * np.pi) ** 2])
    # the small rate is a difference of O(1e9) numbers: relative rounding ~1e-8
    assert np.allclose(np.sort(np.linalg.eigvals(J).real), frozen, rtol=1e-7)


# ---------------------------------------------------------------- the 3D linear-mode seed
@pytest.mark.parametrize("case", ["table2_weak", "table3_strong"])
def test_fast_mode_is_the_printed_fast_eigenvalue(case):
    # fast_mode picks the forward fast wave: on the paper's two backgrounds its frequency
    # is the printed fast eigenvalue of Table 2 / Table 3
    w, u = Disp.fast_mode(_bg(case))
    re, im = GOLD[case]["fast"]
    assert w.real == pytest.approx(re, rel=2e-5)
    assert w.imag == pytest.approx(im, rel=5e-4)


@pytest.mark.parametrize("ratio", [0.1, 1.0])
def test_fast_mode_eigenpair_code_units(ratio):
    bg = Disp.code_units_background(ratio)
    M = Disp.mode_matrix(bg)
    w, u = Disp.fast_mode(bg)
    # an eigenpair of the Appendix-B matrix, scaled to a unit relative density amplitude
    # (M spans 1 to 1e9: the eigensolver's backward error is ~1e-12 of its norm)
    assert np.linalg.norm(M @ u - w * u) <= 1e-10 * np.linalg.norm(M) * np.linalg.norm(u)
    assert u[0] == bg["rho0"]
    # the forward fast wave: a root of the octic, the largest real part of all modes
    r = np.roots(Disp.octic(bg))
    assert np.min(np.abs(r - w)) <= 1e-6 * abs(w)     # the octic's roots to its conditioning
    assert w.real >= np.max(Disp.eigenfrequencies(bg).real) * (1 - 1e-12)
    # slower than light-speed-free ideal MHD would allow and damped
    assert w.imag < 0
    # optically thick (kappa rho L = 1e4): radiation locked to the gas, E_1/E0 = 4 T_1/T0
    # up to the exchange lag O(omega / (c kappa rho)) ~ 1e-7
    T1 = Disp.gas_temperature_amplitude(bg, u)
    assert abs(u[7] / bg["E0"] - 4 * T1 / bg["T0"]) <= 1e-5 * abs(u[7] / bg["E0"])
    # B at 45 degrees to k in the x-z plane: no y components
    assert abs(u[2]) < 1e-10 and abs(u[5]) < 1e-10


@pytest.mark.parametrize("ratio", [0.1, 1.0])
def test_stored_linmode_amplitudes(ratio):
    # the recipe's stored eigenmode (linmode_eigen.json) is the oracle's, recomputed
    from oracle import write_linmode_eigen as W
    from paper_2503_02764_gb300 import inputs as I
    a = W.amplitudes(ratio)
    T1, E1 = I.linmode_amplitudes(ratio)
    assert T1 == pytest.approx(complex(*a["T1"]), rel=1e-12)
    assert E1 == pytest.approx(complex(*a["E1"]), rel=1e-12)


@pytest.mark.parametrize("ratio", [0.1, 1.0])
def test_hydro_frozen_slow_rate_is_effective_diffusion(ratio):
    # with the gas held (rho_1 = v_1 = B_1 = 0) and radiation locked to it, energy diffuses
    # at D k^2 times the radiation's share of the heat capacity,
    # f = (4 E0/T0) / (p0/((gamma - 1) T0) + 4 E0/T0), up to O(D k^2 / (c kappa rho))
    bg = Disp.code_units_background(ratio)
    slow = Disp.hydro_frozen(bg)
    slow = slow[np.argmax(slow.imag)]
    D = bg["c"] / (3 * bg["kappa"] * bg["rho0"])
    f = 4 * bg["E0"] / (bg["p0"] / (bg["gamma"] - 1) + 4 * bg["E0"])
    assert abs(slow.real) < 1e-6 * abs(slow)
    assert -slow.imag == pytest.approx(D * bg["k"] ** 2 * f, rel=1e-6)


@pytest.mark.parametrize("ratio", [0.1, 1.0])
def test_substep_decay_tracks_hydro_frozen_rate(ratio):
    # the split substep's amplification G (dt = 1e-3, 512 cells) on the radiation-locked
    # direction: the diffusion removes a / (1 + a) of E_1 (a = dt D ktilde^2), the exchange
    # shares the loss of total energy back so that the radiation keeps its share f of the
    # heat capacity, so the slow eigenvalue is 1 - f a / (1 + a) (up to O(a / chi),
    # chi = dt c kappa rho = 1e5). Over N steps it follows the continuum exp(-N dt f D k^2)
    # of the hydro-frozen rate to the scheme's first-order error N f a^2 (1 - f/2).
    bg = Disp.code_units_background(ratio)
    dt, N, n = 1e-3, 100, 512
    D = bg["c"] / (3 * bg["kappa"] * bg["rho0"])
    k2 = Disp.discrete_k2(bg["k"], 1.0 / n)
    G = Disp.substep_amplification(dt, bg["c"], bg["kappa"], bg["rho0"], bg["a_r"], bg["T0"],
                                   bg["gamma"], bg["R_gas"], D, k2)
    g = np.linalg.eigvals(G)
    gs = g[np.argmax(np.abs(g))].real
    f = 4 * bg["E0"] / (bg["p0"] / (bg["gamma"] - 1) + 4 * bg["E0"])
    a = dt * D * k2
    assert gs == pytest.approx(1.0 - f * a / (1.0 + a), rel=1e-6)
    lam = -np.max(Disp.hydro_frozen(bg).imag)
    cont = np.exp(-N * dt * lam)
    err = N * f * a * a * (1 - f / 2) * cont
    assert 0.8 * err <= gs ** N - cont <= 1.2 * err
