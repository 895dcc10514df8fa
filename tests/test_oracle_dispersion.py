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
