"""Pins of the oracle's implicit gas-radiation exchange (Eqs. heating, qdot;
Eqs. energy_density and ideal_gas_law for e(T); Sect. 3 for the implicit quartic)."""
import json
import os

import mpmath as mp
import numpy as np
import pytest

from oracle import fld as O
from oracle import dispersion as Disp
from paper_2503_02764_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
CONST = (0, 1.0, 0.0, 0.0)     # kappa supplied per cell below


def _bisect(f, lo, hi, n=250):
    """Root of an increasing f on [lo, hi] by bisection in mpmath arithmetic."""
    lo, hi = mp.mpf(lo), mp.mpf(hi)
    for _ in range(n):
        mid = (lo + hi) / 2
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    return (lo + hi) / 2


def _ex(rho, T, E, kappa, dt, c=1.0, a_r=1.0, gamma=5.0 / 3.0, R_gas=1.0):
    return O.exchange(rho, T, E, dt, c, a_r, gamma, R_gas, ("field", kappa))


def test_fixed_point_table1_states():
    # Table 1 states are in radiative equilibrium (T_g = T_r): E = a_r T^4 must not move.
    t1 = GOLD["table1_states"]
    R_gas = Disp.K_B / (t1["mu"] * Disp.M_P)
    for st in t1["states"]:
        rho, T = np.array([st["rho"]]), np.array([st["T"]])
        # the printed E is a_r T^4 to the printed digits (a_r = 4 sigma / c, Sect. 2)
        if "_note" not in st:
            assert Disp.A_RAD * st["T"] ** 4 == pytest.approx(st["E"], rel=2e-5)
        E = Disp.A_RAD * T ** 4
        for dt in (1e-12, 1e-3, 1e6):
            T2, E2 = O.exchange(rho, T, E, dt, Disp.C_LIGHT, Disp.A_RAD, st["gamma"], R_gas,
                                ("field", np.array([0.4])))
            assert abs(T2[0] / T[0] - 1) <= 4e-16 and abs(E2[0] / E[0] - 1) <= 8e-16


def test_dt_zero_and_infinite():
    mp.mp.dps = 40
    rho, T, E, kap = I.random_cells(2000, seed=1)
    T0, E0 = _ex(rho, T, E, kap, 0.0)
    assert np.array_equal(T0, T) and np.max(np.abs(E0 / E - 1)) < 1e-15
    # dt -> infinity: radiative equilibrium of the total, rho c_v T + a_r T^4 = e + E
    Ti, Ei = _ex(rho, T, E, kap, 1e30)
    cv = 1.0 / (2.0 / 3.0)
    for i in range(0, 2000, 97):
        S = mp.mpf(rho[i]) * cv * mp.mpf(T[i]) + mp.mpf(E[i])
        r = _bisect(lambda t: mp.mpf(rho[i]) * cv * t + t ** 4 - S, 0, S / (mp.mpf(rho[i]) * cv))
        assert abs(Ti[i] / float(r) - 1) < 1e-14
        assert abs(Ei[i] / float(r) ** 4 - 1) < 1e-13


def _ferrari_positive_root(p, q):
    """Positive root of x^4 + p x - q = 0 (p, q > 0) by Ferrari's method in mpmath."""
    # x^4 + p x - q = (x^2 + m)^2 - (2m x^2 - p x + m^2 + q); the bracket is a square
    # when its discriminant vanishes: m^3 + q m - p^2/8 = 0 (Cardano, one real root).
    a, b = q, -p * p / 8
    disc = mp.sqrt(b * b / 4 + a ** 3 / 27)
    def rcbrt(v):                       # real cube root
        return mp.sign(v) * mp.cbrt(abs(v))
    m = rcbrt(-b / 2 + disc) + rcbrt(-b / 2 - disc)
    s = mp.sqrt(2 * m)
    # x^2 + s x + m - p/(2s) = 0 carries the positive root
    return (-s + mp.sqrt(s * s - 4 * (m - p / (2 * s)))) / 2


def test_closed_form_ferrari():
    mp.mp.dps = 60
    rho, T, E, kap = I.random_cells(300, seed=2)
    dt = 10.0 ** np.random.default_rng(0).uniform(-6, 4, 300)
    cv = 1.5
    for i in range(300):
        T2, E2 = _ex(rho[i:i + 1], T[i:i + 1], E[i:i + 1], kap[i:i + 1], dt[i])
        chi = mp.mpf(dt[i]) * mp.mpf(kap[i]) * mp.mpf(rho[i])
        w = chi / (1 + chi)
        alpha = mp.mpf(rho[i]) * cv
        q = alpha * mp.mpf(T[i]) + w * mp.mpf(E[i])
        x = _ferrari_positive_root(alpha / w, q / w)
        assert abs(T2[0] / float(x) - 1) < 1e-15, (i, T2[0], x)
        Ex = (mp.mpf(E[i]) + chi * x ** 4) / (1 + chi)
        assert abs(E2[0] / float(Ex) - 1) < 2e-15


def test_bruteforce_bisection_wide_chi():
    # chi = dt c kappa rho over [1e-6, 1e12]; bisection in 40-digit arithmetic
    mp.mp.dps = 40
    rng = np.random.default_rng(7)
    n = 400
    rho = 10 ** rng.uniform(-2, 2, n)
    T = 10 ** rng.uniform(-1, 1, n)
    E = 10 ** rng.uniform(-3, 5, n)
    chi = 10 ** rng.uniform(-6, 12, n)
    kap = np.ones(n)
    dt = chi / rho
    for i in range(n):
        T2, _ = _ex(rho[i:i + 1], T[i:i + 1], E[i:i + 1], kap[i:i + 1], dt[i])
        c_ = mp.mpf(dt[i]) * mp.mpf(rho[i])
        w = c_ / (1 + c_)
        alpha = mp.mpf(rho[i]) * mp.mpf(1.5)
        q = alpha * mp.mpf(T[i]) + w * mp.mpf(E[i])
        lo, hi = mp.mpf(0), q / alpha
        for _ in range(200):
            mid = (lo + hi) / 2
            if w * mid ** 4 + alpha * mid - q > 0:
                hi = mid
            else:
                lo = mid
        assert abs(T2[0] / float(lo) - 1) < 1e-15


def test_conservation_per_cell():
    rho, T, E, kap = I.random_cells(5000, seed=3)
    T2, E2 = _ex(rho, T, E, kap, 0.37)
    e, e2 = O.internal_energy(rho, T, 5 / 3, 1.0), O.internal_energy(rho, T2, 5 / 3, 1.0)
    assert np.max(np.abs((e2 + E2) - (e + E)) / (e + E)) < 1e-14
    # the exchange moves both temperatures toward each other
    Tr = E ** 0.25
    assert np.all((T2 - T) * (Tr - T) >= 0)


def test_heatcool_equilibrium_and_relaxation():
    # Sect. 4.2: rho = 1e-7, kappa = 0.4, mu = 0.6, e + E = 1e12 (CGS).
    hc = GOLD["heatcool"]
    R_gas = Disp.K_B / (hc["mu"] * Disp.M_P)
    gam, rho, kap = hc["gamma"], hc["rho0"], hc["kappa"]
    cv = R_gas / (gam - 1)
    S = hc["e_plus_E"]
    # equilibrium with e = rho c_v T (Eq. energy_density): within 2% of the printed
    # e_equi (the text's formula omits 1/(gamma-1), which the printed number does not).
    Teq = float(_bisect(lambda t: rho * cv * t + Disp.A_RAD * t ** 4 - S, 0, S / (rho * cv)))
    e_eq = rho * cv * Teq
    assert e_eq == pytest.approx(hc["e_equi"], rel=0.02)
    # oracle with a huge dt lands on it
    e_i = 1e-2 * hc["e_equi"]
    T_i = e_i / (rho * cv)
    T2, E2 = O.exchange(np.array([rho]), np.array([T_i]), np.array([S - e_i]), 1e9,
                        Disp.C_LIGHT, Disp.A_RAD, gam, R_gas, ("field", np.array([kap])))
    assert rho * cv * T2[0] == pytest.approx(e_eq, rel=1e-12)
    # backward Euler converges at first order to the ODE de/dt = c kappa rho (S - e - a_r T(e)^4)
    from scipy.integrate import solve_ivp
    k = Disp.C_LIGHT * kap * rho

    def rhs(t, y):
        e = y[0]
        return [k * (S - e - Disp.A_RAD * (e / (rho * cv)) ** 4)]

    for e0 in (1e-2 * hc["e_equi"], 1e2 * hc["e_equi"]):
        tend = 3.0 / (k * (1 + 4 * Disp.A_RAD * Teq ** 3 / (rho * cv)))
        ref = solve_ivp(rhs, (0, tend), [e0], method="Radau", rtol=1e-13, atol=1e-3).y[0, -1]
        errs = []
        for nsteps in (40, 80, 160):
            T_, E_ = np.array([e0 / (rho * cv)]), np.array([S - e0])
            for _ in range(nsteps):
                T_, E_ = O.exchange(np.array([rho]), T_, E_, tend / nsteps, Disp.C_LIGHT,
                                    Disp.A_RAD, gam, R_gas, ("field", np.array([kap])))
            errs.append(abs(rho * cv * T_[0] - ref))
        orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert np.all((orders > 0.9) & (orders < 1.1)), orders


def test_rejects_nonpositive():
    with pytest.raises(ValueError):
        _ex(np.array([1.0]), np.array([-1.0]), np.array([1.0]), np.array([1.0]), 1.0)
