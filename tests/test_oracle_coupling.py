"""Pins of the oracle's explicit coupling terms (Sect. 3; Eqs. fld_F, rad_force, fld_f,
fld_Eddington_tensor, fld_P) against what the paper and the mathematics fix: the limits
of the Eddington factor, the unit trace of the Eddington tensor, the free-streaming bound
on the flux, the two forms of the radiation force, closed forms in the isotropic and
free-streaming limits, and exact gradients of linear fields."""
import numpy as np
import pytest

from oracle import fld as O

NEU = ((1, 1),)


def _fields(shape, seed, kappa=1.0):
    rng = np.random.default_rng(seed)
    E = 1.0 + rng.uniform(0, 1, shape)
    rho = 0.5 + rng.uniform(0, 1, shape)
    T = 1.0 + rng.uniform(0, 1, shape)
    v = [rng.standard_normal(shape) for _ in shape]
    return E, rho, T, v, (0, kappa, 0.0, 0.0)


def _bc_neumann(nd):
    return tuple((1, 1) for _ in range(nd))


def test_eddington_factor_values_and_limits():
    # f(R) = lambda + lambda^2 R^2 with lambda = (2 + R)/(6 + 3R + R^2): f(0) = 1/3,
    # f(1) = 3/10 + 9/100, f -> 1 as R -> infinity (lambda R -> 1, lambda -> 0)
    assert O.eddington_factor(O.lp_lambda(0.0), 0.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert O.eddington_factor(O.lp_lambda(1.0), 1.0) == pytest.approx(0.39, rel=1e-15)
    R = np.array([1e3, 1e5, 1e8])
    assert np.all(1.0 - O.eddington_factor(O.lp_lambda(R), R) < 3.0 / R)
    R = np.logspace(-6, 6, 400)
    f = O.eddington_factor(O.lp_lambda(R), R)
    assert np.all(f >= 1.0 / 3.0 - 1e-15) and np.all(f <= 1.0)
    assert np.all(np.diff(f) >= -1e-15)       # monotone from diffusion to free streaming


@pytest.mark.parametrize("kappa", [1e-3, 1.0, 1e3])
def test_tensor_trace_bound_and_force_forms(kappa):
    shape = (6, 7, 9)
    E, rho, T, v, op = _fields(shape, 3, kappa)
    h = (0.1, 0.12, 0.09)
    o = O.coupling(E, rho, T, h, _bc_neumann(3), {}, 2.0, op, v)
    P = o["P"]
    trace = sum(P[i][i] for i in range(3)) / E
    assert np.max(np.abs(trace - 1.0)) < 1e-14                     # tr f = 1
    for i in range(3):
        for j in range(3):
            assert np.max(np.abs(P[i][j] - P[j][i]) / E) < 1e-15    # symmetric
    Fmag = np.sqrt(sum(Fi * Fi for Fi in o["F"]))
    assert np.all(Fmag <= 2.0 * E * (1 + 1e-14))                   # |F| <= c E
    kap = O.opacity(op, rho, T)
    for d in range(3):                                              # f_r = rho kappa F / c
        np.testing.assert_allclose(o["fr"][d], rho * kap * o["F"][d] / 2.0, rtol=1e-13,
                                   atol=1e-300)
    assert np.all(o["f"] >= 1.0 / 3.0 - 1e-15) and np.all(o["f"] <= 1.0)


def test_uniform_field_isotropic_closed_form():
    # grad E = 0: no flux, f = 1/3, P = E/3 I, P : grad v = (E/3) div v
    shape = (5, 6, 8)
    _, rho, T, v, op = _fields(shape, 5)
    E = np.full(shape, 2.5)
    h = (0.2, 0.25, 0.3)
    bc = ((0, 0), (0, 0), (0, 0))
    o = O.coupling(E, rho, T, h, bc, {}, 1.0, op, v)
    assert all(np.all(Fi == 0.0) for Fi in o["F"])
    assert np.all(o["f"] == 1.0 / 3.0)
    div = sum(O.gradient5(v[d], h, bc, {})[d] for d in range(3))
    np.testing.assert_allclose(o["ptire"], E / 3.0 * div, rtol=1e-13, atol=1e-13)


def test_linear_fields_interior_exact():
    # E linear in x (1D): the 5-point gradient is exact away from the walls, so
    # F = -D s, f_r = -lambda s; v = a x gives P : grad v = P_xx a = f E a
    n, hx, s, a = 40, 0.05, 0.3, 1.7
    x = (np.arange(n) + 0.5) * hx
    E = 2.0 + s * x
    rho = np.full(n, 1.3)
    T = np.ones(n)
    op = (0, 2.0, 0.0, 0.0)
    o = O.coupling(E, rho, T, (hx,), NEU, {}, 1.0, op, [a * x])
    D, lam, R = O.limiter(E, rho, T, (hx,), NEU, {}, 1.0, op)
    inner = slice(2, n - 2)
    np.testing.assert_allclose(o["F"][0][inner], -D[inner] * s, rtol=1e-13)
    np.testing.assert_allclose(o["fr"][0][inner], -lam[inner] * s, rtol=1e-13)
    # R from its definition, |grad E| / (kappa rho E)
    np.testing.assert_allclose(R[inner], s / (2.0 * 1.3 * E[inner]), rtol=1e-13)
    np.testing.assert_allclose(o["ptire"][inner], o["f"][inner] * E[inner] * a, rtol=1e-13)


def test_free_streaming_limit():
    # kappa rho -> 0: f -> 1 and P -> E n n, so P : grad v -> E n . (grad v) n
    shape = (4, 6, 7)
    E, rho, T, v, _ = _fields(shape, 9)
    h = (0.1, 0.1, 0.1)
    bc = _bc_neumann(3)
    o = O.coupling(E, rho, T, h, bc, {}, 1.0, (0, 1e-9, 0.0, 0.0), v)
    assert np.all(o["f"] > 1 - 1e-6)
    g = O.gradient5(E, h, bc, {})
    gn = np.sqrt(sum(gi * gi for gi in g))
    n = [gi / gn for gi in g]
    gv = [O.gradient5(v[i], h, bc, {}) for i in range(3)]
    proj = E * sum(n[i] * gv[i][j] * n[j] for i in range(3) for j in range(3))
    np.testing.assert_allclose(o["ptire"], proj, rtol=1e-5, atol=1e-8 * np.max(np.abs(proj)))


def test_force_work_sign_against_the_gradient():
    # v antiparallel to grad E: v . f_r = lambda |grad E| |v| >= 0
    shape = (6, 8)
    E, rho, T, _, op = _fields(shape, 11)
    h = (0.1, 0.1)
    bc = _bc_neumann(2)
    g = O.gradient5(E, h, bc, {})
    v = [-gi for gi in g]
    o = O.coupling(E, rho, T, h, bc, {}, 1.0, op, v)
    D, lam, R = O.limiter(E, rho, T, h, bc, {}, 1.0, op)
    np.testing.assert_allclose(o["vfr"], lam * (g[0] ** 2 + g[1] ** 2), rtol=1e-13)
    assert np.all(o["vfr"] >= 0)
