"""Pins of the oracle's limiter (Eqs. fld_lambda, fld_R, fld_F, fld_f; Sect. 3 gradient).

Each check is fixed by the paper or by mathematics, not by the oracle itself.
"""
import numpy as np
import pytest

from oracle import fld as O


def test_lambda_special_values():
    # Eq. fld_lambda: lambda(0) = 2/6, lambda(1) = 3/10, lambda(2) = 4/16
    assert O.lp_lambda(0.0) == pytest.approx(1.0 / 3.0, rel=1e-16)
    assert O.lp_lambda(1.0) == pytest.approx(0.3, rel=1e-16)
    assert O.lp_lambda(2.0) == pytest.approx(0.25, rel=1e-16)
    # free-streaming limit (text after Eq. fld_R): lambda -> 1/R, |F| -> c E
    for R in (1e4, 1e6, 1e9):
        assert O.lp_lambda(R) * R == pytest.approx(1.0, rel=2.0 / R)


def test_lambda_invariants():
    rng = np.random.default_rng(1)
    R = np.sort(10.0 ** rng.uniform(-8, 8, 1_000_000))
    lam = O.lp_lambda(R)
    assert np.all(np.diff(lam) <= 4e-16 * lam[1:])   # monotone decreasing (to rounding;
    # lambda is flat at R = 0, so neighbours can differ by an ulp either way)
    assert np.all(lam * R < 1.0)              # flux never exceeds c E
    assert np.all(lam <= 1.0 / 3.0 + 1e-16)
    f = O.eddington_factor(lam, R)            # Eq. fld_f: thick 1/3 .. thin 1
    assert np.all(f >= 1.0 / 3.0 - 1e-15) and np.all(f <= 1.0)
    assert O.eddington_factor(O.lp_lambda(1e-9), 1e-9) == pytest.approx(1.0 / 3.0, rel=1e-8)
    assert O.eddington_factor(O.lp_lambda(1e9), 1e9) == pytest.approx(1.0, rel=1e-8)


@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_gradient_exact_for_quartics_in_interior(deg):
    # The 5-point 4th-order central difference (Sect. 3, Fornberg) is exact for
    # polynomials of degree <= 4; check every interior cell (2 away from a wall).
    n, h = 23, 0.37
    x = (np.arange(n) + 0.5) * h
    coef = np.arange(1, deg + 2) * 0.7
    E = np.polyval(coef, x)
    dE = np.polyval(np.polyder(coef), x) if deg > 0 else np.zeros(n)
    g = O.gradient5(E, (h,), ((1, 1),), {})[0]
    scale = np.abs(dE).max() + 1.0
    assert np.max(np.abs(g[2:-2] - dE[2:-2])) / scale < 1e-13


@pytest.mark.parametrize("kind", ["periodic", "neumann", "dirichlet"])
def test_gradient_fourth_order_with_ghosts(kind):
    # Boundary ghosts: periodic wrap, even mirror (Neumann) for a field even about
    # the wall, odd reflection (Dirichlet) for a field odd about the wall value.
    # With the right ghost rule the error is O(h^4) everywhere, walls included.
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        if kind == "periodic":
            E, dE, bc, Eb = np.sin(2 * np.pi * x), 2 * np.pi * np.cos(2 * np.pi * x), ((0, 0),), {}
        elif kind == "neumann":
            E, dE, bc, Eb = np.cos(np.pi * x), -np.pi * np.sin(np.pi * x), ((1, 1),), {}
        else:
            E = 2.0 + np.sin(np.pi * x)
            dE = np.pi * np.cos(np.pi * x)
            bc, Eb = ((2, 2),), {(0, 0): np.array(2.0), (0, 1): np.array(2.0)}
        g = O.gradient5(E, (h,), bc, Eb)[0]
        errs.append(np.max(np.abs(g - dE)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 3.7), orders


def test_limiter_linear_field_closed_form():
    # E linear in 3D: the 5-point gradient is exact in the interior, so
    # R = |g| / (kappa rho E) and D = c lambda(R) / (kappa rho) in closed form.
    nz, ny, nx = 9, 10, 11
    h = (0.1, 0.2, 0.3)
    g = np.array([0.3, -0.2, 0.5])
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) * hh for n, hh in zip((nz, ny, nx), h[::-1])],
                          indexing="ij")
    E = 5.0 + g[0] * x + g[1] * y + g[2] * z
    rng = np.random.default_rng(3)
    rho = 10 ** rng.uniform(-1, 1, E.shape)
    T = 10 ** rng.uniform(-0.5, 0.5, E.shape)
    op = (1, 0.7, 1.0, -3.5)
    bc = ((1, 1),) * 3
    D, lam, R = O.limiter(E, rho, T, h, bc, {}, 2.5, op)
    kap = 0.7 * rho * T ** -3.5
    Rx = np.linalg.norm(g) / (kap * rho * E)
    Dx = 2.5 * (2 + Rx) / (6 + 3 * Rx + Rx ** 2) / (kap * rho)
    inner = (slice(2, -2),) * 3
    assert np.max(np.abs(D[inner] / Dx[inner] - 1)) < 1e-13
    # diffusion-limit mode: lambda = 1/3 everywhere
    D3, lam3, _ = O.limiter(E, rho, T, h, bc, {}, 2.5, op, mode=1)
    assert np.allclose(D3, 2.5 / (3 * kap * rho), rtol=1e-15)


def test_limiter_flat_field_is_diffusion_limit():
    E = np.full((6, 7), 3.0)
    rho = np.full((6, 7), 2.0)
    D, lam, R = O.limiter(E, rho, E, (1.0, 1.0), ((0, 0), (0, 0)), {}, 1.0, (0, 4.0, 0, 0))
    assert np.all(R == 0) and np.all(lam == 1.0 / 3.0)
    assert np.allclose(D, 1.0 / (3 * 8.0), rtol=1e-16)


def test_limiter_symmetry():
    # transposing the inputs (with h and bc swapped) transposes the output
    rng = np.random.default_rng(5)
    E = 1 + rng.uniform(0, 1, (12, 17))
    rho = 1 + rng.uniform(0, 1, (12, 17))
    bc = ((0, 0), (1, 2))
    Eb = {(1, 1): np.full(17, 1.5)}
    D, _, _ = O.limiter(E, rho, rho, (0.3, 0.7), bc, Eb, 1.0, (0, 2.0, 0, 0))
    Dt, _, _ = O.limiter(E.T.copy(), rho.T.copy(), rho.T.copy(), (0.7, 0.3), (bc[1], bc[0]),
                         {(0, 1): np.full(17, 1.5)}, 1.0, (0, 2.0, 0, 0))
    assert np.allclose(D, Dt.T, rtol=1e-15, atol=0)
    # mirror in x with swapped boundary sides
    Dm, _, _ = O.limiter(E[:, ::-1].copy(), rho[:, ::-1].copy(), rho[:, ::-1].copy(), (0.3, 0.7),
                         bc, Eb, 1.0, (0, 2.0, 0, 0))
    assert np.allclose(D, Dm[:, ::-1], rtol=1e-14, atol=0)


def test_limiter_rejects_nonpositive():
    E = np.ones(8)
    E[3] = -1.0
    with pytest.raises(ValueError):
        O.limiter(E, np.ones(8), np.ones(8), (1.0,), ((0, 0),), {}, 1.0, (0, 1.0, 0, 0))


def test_minerbo_limiter_pins():
    # the published closed form: lambda(0) = 1/3; the two branches meet at R = 3/2 with the
    # value 2/9 and the same slope; lambda R -> 1 as R -> infinity; lambda R < 1
    assert O.minerbo_lambda(0.0) == pytest.approx(1.0 / 3.0, rel=1e-15)
    lo = lambda R: 2.0 / (3.0 + np.sqrt(9.0 + 12.0 * R * R))
    hi = lambda R: 1.0 / (1.0 + R + np.sqrt(1.0 + 2.0 * R))
    assert lo(1.5) == pytest.approx(2.0 / 9.0, rel=1e-15)
    assert hi(1.5) == pytest.approx(2.0 / 9.0, rel=1e-15)
    eps = 1e-6
    slope_lo = (lo(1.5) - lo(1.5 - eps)) / eps
    slope_hi = (hi(1.5 + eps) - hi(1.5)) / eps
    assert slope_lo == pytest.approx(slope_hi, rel=1e-4)
    R = np.logspace(-6, 9, 500)
    lam = O.minerbo_lambda(R)
    assert np.all(lam * R < 1.0) and np.all(np.diff(lam) < 0)
    assert abs(O.minerbo_lambda(1e9) * 1e9 - 1.0) < 1e-4
    # both limiters agree at the two ends and differ in between
    assert abs(O.minerbo_lambda(1e-8) - O.lp_lambda(1e-8)) < 1e-8
    assert abs(O.minerbo_lambda(1.0) - O.lp_lambda(1.0)) > 1e-3


def test_limiter_mode_minerbo_in_the_field():
    rng = np.random.default_rng(4)
    E = 1.0 + rng.uniform(0, 1, (6, 9))
    rho = np.full(E.shape, 0.3)
    T = np.ones(E.shape)
    bc = ((0, 0), (1, 1))
    D, lam, R = O.limiter(E, rho, T, (0.1, 0.1), bc, {}, 2.0, (0, 1.0, 0.0, 0.0), mode=2)
    np.testing.assert_allclose(lam, O.minerbo_lambda(R), rtol=1e-15)
    np.testing.assert_allclose(D, 2.0 * lam / 0.3, rtol=1e-15)
