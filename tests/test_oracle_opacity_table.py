"""Pins of the oracle's tabulated opacity (the opacity tables the paper names as the next
step, Sect. 5): bilinear interpolation of log10 kappa on a uniform (log10 rho, log10 T)
grid, clamped at the table's edges. Checked against scipy's regular-grid interpolator,
against fields the bilinear interpolant reproduces exactly (power laws and bilinear
functions of the logs), at the nodes, across cell boundaries and outside the table."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I

GRID = (-2.0, 0.1, -0.1, 0.05)      # log_rho0, dlog_rho, log_T0, dlog_T


def _nodes(n_rho, n_T, grid=GRID):
    lr = grid[0] + grid[1] * np.arange(n_rho)
    lt = grid[2] + grid[3] * np.arange(n_T)
    return lr, lt


def _inside(rng, n, n_rho, n_T, grid=GRID):
    lr, lt = _nodes(n_rho, n_T, grid)
    return 10.0 ** rng.uniform(lr[0], lr[-1], n), 10.0 ** rng.uniform(lt[0], lt[-1], n)


def test_matches_scipy_regular_grid_interpolator():
    interp = pytest.importorskip("scipy.interpolate")
    table, grid = I.opacity_table(3.0e4)
    n_T, n_rho = table.shape
    lr, lt = _nodes(n_rho, n_T, grid)
    rng = np.random.default_rng(1)
    # inside the table and beyond every edge
    rho = 10.0 ** rng.uniform(lr[0] - 0.5, lr[-1] + 0.5, 20000)
    T = 10.0 ** rng.uniform(lt[0] - 0.5, lt[-1] + 0.5, 20000)
    ref = interp.RegularGridInterpolator((lt, lr), table, method="linear")
    pts = np.stack([np.clip(np.log10(T), lt[0], lt[-1]),
                    np.clip(np.log10(rho), lr[0], lr[-1])], axis=-1)
    want = 2.5 * 10.0 ** ref(pts)
    got = O.opacity_table(2.5, table, grid, rho, T)
    np.testing.assert_allclose(got, want, rtol=1e-13)


def test_bilinear_log_fields_are_reproduced_exactly():
    # log10 kappa = a + b X + c Y + d X Y (X = log10 rho, Y = log10 T) is bilinear, so its
    # interpolant from the nodes equals it everywhere inside; d != 0 tests the cross weights
    n_rho, n_T = 13, 9
    lr, lt = _nodes(n_rho, n_T)
    a, b, c, d = 0.7, 1.3, -2.9, 0.45
    X, Y = np.meshgrid(lr, lt, indexing="xy")
    table = a + b * X + c * Y + d * X * Y
    rho, T = _inside(np.random.default_rng(2), 5000, n_rho, n_T)
    Xs, Ys = np.log10(rho), np.log10(T)
    got = np.log10(O.opacity_table(1.0, table, GRID, rho, T))
    np.testing.assert_allclose(got, a + b * Xs + c * Ys + d * Xs * Ys, rtol=0, atol=1e-12)


@pytest.mark.parametrize("a_rho,a_T", [(1.0, -3.5), (0.5, 2.0), (0.0, 0.0)])
def test_power_law_table_equals_the_power_law(a_rho, a_T):
    n_rho, n_T = 17, 21
    lr, lt = _nodes(n_rho, n_T)
    kappa0 = 40.0
    X, Y = np.meshgrid(lr, lt, indexing="xy")
    table = np.log10(kappa0) + a_rho * X + a_T * Y
    rho, T = _inside(np.random.default_rng(3), 5000, n_rho, n_T)
    got = O.opacity((2, 1.0, table, GRID), rho, T)
    np.testing.assert_allclose(got, O.opacity((1, kappa0, a_rho, a_T), rho, T), rtol=1e-13)


def test_node_values_and_continuity_across_cells():
    table, grid = I.opacity_table(1.0, n_rho=8, n_T=6)
    n_T, n_rho = table.shape
    lr, lt = _nodes(n_rho, n_T, grid)
    R, Tt = np.meshgrid(10.0 ** lr, 10.0 ** lt, indexing="xy")
    np.testing.assert_allclose(O.opacity_table(1.0, table, grid, R, Tt), 10.0 ** table,
                               rtol=1e-14)
    # just below and just above every interior rho node, at an off-node T
    eps = 1e-11
    T = np.full(n_rho - 2, 10.0 ** (lt[2] + 0.3 * grid[3]))
    lo = O.opacity_table(1.0, table, grid, 10.0 ** (lr[1:-1] - eps), T)
    hi = O.opacity_table(1.0, table, grid, 10.0 ** (lr[1:-1] + eps), T)
    np.testing.assert_allclose(lo, hi, rtol=1e-8)


def test_clamped_outside_the_table():
    table, grid = I.opacity_table(1.0, n_rho=8, n_T=6)
    n_T, n_rho = table.shape
    lr, lt = _nodes(n_rho, n_T, grid)
    T = np.array([10.0 ** (lt[0] + 0.37 * grid[3])] * 3)
    far = O.opacity_table(1.0, table, grid, np.array([1e-30, 1e-5, 10.0 ** (lr[0] - 1e-3)]), T)
    edge = O.opacity_table(1.0, table, grid, np.full(3, 10.0 ** lr[0]), T)
    np.testing.assert_allclose(far, edge, rtol=1e-14)
    # above the top corner: the corner node
    top = O.opacity_table(1.0, table, grid, np.array([1e30]), np.array([1e30]))
    assert top[0] == pytest.approx(10.0 ** table[-1, -1], rel=1e-14)


def test_axis_order_matters():
    # rho runs along the table's last axis: a table that rises only with rho must give an
    # opacity that rises with rho and ignores T
    n_rho, n_T = 6, 5
    lr, lt = _nodes(n_rho, n_T)
    table = np.tile(np.arange(n_rho, dtype=float), (n_T, 1))
    rho = 10.0 ** np.array([lr[1], lr[3]])
    for T in (10.0 ** lt[0], 10.0 ** lt[-1]):
        k = O.opacity_table(1.0, table, GRID, rho, np.full(2, T))
        np.testing.assert_allclose(k, [10.0, 1000.0], rtol=1e-14)


def test_table_workload_covers_interior_and_clamped_cells():
    P = I.stratified_3d_table()
    kind, kappa0, table, grid = P.opacity
    assert kind == I.OPACITY_TABLE and table.shape == (30, 24)
    x = (np.log10(P.rho) - grid[0]) / grid[1]
    y = (np.log10(P.T) - grid[2]) / grid[3]
    assert np.any(x < 0) and np.any((x > 0) & (x < table.shape[1] - 1))
    assert np.all((y > 0) & (y < table.shape[0] - 1))
    k = O.opacity(P.opacity, P.rho, P.T)
    assert np.all(np.isfinite(k)) and np.all(k > 0)
