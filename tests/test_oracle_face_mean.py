"""Pins of the oracle's harmonic face mean (face_mean="harm": w_f = 2 D_i D_j/(D_i + D_j)).
The closed form: in a layered medium between two Dirichlet walls the steady flux is that
of resistances h/D in series, and the cell-centre values of that piecewise-linear profile
satisfy the harmonic-mean discretisation exactly, so they are a fixed point of the
backward-Euler step for any dt (the arithmetic mean misses it, which the last test shows).
Also: constant D gives the arithmetic operator, the flux form stays symmetric and
conservative, and the matrix-free statement agrees with the assembled one."""
import numpy as np
import pytest

from oracle import fld as O


def _faces(shape, bc, value=1.0):
    nd = len(shape)
    return {(d, side): np.full(tuple(n for a, n in enumerate(shape) if a != nd - 1 - d), value)
            for d in range(nd) for side in (0, 1) if bc[d][side] == 2}


def _series_profile(D1, h, EL, ER):
    """cell-centre values of the steady profile through cells of conductivity D1 (wall at
    half a cell from the first and last centres), and its flux"""
    R = h / D1
    q = (EL - ER) / R.sum()
    before = np.concatenate(([0.0], np.cumsum(R)[:-1]))
    return EL - q * (before + 0.5 * R), q


@pytest.mark.parametrize("n,sigma", [(7, 0.5), (40, 1.5), (129, 2.5)])
def test_layered_steady_profile_is_a_fixed_point(n, sigma):
    rng = np.random.default_rng(n)
    D = np.exp(sigma * rng.standard_normal(n))
    h = 0.37
    E, _ = _series_profile(D, h, 3.0, 1.0)
    Eb = {(0, 0): np.array(3.0), (0, 1): np.array(1.0)}
    for dt in (0.1, 1e3, 1e8):
        x = O.diffuse(E, D, (h,), ((2, 2),), Eb, dt, method="lu", face_mean="harm")
        assert np.max(np.abs(x - E)) <= 1e-12 * 3.0, dt


def test_layered_profile_in_3d_with_periodic_tangential_axes():
    # D and E vary along x only; y and z periodic (no tangential flux)
    nx, ny, nz = 24, 5, 6
    rng = np.random.default_rng(3)
    Dx = np.exp(2.0 * rng.standard_normal(nx))
    h = (0.5, 0.8, 1.3)
    Ex, _ = _series_profile(Dx, h[0], 2.0, 5.0)
    D = np.broadcast_to(Dx, (nz, ny, nx)).copy()
    E = np.broadcast_to(Ex, (nz, ny, nx)).copy()
    bc = ((2, 2), (0, 0), (0, 0))
    Eb = {(0, 0): np.full((nz, ny), 2.0), (0, 1): np.full((nz, ny), 5.0)}
    x = O.diffuse(E, D, h, bc, Eb, 50.0, method="splu", face_mean="harm")
    assert np.max(np.abs(x - E)) <= 1e-12 * 5.0


def test_arithmetic_mean_misses_the_layered_profile():
    # the pin above discriminates: the arithmetic mean's step moves the series profile
    rng = np.random.default_rng(40)
    D = np.exp(1.5 * rng.standard_normal(40))
    E, _ = _series_profile(D, 0.37, 3.0, 1.0)
    Eb = {(0, 0): np.array(3.0), (0, 1): np.array(1.0)}
    x = O.diffuse(E, D, (0.37,), ((2, 2),), Eb, 1e3, method="lu", face_mean="arith")
    assert np.max(np.abs(x - E)) > 1e-2


def test_constant_D_gives_the_arithmetic_operator():
    D = np.full((6, 5, 7), 1.7)
    bc = ((2, 1), (0, 0), (1, 2))
    Eb = {(0, 0): np.ones((6, 5)), (2, 1): np.ones((5, 7))}
    A1, g1 = O.assemble(D, (0.3, 0.2, 0.4), bc, Eb, 0.9, "arith")
    A2, g2 = O.assemble(D, (0.3, 0.2, 0.4), bc, Eb, 0.9, "harm")
    assert abs(A1 - A2).max() <= 1e-15 * abs(A1).max()
    assert np.max(np.abs(g1 - g2)) == 0.0


@pytest.mark.parametrize("bc", [((0, 0), (0, 0)), ((1, 1), (0, 0)), ((2, 2), (1, 2))])
def test_symmetric_conservative_and_between_the_means(bc):
    rng = np.random.default_rng(9)
    shape = (9, 11)
    D = np.exp(2.0 * rng.standard_normal(shape))
    Eb = _faces(shape, bc)
    A, _ = O.assemble(D, (1.0, 1.0), bc, Eb, 0.4, "harm")
    Ad = A.toarray()
    assert np.max(np.abs(Ad - Ad.T)) <= 1e-15 * np.max(np.abs(Ad))
    assert np.min(np.linalg.eigvalsh(Ad)) >= 1 - 1e-12
    if all(b != 2 for side in bc for b in side):
        # no Dirichlet wall: column sums are one, so the step conserves sum(E)
        assert np.max(np.abs(Ad.sum(axis=0) - 1.0)) <= 1e-13
    # every off-diagonal coupling lies between the harmonic lower bound min(D) and the
    # arithmetic one
    Aa = O.assemble(D, (1.0, 1.0), bc, Eb, 0.4, "arith")[0].toarray()
    off = ~np.eye(Ad.shape[0], dtype=bool)
    assert np.all(-Ad[off] <= -Aa[off] + 1e-15)


def test_matrix_free_statement_agrees():
    rng = np.random.default_rng(5)
    shape = (5, 6, 7)
    D = np.exp(rng.standard_normal(shape))
    x = rng.uniform(0.5, 2.0, shape)
    bc = ((2, 1), (0, 0), (1, 2))
    h = (0.3, 0.5, 0.7)
    A, _ = O.assemble(D, h, bc, _faces(shape, bc, 0.0), 0.8, "harm")
    y = O.apply_operator(x, D, h, bc, 0.8, "harm")
    assert np.max(np.abs(y.ravel() - A @ x.ravel())) <= 1e-13 * np.max(np.abs(y))
