"""Pins of the oracle's backward-Euler diffusion solve (the div F term of Eq. mhd_r_e
with F = -D grad E, Eq. fld_F), by closed forms, invariants and independent solvers."""
import numpy as np
import pytest

from oracle import fld as O


def _rand_problem(shape, bc, seed, sigma=1.0):
    rng = np.random.default_rng(seed)
    D = np.exp(sigma * rng.standard_normal(shape))
    E = 1.0 + rng.uniform(0, 1, shape)
    Eb = {}
    nd = len(shape)
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1.0 + rng.uniform(0, 1, fs)
    return D, E, Eb


BCS3 = [((0, 0), (0, 0), (0, 0)), ((1, 1), (2, 1), (0, 0)), ((2, 2), (1, 2), (1, 1))]


@pytest.mark.parametrize("bc", BCS3)
def test_dense_lu_equals_pcg(bc):
    shape = (7, 6, 9)
    D, E, Eb = _rand_problem(shape, bc, 11)
    h = (0.11, 0.13, 0.17)
    dt = 0.05
    x_lu = O.diffuse(E, D, h, bc, Eb, dt, method="lu")
    x_cg = O.diffuse(E, D, h, bc, Eb, dt, method="pcg")
    assert np.max(np.abs(x_lu - x_cg)) / np.max(np.abs(x_lu)) < 1e-13
    assert O.relative_residual(x_lu, E, D, h, bc, Eb, dt) < 1e-14


def test_matrix_symmetric_positive():
    bc = BCS3[1]
    D, E, Eb = _rand_problem((5, 4, 6), bc, 2)
    A, g = O.assemble(D, (0.2, 0.3, 0.1), bc, Eb, 0.07)
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T, rtol=0, atol=1e-15 * np.abs(Ad).max())
    assert np.linalg.eigvalsh(Ad).min() >= 1.0 - 1e-12      # A = I + SPD part


def test_spectral_closed_form_constant_D():
    # Constant D on a periodic grid: each Fourier mode is divided by
    # 1 + dt D sum_d (4/h_d^2) sin^2(pi m_d / n_d). Compare with an FFT solve.
    shape = (8, 10, 12)
    h = (1.0 / 12, 1.0 / 10, 0.125)
    dt, Dc = 0.003, 0.7
    rng = np.random.default_rng(4)
    E = rng.standard_normal(shape)
    x = O.diffuse(E, np.full(shape, Dc), h, ((0, 0),) * 3, {}, dt, method="pcg")
    sym = np.ones(shape)
    for d in range(3):
        a = 2 - d
        n = shape[a]
        m = np.fft.fftfreq(n) * n
        sh = [1, 1, 1]
        sh[a] = n
        sym = sym + (dt * Dc * 4.0 / h[d] ** 2 * np.sin(np.pi * m / n) ** 2).reshape(sh)
    xf = np.real(np.fft.ifftn(np.fft.fftn(E) / sym))
    assert np.max(np.abs(x - xf)) / np.max(np.abs(xf)) < 1e-13


def test_gaussian_closed_form_convergence():
    # Continuum Gaussian: E - 1 = A (w0/w) exp(-(x - 0.5)^2 / w^2), w^2 = w0^2 + 4 D t.
    # Backward Euler + 2nd-order space: error ~ C1 h^2 + C2 dt.
    Dc, w0, tend = 1.0 / 3.0, 0.05, 2e-4

    def run(n, nsteps):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        E = 1.0 + 0.1 * np.exp(-((x - 0.5) ** 2) / w0 ** 2)
        for _ in range(nsteps):
            E = O.diffuse(E, np.full(n, Dc), (h,), ((0, 0),), {}, tend / nsteps, method="pcg")
        w = np.sqrt(w0 ** 2 + 4 * Dc * tend)
        ex = 1.0 + 0.1 * (w0 / w) * np.exp(-((x - 0.5) ** 2) / w ** 2)
        return np.max(np.abs(E - ex))

    # time order at fine space
    et = [run(1024, m) for m in (4, 8, 16)]
    ot = np.log2(np.array(et[:-1]) / np.array(et[1:]))
    assert np.all((ot > 0.85) & (ot < 1.2)), ot
    # space order at fine time
    es = [run(n, 400) for n in (64, 128)]
    assert 1.7 < np.log2(es[0] / es[1]) < 2.3, es


@pytest.mark.parametrize("bc", [((0, 0), (0, 0)), ((1, 1), (0, 0)), ((1, 1), (1, 1))])
def test_conservation_without_dirichlet(bc):
    D, E, Eb = _rand_problem((13, 11), bc, 7, sigma=2.0)
    x = O.diffuse(E, D, (0.1, 0.2), bc, Eb, 0.5, method="lu")
    assert abs(x.sum() - E.sum()) / E.sum() < 1e-13


def test_dirichlet_linear_profile_is_fixed_point():
    # Constant D, E linear between two Dirichlet faces holding the linear
    # function's values: the discrete flux is uniform, so E is unchanged.
    # This fixes the half-cell distance h/2 of the boundary flux.
    n, h = 17, 0.1
    x = (np.arange(n) + 0.5) * h
    E = 2.0 + 3.0 * x
    Eb = {(0, 0): np.array(2.0), (0, 1): np.array(2.0 + 3.0 * n * h)}
    xs = O.diffuse(E, np.full(n, 0.9), (h,), ((2, 2),), Eb, 0.4, method="lu")
    assert np.max(np.abs(xs - E)) < 1e-13
    # same in 3D along z with x, y periodic
    shape = (n, 4, 5)
    E3 = np.broadcast_to(E[:, None, None], shape).copy()
    Eb3 = {(2, 0): np.full((4, 5), 2.0), (2, 1): np.full((4, 5), 2.0 + 3.0 * n * h)}
    xs3 = O.diffuse(E3, np.full(shape, 0.9), (0.3, 0.2, h), ((0, 0), (0, 0), (2, 2)), Eb3, 0.4,
                    method="lu")
    assert np.max(np.abs(xs3 - E3)) < 1e-13


def test_reflection_and_transpose_invariance():
    bc = ((2, 1), (0, 0))
    D, E, Eb = _rand_problem((9, 9), bc, 9)
    h = (0.2, 0.2)
    x = O.diffuse(E, D, h, bc, Eb, 0.3, method="lu")
    # mirror x: swap low/high boundary kinds and values
    xm = O.diffuse(E[:, ::-1].copy(), D[:, ::-1].copy(), h, ((1, 2), (0, 0)),
                   {(0, 1): Eb[(0, 0)]}, 0.3, method="lu")
    assert np.allclose(xm[:, ::-1], x, rtol=1e-13, atol=0)
    # transpose (x <-> y)
    xt = O.diffuse(E.T.copy(), D.T.copy(), h, ((0, 0), (2, 1)), {(1, 0): Eb[(0, 0)]}, 0.3,
                   method="lu")
    assert np.allclose(xt.T, x, rtol=1e-13, atol=0)


def test_matrix_free_operator_agrees_with_matrix():
    bc = ((2, 1), (0, 0), (1, 2))
    D, E, Eb = _rand_problem((6, 5, 7), bc, 3)
    h = (0.3, 0.2, 0.4)
    A, _ = O.assemble(D, h, bc, Eb, 0.2)
    y = O.apply_operator(E, D, h, bc, 0.2)
    scale = abs(A) @ np.abs(E.ravel())          # size of the terms being summed
    assert np.all(np.abs(y.ravel() - A @ E.ravel()) <= 1e-14 * scale)
