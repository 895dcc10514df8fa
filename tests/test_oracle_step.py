"""Pins of the oracle's whole substep (limiter -> diffusion -> exchange) and of the
seeded workload recipes."""
import numpy as np
import pytest

from oracle import fld as O
from oracle import dispersion as Disp
from paper_2503_02764_gb300 import inputs as I


def _run(P, nsteps=None, method="auto"):
    T, E = P.T.copy(), P.E.copy()
    for _ in range(P.steps if nsteps is None else nsteps):
        T, E, _ = O.step(P.rho, T, E, P.h, P.bc, P.E_bc, P.dt, P.c, P.a_r, P.gamma, P.R_gas,
                         P.opacity, P.limiter, method)
    return T, E


@pytest.mark.parametrize("ratio", [0.1, 1.0])
def test_linear_mode_amplification(ratio):
    # A small cos(2 pi x) perturbation about radiative equilibrium evolves by the exact
    # per-step matrix G = (I - dt J)^-1 diag(1, 1/(1 + dt D ktilde^2)) (exchange after
    # diffusion; lambda = 1/3 + O(R^2) for R ~ 1e-10).
    amp = 1e-7
    P = I.linear_mode_3d(16, ratio=ratio, amp=amp, ny=2, nz=2, steps=6, mode="excess")
    n = 16
    x = (np.arange(n) + 0.5) / n
    cosx = np.cos(2 * np.pi * x)

    def modes(T, E):
        e = P.rho * P.R_gas * T / (P.gamma - 1)
        return np.array([2.0 / n * np.sum(e[0, 0] * cosx), 2.0 / n * np.sum(E[0, 0] * cosx)])

    v0 = modes(P.T, P.E)
    T, E = _run(P)
    D = P.c / (3.0 * 1e4 * 1.0)
    G = Disp.substep_amplification(P.dt, P.c, 1e4, 1.0, P.a_r, 1.0, P.gamma, P.R_gas, D,
                                   Disp.discrete_k2(2 * np.pi, 1.0 / n))
    v = np.linalg.matrix_power(G, P.steps) @ v0
    got = modes(T, E)
    # agreement is ~1e-9 of the amplitude; swapping the split order misses by ~1e-3
    assert np.all(np.abs(got - v) <= 1e-7 * np.abs(v).max())
    # the y/z structure stays uniform
    assert np.ptp(E, axis=(0, 1)).max() < 1e-13 * E.max()


def test_total_energy_conserved_periodic():
    P = I.lognormal_2d(40, ny=36, steps=2)
    e0 = O.internal_energy(P.rho, P.T, P.gamma, P.R_gas) + P.E
    T, E = _run(P)
    e1 = O.internal_energy(P.rho, T, P.gamma, P.R_gas) + E
    assert abs(e1.sum() - e0.sum()) / e0.sum() < 1e-13


@pytest.mark.parametrize("cfg", [1, 2, 3, 5])
def test_small_workloads_run_and_stay_positive(cfg):
    P = I.make_config(cfg, small=True)
    T, E = _run(P, nsteps=1)
    assert np.all(T > 0) and np.all(E > 0) and np.all(np.isfinite(E))


def test_pulse_diffusion_limit_matches_gaussian_solution():
    # Workload 1 in the diffusion-limit mode is the constant-D Gaussian problem: one
    # backward-Euler step at 10x the explicit limit stays within the O(dt) error of
    # the continuum solution E - 1 = 0.1 (w0/w) exp(-(x-0.5)^2/w^2), w^2 = w0^2 + 4 D dt.
    P = I.gaussian_pulse_1d(256)
    D, _, _ = O.limiter(P.E, P.rho, P.T, P.h, P.bc, P.E_bc, P.c, P.opacity, mode=1)
    E1 = O.diffuse(P.E, D, P.h, P.bc, P.E_bc, P.dt)
    x = (np.arange(256) + 0.5) / 256
    w0 = 0.01
    w = np.sqrt(w0 ** 2 + 4 * D[0] * P.dt)
    ex = 1 + 0.1 * (w0 / w) * np.exp(-((x - 0.5) ** 2) / w ** 2)
    assert np.max(np.abs(E1 - ex)) < 0.1 * 0.1     # within 10% of the pulse height
    assert abs(E1.sum() - P.E.sum()) / P.E.sum() < 1e-14


def test_recipes_are_seeded_and_shaped():
    a, b = I.stratified_3d(16, nz=12, ny=10), I.stratified_3d(16, nz=12, ny=10)
    assert np.array_equal(a.rho, b.rho) and a.shape == (12, 10, 16)
    assert a.E_bc[(2, 0)].shape == (10, 16)
    g = I.correlated_gaussian(np.random.default_rng(0), (64, 64), 8.0)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1) < 1e-12
    m = I.batch(4, nmin=32, nmax=40)
    assert all(32 <= s <= 40 for p in m for s in p.shape)
    packed = I.pack_dirichlet(a.shape, a.bc, a.E_bc)
    assert packed.size == 2 * 10 * 16


def test_batch_shapes_without_fields_match_the_members():
    # the autotuner's signature of the 512-member batch is computed from these shapes
    for p in (0, 1, 7, 300, 511):
        assert I.batch_member_shape(p) == I.batch_member(p).shape
    assert [m.shape for m in I.batch_shapes(4, nmin=32, nmax=40)] == \
        [m.shape for m in I.batch(4, nmin=32, nmax=40)]
