"""Seeded synthetic inputs for the FLD radiation substep.

This module is shared by the CPU oracle's tests and by the CUDA path's tests and
benchmark. It holds input recipes only (shapes, random fields, boundary kinds,
time steps) and none of the substep's arithmetic (no limiter, no diffusion
operator, no exchange).

Conventions
-----------
* Arrays are float64, C-contiguous, numpy axis order (z, y, x): x is fastest.
  A 1D problem has shape (nx,), 2D (ny, nx), 3D (nz, ny, nx).
* ``h`` and ``bc`` are given in physical axis order (x, y, z).
* Boundary codes: 0 periodic, 1 Neumann (zero flux), 2 Dirichlet (face value).
* Dirichlet face values are a dict ``{(axis, side): face_array}`` with
  ``side`` 0 = low, 1 = high and ``face_array`` the field's shape with that
  axis removed. ``pack_dirichlet`` flattens them in the order x-lo, x-hi,
  y-lo, y-hi, z-lo, z-hi (Dirichlet sides only), which is the layout the C
  library takes.
* Seeds: 250302764 + workload index; member p of the batched workload uses
  base seed + 1000 * p.

The time steps are stated as multiples of the explicit diffusion limit
h^2 / (2 d D_ref) with the diffusion-limit bound D_ref = c / (3 min(kappa rho))
(the limiter never exceeds 1/3), so dt is a plain input number.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

SEED_BASE = 250302764
PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2
OPACITY_CONST, OPACITY_POWER, OPACITY_TABLE = 0, 1, 2
LIMITER_LP, LIMITER_DIFFUSION = 0, 1


@dataclass
class Problem:
    name: str
    shape: tuple            # numpy order (z, y, x) restricted to ndim
    h: tuple                # (hx, hy, hz)[:ndim]
    bc: tuple               # ((xlo, xhi), (ylo, yhi), ...)[:ndim]
    c: float
    a_r: float
    gamma: float
    R_gas: float
    opacity: tuple          # (kind, kappa0, a_rho, a_T): kappa = kappa0 rho^a_rho T^a_T, or
                            # (OPACITY_TABLE, kappa0, log10 kappa table, grid): see opacity_table
    dt: float
    rho: np.ndarray
    T: np.ndarray
    E: np.ndarray
    E_bc: dict = field(default_factory=dict)
    limiter: int = LIMITER_LP
    tol: float = 1e-10
    steps: int = 1

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def ncells(self):
        return int(np.prod(self.shape))

    def n_xyz(self):
        """(nx, ny, nz) with 1 for absent axes."""
        n = list(reversed(self.shape)) + [1] * (3 - self.ndim)
        return tuple(int(v) for v in n)


def pack_dirichlet(shape, bc, E_bc):
    """Flatten Dirichlet face arrays in x-lo, x-hi, y-lo, y-hi, z-lo, z-hi order."""
    parts = []
    for d in range(len(shape)):
        for s in (0, 1):
            if bc[d][s] == DIRICHLET:
                parts.append(np.ascontiguousarray(E_bc[(d, s)], dtype=np.float64).ravel())
    if not parts:
        return np.zeros(0, dtype=np.float64)
    return np.concatenate(parts)


def correlated_gaussian(rng, shape, ell):
    """Zero-mean, unit-variance Gaussian field with correlation exp(-r^2/(2 ell^2)).

    White noise is filtered by exp(-|k|^2 ell^2 / 4) in Fourier space (k in
    radians per cell) and normalised to sample mean 0 and sample std 1.
    """
    w = rng.standard_normal(shape)
    k2 = np.zeros(shape)
    for a, n in enumerate(shape):
        k = 2.0 * np.pi * np.fft.fftfreq(n)
        sh = [1] * len(shape)
        sh[a] = n
        k2 = k2 + (k.reshape(sh)) ** 2
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * np.exp(-k2 * ell * ell / 4.0)))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal(rng, shape, sigma, ell):
    g = correlated_gaussian(rng, shape, ell)
    return np.exp(sigma * g - 0.5 * sigma * sigma)


def _cell_centres(n, L=1.0):
    return (np.arange(n) + 0.5) * (L / n)


def gaussian_pulse_1d(n=256, seed=None):
    """1D periodic, n cells, unit box: rho = 1, kappa = 1e3, T = 1,
    E = 1 + 0.1 exp(-(x - 0.5)^2 / 0.01^2); dt = 10 x the explicit limit."""
    h = 1.0 / n
    x = _cell_centres(n)
    c, kappa = 1.0, 1.0e3
    D_ref = c / (3.0 * kappa * 1.0)
    dt = 10.0 * h * h / (2.0 * D_ref)
    return Problem(
        name="pulse1d_%d" % n, shape=(n,), h=(h,), bc=((PERIODIC, PERIODIC),),
        c=c, a_r=1.0, gamma=5.0 / 3.0, R_gas=1.0,
        opacity=(OPACITY_CONST, kappa, 0.0, 0.0), dt=dt,
        rho=np.ones(n), T=np.ones(n), E=1.0 + 0.1 * np.exp(-((x - 0.5) ** 2) / 0.01 ** 2),
        tol=1e-12, steps=1)


def lognormal_2d(n=1024, seed=None, ny=None, steps=10):
    """2D periodic n x n (or ny x n), h = 1: log-normal rho (sigma = 1,
    correlation 32 cells), kappa = 0.4, T = p0/(R_gas rho) with p0 = 1,
    E = a_r T^4 (1 + 0.05 U(-1, 1)); dt = 10 x the explicit limit."""
    ny = n if ny is None else ny
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 2 if seed is None else seed))
    shape = (ny, n)
    rho = lognormal(rng, shape, 1.0, 32.0)
    c, a_r, R_gas, kappa = 1.0, 1.0, 1.0, 0.4
    T = 1.0 / (R_gas * rho)
    E = a_r * T ** 4 * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, shape))
    D_ref = c / (3.0 * kappa * rho.min())
    dt = 10.0 * 1.0 / (2.0 * 2 * D_ref)
    return Problem(
        name="lognormal2d_%dx%d" % (n, ny), shape=shape, h=(1.0, 1.0),
        bc=((PERIODIC, PERIODIC), (PERIODIC, PERIODIC)),
        c=c, a_r=a_r, gamma=5.0 / 3.0, R_gas=R_gas,
        opacity=(OPACITY_CONST, kappa, 0.0, 0.0), dt=dt, rho=rho, T=T, E=E,
        tol=1e-10, steps=steps)


def stratified_3d(n=256, seed=None, nz=None, ny=None):
    """3D stratified box, unit cube, x/y periodic, z Dirichlet.

    rho = exp(-z/0.2), T = 10 - 9 z (10x contrast), both times (1 + 0.01 U(-1,1));
    Kramers-like kappa = kappa0 rho T^-3.5 with kappa0 set so that the
    unperturbed kappa rho h = 1 at z = 0.5; E = a_r T^4; the z faces hold E of
    the adjacent cells (radiation temperature pinned to the gas temperature);
    dt = 10 x the explicit limit of the unperturbed profile.
    """
    nz = n if nz is None else nz
    ny = n if ny is None else ny
    nx = n
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 3 if seed is None else seed))
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    z = _cell_centres(nz)[:, None, None] * np.ones((nz, ny, nx))
    rho0 = np.exp(-z / 0.2)
    T0 = 10.0 - 9.0 * z
    rho = rho0 * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, rho0.shape))
    T = T0 * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, T0.shape))
    c, a_r = 1.0, 1.0
    # kappa rho = kappa0 rho^2 T^-3.5 ; equal to 1/h_z at z = 0.5 (unperturbed)
    kappa0 = (1.0 / h[2]) / (np.exp(-0.5 / 0.2) ** 2 * (10.0 - 4.5) ** -3.5)
    zc = _cell_centres(nz)
    kr_min = np.min(kappa0 * np.exp(-zc / 0.2) ** 2 * (10.0 - 9.0 * zc) ** -3.5)
    D_ref = c / (3.0 * kr_min)
    hmin = min(h)
    dt = 10.0 * hmin * hmin / (2.0 * 3 * D_ref)
    E = a_r * T ** 4
    E_bc = {(2, 0): E[0].copy(), (2, 1): E[-1].copy()}
    return Problem(
        name="stratified3d_%dx%dx%d" % (nx, ny, nz), shape=(nz, ny, nx), h=h,
        bc=((PERIODIC, PERIODIC), (PERIODIC, PERIODIC), (DIRICHLET, DIRICHLET)),
        c=c, a_r=a_r, gamma=5.0 / 3.0, R_gas=1.0,
        opacity=(OPACITY_POWER, kappa0, 1.0, -3.5), dt=dt, rho=rho, T=T, E=E,
        E_bc=E_bc, tol=1e-10, steps=1)


def batch_member_shape(p, seed_base=None, nmin=32, nmax=512):
    """(ny, nx) of member p of the batched workload without building its fields (the
    first two draws of the member's generator, as in batch_member)."""
    base = SEED_BASE + 4 if seed_base is None else seed_base
    rng = np.random.Generator(np.random.PCG64(base + 1000 * p))
    nx = int(rng.integers(nmin, nmax + 1))
    ny = int(rng.integers(nmin, nmax + 1))
    return (ny, nx)


def batch_shapes(nprob=512, seed_base=None, nmin=32, nmax=512):
    """Shapes and boundary kinds of the batched workload's members (what the autotuner's
    workload signature reads), without building their fields."""
    from types import SimpleNamespace
    bc = ((PERIODIC, PERIODIC), (PERIODIC, PERIODIC))
    return [SimpleNamespace(shape=batch_member_shape(p, seed_base, nmin, nmax), bc=bc)
            for p in range(nprob)]


def batch_member(p, seed_base=None, nmin=32, nmax=512):
    """Member p of the batched 2D workload: sides U{nmin..nmax}, periodic, h = 1,
    log-normal rho (sigma ~ U[0.5, 2], correlation 8 cells), kappa = 10^U[0,4],
    T = 1/rho, E = T^4 (1 + 0.05 U(-1,1)), dt = s x the explicit limit with
    s = 10^U[0, 2]."""
    base = SEED_BASE + 4 if seed_base is None else seed_base
    rng = np.random.Generator(np.random.PCG64(base + 1000 * p))
    nx = int(rng.integers(nmin, nmax + 1))
    ny = int(rng.integers(nmin, nmax + 1))
    sigma = float(rng.uniform(0.5, 2.0))
    kappa = float(10.0 ** rng.uniform(0.0, 4.0))
    s = float(10.0 ** rng.uniform(0.0, 2.0))
    shape = (ny, nx)
    rho = lognormal(rng, shape, sigma, 8.0)
    T = 1.0 / rho
    E = T ** 4 * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, shape))
    c = 1.0
    D_ref = c / (3.0 * kappa * rho.min())
    dt = s * 1.0 / (2.0 * 2 * D_ref)
    return Problem(
        name="batch2d_p%d_%dx%d" % (p, nx, ny), shape=shape, h=(1.0, 1.0),
        bc=((PERIODIC, PERIODIC), (PERIODIC, PERIODIC)),
        c=c, a_r=1.0, gamma=5.0 / 3.0, R_gas=1.0,
        opacity=(OPACITY_CONST, kappa, 0.0, 0.0), dt=dt, rho=rho, T=T, E=E,
        tol=1e-10, steps=1)


def batch(nprob=512, seed_base=None, nmin=32, nmax=512):
    return [batch_member(p, seed_base, nmin, nmax) for p in range(nprob)]


def linmode_amplitudes(ratio):
    """Complex amplitudes (T_1, E_1) per unit relative density amplitude of the fast
    magnetosonic eigenmode for the radiation-to-gas pressure ratio 0.1 or 1, as stored in
    linmode_eigen.json (written by the oracle's write_linmode_eigen script from the
    Appendix-B system: B = 1 at 45 degrees to k = 2 pi, rho0 = T0 = 1, kappa = c = 1e4)."""
    import json
    import os
    d = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                    "linmode_eigen.json")))
    m = d["modes"]["%g" % ratio]
    return complex(*m["T1"]), complex(*m["E1"])


def linear_mode_3d(n=512, ratio=1.0, amp=1e-4, seed=None, ny=None, nz=None,
                   steps=100, dt=1e-3, mode="eigen"):
    """3D periodic unit box driven by a linear perturbation along x.

    rho = 1, T0 = 1, R_gas = 1, gamma = 5/3, a_r = 3 x ratio (so that the
    radiation-to-gas pressure ratio a_r T^4/3 / (rho R_gas T) equals ratio),
    kappa = 1e4, c = 1e4 (D = 1/3 in the diffusion limit, c kappa rho = 1e8).
    The mode is k = 2 pi x-hat with, per cell, X = X0 + amp Re(X_1 exp(i k x)):
    mode "eigen" (ratio 0.1 or 1): T_1 and E_1 of the fast magnetosonic eigenmode with
      B = 1 at 45 degrees to k, per unit relative density amplitude (so amp is the
      relative density amplitude of the wave; the substep keeps rho fixed);
    mode "excess": T_1 = 1/2, E_1 = 4 E0 (a radiation-temperature excess over the gas,
      so that both the diffusion and the exchange act on it).
    """
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    nx = n
    a_r = 3.0 * ratio
    E0 = a_r * 1.0
    if mode == "eigen":
        T1, E1 = linmode_amplitudes(ratio)
    else:
        T1, E1 = complex(0.5), complex(4.0 * E0)
    x = _cell_centres(nx)
    ph = np.exp(1j * 2.0 * np.pi * x)
    ones = np.ones((nz, ny, 1))
    T = (1.0 + amp * np.real(T1 * ph))[None, None, :] * ones
    E = (E0 + amp * np.real(E1 * ph))[None, None, :] * ones
    return Problem(
        name="linmode3d_%d_r%g_%s" % (n, ratio, mode), shape=(nz, ny, nx),
        h=(1.0 / nx, 1.0 / ny, 1.0 / nz),
        bc=((PERIODIC, PERIODIC),) * 3, c=1.0e4, a_r=a_r, gamma=5.0 / 3.0, R_gas=1.0,
        opacity=(OPACITY_CONST, 1.0e4, 0.0, 0.0), dt=dt,
        rho=np.ones((nz, ny, nx)), T=np.ascontiguousarray(T), E=np.ascontiguousarray(E),
        tol=1e-10, steps=steps)


def opacity_table(kappa0, log_rho=(-2.0, 0.3), log_T=(-0.1, 1.05), n_rho=24, n_T=30,
                  bump=2.0, bump_logT=0.6, bump_width=0.1, noise=0.02, seed=None):
    """A synthetic opacity table with the structure of tabulated stellar opacities.

    log10 kappa on a uniform grid in (log10 rho, log10 T): a Kramers-like law
    kappa0 rho T^-3.5, raised by a Gaussian bump in log10 T (factor 1 + bump at
    its peak, the shape of the iron bump of real tables), plus seeded noise of
    ``noise`` dex so that the table is not bilinear in the logs. Returns
    (table, grid) with table[j, i] at log10 rho = log_rho0 + i dlog_rho,
    log10 T = log_T0 + j dlog_T, and grid = (log_rho0, dlog_rho, log_T0, dlog_T).
    """
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 91 if seed is None else seed))
    lr = np.linspace(log_rho[0], log_rho[1], n_rho)
    lt = np.linspace(log_T[0], log_T[1], n_T)
    LR, LT = np.meshgrid(lr, lt, indexing="xy")          # (n_T, n_rho), rho fastest
    table = (np.log10(kappa0) + LR - 3.5 * LT
             + np.log10(1.0 + bump * np.exp(-0.5 * ((LT - bump_logT) / bump_width) ** 2))
             + noise * rng.uniform(-1.0, 1.0, LR.shape))
    grid = (float(lr[0]), float(lr[1] - lr[0]), float(lt[0]), float(lt[1] - lt[0]))
    return np.ascontiguousarray(table), grid


def stratified_3d_table(n=32, seed=None, nz=24, ny=20):
    """The stratified box with a tabulated opacity in place of the power law: the
    table of ``opacity_table`` built around the box's own Kramers coefficient. Its
    density range stops above the box's lowest densities, so the top cells take
    the table's edge values (clamped lookups)."""
    P = stratified_3d(n, seed, nz=nz, ny=ny)
    table, grid = opacity_table(P.opacity[1])
    P.opacity = (OPACITY_TABLE, 1.0, table, grid)
    P.name = P.name.replace("stratified3d", "stratified3d_table")
    return P


# CGS constants of the radiation-MHD wave recipes
C_LIGHT = 2.99792458e10
K_B = 1.380649e-16
M_P = 1.67262192e-24
SIGMA_SB = 5.670374e-5
A_RAD = 4.0 * SIGMA_SB / C_LIGHT


# the two backgrounds of the linear-wave tests (Sect. 4.3): weakly radiative and
# radiation-dominant, the same rho_0, B_0, gamma, mu, kappa and optical depth per wavelength
WAVE_BACKGROUNDS = {
    "weak": dict(rho0=3.216e-9, p0=17.34e3, B0_gauss=(330.14, 0.0, 330.14), gamma=5.0 / 3.0,
                 mu=0.5, kappa=0.4, tau=1e3),
    "strong": dict(rho0=3.216e-9, p0=43.35e3, B0_gauss=(330.14, 0.0, 330.14), gamma=5.0 / 3.0,
                   mu=0.5, kappa=0.4, tau=1e3),
}


@dataclass
class Wave1D:
    """A driven 1D wave problem (the linear-wave tests of Sect. 4.3), CGS units, the
    magnetic field in Heaviside-Lorentz form (B_gauss / sqrt(4 pi)). W0 and hat are the
    background and the driving amplitudes of the primitive variables (rho, v_x, v_y,
    v_z, B_y, B_z, p, E); the driven cells hold W0 + hat sin(k x - omega t)."""
    name: str
    n: int
    n_wavelengths: int
    dx: float
    lam: float
    k: float
    omega: float
    phase_speed: float
    gamma: float
    mu: float
    Bx: float
    R_gas: float
    c: float
    a_r: float
    kappa: float
    E0: float
    W0: np.ndarray
    hat: np.ndarray
    n_driven: int
    kind: str
    radiation: bool

    @property
    def x(self):
        return (np.arange(self.n) + 0.5) * self.dx


def wave1d(background, n_cells, n_wavelengths, kind="fast", amp=1e-2, radiation=True):
    """The Sect. 4.3 wave set-up on n_cells cells over n_wavelengths wavelengths.

    ``background``: rho0, p0, B0_gauss, gamma, mu, kappa, tau (optical depth per
    wavelength), as printed for the weakly and strongly radiative cases. T0 from the ideal
    gas law, E0 = a_r T0^4 (radiative equilibrium), lambda_w = tau / (kappa rho0).
    kind "fast"/"slow": the magnetosonic wave with omega/k the ideal-MHD speed built from
    the isothermal sound speed (the adiabatic one when ``radiation`` is False), rho_1 =
    amp rho0, v_x1 = (omega/k) amp, p_1 = c_s^2 rho_1 with that sound speed, v_z1 and B_z1
    from the transverse balance (Sect. 4.3), E_1 = 0. kind "alfven": omega/k = v_Ax,
    v_y1 = amp v_Ax, B_y1 = -(B_x k / omega) v_y1.
    """
    r0, p0, g, mu = background["rho0"], background["p0"], background["gamma"], background["mu"]
    kappa = background["kappa"]
    T0 = p0 * mu * M_P / (r0 * K_B)
    E0 = A_RAD * T0 ** 4
    Bx, By, Bz = (np.asarray(background["B0_gauss"], dtype=float) / np.sqrt(4.0 * np.pi))
    lam = background["tau"] / (kappa * r0)
    k = 2.0 * np.pi / lam
    vax2 = Bx * Bx / r0
    hat = np.zeros(8)
    if kind == "alfven":
        cw = np.sqrt(vax2)
        hat[2] = amp * cw
        hat[4] = -(Bx / cw) * hat[2]
    else:
        cs2 = p0 / r0 if radiation else g * p0 / r0
        va2 = (Bx * Bx + By * By + Bz * Bz) / r0
        s = cs2 + va2
        root = np.sqrt(s * s - 4.0 * cs2 * vax2)
        cw = np.sqrt(0.5 * (s + root) if kind == "fast" else 0.5 * (s - root))
        hat[0] = amp * r0
        hat[1] = cw * amp
        hat[3] = (Bz / Bx) * cw / (1.0 - cw * cw / vax2) * amp
        hat[5] = Bz / (1.0 - vax2 / (cw * cw)) * amp
        hat[6] = cs2 * hat[0]
    dx = n_wavelengths * lam / n_cells
    x = (np.arange(n_cells) + 0.5) * dx
    return Wave1D(name="wave1d_%s_%d" % (kind, n_cells), n=n_cells, n_wavelengths=n_wavelengths,
                  dx=dx, lam=lam, k=k, omega=k * cw, phase_speed=cw, gamma=g, mu=mu, Bx=Bx,
                  R_gas=K_B / (mu * M_P), c=C_LIGHT, a_r=A_RAD, kappa=kappa, E0=E0,
                  W0=np.array([r0, 0.0, 0.0, 0.0, By, Bz, p0, E0]), hat=hat,
                  n_driven=int(np.count_nonzero(x < lam)), kind=kind, radiation=radiation)


def random_cells(ncell, seed=0):
    """Random per-cell exchange inputs spanning chi = dt c kappa rho in [1e-6, 1e12]
    and gas/radiation energy ratios over many decades."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 77 + seed))
    rho = 10.0 ** rng.uniform(-3, 3, ncell)
    T = 10.0 ** rng.uniform(-1, 2, ncell)
    E = 10.0 ** rng.uniform(-4, 8, ncell)
    kappa = 10.0 ** rng.uniform(-2, 4, ncell)
    return rho, T, E, kappa


def make_config(i, seed=None, small=False):
    """Workload by index: 1 pulse1d, 2 lognormal2d, 3 stratified3d, 4 batch, 5 linmode3d.
    ``small`` selects a reduced size the oracle solves in seconds."""
    if i == 1:
        return gaussian_pulse_1d(256)
    if i == 2:
        return lognormal_2d(96 if small else 1024, seed, ny=80 if small else None,
                            steps=2 if small else 10)
    if i == 3:
        return stratified_3d(32 if small else 256, seed, nz=24 if small else None,
                             ny=20 if small else None)
    if i == 4:
        return batch(6 if small else 512, seed, 32 if small else 32, 64 if small else 512)
    if i == 5:
        return linear_mode_3d(16 if small else 512, 1.0, steps=5 if small else 100)
    raise ValueError("workload index must be 1..5")
