"""One-dimensional radiation-MHD travelling waves: the FLD substep inside a whole step.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; never imported by the library).

The paper's linear-wave tests (Sect. 4.3) excite a right-travelling magnetosonic wave
at the left end of a uniform medium in radiative equilibrium and compare the spatial
damping of its amplitude with the dispersion relation of Appendix B. This module
advances that 1D problem with the scheme of Sect. 3, split into two parts per step of
length dt:

1. the hyperbolic terms (the left-hand sides of Eqs. mhd_mass, mhd_mom, mhd_energy and
   mhd_mag, and the advection term of Eq. mhd_r_e) together with the explicit coupling
   terms (the radiation force f_r = -lambda grad E in the momentum equation, its work
   v . f_r in the energy equation, photon tiring P : grad v in Eq. mhd_r_e), by the
   three-stage strong-stability-preserving Runge-Kutta scheme of Shu and Osher, with
   HLL interface fluxes (Einfeldt's signal speeds from the fast magnetosonic speed) and
   third-order WENO reconstruction (Jiang-Shu weights) of the primitive variables;
2. the FLD substep on (rho, T_g, E): the limiter and the coupling terms of
   ``oracle.fld``, a backward-Euler diffusion solve of the system ``oracle.fld.assemble``
   builds (here as a banded solve along the single axis), and ``oracle.fld.exchange``;
   the gas internal energy is then replaced by the exchange's.

Units are CGS with the magnetic field in Heaviside-Lorentz units (magnetic pressure
B^2/2, as the paper writes it); B_x is constant in 1D.

Readings where the paper is silent (it names the solver family only):
* the time integrator and the split: SSP-RK3 for part 1, then part 2 (first order);
* WENO3 acts on the primitive variables, with epsilon = 1e-6 added to the smoothness
  indicators divided by the largest square of the four cells the interface uses, so
  that the weights do not depend on the units;
* the HLL signal speeds use the gas fast speed (radiation pressure acts through f_r);
* boundaries: the cells within one wavelength of the left end, and the left ghost
  cells, hold the ideal-MHD wave of Sect. 4.3 at every stage (the paper's interior
  boundary); on the right, zero gradient for gas and field, and for E a Dirichlet face
  value E_0 in the diffusion solve and the gradient, zero gradient in its advection.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded

from . import dispersion as Disp
from . import fld as F

# primitive layout; the conservative one keeps rho, B_y, B_z, E and holds the momenta
# at VX..VZ and the total gas energy (Eq. energy_density) at PG
RHO, VX, VY, VZ, BY, BZ, PG, ER = range(8)
NV = 8


def conserved(W, Bx, gamma):
    rho, vx, vy, vz, By, Bz, p, E = W
    e = (p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
         + 0.5 * (Bx * Bx + By * By + Bz * Bz))
    return np.stack([rho, rho * vx, rho * vy, rho * vz, By, Bz, e, E])


def primitive(U, Bx, gamma):
    rho = U[RHO]
    vx, vy, vz = U[VX] / rho, U[VY] / rho, U[VZ] / rho
    By, Bz = U[BY], U[BZ]
    p = (gamma - 1.0) * (U[PG] - 0.5 * rho * (vx * vx + vy * vy + vz * vz)
                         - 0.5 * (Bx * Bx + By * By + Bz * Bz))
    return np.stack([rho, vx, vy, vz, By, Bz, p, U[ER]])


def flux(W, Bx, gamma):
    """x-fluxes of Eqs. mhd_mass, mhd_mom, mhd_mag, mhd_energy and of E v (Eq. mhd_r_e)."""
    rho, vx, vy, vz, By, Bz, p, E = W
    B2 = Bx * Bx + By * By + Bz * Bz
    pt = p + 0.5 * B2
    e = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * B2
    Bv = Bx * vx + By * vy + Bz * vz
    return np.stack([rho * vx,
                     rho * vx * vx + pt - Bx * Bx,
                     rho * vx * vy - Bx * By,
                     rho * vx * vz - Bx * Bz,
                     vx * By - Bx * vy,
                     vx * Bz - Bx * vz,
                     (e + pt) * vx - Bv * Bx,
                     E * vx])


def fast_speed(W, Bx, gamma):
    """Fast magnetosonic speed along x from the gas sound speed sqrt(gamma p / rho)."""
    rho = W[RHO]
    cs2 = gamma * W[PG] / rho
    va2 = (Bx * Bx + W[BY] ** 2 + W[BZ] ** 2) / rho
    vax2 = Bx * Bx / rho
    s = cs2 + va2
    return np.sqrt(0.5 * (s + np.sqrt(np.maximum(s * s - 4.0 * cs2 * vax2, 0.0))))


def weno3(q, eps=1e-6):
    """Left and right states at the interfaces m + 1/2, m = 1 .. M - 3, of arrays with M
    cells along the last axis: third-order WENO from two two-cell stencils per side."""
    qm, q0, qp, qpp = q[..., :-3], q[..., 1:-2], q[..., 2:-1], q[..., 3:]
    # indicators relative to the stencils' largest square: bounded by 4, unit-free
    scale = np.maximum(np.maximum(qm * qm, q0 * q0), np.maximum(qp * qp, qpp * qpp)) + 1e-300
    # left state: stencil {m-1, m} (linear weight 1/3) and stencil {m, m+1} (2/3)
    a0 = (1.0 / 3.0) / (eps + (q0 - qm) ** 2 / scale) ** 2
    a1 = (2.0 / 3.0) / (eps + (qp - q0) ** 2 / scale) ** 2
    qL = (a0 * (1.5 * q0 - 0.5 * qm) + a1 * (0.5 * q0 + 0.5 * qp)) / (a0 + a1)
    # right state: stencil {m+1, m+2} (1/3) and stencil {m, m+1} (2/3)
    b0 = (1.0 / 3.0) / (eps + (qpp - qp) ** 2 / scale) ** 2
    b1 = (2.0 / 3.0) / (eps + (qp - q0) ** 2 / scale) ** 2
    qR = (b0 * (1.5 * qp - 0.5 * qpp) + b1 * (0.5 * q0 + 0.5 * qp)) / (b0 + b1)
    return qL, qR


def hll(WL, WR, Bx, gamma):
    """HLL flux between primitive states WL | WR, signal speeds min/max of v_x -+ c_f."""
    UL, UR = conserved(WL, Bx, gamma), conserved(WR, Bx, gamma)
    FL, FR = flux(WL, Bx, gamma), flux(WR, Bx, gamma)
    cL, cR = fast_speed(WL, Bx, gamma), fast_speed(WR, Bx, gamma)
    SL = np.minimum(np.minimum(WL[VX] - cL, WR[VX] - cR), 0.0)
    SR = np.maximum(np.maximum(WL[VX] + cL, WR[VX] + cR), 0.0)
    return (SR * FL - SL * FR + SL * SR * (UR - UL)) / (SR - SL)


def diffuse_1d(E, D, h, bc, E_bc, dt):
    """Backward-Euler diffusion along one non-periodic axis: the tridiagonal system of
    ``oracle.fld.assemble`` (face weight dt/h^2 (D_i + D_{i+1})/2, a Dirichlet face
    2 dt D_i/h^2 with the face value on the right-hand side), solved as a banded system."""
    if bc[0][0] == F.PERIODIC:
        raise ValueError("diffuse_1d takes non-periodic axes only")
    n = E.size
    s = dt / (h * h)
    w = s * 0.5 * (D[:-1] + D[1:])
    diag = np.ones(n)
    diag[:-1] += w
    diag[1:] += w
    rhs = np.array(E, dtype=np.float64)
    for side, cell in ((0, 0), (1, n - 1)):
        if bc[0][side] == F.DIRICHLET:
            wd = s * 2.0 * D[cell]
            diag[cell] += wd
            rhs[cell] += wd * float(E_bc[(0, side)])
    ab = np.zeros((3, n))
    ab[0, 1:] = -w
    ab[1] = diag
    ab[2, :-1] = -w
    return solve_banded((1, 1), ab, rhs)


class Wave:
    """The oracle's run of a driven 1D wave problem (``inputs.wave1d``: background, grid
    and driving wave of Sect. 4.3). The driven cells and the left ghost cells hold the
    problem's W0 + hat sin(k x - omega t) at every stage. With ``problem.radiation``
    False the coupling terms and the FLD substep are off (ideal MHD)."""

    def __init__(self, problem, cfl=0.8, mode=0, scheme="split"):
        P = problem
        self.scheme = scheme
        self.P = P
        self.gamma = P.gamma
        self.R_gas = P.R_gas
        self.c, self.a_r = P.c, P.a_r
        self.Bx = P.Bx
        self.k = P.k
        self.lam = P.lam
        self.n = P.n
        self.nw = P.n_wavelengths
        self.dx = P.dx
        self.x = P.x
        self.cfl = cfl
        self.mode = mode
        self.radiation = P.radiation
        self.op = (0, P.kappa, 0.0, 0.0)          # constant opacity
        self.bcE = ((F.NEUMANN, F.DIRICHLET),)
        self.E_bc = {(0, 1): np.array(P.E0)}
        self.kind = P.kind
        self.phase_speed = P.phase_speed
        self.omega = P.omega
        self.hat = np.asarray(P.hat, dtype=float)
        self.W0 = np.asarray(P.W0, dtype=float)
        self.driven = np.arange(P.n) < P.n_driven

    def analytic(self, x, t):
        return self.W0[:, None] + self.hat[:, None] * np.sin(self.k * x - self.omega * t)[None, :]

    def initial(self):
        W = np.repeat(self.W0[:, None], self.n, axis=1)
        W[:, self.driven] = self.analytic(self.x[self.driven], 0.0)
        return conserved(W, self.Bx, self.gamma)

    def drive(self, U, t):
        U[:, self.driven] = conserved(self.analytic(self.x[self.driven], t), self.Bx, self.gamma)

    def T_gas(self, W):
        return W[PG] / (W[RHO] * self.R_gas)

    def rhs(self, U, t):
        W = primitive(U, self.Bx, self.gamma)
        left = self.analytic(self.x[0] - self.dx * np.array([2.0, 1.0]), t)
        right = np.repeat(W[:, -1:], 2, axis=1)
        qL, qR = weno3(np.concatenate([left, W, right], axis=1))
        Fi = hll(qL, qR, self.Bx, self.gamma)
        dU = -(Fi[:, 1:] - Fi[:, :-1]) / self.dx
        if self.radiation:
            cp = F.coupling(W[ER], W[RHO], self.T_gas(W), (self.dx,), self.bcE, self.E_bc,
                            self.c, self.op, v=[W[VX]], mode=self.mode)
            dU[VX] += cp["fr"][0]
            dU[PG] += cp["vfr"]
            dU[ER] -= cp["ptire"]
        return dU

    def implicit(self, P, tau, t):
        """The FLD substep over tau on the state P (the stage solve of the IMEX scheme):
        limiter, backward-Euler diffusion, exchange; the exchange's change of T_g goes to
        the gas energy. Returns the new state, its driven cells at time t. Without radiation
        there is no implicit term: the stage value is the predictor."""
        if not self.radiation:
            U = P.copy()
            self.drive(U, t)
            return U
        W = primitive(P, self.Bx, self.gamma)
        T = self.T_gas(W)
        D, _, _ = F.limiter(W[ER], W[RHO], T, (self.dx,), self.bcE, self.E_bc, self.c,
                            self.op, self.mode)
        E1 = diffuse_1d(W[ER], D, self.dx, self.bcE, self.E_bc, tau)
        T2, E2 = F.exchange(W[RHO], T, E1, tau, self.c, self.a_r, self.gamma, self.R_gas,
                            self.op)
        U = P.copy()
        U[PG] += W[RHO] * self.R_gas * (T2 - T) / (self.gamma - 1.0)
        U[ER] = E2
        self.drive(U, t)
        return U

    def step_ars3(self, U, t, dt):
        """One step of the ARS(2,3,3) IMEX scheme (Ascher, Ruuth and Spiteri 1997), the
        ARS3 of Sect. 3: explicit hyperbolic and coupling terms L, implicit FLD substep.
        gamma = (3 + sqrt 3)/6; stage predictors
          P1 = U + dt gamma L(U),
          P2 = U + dt ((gamma - 1) L(U) + 2 (1 - gamma) L(U2)) + dt (1 - 2 gamma) G2,
        stage values U_{s+1} = the substep over gamma dt from P_s, G = (U_{s+1} - P_s)/(gamma
        dt) its implicit increment, and U^{n+1} = U + dt/2 (L(U2) + L(U3)) + dt/2 (G2 + G3).
        Each predictor and stage value takes the driving wave at its stage time."""
        g = (3.0 + np.sqrt(3.0)) / 6.0
        L1 = self.rhs(U, t)
        P1 = U + dt * g * L1
        self.drive(P1, t + g * dt)
        U2 = self.implicit(P1, g * dt, t + g * dt)
        G2 = (U2 - P1) / (g * dt)
        L2 = self.rhs(U2, t + g * dt)
        P2 = U + dt * ((g - 1.0) * L1 + 2.0 * (1.0 - g) * L2) + dt * (1.0 - 2.0 * g) * G2
        self.drive(P2, t + (1.0 - g) * dt)
        U3 = self.implicit(P2, g * dt, t + (1.0 - g) * dt)
        G3 = (U3 - P2) / (g * dt)
        L3 = self.rhs(U3, t + (1.0 - g) * dt)
        Un = U + 0.5 * dt * (L2 + L3) + 0.5 * dt * (G2 + G3)
        self.drive(Un, t + dt)
        return Un

    def step(self, U, t, dt):
        if self.scheme == "ars3":
            return self.step_ars3(U, t, dt)
        U1 = U + dt * self.rhs(U, t)
        self.drive(U1, t + dt)
        U2 = 0.75 * U + 0.25 * (U1 + dt * self.rhs(U1, t + dt))
        self.drive(U2, t + 0.5 * dt)
        U3 = U / 3.0 + 2.0 / 3.0 * (U2 + dt * self.rhs(U2, t + 0.5 * dt))
        self.drive(U3, t + dt)
        if self.radiation:
            W = primitive(U3, self.Bx, self.gamma)
            T = self.T_gas(W)
            D, _, _ = F.limiter(W[ER], W[RHO], T, (self.dx,), self.bcE, self.E_bc, self.c,
                                self.op, self.mode)
            E1 = diffuse_1d(W[ER], D, self.dx, self.bcE, self.E_bc, dt)
            T2, E2 = F.exchange(W[RHO], T, E1, dt, self.c, self.a_r, self.gamma, self.R_gas,
                                self.op)
            U3[PG] += W[RHO] * self.R_gas * (T2 - T) / (self.gamma - 1.0)
            U3[ER] = E2
            self.drive(U3, t + dt)
        return U3

    def dt_max(self, U):
        W = primitive(U, self.Bx, self.gamma)
        return self.cfl * self.dx / np.max(np.abs(W[VX]) + fast_speed(W, self.Bx, self.gamma))

    def run(self, t_end, U=None, t=0.0):
        U = self.initial() if U is None else U
        steps = 0
        while t < t_end * (1.0 - 1e-12):
            dt = min(self.dt_max(U), t_end - t)
            U = self.step(U, t, dt)
            t += dt
            steps += 1
        return U, t, steps

    def amplitudes(self, U, var=RHO):
        """Half the peak-to-peak perturbation of a primitive variable in each wavelength."""
        W = primitive(U, self.Bx, self.gamma)
        d = (W[var] - self.W0[var]).reshape(self.nw, -1)
        return 0.5 * (d.max(axis=1) - d.min(axis=1))

    def damping(self, U, first, last, var=RHO):
        """Spatial damping rate (1/cm): minus the slope of a least-squares line through
        log amplitude against the centres of wavelengths first .. last - 1."""
        a = self.amplitudes(U, var)[first:last]
        x = (np.arange(first, last) + 0.5) * self.lam
        return -np.polyfit(x, np.log(a), 1)[0]


def spatial_damping(bg, omega, k0, iters=60):
    """Complex wavenumber k of the wave driven at real frequency omega: omega is an
    eigenvalue of the Appendix-B matrix M(k). Secant iteration from k0 on the eigenvalue
    of M(k) nearest omega; amplitudes then fall as exp(-Im(k) x)."""
    def g(k):
        b = dict(bg)
        b["k"] = k
        w = np.linalg.eigvals(Disp.mode_matrix(b))
        return w[np.argmin(np.abs(w - omega))] - omega

    k1, k2 = complex(k0), complex(k0) * (1.0 + 1e-3)
    g1, g2 = g(k1), g(k2)
    for _ in range(iters):
        if g2 == g1:
            break
        k3 = k2 - g2 * (k2 - k1) / (g2 - g1)
        k1, g1, k2, g2 = k2, g2, k3, g(k3)
        if abs(k2 - k1) <= 1e-13 * abs(k2):
            break
    return k2
