"""Linear RMHD modes about a uniform radiative-equilibrium background.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; never imported by the
library).

Follows the paper's Appendix B: the linearised equations eigen_mass,
eigen_mom, eigen_energy, eigen_mag and eigen_r_e with k along x, lambda = 1/3,
the linearised ideal-gas law (ideal_gas_law_lin) and E_1/E_0 = 4 T_r1/T_r0
(rad_temp_lin). The eight unknowns are (rho, v_x, v_y, v_z, p, B_y, B_z, E);
omega u = M u, so the eigenfrequencies are the eigenvalues of M.

The magnetic field enters in Heaviside-Lorentz units (the paper writes the
magnetic pressure as B^2/2), so a field given in Gauss is divided by
sqrt(4 pi).

The printed octic (Eq. dispersion_relation_simplified) is also provided. Its
omega^1 coefficient is read with qdot_{T_r} in the last bracket (printed as
qdot_{T_g}); with that reading its roots equal the eigenvalues of M, while the
printed form makes the slow mode grow.

Also here: the hydro-frozen 2x2 block (rho_1 = v_1 = B_1 = 0) in (p, E) and
the exact per-step amplification of a Fourier mode under the split FLD
substep (backward-Euler diffusion, then backward-Euler exchange), both in the
diffusion limit lambda = 1/3.
"""
from __future__ import annotations

import numpy as np

# CGS constants
C_LIGHT = 2.99792458e10
K_B = 1.380649e-16
M_P = 1.67262192e-24
SIGMA_SB = 5.670374e-5
A_RAD = 4.0 * SIGMA_SB / C_LIGHT


def background(rho0, p0, B0_gauss, gamma, mu, kappa, tau=None, k=None):
    """Equilibrium state with T_r = T_g; k from the optical depth per wavelength
    tau = kappa rho0 lambda_w when not given."""
    T0 = p0 * mu * M_P / (rho0 * K_B)
    E0 = A_RAD * T0 ** 4
    B = np.asarray(B0_gauss, dtype=float) / np.sqrt(4.0 * np.pi)
    if k is None:
        lam_w = tau / (kappa * rho0)
        k = 2.0 * np.pi / lam_w
    return dict(rho0=rho0, p0=p0, B=B, gamma=gamma, mu=mu, kappa=kappa, T0=T0,
                E0=E0, k=k, c=C_LIGHT, a_r=A_RAD)


def qdot_derivatives(bg):
    """Eqs. qdot_rho, qdot_Tr, qdot_Tg at radiative equilibrium."""
    c, k_, r0, T0, ar = bg["c"], bg["kappa"], bg["rho0"], bg["T0"], bg["a_r"]
    q_rho = c * k_ * ar * (T0 ** 4 - T0 ** 4)
    q_Tr = 4.0 * c * r0 * k_ * ar * T0 ** 3
    q_Tg = -4.0 * c * r0 * k_ * ar * T0 ** 3
    return q_rho, q_Tr, q_Tg


def mode_matrix(bg):
    """M with omega u = M u, u = (rho, vx, vy, vz, p, By, Bz, E)."""
    r0, p0, g, k = bg["rho0"], bg["p0"], bg["gamma"], bg["k"]
    T0, E0, c, kap = bg["T0"], bg["E0"], bg["c"], bg["kappa"]
    Bx, By, Bz = bg["B"]
    q_rho, q_Tr, q_Tg = qdot_derivatives(bg)
    M = np.zeros((8, 8), dtype=complex)
    RHO, VX, VY, VZ, P, BY, BZ, EE = range(8)
    # Q = qdot_rho rho + qdot_Tg T_g + qdot_Tr T_r,
    # T_g = T0 (p/p0 - rho/rho0) (ideal_gas_law_lin), T_r = T0 E/(4 E0) (rad_temp_lin)
    Q = np.zeros(8, dtype=complex)
    Q[RHO] = q_rho - q_Tg * T0 / r0
    Q[P] = q_Tg * T0 / p0
    Q[EE] = q_Tr * T0 / (4.0 * E0)
    # eigen_mass: omega rho = rho0 k vx
    M[RHO, VX] = r0 * k
    # eigen_mom (x): omega rho0 vx = k (p + E/3) + k (B . B0) - (B0 . k) Bx, Bx = 0
    M[VX, P] = k / r0
    M[VX, EE] = k / (3.0 * r0)
    M[VX, BY] = k * By / r0
    M[VX, BZ] = k * Bz / r0
    # eigen_mom (y, z): omega rho0 v = -(B0x k) B
    M[VY, BY] = -Bx * k / r0
    M[VZ, BZ] = -Bx * k / r0
    # eigen_energy: omega p = gamma p0 k vx + i (gamma - 1) Q
    M[P, VX] = g * p0 * k
    M[P, :] += 1j * (g - 1.0) * Q
    # eigen_mag: omega B = B0 (k vx) - (B0x k) v
    M[BY, VX] = By * k
    M[BY, VY] = -Bx * k
    M[BZ, VX] = Bz * k
    M[BZ, VZ] = -Bx * k
    # eigen_r_e: omega E = 4/3 E0 k vx - i Q - i k^2 c E / (3 rho0 kappa)
    M[EE, VX] = 4.0 / 3.0 * E0 * k
    M[EE, :] += -1j * Q
    M[EE, EE] += -1j * k * k * c / (3.0 * r0 * kap)
    return M


def eigenfrequencies(bg):
    w = np.linalg.eigvals(mode_matrix(bg))
    return w[np.argsort(w.real + 1e-30 * w.imag)]


def char_speeds(bg):
    """Eq. char_speeds (squares)."""
    r0 = bg["rho0"]
    Bx, By, Bz = bg["B"]
    cg2 = bg["gamma"] * bg["p0"] / r0
    cr2 = 4.0 * bg["E0"] / (9.0 * r0)
    vA2 = (Bx * Bx + By * By + Bz * Bz) / r0
    vAx2 = Bx * Bx / r0
    return cg2, cr2, vA2, vAx2


def magnetosonic_speed(bg, fast=True, isothermal=True):
    """Ideal-MHD fast/slow speed (Eq. cfs_speed read without its stray square),
    with the isothermal sound speed when ``isothermal``."""
    cg2, _, vA2, vAx2 = char_speeds(bg)
    if isothermal:
        cg2 = bg["p0"] / bg["rho0"]
    s = cg2 + vA2
    root = np.sqrt(s * s - 4.0 * cg2 * vAx2)
    return np.sqrt(0.5 * (s + root) if fast else 0.5 * (s - root))


def octic(bg):
    """Coefficients (highest power first) of Eq. dispersion_relation_simplified,
    with qdot_{T_r} in the omega^1 coefficient's last bracket."""
    r0, p0, g, k = bg["rho0"], bg["p0"], bg["gamma"], bg["k"]
    T0, E0, c, kap = bg["T0"], bg["E0"], bg["c"], bg["kappa"]
    _, q_Tr, q_Tg = qdot_derivatives(bg)
    cg2, cr2, vA2, vAx2 = char_speeds(bg)
    dk = c / (3.0 * r0 * kap)
    k2 = k * k
    a6 = 1.0
    a5 = 1j * (dk * k2 + q_Tr * T0 / (4.0 * E0) - (g - 1.0) * q_Tg * T0 / p0)
    a4 = -k2 * (cr2 + cg2 + vA2 - (g - 1.0) * q_Tg * T0 / p0 * dk)
    a3 = 1j * k2 * (-dk * k2 * (cg2 + vA2)
                    + (g - 1.0) * q_Tg * T0 / r0 * (4.0 / 3.0 + g * cr2 / cg2 + g * vA2 / cg2)
                    - q_Tr * T0 / r0 * (cg2 / (9.0 * cr2) + (g - 1.0) / 3.0 + vA2 / (9.0 * cr2)))
    a2 = k2 * k2 * ((g - 1.0) * (-q_Tg * T0 / r0 * dk) * (1.0 + g * vA2 / cg2)
                    + vAx2 * (cr2 + cg2))
    a1 = 1j * k2 * k2 * vAx2 * (k2 * cg2 * dk
                                - q_Tg * T0 / r0 * (g - 1.0) * (g * cr2 / cg2 + 4.0 / 3.0)
                                + q_Tr * T0 / r0 * ((g - 1.0) / 3.0 + cg2 / (9.0 * cr2)))
    a0 = k2 ** 3 * (g - 1.0) * vAx2 * q_Tg * T0 / r0 * dk
    hexic = np.array([a6, a5, a4, a3, a2, a1, a0], dtype=complex)
    alfven = np.array([1.0, 0.0, -k2 * vAx2], dtype=complex)
    return np.polymul(alfven, hexic)


def hydro_frozen(bg):
    """Eigenfrequencies of the (p, E) block with rho_1 = v_1 = B_1 = 0."""
    M = mode_matrix(bg)
    idx = [4, 7]
    return np.linalg.eigvals(M[np.ix_(idx, idx)])


def substep_amplification(dt, c, kappa, rho, a_r, T0, gamma, R_gas, D, ktilde2):
    """Per-step amplification of a Fourier mode (e_1, E_1) under the split substep.

    Diffusion multiplies E_1 by 1/(1 + dt D ktilde^2); the backward-Euler exchange
    linearised about E_0 = a_r T0^4 multiplies (e_1, E_1) by (I - dt J)^-1 with
    J = c kappa rho [[-beta, 1], [beta, -1]], beta = 4 a_r T0^3 / (rho c_v).
    """
    cv = R_gas / (gamma - 1.0)
    beta = 4.0 * a_r * T0 ** 3 / (rho * cv)
    J = c * kappa * rho * np.array([[-beta, 1.0], [beta, -1.0]])
    Dif = np.diag([1.0, 1.0 / (1.0 + dt * D * ktilde2)])
    return np.linalg.solve(np.eye(2) - dt * J, Dif)


def discrete_k2(k, h):
    """Eigenvalue of the 3-point second difference: (4/h^2) sin^2(k h / 2)."""
    return 4.0 / (h * h) * np.sin(0.5 * k * h) ** 2


# ----------------------------------------------------------------- code-unit linear mode
def code_units_background(ratio, B=1.0, angle_deg=45.0, rho0=1.0, T0=1.0, R_gas=1.0,
                          gamma=5.0 / 3.0, kappa=1.0e4, c=1.0e4, k=2.0 * np.pi):
    """Uniform radiative-equilibrium background in code units for the 3D linear-mode
    workload: p0 = rho0 R_gas T0, E0 = a_r T0^4 with a_r set by the radiation-to-gas
    pressure ratio (E0/3)/p0 = ratio, B of strength B in the x-z plane at angle_deg to
    k = k x-hat (Heaviside-Lorentz form, as in Appendix B)."""
    p0 = rho0 * R_gas * T0
    a_r = 3.0 * ratio * p0 / T0 ** 4
    th = np.deg2rad(angle_deg)
    return dict(rho0=rho0, p0=p0, B=np.array([B * np.cos(th), 0.0, B * np.sin(th)]),
                gamma=gamma, mu=None, kappa=kappa, T0=T0, E0=a_r * T0 ** 4, k=k, c=c,
                a_r=a_r, R_gas=R_gas)


def fast_mode(bg):
    """The forward fast magnetosonic eigenpair of the Appendix-B system: the eigenvalue
    with the largest real part, its eigenvector scaled so that the density component is
    rho0 (a unit relative density amplitude). Returns (omega, u) with u over
    (rho, v_x, v_y, v_z, p, B_y, B_z, E)."""
    w, V = np.linalg.eig(mode_matrix(bg))
    i = int(np.argmax(w.real))
    u = V[:, i] / V[0, i] * bg["rho0"]
    return w[i], u


def gas_temperature_amplitude(bg, u):
    """T_g,1 from the linearised ideal-gas law (Eq. ideal_gas_law_lin):
    T_1 = T0 (p_1/p0 - rho_1/rho0)."""
    return bg["T0"] * (u[4] / bg["p0"] - u[0] / bg["rho0"])


def hydro_frozen_code(bg):
    """Hydro-frozen (p, E) rates of a code-unit background (see hydro_frozen)."""
    return hydro_frozen(bg)
