"""Plain FP64 CPU oracle for the flux-limited-diffusion (FLD) radiation substep.

TEST INFRASTRUCTURE ONLY. This module is the slow, obviously correct reference
that the CUDA library is checked against. Only the tests, the smoke check and
the benchmark's CPU-baseline leg may import it; the library never does.

What it computes (paper: Sect. 2, Eqs. heating, qdot, fld_F, fld_lambda,
fld_R; Sect. 3 for the gradient stencil and for the implicit treatment of the
diffusion and exchange terms):

1. limiter:   grad E by the 4th-order 5-point central difference per axis
              (Sect. 3), R = |grad E| / (kappa rho E) (Eq. fld_R),
              lambda = (2 + R) / (6 + 3R + R^2) (Eq. fld_lambda, Levermore-
              Pomraning), D = c lambda / (kappa rho) (Eq. fld_F).
2. diffuse:   one backward-Euler step of dE/dt = div(D grad E) (the div F
              term of Eq. mhd_r_e with F = -D grad E), cell-centred finite
              volumes, face D = arithmetic mean of the two cell values (the
              harmonic mean 2 D_i D_j / (D_i + D_j) as an option);
              the linear system A x = b is solved directly (dense LU) or by
              Jacobi-preconditioned CG to a relative residual of 1e-14.
3. exchange:  backward Euler on de/dt = +qdot, dE/dt = -qdot with
              qdot = c rho kappa (E - a_r T^4) (Eqs. heating, qdot with equal
              opacities and E = a_r T_r^4), e = rho R_gas T / (gamma - 1)
              (Eqs. energy_density, ideal_gas_law). Eliminating E' gives the
              quartic rho c_v T' + (chi/(1+chi)) a_r T'^4 = e + chi E/(1+chi)
              with chi = dt c kappa rho, solved per cell by safeguarded Newton
              in extended precision; E' = (E + chi a_r T'^4)/(1 + chi).

Readings where the paper is silent (it defers to its multigrid library and to
the cited exchange papers): R and lambda are cell-centred; D is lagged (frozen
from E^n); the opacity is evaluated once from (rho, T^n); ghost values for the
gradient: periodic wrap, Neumann even mirror (E_-1 = E_0, E_-2 = E_1),
Dirichlet odd reflection about the face value E_b (E_-k = 2 E_b - E_{k-1});
the Dirichlet face flux in the solve is D_0 (x_0 - E_b) / (h/2); |grad E| = 0
gives R = 0.

Conventions: arrays in numpy order (z, y, x); h and bc in (x, y, z) order;
bc codes 0 periodic, 1 Neumann, 2 Dirichlet; E_bc maps (axis, side) to the
face array (the field's shape with that axis removed).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2


# ----------------------------------------------------------------- opacity
def opacity_table(kappa0, table, grid, rho, T):
    """Tabulated opacity: kappa0 times 10 to the bilinear interpolant of log10 kappa.

    The paper uses constant opacities and names opacity tables as the next step
    (Sect. 5). Reading taken here: ``table[j, i]`` holds log10 kappa at
    log10 rho = log_rho0 + i dlog_rho and log10 T = log_T0 + j dlog_T; a point is
    located by its fractional grid coordinates, clamped to the table (outside it the
    edge value holds), and log10 kappa is the bilinear interpolant of the four
    surrounding nodes.
    """
    log_rho0, dlog_rho, log_T0, dlog_T = grid
    n_T, n_rho = table.shape
    x = np.clip((np.log10(rho) - log_rho0) / dlog_rho, 0.0, n_rho - 1.0)
    y = np.clip((np.log10(T) - log_T0) / dlog_T, 0.0, n_T - 1.0)
    i = np.minimum(np.floor(x).astype(np.int64), n_rho - 2)
    j = np.minimum(np.floor(y).astype(np.int64), n_T - 2)
    fx, fy = x - i, y - j
    logk = ((1.0 - fx) * (1.0 - fy) * table[j, i] + fx * (1.0 - fy) * table[j, i + 1]
            + (1.0 - fx) * fy * table[j + 1, i] + fx * fy * table[j + 1, i + 1])
    return kappa0 * 10.0 ** logk


def opacity(op, rho, T):
    """kappa = kappa0 rho^a_rho T^a_T (constant when kind == 0); kind 2 is a table
    ``(2, kappa0, table, grid)`` read by ``opacity_table``.

    ``op = ("field", kappa)`` passes an already evaluated opacity through.
    """
    if op[0] == "field":
        return np.asarray(op[1])
    if op[0] == 2:
        return opacity_table(op[1], np.asarray(op[2]), op[3], np.asarray(rho, dtype=float),
                             np.asarray(T, dtype=float))
    kind, kappa0, a_rho, a_T = op
    if kind == 0:
        return np.full(np.shape(rho), kappa0, dtype=np.asarray(rho).dtype)
    return kappa0 * rho ** a_rho * T ** a_T


# ----------------------------------------------------------------- limiter
def lp_lambda(R):
    """Levermore-Pomraning flux limiter, Eq. fld_lambda."""
    return (2.0 + R) / (6.0 + 3.0 * R + R * R)


def minerbo_lambda(R):
    """Minerbo's flux limiter, which the paper implements (Sect. 2) but does not print; the
    published closed form: 2 / (3 + sqrt(9 + 12 R^2)) for R <= 3/2, else
    1 / (1 + R + sqrt(1 + 2R))."""
    R = np.asarray(R, dtype=float)
    lo = 2.0 / (3.0 + np.sqrt(9.0 + 12.0 * R * R))
    hi = 1.0 / (1.0 + R + np.sqrt(1.0 + 2.0 * R))
    return np.where(R <= 1.5, lo, hi)


def eddington_factor(lam, R):
    """Scalar Eddington factor f = lambda + lambda^2 R^2, Eq. fld_f."""
    return lam + lam * lam * R * R


def _npaxis(ndim, d):
    return ndim - 1 - d


def pad_ghosts(E, d, bc, E_bc, width=2):
    """Append `width` ghost layers on both sides of physical axis d."""
    ndim = E.ndim
    a = _npaxis(ndim, d)
    n = E.shape[a]

    def take(idx):
        return np.take(E, idx, axis=a)

    lo_kind, hi_kind = bc[d]
    lo, hi = [], []
    for k in range(1, width + 1):
        # low ghost at index -k, high ghost at index n-1+k
        if lo_kind == PERIODIC:
            lo.append(take((-k) % n))
        elif lo_kind == NEUMANN:
            lo.append(take(k - 1))
        else:
            lo.append(2.0 * E_bc[(d, 0)] - take(k - 1))
        if hi_kind == PERIODIC:
            hi.append(take((n - 1 + k) % n))
        elif hi_kind == NEUMANN:
            hi.append(take(n - k))
        else:
            hi.append(2.0 * E_bc[(d, 1)] - take(n - k))
    lo = [np.expand_dims(v, a) for v in reversed(lo)]     # order -width .. -1
    hi = [np.expand_dims(v, a) for v in hi]               # order n .. n-1+width
    return np.concatenate(lo + [E] + hi, axis=a)


def gradient5(E, h, bc, E_bc):
    """Per-axis 4th-order central difference (E_{i-2} - 8E_{i-1} + 8E_{i+1} - E_{i+2})/(12h)."""
    out = []
    ndim = E.ndim
    for d in range(ndim):
        a = _npaxis(ndim, d)
        P = pad_ghosts(E, d, bc, E_bc, 2)
        n = E.shape[a]

        def sl(off):
            idx = [slice(None)] * ndim
            idx[a] = slice(2 + off, 2 + off + n)
            return P[tuple(idx)]

        out.append((sl(-2) - 8.0 * sl(-1) + 8.0 * sl(1) - sl(2)) / (12.0 * h[d]))
    return out


def limiter(E, rho, T, h, bc, E_bc, c, op, mode=0):
    """Cell-centred D = c lambda / (kappa rho); returns (D, lambda, R).

    mode 0: Levermore-Pomraning lambda(R); mode 1: diffusion limit lambda = 1/3;
    mode 2: Minerbo lambda(R).
    """
    if np.any(~(E > 0)) or np.any(~(rho > 0)) or np.any(~(T > 0)):
        raise ValueError("E, rho and T must be positive and finite")
    kappa = opacity(op, rho, T)
    g = gradient5(E, h, bc, E_bc)
    gnorm = np.sqrt(sum(gi * gi for gi in g))
    R = gnorm / (kappa * rho * E)
    if mode == 0:
        lam = lp_lambda(R)
    elif mode == 2:
        lam = minerbo_lambda(R)
    else:
        lam = np.full(E.shape, 1.0 / 3.0)
    D = c * lam / (kappa * rho)
    return D, lam, R


def coupling(E, rho, T, h, bc, E_bc, c, op, v=None, mode=0):
    """Explicit coupling terms of the limiter pass (Sect. 3), from the same gradient.

    F = -D grad E (Eq. fld_F); the radiation force f_r = rho kappa F / c = -lambda grad E
    (Eq. rad_force with Eq. fld_F); the scalar Eddington factor f = lambda + lambda^2 R^2
    (Eq. fld_f); the Eddington tensor ((1 - f) I + (3f - 1) n n) / 2 with n = grad E /
    |grad E| (Eq. fld_Eddington_tensor; n n drops out where grad E = 0, since f = 1/3
    there); P = tensor E (Eq. fld_P). With a velocity field v (ndim components, v[d] along
    physical axis d): v . f_r and the photon-tiring term P : grad v = sum_ij P_ij d_j v_i,
    grad v by the same 5-point stencil with velocity ghosts wrapping on periodic axes and
    mirroring evenly at walls (zero gradient; the paper does not fix them).

    Returns a dict with F, fr (lists of ndim arrays), f, P (ndim x ndim nested lists),
    and vfr, ptire when v is given.
    """
    D, lam, R = limiter(E, rho, T, h, bc, E_bc, c, op, mode)
    g = gradient5(E, h, bc, E_bc)
    nd = E.ndim
    gnorm = np.sqrt(sum(gi * gi for gi in g))
    safe = np.where(gnorm > 0, gnorm, 1.0)
    n = [np.where(gnorm > 0, gi / safe, 0.0) for gi in g]
    f = eddington_factor(lam, R)
    P = [[(0.5 * (1.0 - f) * (1.0 if i == j else 0.0) + 0.5 * (3.0 * f - 1.0) * n[i] * n[j]) * E
          for j in range(nd)] for i in range(nd)]
    out = {"F": [-D * gi for gi in g], "fr": [-lam * gi for gi in g], "f": f, "P": P}
    if v is not None:
        out["vfr"] = sum(v[d] * out["fr"][d] for d in range(nd))
        bcv = tuple((PERIODIC, PERIODIC) if b[0] == PERIODIC else (NEUMANN, NEUMANN) for b in bc)
        gv = [gradient5(v[i], h, bcv, {}) for i in range(nd)]       # gv[i][j] = d_j v_i
        out["ptire"] = sum(P[i][j] * gv[i][j] for i in range(nd) for j in range(nd))
    return out


# ----------------------------------------------------------------- diffusion
def face_coefficient(Di, Dj, face_mean="arith"):
    """Face D between two cells: the arithmetic mean (D_i + D_j)/2, or the harmonic mean
    2 D_i D_j / (D_i + D_j), the face value for which the flux through cells of unequal
    D equals that of resistances h/D in series."""
    if face_mean == "arith":
        return 0.5 * (Di + Dj)
    if face_mean == "harm":
        return 2.0 * Di * Dj / (Di + Dj)
    raise ValueError(face_mean)


def assemble(D, h, bc, E_bc, dt, face_mean="arith"):
    """Backward-Euler matrix A and the Dirichlet right-hand-side term g.

    (A x)_i = x_i + sum over faces f of i of (dt/h_d^2) w_f (x_i - x_j),
    w_f = face_coefficient(D_i, D_j) for interior/periodic faces; a Dirichlet face adds
    (dt/h_d^2) 2 D_i (x_i - E_b), i.e. 2 dt D_i/h_d^2 to A_ii and
    2 dt D_i E_b/h_d^2 to g_i. Neumann faces carry no flux.
    """
    shape = D.shape
    ndim = D.ndim
    N = D.size
    idx = np.arange(N).reshape(shape)
    Df = D.ravel()
    rows, cols, vals = [], [], []
    diag = np.ones(N)
    g = np.zeros(N)
    for d in range(ndim):
        a = _npaxis(ndim, d)
        n = shape[a]
        s = dt / (h[d] * h[d])
        periodic = bc[d][0] == PERIODIC
        nfaces = n if periodic else n - 1
        for f in range(nfaces):
            i = np.take(idx, f, axis=a).ravel()
            j = np.take(idx, (f + 1) % n, axis=a).ravel()
            w = s * face_coefficient(Df[i], Df[j], face_mean)
            np.add.at(diag, i, w)
            np.add.at(diag, j, w)
            rows += [i, j]
            cols += [j, i]
            vals += [-w, -w]
        for side, cell in ((0, 0), (1, n - 1)):
            if bc[d][side] == DIRICHLET:
                i = np.take(idx, cell, axis=a).ravel()
                w = s * 2.0 * Df[i]
                np.add.at(diag, i, w)
                g[i] += w * np.asarray(E_bc[(d, side)]).ravel()
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A, g


def pcg(A, b, x0, rtol=1e-14, maxiter=100000):
    """Jacobi-preconditioned conjugate gradients (textbook form)."""
    Minv = 1.0 / A.diagonal()
    x = x0.copy()
    r = b - A @ x
    z = Minv * r
    p = z.copy()
    rz = r @ z
    bnorm = np.linalg.norm(b)
    it = 0
    while np.linalg.norm(r) > rtol * bnorm and it < maxiter:
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        z = Minv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


def diffuse(E, D, h, bc, E_bc, dt, method="auto", face_mean="arith"):
    """E^{n+1} = A^{-1}(E^n + g) for the backward-Euler diffusion step."""
    A, g = assemble(D, h, bc, E_bc, dt, face_mean)
    b = E.ravel() + g
    if method == "auto":
        method = "lu" if E.size <= 4096 else "pcg"
    if method == "lu":
        x = np.linalg.solve(A.toarray(), b)
    elif method == "splu":
        import scipy.sparse.linalg as sla
        x = sla.spsolve(A.tocsc(), b)
    else:
        x, _ = pcg(A, b, E.ravel().astype(np.float64))
    return x.reshape(E.shape)


def relative_residual(x, E, D, h, bc, E_bc, dt, face_mean="arith"):
    """||b - A x||_2 / ||b||_2 with b = E^n + g (plain sparse matvec)."""
    A, g = assemble(D, h, bc, E_bc, dt, face_mean)
    b = E.ravel() + g
    return np.linalg.norm(b - A @ x.ravel()) / np.linalg.norm(b)


def apply_operator(x, D, h, bc, dt, face_mean="arith"):
    """A x without boundary data (homogeneous Dirichlet), by direct stencil sums.

    A second, matrix-free statement of the same operator, used to check any
    subset of cells of a large grid one by one.
    """
    ndim = x.ndim
    out = x.copy()
    for d in range(ndim):
        a = _npaxis(ndim, d)
        s = dt / (h[d] * h[d])
        n = x.shape[a]
        for off in (-1, 1):
            xn = np.roll(x, -off, axis=a)
            Dn = np.roll(D, -off, axis=a)
            w = s * face_coefficient(D, Dn, face_mean)
            contrib = w * (x - xn)
            edge = [slice(None)] * ndim
            edge[a] = (n - 1) if off == 1 else 0
            side = 1 if off == 1 else 0
            if bc[d][side] != PERIODIC:
                contrib[tuple(edge)] = (2.0 * s * D[tuple(edge)] * x[tuple(edge)]
                                        if bc[d][side] == DIRICHLET else 0.0)
            out = out + contrib
    return out


# ----------------------------------------------------------------- exchange
def exchange(rho, T, E, dt, c, a_r, gamma, R_gas, op, return_iters=False):
    """Implicit gas-radiation energy exchange, cell by cell, in long double.

    f(T') = alpha T' + beta T'^4 - q = 0, alpha = rho c_v, beta = a_r chi/(1+chi),
    q = e + chi E/(1+chi). f is increasing and convex for T' > 0 with f(0) < 0,
    so there is exactly one positive root; min(q/alpha, (q/beta)^(1/4)) bounds
    it from above. Newton steps from that bound are kept inside the bracket
    [lo, hi] (bisection otherwise) until the step is below 4 ulp.
    """
    L = np.longdouble
    rho = np.asarray(rho, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    if np.any(~(rho > 0)) or np.any(~(T > 0)) or np.any(~(E > 0)):
        raise ValueError("rho, T and E must be positive and finite")
    kappa = opacity(op, rho, T).astype(L)
    rhoL, TL, EL = rho.astype(L), T.astype(L), E.astype(L)
    chi = L(dt) * L(c) * kappa * rhoL
    cv = L(R_gas) / (L(gamma) - L(1))
    alpha = rhoL * cv
    e = alpha * TL
    w = chi / (L(1) + chi)
    beta = w * L(a_r)
    q = e + w * EL
    hi = q / alpha
    with np.errstate(divide="ignore"):
        hi4 = np.where(beta > 0, np.sqrt(np.sqrt(q / np.where(beta > 0, beta, L(1)))), hi)
    hi = np.minimum(hi, hi4)
    lo = np.zeros_like(hi)
    t = hi.copy()
    eps = np.finfo(L).eps
    active = np.ones(t.shape, dtype=bool)
    iters = 0
    for iters in range(1, 400):
        t2 = t * t
        f = beta * t2 * t2 + alpha * t - q
        fp = L(4) * beta * t2 * t + alpha
        lo = np.where(f < 0, t, lo)
        hi = np.where(f > 0, t, hi)
        tn = t - f / fp
        bad = ~((tn > lo) & (tn < hi))
        tn = np.where(bad, L(0.5) * (lo + hi), tn)
        done = np.abs(tn - t) <= L(4) * eps * t
        t = np.where(active, tn, t)
        active &= ~done
        if not active.any():
            break
    En = (EL + chi * L(a_r) * t ** 4) / (L(1) + chi)
    out = (t.astype(np.float64), En.astype(np.float64))
    return out + (iters,) if return_iters else out


def internal_energy(rho, T, gamma, R_gas):
    return rho * R_gas * T / (gamma - 1.0)


# ----------------------------------------------------------------- substep
def step(rho, T, E, h, bc, E_bc, dt, c, a_r, gamma, R_gas, op, mode=0, method="auto",
         face_mean="arith"):
    """limiter -> backward-Euler diffusion -> exchange (opacity frozen at T^n).

    Returns (T', E', D). The exchange uses kappa(rho, T^n), the same value the
    limiter used.
    """
    D, _, _ = limiter(E, rho, T, h, bc, E_bc, c, op, mode)
    E1 = diffuse(E, D, h, bc, E_bc, dt, method, face_mean)
    kappa = opacity(op, rho, T)
    T2, E2 = exchange(rho, T, E1, dt, c, a_r, gamma, R_gas, ("field", kappa))
    return T2, E2, D
