"""The rounding bound of the recursive refinement residual, checked on the CPU.

The MIXED refinement updates its residual as r - A e with A e evaluated in FP32 on the
level's FP32 coefficients, and bounds what that adds to the gap to the true residual by
beta = 2^-20 (|r| + |e_c| + sum_d (w_d/2) sum_faces |(K_c + K_q)(e_c - e_q)|) per cell, plus
2^-53 ||A||_2 ||x + e||_2 for the FP64 rounding of x + e, with ||A||_2 bounded by the largest
absolute row sum and ||x + e||_2 by ||b||_2. Here the update is restated in numpy FP32
(every operation rounded to FP32; the kernel's fused multiply-adds round once where this
rounds twice, so its error is no larger), on inputs chosen to stress the bound: a rough
correction, K contrasts of several decades, every wall kind. The exact values are formed in
extended precision."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I

LD = np.longdouble
U53 = 2.0 ** -53


def _nb(a, d, side, bc, ghost):
    """Neighbour of every cell along axis d (x = 0; arrays are (z, y, x)) on `side` (-1/+1):
    a periodic wrap, or at a wall the ghost value `ghost(a_wall_cells, kind)`."""
    ax = a.ndim - 1 - d
    q = np.roll(a, -side, axis=ax)
    kind = bc[d][0 if side < 0 else 1]
    if kind != 0:
        sl = [slice(None)] * a.ndim
        sl[ax] = 0 if side < 0 else a.shape[ax] - 1
        q[tuple(sl)] = ghost(a[tuple(sl)], kind)
    return q


def _faces(e, K, bc, nd):
    """Per axis and side: (K_c + K_q, e_c - e_q) with the wall ghosts of the kernels
    (e = 0; K = 3 K_wall for Dirichlet, -K_wall for Neumann), in the arrays' own type."""
    out = []
    for d in range(nd):
        for side in (-1, 1):
            eq = _nb(e, d, side, bc, lambda v, kind: np.zeros_like(v))
            kq = _nb(K, d, side, bc,
                     lambda v, kind: (v * v.dtype.type(3)) if kind == 2 else -v)
            out.append((d, K + kq, e - eq))
    return out


def _problem(shape, bc, sigma, kmax, seed):
    rng = np.random.default_rng(seed)
    h = tuple(1.0 / n for n in shape[::-1])
    D = I.lognormal(rng, shape, sigma, 3.0)
    dt = kmax * h[0] * h[0] / float(D.max())
    E = 1.0 + rng.uniform(0, 1, shape)
    nd = len(shape)
    Eb = {}
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1.0 + rng.uniform(0, 1, fs)
    return h, D, dt, E, Eb


CASES = [
    ((12, 10, 14), ((0, 0), (1, 2), (2, 1)), 1.0, 2.0),
    ((9, 16, 8), ((2, 2), (0, 0), (1, 1)), 2.5, 300.0),
    ((8, 8, 12), ((0, 0), (0, 0), (0, 0)), 0.5, 0.05),
]


@pytest.mark.parametrize("shape,bc,sigma,kmax", CASES)
def test_recursive_residual_rounding_bound(shape, bc, sigma, kmax):
    nd = len(shape)
    h, D, dt, E, Eb = _problem(shape, bc, sigma, kmax, 11 + shape[0])
    w = [(h[0] / h[d]) ** 2 for d in range(nd)]
    K64 = dt * D / (h[0] * h[0])
    A, g = O.assemble(D, h, bc, Eb, dt)
    b = E.ravel() + g
    x_star = O.diffuse(E, D, h, bc, Eb, dt, method="lu").ravel()
    rng = np.random.default_rng(5)
    # an iterate near the solution, its FP64 residual, and a rough FP32 correction of the
    # residual's size
    x1 = x_star * (1.0 + 3e-8 * rng.standard_normal(x_star.size))
    r1 = b - A @ x1
    e = (np.abs(r1).max() * rng.standard_normal(shape)).astype(np.float32)

    # the update restated in FP32, in the kernel's order
    f32 = np.float32
    K32 = K64.astype(f32)
    hs = [f32(0.5) * f32(w[d]) for d in range(nd)]
    r1h = r1.reshape(shape).astype(f32)
    fac = _faces(e, K32, bc, nd)
    rv = r1h - e
    bnd = np.abs(r1h) + np.abs(e)
    rsum = np.zeros(shape, f32)
    for d in range(nd):
        (_, a1, d1), (_, a2, d2) = fac[2 * d], fac[2 * d + 1]
        p1, p2 = a1 * d1, a2 * d2
        rv = rv - hs[d] * (p1 + p2)
        bnd = bnd + hs[d] * (np.abs(p1) + np.abs(p2))
        rsum = rsum + hs[d] * (np.abs(a1) + np.abs(a2))
    amax = float((f32(1) + f32(2) * rsum).max())
    beta = 2.0 ** -20 * bnd.astype(np.float64)

    # exact: r1 - A64 e from the FP64 residual, the FP32 correction and the FP64 K
    eL, KL = e.astype(LD), K64.astype(LD)
    Ae = eL.copy()
    for d, a, df in _faces(eL, KL, bc, nd):
        Ae += LD(0.5 * w[d]) * a * df
    exact = r1.reshape(shape).astype(LD) - Ae
    gap = np.abs(rv.astype(LD) - exact)
    assert np.all(gap <= beta.astype(LD) * (1 + 1e-6)), float((gap / beta).max())
    # the bound is not vacuous: it is within a few decades of the actual rounding
    assert float((gap / beta).max()) > 1e-4

    # the FP64 rounding of x + e moves the true residual by at most 2^-53 amax ||b||
    x2 = x1 + e.ravel().astype(np.float64)
    delta = x2.astype(LD) - (x1.astype(LD) + e.ravel().astype(LD))
    Ad = _matvec_ld(A, delta)
    phi = 1.01 * U53 * amax * np.linalg.norm(b)
    assert float(np.sqrt(np.sum(Ad * Ad))) <= phi
    # the largest row sum bounds the operator's infinity norm (FP64 coefficients)
    assert np.asarray(abs(A).sum(axis=1)).ravel().max() <= 1.01 * amax
    # together: the recursive residual is within ||beta|| + phi of r1 - A (x2 - x1), the
    # residual of x2 taken from the FP64 residual of x1 (whose own rounding every
    # refinement scheme has)
    lhs = float(np.sqrt(np.sum((rv.ravel().astype(LD) - (exact.ravel() - Ad)) ** 2)))
    assert lhs <= (np.linalg.norm(beta) + phi) * (1 + 1e-6)


def _matvec_ld(A, v):
    """A v in extended precision (A's FP64 entries exact)."""
    A = A.tocsr()
    out = np.zeros(A.shape[0], dtype=LD)
    data = A.data.astype(LD)
    for i in range(A.shape[0]):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        out[i] = np.sum(data[lo:hi] * v[A.indices[lo:hi]])
    return out
