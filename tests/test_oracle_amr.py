"""Pins of the oracle's composite-grid diffusion step (oracle/amr.py: a coarse block with
one patch refined by 2): the uniform fine grid when the patch covers the block, exact
conservation, symmetry of the flux form, constant and linear fields as fixed points (the
second pins the coarse-fine face's distance and area), and planted mistakes that these
catch."""
import numpy as np
import pytest

from oracle import amr as A
from oracle import fld as O


def _fields(shape_c, lo, hi, seed, sigma=1.0):
    rng = np.random.default_rng(seed)
    nd = len(shape_c)
    shape_f = tuple(2 * (hi[nd - 1 - a] - lo[nd - 1 - a]) for a in range(nd))
    Dc = np.exp(sigma * rng.standard_normal(shape_c))
    Df = np.exp(sigma * rng.standard_normal(shape_f))
    Ec = 1.0 + rng.uniform(0, 1, shape_c)
    Ef = 1.0 + rng.uniform(0, 1, shape_f)
    return Dc, Df, Ec, Ef


def _faces(shape, bc, rng):
    nd = len(shape)
    Eb = {}
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1.0 + rng.uniform(0, 1, fs)
    return Eb


def _fine_faces(Eb, nd):
    # the coarse face values under each fine face (every coarse face value repeated 2x per
    # tangential axis)
    out = {}
    for k, v in Eb.items():
        f = np.asarray(v)
        for ax in range(f.ndim):
            f = np.repeat(f, 2, axis=ax)
        out[k] = f
    return out


@pytest.mark.parametrize("shape,H,bc", [
    ((6, 8), (0.5, 0.25), ((0, 0), (2, 1))),
    ((4, 6, 5), (1.0, 1.0, 1.0), ((1, 2), (0, 0), (2, 2))),
])
def test_full_patch_is_the_uniform_fine_grid(shape, H, bc):
    nd = len(shape)
    nc = tuple(reversed(shape))
    G = A.Composite(shape, H, bc, (0,) * nd, nc)
    rng = np.random.default_rng(1)
    Dc, Df, Ec, Ef = _fields(shape, (0,) * nd, nc, 2)
    Eb = _faces(shape, bc, rng)
    dt = 0.3
    Mc, g = A.assemble(G, Dc, Df, Eb, dt)
    h = tuple(0.5 * v for v in H)
    Mu, gu = O.assemble(Df, h, bc, _fine_faces(Eb, nd), dt)
    assert abs(Mc - Mu).max() <= 1e-13 * abs(Mu).max()
    assert np.max(np.abs(g - gu)) <= 1e-13 * max(np.max(np.abs(gu)), 1.0)
    _, xf = A.diffuse(G, Ec, Ef, Dc, Df, Eb, dt)
    xu = O.diffuse(Ef, Df, h, bc, _fine_faces(Eb, nd), dt, method="lu")
    assert np.max(np.abs(xf - xu)) <= 1e-13 * np.max(np.abs(xu))


CASES = [
    ((8, 10), (1.0, 1.0), ((0, 0), (0, 0)), (3, 2), (7, 5)),           # periodic 2D
    ((8, 10), (0.5, 0.7), ((1, 1), (0, 0)), (2, 1), (5, 7)),           # Neumann x
    ((6, 7, 8), (1.0, 0.8, 1.2), ((0, 0), (1, 1), (0, 0)), (2, 1, 1), (5, 4, 3)),
    ((8, 6), (1.0, 1.0), ((0, 0), (1, 1)), (0, 2), (6, 6)),            # patch spans x
]


@pytest.mark.parametrize("shape,H,bc,lo,hi", CASES)
def test_conservation_and_symmetry(shape, H, bc, lo, hi):
    G = A.Composite(shape, H, bc, lo, hi)
    Dc, Df, Ec, Ef = _fields(shape, lo, hi, 3)
    dt = 2.0
    xc, xf = A.diffuse(G, Ec, Ef, Dc, Df, {}, dt)
    t0, t1 = A.total(G, Ec, Ef), A.total(G, xc, xf)
    assert abs(t1 - t0) <= 1e-13 * abs(t0)
    M, _ = A.assemble(G, Dc, Df, {}, dt)
    V = G.volumes()
    S = (sp_diag(V) @ (M - sp_eye(G.N))).toarray()
    assert np.max(np.abs(S - S.T)) <= 1e-14 * np.max(np.abs(S))
    # A = I + dt V^-1 L with L symmetric positive semi-definite: smallest eigenvalue >= 1
    Msym = np.diag(np.sqrt(V)) @ M.toarray() @ np.diag(1 / np.sqrt(V))
    assert np.min(np.linalg.eigvalsh(0.5 * (Msym + Msym.T))) >= 1 - 1e-12
    # a constant field is a fixed point
    cc, cf = A.diffuse(G, np.full(shape, 3.0), np.full(Ef.shape, 3.0), Dc, Df, {}, dt)
    assert np.max(np.abs(cf - 3.0)) < 1e-13 and np.max(np.abs(cc - 3.0)) < 1e-13


def sp_diag(v):
    import scipy.sparse as sp
    return sp.diags(v)


def sp_eye(n):
    import scipy.sparse as sp
    return sp.eye(n)


@pytest.mark.parametrize("axis", [0, 1])
def test_linear_field_along_an_axis_is_a_fixed_point(axis):
    # constant D, E linear along `axis` with Dirichlet walls carrying its face values: every
    # face flux, coarse-fine ones included, is D times the slope, so the step changes
    # nothing. This pins the coarse-fine face's centre distance (h + H)/2 and its area.
    # the patch spans the other (periodic) axis, so every coarse-fine face is normal to
    # `axis` (across a face normal to the other axis the two-point flux would see the
    # fine cells' tangential offset from the coarse centre)
    shape, H = (10, 12), (1.0, 1.0)
    bc = [(0, 0), (0, 0)]
    bc[axis] = (2, 2)
    bc = tuple(bc)
    lo, hi = [0, 0], [12, 10]
    lo[axis], hi[axis] = (4, 8) if axis == 0 else (3, 6)
    G = A.Composite(shape, H, bc, tuple(lo), tuple(hi))
    nd = 2
    nc = tuple(reversed(shape))
    xs_c = (np.arange(nc[axis]) + 0.5) * H[axis]
    xs_f = lo[axis] * H[axis] + (np.arange(2 * (hi[axis] - lo[axis])) + 0.5) * 0.5 * H[axis]
    slope, off = 0.37, 2.0

    def field(shape_np, xs):
        f = off + slope * xs
        sh = [1] * nd
        sh[nd - 1 - axis] = -1
        return np.broadcast_to(f.reshape(sh), shape_np).copy()

    shape_f = tuple(2 * (hi[nd - 1 - a] - lo[nd - 1 - a]) for a in range(nd))
    Ec, Ef = field(shape, xs_c), field(shape_f, xs_f)
    fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - axis)
    Eb = {(axis, 0): np.full(fs, off), (axis, 1): np.full(fs, off + slope * nc[axis] * H[axis])}
    Dc, Df = np.full(shape, 1.7), np.full(shape_f, 1.7)
    xc, xf = A.diffuse(G, Ec, Ef, Dc, Df, Eb, 5.0)
    assert np.max(np.abs(xf - Ef)) < 1e-12 and np.max(np.abs(xc - Ec)) < 1e-12


def test_planted_mistakes_fail_the_pins(monkeypatch):
    # a coarse-fine distance of h (instead of (h + H)/2) breaks the linear fixed point; a
    # flux counted on one side only breaks conservation
    orig = A.Composite.faces

    def wrong_distance(self, Dc, Df):
        inner, walls = orig(self, Dc, Df)
        out = []
        for p, q, a in inner:
            cf = (p >= self.ncoarse) != (q >= self.ncoarse)
            out.append((p, q, a * 1.5 if cf else a))
        return out, walls

    monkeypatch.setattr(A.Composite, "faces", wrong_distance)
    with pytest.raises(AssertionError):
        test_linear_field_along_an_axis_is_a_fixed_point(0)
    monkeypatch.setattr(A.Composite, "faces", orig)

    def one_sided(G, Dc, Df, E_bc, dt):
        inner, walls = G.faces(Dc, Df)
        V = G.volumes()
        import scipy.sparse as sp
        M = sp.lil_matrix((G.N, G.N))
        for i in range(G.N):
            M[i, i] = 1.0
        for p, q, a in inner:
            M[p, p] += dt * a / V[p]
            M[p, q] -= dt * a / V[p]
            M[q, q] += dt * a / V[p]           # wrong volume on the q side
            M[q, p] -= dt * a / V[p]
        return M.tocsr(), np.zeros(G.N)

    monkeypatch.setattr(A, "assemble", one_sided)
    with pytest.raises(AssertionError):
        test_conservation_and_symmetry(*CASES[0])
