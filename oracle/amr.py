"""Composite-grid backward-Euler diffusion on a coarse block with one refined patch.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; never imported by the library).

The paper solves the implicit div F term over MPI-AMRVAC's block-adaptive hierarchy with
its octree multigrid library (Sect. 3) and refines by Loehner's criterion; it states
neither the coarse-fine discretisation nor the solver. Reading taken here (the smallest
block-structured case): a uniform coarse block of cells H_d and one box of it, the patch,
refined by 2 in every axis (cells h_d = H_d / 2). The unknowns are the coarse cells the
patch does not cover and every fine cell. For each cell p of volume V_p,

    (A x)_p = x_p + (dt / V_p) sum_faces a_f (x_p - x_q)
                  + (dt / V_p) sum_Dirichlet a_w (x_p - E_b),

with the face conductance a_f = (D_p + D_q)/2 * area_f / dist_f, dist_f the distance of the
two cell centres along the face normal: H_d between coarse cells, h_d between fine cells,
(h_d + H_d)/2 = 3 h_d / 2 between a fine cell and the coarse cell across the patch's edge,
where one coarse face meets 2^(d-1) fine faces (area h^(d-1) each); a Dirichlet wall face
has dist H_d / 2 (coarse) or h_d / 2 (fine). Every face flux enters the two cells it
separates with opposite signs, so the scheme conserves sum_p V_p x_p (periodic and Neumann
walls), V (A - I) / dt is symmetric, and with the patch covering the whole block the system
is the uniform fine grid's (oracle.fld.assemble at spacing h).

Patch placement: along each axis the patch either lies strictly inside the block (at least
one coarse cell from each wall) or spans the axis, in which case the axis's boundary
conditions apply to the fine cells (Dirichlet face values of the coarse face under each
fine face).

Conventions as oracle/fld.py: arrays in numpy order (z, y, x); h, bc and the patch box in
(x, y, z) order; lo/hi coarse indices of the box (hi exclusive); bc codes 0 periodic,
1 Neumann, 2 Dirichlet; E_bc maps (axis, side) to the coarse face array.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2


class Composite:
    """Index maps and geometry of a coarse block (numpy shape `shape`, cell sizes H in
    (x, y, z) order) with the patch [lo, hi) refined by 2."""

    def __init__(self, shape, H, bc, lo, hi):
        self.nd = len(shape)
        self.nc = tuple(int(v) for v in reversed(shape))              # (nx, ny, nz)[:nd]
        self.H = tuple(float(v) for v in H)
        self.h = tuple(0.5 * v for v in self.H)
        self.bc = tuple(tuple(b) for b in bc)
        self.lo, self.hi = tuple(lo), tuple(hi)
        for d in range(self.nd):
            n = self.nc[d]
            full = self.lo[d] == 0 and self.hi[d] == n
            inside = 1 <= self.lo[d] < self.hi[d] <= n - 1
            if not (full or inside):
                raise ValueError("patch must lie inside the block or span the axis")
        self.nf = tuple(2 * (self.hi[d] - self.lo[d]) for d in range(self.nd))
        self.Vc = float(np.prod(self.H))
        self.Vf = float(np.prod(self.h))
        # unknown numbering: uncovered coarse cells (coarse linear order), then fine cells
        self.cidx = {}
        k = 0
        for c in self.cells(self.nc):
            if not self.covered(c):
                self.cidx[c] = k
                k += 1
        self.ncoarse = k
        self.fidx = {}
        for f in self.cells(self.nf):
            self.fidx[f] = k
            k += 1
        self.N = k

    @staticmethod
    def cells(n):
        """(x, y, z) index tuples in the arrays' memory order (x fastest)."""
        for t in itertools.product(*[range(v) for v in reversed(n)]):
            yield tuple(reversed(t))

    def covered(self, c):
        return all(self.lo[d] <= c[d] < self.hi[d] for d in range(self.nd))

    def parent(self, f):
        return tuple(self.lo[d] + f[d] // 2 for d in range(self.nd))

    def coarse_neighbour(self, c, d, s):
        """Coarse cell across face (d, s) of coarse cell c, or None at a wall."""
        m = list(c)
        m[d] += s
        n = self.nc[d]
        if not 0 <= m[d] < n:
            if self.bc[d][0] != PERIODIC:
                return None
            m[d] %= n
        return tuple(m)

    def fine_neighbour(self, f, d, s):
        """('f', fine cell), ('c', coarse cell) or None (a wall) across face (d, s) of f."""
        m = list(f)
        m[d] += s
        if 0 <= m[d] < self.nf[d]:
            return ("f", tuple(m))
        if self.lo[d] == 0 and self.hi[d] == self.nc[d]:       # the patch spans this axis
            if self.bc[d][0] != PERIODIC:
                return None
            m[d] %= self.nf[d]
            return ("f", tuple(m))
        c = list(self.parent(f))
        c[d] += s
        return ("c", tuple(c))

    # ---- face lists: (p, q, a) with unknown indices p, q and conductance a
    def faces(self, Dc, Df):
        """Interior faces as (p, q, a_f) and wall faces as (p, a_w, E_b index info)."""
        Dcx = np.asarray(Dc).transpose()                     # index as [x, y, z]
        Dfx = np.asarray(Df).transpose()
        inner, walls = [], []
        nd = self.nd
        for c, p in self.cidx.items():
            for d in range(nd):
                area = self.Vc / self.H[d]
                for s in (-1, 1):
                    q = self.coarse_neighbour(c, d, s)
                    if q is None:
                        if self.bc[d][0 if s < 0 else 1] == DIRICHLET:
                            walls.append((p, Dcx[c] * area / (0.5 * self.H[d]), ("c", c, d, s)))
                        continue
                    if s < 0:
                        continue                      # each face once: from its low side
                    if not self.covered(q):
                        a = 0.5 * (Dcx[c] + Dcx[q]) * area / self.H[d]
                        inner.append((p, self.cidx[q], a))
            # coarse-fine faces are listed from the fine side below
        for f, p in self.fidx.items():
            for d in range(nd):
                area = self.Vf / self.h[d]
                for s in (-1, 1):
                    nb = self.fine_neighbour(f, d, s)
                    if nb is None:
                        if self.bc[d][0 if s < 0 else 1] == DIRICHLET:
                            walls.append((p, Dfx[f] * area / (0.5 * self.h[d]), ("f", f, d, s)))
                        continue
                    kind, g = nb
                    if kind == "f":
                        if s > 0:
                            a = 0.5 * (Dfx[f] + Dfx[g]) * area / self.h[d]
                            inner.append((p, self.fidx[g], a))
                    else:
                        a = 0.5 * (Dfx[f] + Dcx[g]) * area / (0.5 * (self.h[d] + self.H[d]))
                        inner.append((p, self.cidx[g], a))
        return inner, walls

    def volumes(self):
        V = np.empty(self.N)
        V[:self.ncoarse] = self.Vc
        V[self.ncoarse:] = self.Vf
        return V

    def wall_value(self, info, E_bc):
        """E_b at a wall face: the coarse face value (a fine face takes the value of the
        coarse face it lies in)."""
        kind, cell, d, s = info
        c = cell if kind == "c" else self.parent(cell)
        face = np.asarray(E_bc[(d, 0 if s < 0 else 1)])
        other = [c[e] for e in range(self.nd) if e != d]
        return float(face[tuple(reversed(other))]) if other else float(face)

    # ---- vectors: coarse and fine arrays <-> unknowns
    def pack(self, Ec, Ef):
        Ecx, Efx = np.asarray(Ec).transpose(), np.asarray(Ef).transpose()
        v = np.empty(self.N)
        for c, p in self.cidx.items():
            v[p] = Ecx[c]
        for f, p in self.fidx.items():
            v[p] = Efx[f]
        return v

    def unpack(self, v):
        """Coarse array (covered cells: the volume average of their fine cells) and the
        fine patch array, numpy order."""
        Ec = np.zeros(self.nc)
        Ef = np.zeros(self.nf)
        for c, p in self.cidx.items():
            Ec[c] = v[p]
        for f, p in self.fidx.items():
            Ef[f] = v[p]
        cnt = 2 ** self.nd
        for f in self.fidx:
            Ec[self.parent(f)] += Ef[f] / cnt
        return Ec.transpose().copy(), Ef.transpose().copy()


def assemble(G, Dc, Df, E_bc, dt):
    """The composite matrix A and the wall term g (b = E^n + g)."""
    inner, walls = G.faces(Dc, Df)
    V = G.volumes()
    rows, cols, vals = [], [], []
    diag = np.ones(G.N)
    g = np.zeros(G.N)
    for p, q, a in inner:
        diag[p] += dt * a / V[p]
        diag[q] += dt * a / V[q]
        rows += [p, q]
        cols += [q, p]
        vals += [-dt * a / V[p], -dt * a / V[q]]
    for p, a, info in walls:
        diag[p] += dt * a / V[p]
        g[p] += dt * a / V[p] * G.wall_value(info, E_bc)
    rows += list(range(G.N))
    cols += list(range(G.N))
    vals += list(diag)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(G.N, G.N)).tocsr()
    A.sum_duplicates()
    return A, g


def diffuse(G, Ec, Ef, Dc, Df, E_bc, dt):
    """One backward-Euler step on the composite grid (sparse LU). Returns (Ec', Ef')."""
    A, g = assemble(G, Dc, Df, E_bc, dt)
    x = sla.spsolve(A.tocsc(), G.pack(Ec, Ef) + g)
    return G.unpack(x)


def relative_residual(G, Ec, Ef, En_c, En_f, Dc, Df, E_bc, dt):
    """||b - A x||_2 / ||b||_2 of (Ec, Ef) for the step from (En_c, En_f)."""
    A, g = assemble(G, Dc, Df, E_bc, dt)
    b = G.pack(En_c, En_f) + g
    return float(np.linalg.norm(b - A @ G.pack(Ec, Ef)) / np.linalg.norm(b))


def total(G, Ec, Ef):
    """sum_p V_p x_p over the composite grid's cells."""
    v = G.pack(Ec, Ef)
    return float(np.dot(G.volumes(), v))
