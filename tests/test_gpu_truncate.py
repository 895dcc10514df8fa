"""V-cycle depth chosen from the operator (the truncate option): the solve stops coarsening
at the first level where a few red-black sweeps solve the coarse problem. Its iterate
solves the same system as the full-depth V-cycle's, to the tolerance, in every precision
mode; a stiff operator keeps every level."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host

pytestmark = pytest.mark.gpu


def _pyramid(shape, h):
    """(n, w, kdown) per level: the coarsening of an axis with n >= 4 to ceil(n/2) until
    at most 8 cells remain, w_d = (H_x/H_d)^2, kdown the K rescaling (H_x old / new)^2."""
    nd = len(shape)
    n = [shape[nd - 1 - d] for d in range(nd)]           # x first
    H = [h[d] for d in range(nd)]
    ln = [H[d] * n[d] for d in range(nd)]
    levels = []
    while True:
        levels.append((list(n), [(H[0] / H[d]) ** 2 for d in range(nd)]))
        if not any(v >= 4 for v in n) or np.prod(n) <= 8:
            break
        hx = H[0]
        for d in range(nd):
            if n[d] >= 4:
                n[d] = (n[d] + 1) // 2
                H[d] = ln[d] / n[d]
        levels[-1] = levels[-1] + ((hx / H[0]) ** 2,)
    return levels


def _expected_depth(shape, h, dt, D):
    """The depth rule restated: K_l <= max K times the rescalings, off-diagonal row sums
    s_l <= 2 K_l sum_d w_d, a sweep contracts by (s/(1+s))^2, at most 4 sweeps to 1e-2,
    above the first level of at most 512 cells (the single-block tail)."""
    lv = _pyramid(shape, h)
    kmax = float(np.float32(np.max(dt * D / (h[0] * h[0])))) * (1 + 1e-6)
    stop = next((l for l in range(len(lv) - 1) if np.prod(lv[l][0]) <= 512), len(lv) - 1)
    k = kmax
    for c in range(1, stop):
        k *= lv[c - 1][2]
        sw = 2.0 * k * sum(lv[c][1])
        rho = sw / (1.0 + sw)
        n = int(np.ceil(np.log(0.01) / (2.0 * np.log(rho)))) if rho > 0 else 1
        if 1 <= n <= 4:
            return c + 1, len(lv)
    return len(lv), len(lv)


CASES = [
    # (shape, h, bc, K_max target): a moderate K (truncated two levels below the finest),
    # a small one (truncated at level 1), a stiff one (every level)
    ((48, 40, 64), (1 / 64, 1 / 40, 1 / 48), ((0, 0), (0, 0), (2, 2)), 1.5),
    ((40, 36, 128), (1.0, 1.0, 1.0), ((0, 0), (1, 2), (2, 1)), 0.1),
    ((33, 45, 70), (1.0, 1.0, 1.0), ((1, 1), (2, 2), (0, 0)), 400.0),
    ((96, 112), (1.0, 1.0), ((0, 0), (1, 2)), 2.0),
]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("shape,h,bc,kmax", CASES)
def test_truncated_vcycle_solves_the_same_system(shape, h, bc, kmax, precision):
    torch = torch_cuda()
    fld = library()
    rng = np.random.default_rng(31 + len(shape) + shape[0])
    D = I.lognormal(rng, shape, 0.8, 4.0)
    dt = kmax * h[0] * h[0] / float(D.max())
    E = 1.0 + rng.uniform(0, 1, shape)
    Eb = {}
    nd = len(shape)
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1.0 + rng.uniform(0, 1, fs)
    packed = I.pack_dirichlet(shape, bc, Eb)
    depth, nlev = _expected_depth(shape, h, dt, D)
    tol = 1e-12 if precision == 0 else 1e-10
    A, g = O.assemble(D, h, bc, Eb, dt)
    bn = np.linalg.norm(E.ravel() + g)
    out = {}
    for truncate in (1, 0):
        hd = fld.Handle(shape, h, bc, precision=precision, tol=tol, max_cycles=60,
                        smoother=2, truncate=truncate)
        assert hd.levels == nlev
        Ed = dev(torch, E)
        st = hd.diffuse(dt, dev(torch, D), dev(torch, packed) if packed.size else None, Ed)
        assert st["levels"] == (depth if truncate else nlev), (st["levels"], depth, nlev)
        x = host(Ed).reshape(shape)
        true = O.relative_residual(x, E, D, h, bc, Eb, dt)
        assert true <= max(tol, st["rel_resid"]) * (1 + 1e-6) + 1e-14, (truncate, true, st)
        out[truncate] = (x, st)
        hd.close()
    (x1, s1), (x0, s0) = out[1], out[0]
    # the coarse solve to 1e-2 keeps the V-cycle's contraction: at most one more cycle
    assert s1["cycles"] <= s0["cycles"] + 1, (s1["cycles"], s0["cycles"])
    # both iterates solve A x = b to their residuals (||A^-1||_2 <= 1)
    dx = np.linalg.norm((x1 - x0).ravel())
    assert dx <= (s1["rel_resid"] + s0["rel_resid"]) * bn * (1 + 1e-6) + 2e-14 * bn


def test_depth_rule_cases_cover_truncated_and_full():
    # the cases above exercise a truncation at level 1, one deeper, and none
    depths = []
    for shape, h, bc, kmax in CASES:
        rng = np.random.default_rng(31 + len(shape) + shape[0])
        D = I.lognormal(rng, shape, 0.8, 4.0)
        dt = kmax * h[0] * h[0] / float(D.max())
        depths.append(_expected_depth(shape, h, dt, D))
    assert any(d == 2 for d, n in depths)
    assert any(2 < d < n for d, n in depths)
    assert any(d == n for d, n in depths)
