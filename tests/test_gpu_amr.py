"""The composite-grid diffusion solve (fld_amr_*: a coarse block with one box refined by 2,
two-level scheme over the block's multigrid) against the oracle's assembled composite
system (oracle/amr.py, sparse LU), cell by cell on both grids, in 2D and 3D with every
boundary kind, a box inside the block and a box spanning an axis; conservation; the
NOT_CONVERGED status."""
import numpy as np
import pytest

from oracle import amr as A
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, maxrel

pytestmark = pytest.mark.gpu

# numpy shape of the coarse block, cell sizes and boundary kinds in (x, y, z) order, box
CASES = [
    ((24, 32), (1.0, 1.0), ((0, 0), (0, 0)), (10, 6), (22, 18), 2.0),
    ((20, 24), (0.5, 0.4), ((1, 2), (2, 1)), (4, 3), (15, 12), 0.05),
    ((16, 20, 12), (1.0, 1.0, 1.0), ((0, 0), (1, 2), (2, 2)), (3, 4, 2), (9, 12, 10), 1.0),
    ((18, 16), (1.0, 1.0), ((0, 0), (1, 1)), (0, 5), (16, 11), 3.0),     # box spans x
    ((8, 12, 16), (1.0, 1.0, 1.0), ((2, 2), (0, 0), (0, 0)), (0, 3, 2), (16, 9, 6), 0.7),
]


def _case(shape, bc, lo, hi, seed):
    rng = np.random.default_rng(seed)
    nd = len(shape)
    shape_f = tuple(2 * (hi[nd - 1 - a] - lo[nd - 1 - a]) for a in range(nd))
    Dc = I.lognormal(rng, shape, 1.0, 3.0)
    Df = I.lognormal(rng, shape_f, 1.0, 6.0)
    Ec = 1.0 + rng.uniform(0, 1, shape)
    Ef = 1.0 + rng.uniform(0, 1, shape_f)
    Eb = {}
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1.0 + rng.uniform(0, 1, fs)
    return Dc, Df, Ec, Ef, Eb


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("shape,h,bc,lo,hi,dt", CASES)
def test_amr_matches_composite_oracle(shape, h, bc, lo, hi, dt, precision):
    torch = torch_cuda()
    fld = library()
    Dc, Df, Ec, Ef, Eb = _case(shape, bc, lo, hi, sum(shape) + lo[0])
    G = A.Composite(shape, h, bc, lo, hi)
    xc, xf = A.diffuse(G, Ec, Ef, Dc, Df, Eb, dt)
    am = fld.Amr(shape, h, bc, lo, hi, precision=precision, tol=1e-13, max_cycles=100)
    packed = I.pack_dirichlet(shape, bc, Eb)
    Ecd, Efd = dev(torch, Ec), dev(torch, Ef)
    st = am.diffuse(dt, dev(torch, Dc), dev(torch, Df), dev(torch, packed) if packed.size else None,
                    Ecd, Efd, raise_on_error=False)
    assert st["status"] == 0, st
    # the two-level iteration contracts by a steady factor
    hist = st["resid_hist"]
    assert all(hist[i + 1] < 0.5 * hist[i] for i in range(len(hist) - 1)), hist
    gc, gf = host(Ecd).reshape(shape), host(Efd).reshape(xf.shape)
    assert maxrel(gf, xf) < 1e-12, maxrel(gf, xf)
    assert maxrel(gc, xc) < 1e-12, maxrel(gc, xc)
    am.close()


def test_amr_conserves_and_reports_not_converged():
    torch = torch_cuda()
    fld = library()
    shape, h, bc, lo, hi, dt = CASES[0]
    Dc, Df, Ec, Ef, _ = _case(shape, bc, lo, hi, 7)
    G = A.Composite(shape, h, bc, lo, hi)
    am = fld.Amr(shape, h, bc, lo, hi, tol=1e-14, max_cycles=100)
    Ecd, Efd = dev(torch, Ec), dev(torch, Ef)
    am.diffuse(dt, dev(torch, Dc), dev(torch, Df), None, Ecd, Efd, raise_on_error=False)
    t0 = A.total(G, Ec, Ef)
    t1 = A.total(G, host(Ecd).reshape(shape), host(Efd).reshape(Ef.shape))
    assert abs(t1 - t0) <= 1e-13 * abs(t0)
    am2 = fld.Amr(shape, h, bc, lo, hi, tol=1e-14, max_cycles=1)
    Ecd, Efd = dev(torch, Ec), dev(torch, Ef)
    st = am2.diffuse(dt, dev(torch, Dc), dev(torch, Df), None, Ecd, Efd, raise_on_error=False)
    assert st["status"] == fld.FLD_ERR_NOT_CONVERGED and st["cycles"] == 1
    assert st["rel_resid"] < st["resid_hist"][0]
