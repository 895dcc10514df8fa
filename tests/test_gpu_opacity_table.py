"""Tabulated opacity (FLD_OPACITY_TABLE) through the C ABI against the oracle: limiter,
exchange, explicit coupling terms and the whole substep on the stratified box with a
table opacity; a table sampled from a power law against the power law itself; argument
errors (all caught on the host, before any launch)."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, handle_for, consts_of, ebc_dev, maxrel

pytestmark = pytest.mark.gpu


def _op(fld, torch, opacity):
    return fld.make_opacity(opacity, dev(torch, opacity[2]))


@pytest.mark.parametrize("limiter", [0, 1, 2])
@pytest.mark.parametrize("precision", [0, 2])
def test_limiter_with_table_matches_oracle(limiter, precision):
    torch = torch_cuda()
    fld = library()
    P = I.stratified_3d_table()
    hd = handle_for(fld, P, precision=precision, limiter=limiter)
    n = P.ncells
    D, lam = (torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(2))
    hd.limiter(consts_of(fld, P), _op(fld, torch, P.opacity), dev(torch, P.E), dev(torch, P.rho),
               dev(torch, P.T), ebc_dev(torch, P), D, lam)
    assert hd.status() == 0
    Do, lo, _ = O.limiter(P.E, P.rho, P.T, P.h, P.bc, P.E_bc, P.c, P.opacity, mode=limiter)
    assert maxrel(host(D).reshape(P.shape), Do) < 1e-12
    assert maxrel(host(lam).reshape(P.shape), lo) < 1e-12
    hd.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_exchange_with_table_matches_oracle(precision):
    torch = torch_cuda()
    fld = library()
    rho, T, E, _ = I.random_cells(65536 + 77, seed=9)
    table, grid = I.opacity_table(10.0, log_rho=(-2.0, 2.0), log_T=(-0.5, 1.5), n_rho=33,
                                  n_T=41)
    op = (I.OPACITY_TABLE, 0.5, table, grid)
    hd = fld.Handle((rho.size,), (1.0,), ((0, 0),), precision=precision)
    consts = (1.0, 1.0, 5 / 3, 1.0)
    for dt in (1e-6, 0.37, 1e4):
        Td, Ed = dev(torch, T), dev(torch, E)
        hd.exchange(fld.make_consts(*consts), _op(fld, torch, op), dt, dev(torch, rho), Td, Ed)
        assert hd.status() == 0
        To, Eo = O.exchange(rho, T, E, dt, *consts, op)
        assert np.max(np.abs(host(Td) / To - 1)) < 1e-12
        assert np.max(np.abs(host(Ed) / Eo - 1)) < 1e-12
    hd.close()


def test_coupling_with_table_matches_oracle():
    torch = torch_cuda()
    fld = library()
    P = I.stratified_3d_table()
    rng = np.random.default_rng(12)
    v = [rng.standard_normal(P.shape) for _ in range(3)]
    o = O.coupling(P.E, P.rho, P.T, P.h, P.bc, P.E_bc, P.c, P.opacity, v)
    hd = handle_for(fld, P)
    n = P.ncells
    z = lambda m: torch.zeros(m, dtype=torch.float64, device="cuda")
    Fd, frd, fd, vfrd, ptd = z(3 * n), z(3 * n), z(n), z(n), z(n)
    hd.coupling(consts_of(fld, P), _op(fld, torch, P.opacity), dev(torch, P.E), dev(torch, P.rho),
                dev(torch, P.T), ebc_dev(torch, P), dev(torch, np.concatenate([c.ravel() for c in v])),
                Fd, frd, fd, vfrd, ptd)
    assert hd.status() == 0
    F, fr = host(Fd).reshape((3,) + P.shape), host(frd).reshape((3,) + P.shape)
    for d in range(3):
        assert maxrel(F[d], o["F"][d]) < 1e-12
        assert maxrel(fr[d], o["fr"][d]) < 1e-12
    assert maxrel(host(fd).reshape(P.shape), o["f"]) < 1e-13
    assert maxrel(host(vfrd).reshape(P.shape), o["vfr"]) < 1e-12
    assert maxrel(host(ptd).reshape(P.shape), o["ptire"]) < 1e-12
    hd.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (2, 1e-10)])
def test_step_with_table_matches_oracle(precision, tol):
    torch = torch_cuda()
    fld = library()
    P = I.stratified_3d_table()
    hd = handle_for(fld, P, precision=precision, tol=1e-14, max_cycles=100)
    Td, Ed, rd = dev(torch, P.T), dev(torch, P.E), dev(torch, P.rho)
    ebc = ebc_dev(torch, P)
    op = _op(fld, torch, P.opacity)
    T, E = P.T.copy(), P.E.copy()
    for _ in range(2):
        st = hd.step(consts_of(fld, P), op, P.dt, rd, Td, Ed, ebc, raise_on_error=False)
        assert st["status"] in (0, 3) and st["rel_resid"] < 1e-13, st
        T, E, _ = O.step(P.rho, T, E, P.h, P.bc, P.E_bc, P.dt, P.c, P.a_r, P.gamma, P.R_gas,
                         P.opacity, P.limiter, method="splu")
    assert maxrel(host(Ed).reshape(P.shape), E) < tol
    assert maxrel(host(Td).reshape(P.shape), T) < tol
    hd.close()


def test_power_law_table_matches_power_law_kind():
    # a table sampled from kappa0 rho T^-3.5 over a range holding every cell: the bilinear
    # interpolant of its logs is the law itself, so D and the exchange agree to rounding
    torch = torch_cuda()
    fld = library()
    P = I.stratified_3d(32, nz=24, ny=20)
    kappa0 = P.opacity[1]
    lr = np.linspace(-2.5, 0.5, 7)
    lt = np.linspace(-0.5, 1.5, 5)
    X, Y = np.meshgrid(lr, lt, indexing="xy")
    table = np.log10(kappa0) + X - 3.5 * Y
    tab_op = (I.OPACITY_TABLE, 1.0, table, (lr[0], lr[1] - lr[0], lt[0], lt[1] - lt[0]))
    hd = handle_for(fld, P)
    n = P.ncells
    out = []
    for op in (fld.make_opacity(P.opacity), _op(fld, torch, tab_op)):
        D = torch.zeros(n, dtype=torch.float64, device="cuda")
        hd.limiter(consts_of(fld, P), op, dev(torch, P.E), dev(torch, P.rho), dev(torch, P.T),
                   ebc_dev(torch, P), D)
        Td, Ed = dev(torch, P.T), dev(torch, P.E)
        hd.exchange(consts_of(fld, P), op, P.dt, dev(torch, P.rho), Td, Ed)
        assert hd.status() == 0
        out.append((host(D), host(Td), host(Ed)))
    for a, b in zip(*out):
        assert maxrel(b, a) < 1e-12
    hd.close()


def test_table_argument_errors():
    torch = torch_cuda()
    fld = library()
    P = I.stratified_3d_table()
    kind, k0, table, grid = P.opacity
    td = dev(torch, table)
    n_T, n_rho = table.shape
    hd = handle_for(fld, P)
    D = torch.zeros(P.ncells, dtype=torch.float64, device="cuda")
    args = (dev(torch, P.E), dev(torch, P.rho), dev(torch, P.T), ebc_dev(torch, P), D)
    good = fld.make_opacity(P.opacity, td)
    hd.limiter(consts_of(fld, P), good, *args)
    assert hd.status() == 0
    bad = [
        fld.fld_opacity(kind, k0, 0.0, 0.0, None, n_rho, n_T, *grid),           # no table
        fld.fld_opacity(kind, k0, 0.0, 0.0, td.data_ptr(), 1, n_T, *grid),      # one column
        fld.fld_opacity(kind, k0, 0.0, 0.0, td.data_ptr(), n_rho, n_T, grid[0], 0.0, grid[2],
                        grid[3]),                                               # zero spacing
        fld.fld_opacity(kind, -1.0, 0.0, 0.0, td.data_ptr(), n_rho, n_T, *grid),  # kappa0 <= 0
    ]
    for op in bad:
        with pytest.raises(fld.FldError):
            hd.limiter(consts_of(fld, P), op, *args)
    with pytest.raises(fld.FldError):                       # T is needed by a table
        hd.limiter(consts_of(fld, P), good, args[0], args[1], None, args[3], D)
    with pytest.raises(fld.FldError):                       # the device table is required
        fld.make_opacity(P.opacity)
    with pytest.raises(fld.FldError):                       # and must hold n_T x n_rho values
        fld.make_opacity(P.opacity, td[:-1])
    hd.close()
    # the batched substep does not take tables
    ps = I.batch(2, nmin=32, nmax=40)
    b = fld.Batch([(p.shape, p.h, p.bc) for p in ps])
    cat = lambda xs: dev(torch, np.concatenate([x.ravel() for x in xs]))
    rd, Td, Ed = cat([p.rho for p in ps]), cat([p.T for p in ps]), cat([p.E for p in ps])
    consts = fld.make_consts(ps[0].c, ps[0].a_r, ps[0].gamma, ps[0].R_gas)
    rc, _ = b.step(consts, [good, good], [p.dt for p in ps], rd, Td, Ed, None,
                   raise_on_error=False)
    assert rc == fld.FLD_ERR_ARG
    b.close()
