"""Batched substep (fld_step_batched: one persistent launch for many uneven problems)
against the oracle's substep, problem by problem."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, maxrel

pytestmark = pytest.mark.gpu


def _problems():
    ps = I.batch(5, nmin=32, nmax=70)
    # a Dirichlet-walled 2D member with Kramers opacity and a small 3D member
    s3 = I.stratified_3d(16, nz=12, ny=10)
    ps.append(s3)
    ps.append(I.lognormal_2d(40, ny=33, steps=1))
    return ps


def _concat(ps):
    cat = lambda xs: np.concatenate([np.ascontiguousarray(x).ravel() for x in xs])
    faces = [I.pack_dirichlet(p.shape, p.bc, p.E_bc) for p in ps]
    return cat([p.rho for p in ps]), cat([p.T for p in ps]), cat([p.E for p in ps]), cat(faces)


def _run(fld, torch, ps, **opts):
    b = fld.Batch([(p.shape, p.h, p.bc) for p in ps], **opts)
    rho, T, E, F = _concat(ps)
    rd, Td, Ed = dev(torch, rho), dev(torch, T), dev(torch, E)
    Fd = dev(torch, F) if F.size else None
    consts = fld.make_consts(ps[0].c, ps[0].a_r, ps[0].gamma, ps[0].R_gas)
    rc, st = b.step(consts, [fld.make_opacity(p.opacity) for p in ps], [p.dt for p in ps], rd, Td,
                    Ed, Fd, raise_on_error=False)
    return b, rc, st, (rd, Td, Ed, Fd), host(Td), host(Ed)


def _split(ps, v):
    out, o = [], 0
    for p in ps:
        out.append(v[o:o + p.ncells].reshape(p.shape))
        o += p.ncells
    return out


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("block,cluster", [(256, 1), (512, 1), (1024, 1), (256, 8), (512, 2),
                                           (512, 4), (1024, 8)])
def test_batch_matches_oracle(block, cluster, precision):
    # cluster > 1: a thread-block cluster shares each problem; precision 1 (MIXED): FP64
    # refinement, limiter and exchange, 2 (MIXED_DF): double-FP32
    torch = torch_cuda()
    fld = library()
    ps = _problems()
    b, rc, st, _, T, E = _run(fld, torch, ps, tol=1e-13, max_cycles=60, block=block,
                              cluster=cluster, precision=precision)
    assert rc in (0, 3), st
    for p, Tp, Ep, s in zip(ps, _split(ps, T), _split(ps, E), st):
        assert s["rel_resid"] < 1e-10, s
        To, Eo, _ = O.step(p.rho, p.T, p.E, p.h, p.bc, p.E_bc, p.dt, p.c, p.a_r, p.gamma,
                           p.R_gas, p.opacity, p.limiter, method="splu")
        assert maxrel(Ep, Eo) < 1e-10, (p.name, maxrel(Ep, Eo), s)
        assert maxrel(Tp, To) < 1e-10, (p.name, maxrel(Tp, To))


@pytest.mark.parametrize("cluster", [1, 4])
def test_batch_graph_replay_and_determinism(cluster):
    torch = torch_cuda()
    fld = library()
    ps = _problems()[:5]
    b, rc, st, (rd, Td, Ed, Fd), T1, E1 = _run(fld, torch, ps, tol=1e-10, graph=1,
                                               cluster=cluster)
    # a second step with the same pointers replays the captured graph
    consts = fld.make_consts(1.0, 1.0, 5 / 3, 1.0)
    ops = [fld.make_opacity(p.opacity) for p in ps]
    rc2, st2 = b.step(consts, ops, [p.dt for p in ps], rd, Td, Ed, Fd)
    T2, E2 = host(Td), host(Ed)
    # the same two steps without graphs give bitwise the same fields
    bb = fld.Batch([(p.shape, p.h, p.bc) for p in ps], tol=1e-10, graph=0, cluster=cluster)
    Tn, En = dev(torch, np.concatenate([p.T.ravel() for p in ps])), dev(torch, np.concatenate([p.E.ravel() for p in ps]))
    for _ in range(2):
        bb.step(consts, ops, [p.dt for p in ps], rd, Tn, En, None)
    assert np.array_equal(host(En), E2) and np.array_equal(host(Tn), T2)
    assert all(s["cycles"] >= 1 for s in st2)


def test_batch_domain_error_isolated():
    torch = torch_cuda()
    fld = library()
    ps = I.batch(3, nmin=32, nmax=40)
    ps[1].E = ps[1].E.copy()
    ps[1].E[3, 4] = -1.0
    b, rc, st, _, T, E = _run(fld, torch, ps, tol=1e-10)
    assert rc == fld.FLD_ERR_DOMAIN
    Es = _split(ps, E)
    assert np.array_equal(Es[1], ps[1].E)          # the bad problem is untouched
    assert st[1]["rel_resid"] == -1.0
    assert st[0]["rel_resid"] < 1e-10 and st[2]["rel_resid"] < 1e-10
    assert not np.array_equal(Es[0], ps[0].E)
