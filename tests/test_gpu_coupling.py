"""GPU explicit coupling terms (fld_coupling) against the oracle: flux, radiation force and
its work, Eddington factor, photon tiring, on the seeded workloads."""
import numpy as np
import pytest

from oracle import fld as O
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, maxrel, consts_of, ebc_dev

pytestmark = pytest.mark.gpu


def _velocity(shape, seed):
    rng = np.random.default_rng(seed)
    # smooth-ish fields: a few Fourier modes plus noise, component d along physical axis d
    nd = len(shape)
    grids = np.meshgrid(*[np.linspace(0, 2 * np.pi, n, endpoint=False) for n in shape],
                        indexing="ij")
    out = []
    for d in range(nd):
        v = sum(rng.uniform(-1, 1) * np.sin((m + 1) * g + rng.uniform(0, 6))
                for m, g in enumerate(grids))
        out.append(v + 0.1 * rng.standard_normal(shape))
    return out


@pytest.mark.parametrize("cfg", [1, 2, 3])
@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_coupling_matches_oracle(cfg, limiter):
    torch = torch_cuda()
    fld = library()
    P = I.make_config(cfg, small=True)
    nd = len(P.shape)
    v = _velocity(P.shape, 100 + cfg)
    o = O.coupling(P.E, P.rho, P.T, P.h, P.bc, P.E_bc, P.c, P.opacity, v, mode=limiter)
    hd = fld.Handle(P.shape, P.h, P.bc, limiter=limiter)
    n = P.E.size
    Fd = torch.zeros(nd * n, dtype=torch.float64, device="cuda")
    frd = torch.zeros_like(Fd)
    fd = torch.zeros(n, dtype=torch.float64, device="cuda")
    vfrd, ptd = torch.zeros_like(fd), torch.zeros_like(fd)
    vd = dev(torch, np.concatenate([c.ravel() for c in v]))
    hd.coupling(consts_of(fld, P), fld.make_opacity(P.opacity), dev(torch, P.E), dev(torch, P.rho),
                dev(torch, P.T), ebc_dev(torch, P), vd, Fd, frd, fd, vfrd, ptd)
    torch.cuda.synchronize()
    F, fr = host(Fd).reshape((nd,) + P.shape), host(frd).reshape((nd,) + P.shape)
    for d in range(nd):
        assert maxrel(F[d], o["F"][d]) < 1e-12, ("F", d)
        assert maxrel(fr[d], o["fr"][d]) < 1e-12, ("fr", d)
    assert maxrel(host(fd).reshape(P.shape), o["f"]) < 1e-13
    assert maxrel(host(vfrd).reshape(P.shape), o["vfr"]) < 1e-12
    assert maxrel(host(ptd).reshape(P.shape), o["ptire"]) < 1e-12
    hd.close()


def test_coupling_optional_outputs_and_argument_errors():
    torch = torch_cuda()
    fld = library()
    P = I.make_config(3, small=True)
    o = O.coupling(P.E, P.rho, P.T, P.h, P.bc, P.E_bc, P.c, P.opacity)
    hd = fld.Handle(P.shape, P.h, P.bc)
    fd = torch.zeros(P.E.size, dtype=torch.float64, device="cuda")
    args = (consts_of(fld, P), fld.make_opacity(P.opacity), dev(torch, P.E), dev(torch, P.rho),
            dev(torch, P.T), ebc_dev(torch, P))
    hd.coupling(*args, f_edd=fd)              # only the Eddington factor
    torch.cuda.synchronize()
    assert maxrel(host(fd).reshape(P.shape), o["f"]) < 1e-13
    # the work terms need the velocity; Dirichlet sides need their face values
    with pytest.raises(fld.FldError):
        hd.coupling(*args, vfr=fd)
    with pytest.raises(fld.FldError):
        hd.coupling(*args[:5], None, f_edd=fd)
    hd.close()
