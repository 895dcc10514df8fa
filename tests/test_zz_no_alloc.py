"""The allocation-free solve, fld_diffuse_static, against the handle-based fld_diffuse.

Some callers cannot allocate device memory: host codes that hand every byte of the GPU
to their own allocator, or code running where a call into the CUDA allocator is not
allowed. fld_diffuse_static serves them from a fixed array inside the library. This file
is collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host, maxrel


def _case(shape, bc, seed):
    rng = np.random.default_rng(seed)
    D = I.lognormal(rng, shape, 1.0, 4.0)
    E = 1.0 + rng.uniform(0, 1, shape)
    Eb = {}
    nd = len(shape)
    for d in range(nd):
        for s in (0, 1):
            if bc[d][s] == 2:
                fs = tuple(n for a, n in enumerate(shape) if a != nd - 1 - d)
                Eb[(d, s)] = 1.0 + rng.uniform(0, 1, fs)
    return D, E, I.pack_dirichlet(shape, bc, Eb)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-10), (2, 1e-10)])
def test_static_solve_matches_handle_solve_twice(precision, tol):
    torch = torch_cuda()
    fld = library()
    cases = [((20, 24, 32), (0.1, 0.1, 0.1), ((0, 0), (1, 1), (2, 2)), 0.02),
             ((96, 130), (1.0, 1.0), ((0, 0), (0, 0)), 4.0)]
    for shape, h, bc, dt in cases:
        D, E, packed = _case(shape, bc, sum(shape))
        opts = fld.make_opts(precision=precision, tol=1e-13, max_cycles=80)
        hd = fld.Handle(shape, h, bc, precision=precision, tol=1e-13, max_cycles=80, direct1d=0)
        Eref = dev(torch, E)
        ebc = dev(torch, packed) if packed.size else None
        ref = hd.diffuse(dt, dev(torch, D), ebc, Eref, raise_on_error=False)
        assert ref["status"] in (0, 3)
        grid = fld.make_grid(shape, h, bc)
        for call in range(2):                    # two calls in a row share the array
            Es = dev(torch, E)
            st = fld.fld_diffuse_static(grid, opts, dt, dev(torch, D), ebc, Es,
                                        raise_on_error=False)
            assert st["status"] == ref["status"], (call, st, ref)
            assert st["cycles"] == ref["cycles"], (call, st, ref)
            assert maxrel(host(Es), host(Eref)) < tol, (call, maxrel(host(Es), host(Eref)))


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-10), (2, 1e-10)])
def test_static_solve_at_the_cell_limit_allocates_nothing(precision, tol):
    """A 1D grid of exactly 131072 cells with Dirichlet faces, the deepest level pyramid
    the limit admits (15 levels, where the workspace's fit check and the 256-byte
    alignment of its pieces matter most): the same result as the handle solve on two
    calls in a row, and the device's free memory is unchanged across repeated calls."""
    torch = torch_cuda()
    fld = library()
    n = 131072
    shape, h, bc = (n,), (1.0 / n,), ((2, 2),)
    D, E, packed = _case(shape, bc, 5)
    dt = 10.0 / n ** 2
    opts = fld.make_opts(precision=precision, tol=1e-13, max_cycles=80)
    hd = fld.Handle(shape, h, bc, precision=precision, tol=1e-13, max_cycles=80, direct1d=0)
    Dd, ebc = dev(torch, D), dev(torch, packed)
    Eref = dev(torch, E)
    ref = hd.diffuse(dt, Dd, ebc, Eref, raise_on_error=False)
    assert ref["status"] in (0, 3)
    grid = fld.make_grid(shape, h, bc)
    outs = [dev(torch, E) for _ in range(3)]
    # the first call loads the library's kernels and its array on this device
    fld.fld_diffuse_static(grid, opts, dt, Dd, ebc, outs[0], raise_on_error=False)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for Es in outs[1:]:
        st = fld.fld_diffuse_static(grid, opts, dt, Dd, ebc, Es, raise_on_error=False)
        assert st["status"] == ref["status"] and st["cycles"] == ref["cycles"], (st, ref)
        assert maxrel(host(Es), host(Eref)) < tol, maxrel(host(Es), host(Eref))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_solve_rejects_oversized_grid():
    # the size check runs on the host before any device work
    from paper_2503_02764_gb300 import fld
    L = fld.lib()
    g = fld.make_grid((64, 64, 64), (1.0, 1.0, 1.0), ((0, 0),) * 3)      # 262144 > 131072
    st = fld.fld_stats()
    rc = L.fld_diffuse_static(ctypes.byref(g), None, 1.0, ctypes.c_void_p(16),
                              None, ctypes.c_void_p(16), ctypes.byref(st), None)
    assert rc == fld.FLD_ERR_ARG
