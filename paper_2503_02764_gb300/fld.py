"""Thin ctypes binding of the C ABI in include/fld.h (argument marshalling only).

Every step of the substep runs in the CUDA library libfld_gb300.so; this module
only converts torch tensors to device pointers and Python numbers to the C
structs. Loading fails loudly if the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# the library (FLD_LIBRARY may name another build of it, such as the bounds-checked
# libfld_gb300_debug.so)
LIBPATH = os.environ.get("FLD_LIBRARY") or os.path.join(HERE, "libfld_gb300.so")

FLD_OK, FLD_ERR_ARG, FLD_ERR_DOMAIN, FLD_ERR_NOT_CONVERGED, FLD_ERR_TIMEOUT, FLD_ERR_CUDA, \
    FLD_ERR_NOMEM = range(7)
PREC_FP64, PREC_MIXED, PREC_MIXED_DF = 0, 1, 2
DIAG_ENERGY, DIAG_TIMES = 1, 2
FACE_ARITH, FACE_HARM = 0, 1
PROLONG_LINEAR, PROLONG_CONSTANT = 0, 1
LIMITER_LP, LIMITER_DIFFUSION, LIMITER_MINERBO = 0, 1, 2
OPACITY_CONST, OPACITY_POWER, OPACITY_TABLE = 0, 1, 2


class FldError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (status %d)" % (where, strerror(code), code))


class fld_consts(C.Structure):
    _fields_ = [("c", C.c_double), ("a_r", C.c_double), ("gamma", C.c_double), ("R_gas", C.c_double)]


class fld_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3),
                ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3)]


class fld_opacity(C.Structure):
    _fields_ = [("kind", C.c_int), ("kappa0", C.c_double), ("a_rho", C.c_double), ("a_T", C.c_double),
                ("table", C.c_void_p), ("n_rho", C.c_int), ("n_T", C.c_int),
                ("log_rho0", C.c_double), ("dlog_rho", C.c_double), ("log_T0", C.c_double),
                ("dlog_T", C.c_double)]


class fld_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("max_cycles", C.c_int),
                ("nu1", C.c_int), ("nu2", C.c_int), ("coarse_sweeps", C.c_int),
                ("limiter", C.c_int), ("block", C.c_int), ("smoother", C.c_int),
                ("graph", C.c_int), ("cluster", C.c_int), ("inner", C.c_int),
                ("direct1d", C.c_int), ("diag", C.c_int), ("face_mean", C.c_int),
                ("prolong", C.c_int), ("limiter_df", C.c_int), ("resid_update", C.c_int),
                ("truncate", C.c_int)]


class fld_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("rel_resid", C.c_double), ("resid_hist", C.c_double * 64),
                ("levels", C.c_int), ("energy_before", C.c_double), ("energy_after", C.c_double),
                ("t_ms", C.c_double * 4)]


class fld_prof_entry(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("level", C.c_int), ("launches", C.c_longlong),
                ("cells", C.c_longlong), ("ms", C.c_double)]


class fld_batch_stat(C.Structure):
    _fields_ = [("cycles", C.c_int), ("rel_resid", C.c_double), ("rel_resid0", C.c_double)]


class fld_wave1d_params(C.Structure):
    _fields_ = [("n", C.c_int), ("n_driven", C.c_int), ("dx", C.c_double), ("gamma", C.c_double),
                ("Bx", C.c_double), ("R_gas", C.c_double), ("consts", fld_consts),
                ("opacity", fld_opacity), ("E_right", C.c_double), ("W0", C.c_double * 8),
                ("hat", C.c_double * 8), ("k", C.c_double), ("omega", C.c_double),
                ("opts", fld_opts), ("scheme", C.c_int), ("radiation", C.c_int)]


class fld_patch(C.Structure):
    _fields_ = [("lo", C.c_int * 3), ("hi", C.c_int * 3)]


_lib = None
P = C.c_void_p
H = C.c_void_p


def lib():
    """Load libfld_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise ImportError("%s not built: run paper_2503_02764_gb300/build.py" % LIBPATH)
    L = C.CDLL(LIBPATH)
    sig = {
        "fld_default_opts": (None, [C.POINTER(fld_opts)]),
        "fld_create": (C.c_int, [C.POINTER(H), C.POINTER(fld_grid), C.POINTER(fld_opts)]),
        "fld_destroy": (C.c_int, [H]),
        "fld_debug_flags": (C.c_int, []),
        "fld_set_opts": (C.c_int, [H, C.POINTER(fld_opts)]),
        "fld_num_levels": (C.c_int, [H]),
        "fld_limiter": (C.c_int, [H, C.POINTER(fld_consts), C.POINTER(fld_opacity), P, P, P, P, P,
                                  P, P]),
        "fld_coupling": (C.c_int, [H, C.POINTER(fld_consts), C.POINTER(fld_opacity), P, P, P, P,
                                   P, P, P, P, P, P, P]),
        "fld_diffuse": (C.c_int, [H, C.c_double, P, P, P, C.POINTER(fld_stats), P]),
        "fld_exchange": (C.c_int, [H, C.POINTER(fld_consts), C.POINTER(fld_opacity), C.c_double,
                                   P, P, P, P]),
        "fld_step": (C.c_int, [H, C.POINTER(fld_consts), C.POINTER(fld_opacity), C.c_double, P, P,
                               P, P, C.POINTER(fld_stats), P]),
        "fld_get_status": (C.c_int, [H, P]),
        "fld_strerror": (C.c_char_p, [C.c_int]),
        "fld_prof_enable": (C.c_int, [H, C.c_int, C.c_int]),
        "fld_prof_read": (C.c_int, [H, C.POINTER(fld_prof_entry), C.c_int]),
        "fld_launch_count": (C.c_longlong, []),
        "fld_batch_create": (C.c_int, [C.POINTER(H), C.c_int, C.POINTER(fld_grid),
                                       C.POINTER(fld_opts)]),
        "fld_batch_destroy": (C.c_int, [H]),
        "fld_batch_set_opts": (C.c_int, [H, C.POINTER(fld_opts)]),
        "fld_batch_cells": (C.c_longlong, [H]),
        "fld_step_batched": (C.c_int, [H, C.POINTER(fld_consts), C.POINTER(fld_opacity),
                                       C.POINTER(C.c_double), P, P, P, P, C.POINTER(fld_batch_stat),
                                       P]),
        "fld_diffuse_static": (C.c_int, [C.POINTER(fld_grid), C.POINTER(fld_opts), C.c_double, P,
                                         P, P, C.POINTER(fld_stats), P]),
        "fld_wave1d_create": (C.c_int, [C.POINTER(H), C.POINTER(fld_wave1d_params)]),
        "fld_wave1d_destroy": (C.c_int, [H]),
        "fld_wave1d_max_dt": (C.c_int, [H, P, C.c_double, C.POINTER(C.c_double), P]),
        "fld_wave1d_step": (C.c_int, [H, P, C.c_double, C.c_double, C.POINTER(fld_stats), P]),
        "fld_ars3_tableau": (None, [C.POINTER(C.c_double)] * 4),
        "fld_ars3_stage": (C.c_int, [H, C.POINTER(fld_consts), C.POINTER(fld_opacity), C.c_double,
                                     C.c_int, P, P, P, P, P, P, C.POINTER(fld_stats), P]),
        "fld_amr_create": (C.c_int, [C.POINTER(H), C.POINTER(fld_grid), C.POINTER(fld_patch),
                                     C.POINTER(fld_opts)]),
        "fld_amr_destroy": (C.c_int, [H]),
        "fld_amr_diffuse": (C.c_int, [H, C.c_double, P, P, P, P, P, C.POINTER(fld_stats), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def strerror(code):
    return lib().fld_strerror(int(code)).decode()


def _ptr(t):
    """Device pointer of a contiguous CUDA float64 tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        return int(t)
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("fields must be contiguous float64 CUDA tensors")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _check(rc, where):
    if rc != FLD_OK:
        raise FldError(rc, where)


def make_grid(shape, h, bc):
    """fld_grid from a numpy-order shape, (x, y, z) spacings and ((lo, hi), ...) kinds."""
    g = fld_grid()
    nd = len(shape)
    g.ndim = nd
    n = list(reversed(shape)) + [1] * (3 - nd)
    for d in range(3):
        g.n[d] = int(n[d])
        g.h[d] = float(h[d]) if d < nd else 1.0
        g.bc_lo[d] = int(bc[d][0]) if d < nd else 0
        g.bc_hi[d] = int(bc[d][1]) if d < nd else 0
    return g


def make_opts(precision=PREC_FP64, tol=1e-10, max_cycles=50, nu1=2, nu2=2, coarse_sweeps=32,
              limiter=LIMITER_LP, block=0, smoother=0, graph=1, cluster=0, inner=1, direct1d=1,
              diag=0, face_mean=FACE_ARITH, prolong=PROLONG_LINEAR, limiter_df=0,
              resid_update=1, truncate=1):
    o = fld_opts()
    lib().fld_default_opts(C.byref(o))
    o.precision, o.tol, o.max_cycles = precision, tol, max_cycles
    o.nu1, o.nu2, o.coarse_sweeps, o.limiter, o.block = nu1, nu2, coarse_sweeps, limiter, block
    o.smoother = smoother
    o.graph = graph
    o.cluster = cluster
    o.inner = inner
    o.direct1d = direct1d
    o.diag = diag
    o.face_mean = face_mean
    o.prolong = prolong
    o.limiter_df = limiter_df
    o.resid_update = resid_update
    o.truncate = truncate
    return o


def make_consts(c, a_r, gamma, R_gas):
    return fld_consts(c, a_r, gamma, R_gas)


def make_opacity(op, table=None):
    """fld_opacity from (kind, kappa0, a_rho, a_T), or for a table from
    (OPACITY_TABLE, kappa0, log10 kappa array (n_T, n_rho), (log_rho0, dlog_rho, log_T0, dlog_T))
    with ``table`` the same values on the device (contiguous float64; the returned
    structure keeps a reference to it)."""
    kind = int(op[0])
    if kind != OPACITY_TABLE:
        _, k0, ar, at = op
        return fld_opacity(kind, float(k0), float(ar), float(at))
    _, k0, host_table, grid = op
    n_T, n_rho = host_table.shape
    if table is None or table.numel() != n_rho * n_T:
        raise FldError(FLD_ERR_ARG, "make_opacity: a table opacity needs its device table "
                       "(n_T x n_rho float64)")
    o = fld_opacity(kind, float(k0), 0.0, 0.0, _ptr(table), int(n_rho), int(n_T),
                    *(float(g) for g in grid))
    o._table = table
    return o


def stats_dict(st):
    n = min(st.cycles, 63)
    return {"cycles": st.cycles, "rel_resid": st.rel_resid, "levels": st.levels,
            "resid_hist": [st.resid_hist[i] for i in range(n + 1)],
            "energy_before": st.energy_before, "energy_after": st.energy_after,
            "t_ms": [st.t_ms[i] for i in range(4)]}


# ------------------------------------------------ C entry points, same names
def fld_create(grid, opts):
    h = H()
    _check(lib().fld_create(C.byref(h), C.byref(grid), C.byref(opts)), "fld_create")
    return h


def fld_destroy(h):
    _check(lib().fld_destroy(h), "fld_destroy")


def fld_set_opts(h, opts):
    _check(lib().fld_set_opts(h, C.byref(opts)), "fld_set_opts")


def fld_num_levels(h):
    return lib().fld_num_levels(h)


def fld_limiter(h, consts, opacity, E, rho, T, E_bc, D, lam=None, stream=None):
    _check(lib().fld_limiter(h, C.byref(consts), C.byref(opacity), _ptr(E), _ptr(rho), _ptr(T),
                             _ptr(E_bc), _ptr(D), _ptr(lam), _stream(stream)), "fld_limiter")


def fld_coupling(h, consts, opacity, E, rho, T, E_bc, v=None, F=None, fr=None, f_edd=None,
                 vfr=None, ptire=None, stream=None):
    _check(lib().fld_coupling(h, C.byref(consts), C.byref(opacity), _ptr(E), _ptr(rho), _ptr(T),
                              _ptr(E_bc), _ptr(v), _ptr(F), _ptr(fr), _ptr(f_edd), _ptr(vfr),
                              _ptr(ptire), _stream(stream)), "fld_coupling")


def fld_diffuse(h, dt, D, E_bc, E, stream=None, raise_on_error=True):
    st = fld_stats()
    rc = lib().fld_diffuse(h, float(dt), _ptr(D), _ptr(E_bc), _ptr(E), C.byref(st), _stream(stream))
    if raise_on_error:
        _check(rc, "fld_diffuse")
    return stats_dict(st) | {"status": rc}


def fld_diffuse_static(grid, opts, dt, D, E_bc, E, stream=None, raise_on_error=True):
    """The no-allocation solve: workspace in the library's fixed device array."""
    st = fld_stats()
    rc = lib().fld_diffuse_static(C.byref(grid), C.byref(opts) if opts is not None else None,
                                  float(dt), _ptr(D), _ptr(E_bc), _ptr(E), C.byref(st),
                                  _stream(stream))
    if raise_on_error:
        _check(rc, "fld_diffuse_static")
    return stats_dict(st) | {"status": rc}


def fld_exchange(h, consts, opacity, dt, rho, T, E, stream=None):
    _check(lib().fld_exchange(h, C.byref(consts), C.byref(opacity), float(dt), _ptr(rho), _ptr(T),
                              _ptr(E), _stream(stream)), "fld_exchange")


def fld_step(h, consts, opacity, dt, rho, T, E, E_bc, stream=None, raise_on_error=True):
    st = fld_stats()
    rc = lib().fld_step(h, C.byref(consts), C.byref(opacity), float(dt), _ptr(rho), _ptr(T),
                        _ptr(E), _ptr(E_bc), C.byref(st), _stream(stream))
    if raise_on_error:
        _check(rc, "fld_step")
    return stats_dict(st) | {"status": rc}


def fld_get_status(h, stream=None):
    return lib().fld_get_status(h, _stream(stream))


def fld_prof_enable(h, on=True, capacity=65536):
    _check(lib().fld_prof_enable(h, int(on), int(capacity)), "fld_prof_enable")


def fld_prof_read(h, cap=256):
    buf = (fld_prof_entry * cap)()
    n = lib().fld_prof_read(h, buf, cap)
    return [{"name": e.name.decode(), "level": e.level, "launches": e.launches, "cells": e.cells,
             "ms": e.ms} for e in buf[:n]]


def fld_debug_flags():
    """Bounds flags raised since the last call by the debug build of the library (cleared
    by the call); -1 from the normal build."""
    return lib().fld_debug_flags()


def fld_launch_count():
    return lib().fld_launch_count()


def fld_batch_create(grids, opts):
    h = H()
    arr = (fld_grid * len(grids))(*grids)
    _check(lib().fld_batch_create(C.byref(h), len(grids), arr, C.byref(opts)), "fld_batch_create")
    return h


def fld_batch_destroy(b):
    _check(lib().fld_batch_destroy(b), "fld_batch_destroy")


def fld_batch_set_opts(b, opts):
    _check(lib().fld_batch_set_opts(b, C.byref(opts)), "fld_batch_set_opts")


def fld_batch_cells(b):
    return lib().fld_batch_cells(b)


def fld_step_batched(b, nprob, consts, opacities, dts, rho, T, E, E_bc, stream=None,
                     raise_on_error=True):
    ops = (fld_opacity * nprob)(*opacities)
    dta = (C.c_double * nprob)(*[float(v) for v in dts])
    st = (fld_batch_stat * nprob)()
    rc = lib().fld_step_batched(b, C.byref(consts), ops, dta, _ptr(rho), _ptr(T), _ptr(E),
                                _ptr(E_bc), st, _stream(stream))
    if raise_on_error:
        _check(rc, "fld_step_batched")
    return rc, [{"cycles": x.cycles, "rel_resid": x.rel_resid, "rel_resid0": x.rel_resid0}
                for x in st]


class Batch:
    """Owns an fld_batch of independent grids; fields are concatenated in order."""

    def __init__(self, grids, **opts):
        self.grids = [make_grid(*g) for g in grids]
        self.nprob = len(grids)
        self.opts = make_opts(**opts)
        self.b = fld_batch_create(self.grids, self.opts)

    @property
    def cells(self):
        return fld_batch_cells(self.b)

    def set_opts(self, **opts):
        self.opts = make_opts(**opts)
        fld_batch_set_opts(self.b, self.opts)

    def step(self, consts, opacities, dts, rho, T, E, E_bc=None, stream=None, raise_on_error=True):
        return fld_step_batched(self.b, self.nprob, consts, opacities, dts, rho, T, E, E_bc,
                                stream, raise_on_error)

    def close(self):
        if self.b:
            fld_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Handle:
    """Owns an fld_handle for one grid; the methods are the C entry points."""

    def __init__(self, shape, h, bc, **opts):
        self.grid = make_grid(shape, h, bc)
        self.opts = make_opts(**opts)
        self.h = fld_create(self.grid, self.opts)
        self.shape = tuple(shape)

    def set_opts(self, **opts):
        self.opts = make_opts(**opts)
        fld_set_opts(self.h, self.opts)

    @property
    def levels(self):
        return fld_num_levels(self.h)

    def close(self):
        if self.h:
            fld_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def limiter(self, consts, opacity, E, rho, T, E_bc, D, lam=None, stream=None):
        fld_limiter(self.h, consts, opacity, E, rho, T, E_bc, D, lam, stream)

    def coupling(self, consts, opacity, E, rho, T, E_bc, v=None, F=None, fr=None, f_edd=None,
                 vfr=None, ptire=None, stream=None):
        fld_coupling(self.h, consts, opacity, E, rho, T, E_bc, v, F, fr, f_edd, vfr, ptire,
                     stream)

    def diffuse(self, dt, D, E_bc, E, stream=None, raise_on_error=True):
        return fld_diffuse(self.h, dt, D, E_bc, E, stream, raise_on_error)

    def exchange(self, consts, opacity, dt, rho, T, E, stream=None):
        fld_exchange(self.h, consts, opacity, dt, rho, T, E, stream)

    def step(self, consts, opacity, dt, rho, T, E, E_bc, stream=None, raise_on_error=True):
        return fld_step(self.h, consts, opacity, dt, rho, T, E, E_bc, stream, raise_on_error)

    def status(self, stream=None):
        return fld_get_status(self.h, stream)

    def prof_enable(self, on=True, capacity=65536):
        fld_prof_enable(self.h, on, capacity)

    def prof_read(self, cap=256):
        return fld_prof_read(self.h, cap)


# ------------------------------------------------ 1D radiation-MHD wave step
def fld_wave1d_create(params):
    w = H()
    _check(lib().fld_wave1d_create(C.byref(w), C.byref(params)), "fld_wave1d_create")
    return w


def fld_wave1d_destroy(w):
    _check(lib().fld_wave1d_destroy(w), "fld_wave1d_destroy")


def fld_wave1d_max_dt(w, U, cfl, stream=None):
    dt = C.c_double()
    _check(lib().fld_wave1d_max_dt(w, _ptr(U), float(cfl), C.byref(dt), _stream(stream)),
           "fld_wave1d_max_dt")
    return dt.value


def fld_wave1d_step(w, U, t, dt, stream=None, raise_on_error=True):
    st = fld_stats()
    rc = lib().fld_wave1d_step(w, _ptr(U), float(t), float(dt), C.byref(st), _stream(stream))
    if raise_on_error and rc not in (FLD_OK, FLD_ERR_NOT_CONVERGED):
        _check(rc, "fld_wave1d_step")
    return stats_dict(st) | {"status": rc}


def make_wave1d_params(problem, scheme=0, **opts):
    """fld_wave1d_params from a 1D wave problem (attributes n, n_driven, dx, gamma, Bx,
    R_gas, c, a_r, kappa, E0, W0, hat, k, omega), the time scheme (0 split, 1 ARS3) and the
    FLD substep's options."""
    p = fld_wave1d_params()
    p.scheme = int(scheme)
    p.radiation = 1 if getattr(problem, "radiation", True) else 0
    p.n, p.n_driven = int(problem.n), int(problem.n_driven)
    p.dx, p.gamma, p.Bx, p.R_gas = (float(problem.dx), float(problem.gamma), float(problem.Bx),
                                    float(problem.R_gas))
    p.consts = make_consts(problem.c, problem.a_r, problem.gamma, problem.R_gas)
    p.opacity = make_opacity((OPACITY_CONST, problem.kappa, 0.0, 0.0))
    p.E_right = float(problem.E0)
    for v in range(8):
        p.W0[v] = float(problem.W0[v])
        p.hat[v] = float(problem.hat[v])
    p.k, p.omega = float(problem.k), float(problem.omega)
    p.opts = make_opts(**opts)
    return p


class Wave1D:
    """Owns an fld_wave1d: the 1D radiation-MHD step on a caller's state U (device
    float64 [8][n])."""

    def __init__(self, problem, scheme=0, **opts):
        self.params = make_wave1d_params(problem, scheme, **opts)
        self.n = self.params.n
        self.w = fld_wave1d_create(self.params)

    def _state(self, U):
        if U.numel() != 8 * self.n:
            raise ValueError("the state must hold 8 x n float64 values")
        return U

    def max_dt(self, U, cfl, stream=None):
        return fld_wave1d_max_dt(self.w, self._state(U), cfl, stream)

    def step(self, U, t, dt, stream=None, raise_on_error=True):
        return fld_wave1d_step(self.w, self._state(U), t, dt, stream, raise_on_error)

    def close(self):
        if self.w:
            fld_wave1d_destroy(self.w)
            self.w = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------ ARS3 IMEX stages
def fld_ars3_tableau():
    """(A_ex, A_im, b, c) of ARS(2,3,3) as numpy arrays (3 x 3, 3 x 3, 3, 3)."""
    import numpy as np
    ae, ai, b, c = (C.c_double * 9)(), (C.c_double * 9)(), (C.c_double * 3)(), (C.c_double * 3)()
    lib().fld_ars3_tableau(ae, ai, b, c)
    return (np.array(ae[:]).reshape(3, 3), np.array(ai[:]).reshape(3, 3), np.array(b[:]),
            np.array(c[:]))


def fld_ars3_stage(h, consts, opacity, dt, stage, rho, T, E, E_bc, F_E=None, F_e=None,
                   stream=None, raise_on_error=True):
    st = fld_stats()
    rc = lib().fld_ars3_stage(h, C.byref(consts), C.byref(opacity), float(dt), int(stage),
                              _ptr(rho), _ptr(T), _ptr(E), _ptr(E_bc), _ptr(F_E), _ptr(F_e),
                              C.byref(st), _stream(stream))
    if raise_on_error and rc not in (FLD_OK, FLD_ERR_NOT_CONVERGED):
        _check(rc, "fld_ars3_stage")
    return stats_dict(st) | {"status": rc}


# ------------------------------------------------ composite grid (coarse block + refined box)
def make_patch(lo, hi):
    """fld_patch from (x, y, z)-ordered coarse-index bounds (absent axes: 0, 1)."""
    p = fld_patch()
    for d in range(3):
        p.lo[d] = int(lo[d]) if d < len(lo) else 0
        p.hi[d] = int(hi[d]) if d < len(hi) else 1
    return p


def fld_amr_create(grid, patch, opts):
    a = H()
    _check(lib().fld_amr_create(C.byref(a), C.byref(grid), C.byref(patch), C.byref(opts)),
           "fld_amr_create")
    return a


def fld_amr_destroy(a):
    _check(lib().fld_amr_destroy(a), "fld_amr_destroy")


def fld_amr_diffuse(a, dt, Dc, Df, E_bc, Ec, Ef, stream=None, raise_on_error=True):
    st = fld_stats()
    rc = lib().fld_amr_diffuse(a, float(dt), _ptr(Dc), _ptr(Df), _ptr(E_bc), _ptr(Ec), _ptr(Ef),
                               C.byref(st), _stream(stream))
    if raise_on_error:
        _check(rc, "fld_amr_diffuse")
    return stats_dict(st) | {"status": rc}


class Amr:
    """Owns an fld_amr: the diffusion solve on a coarse block (numpy shape `shape`, cell
    sizes h and boundary kinds bc in (x, y, z) order) with the box [lo, hi) refined by 2."""

    def __init__(self, shape, h, bc, lo, hi, **opts):
        self.grid = make_grid(shape, h, bc)
        self.patch = make_patch(lo, hi)
        self.opts = make_opts(**opts)
        self.a = fld_amr_create(self.grid, self.patch, self.opts)

    def diffuse(self, dt, Dc, Df, E_bc, Ec, Ef, stream=None, raise_on_error=True):
        return fld_amr_diffuse(self.a, dt, Dc, Df, E_bc, Ec, Ef, stream, raise_on_error)

    def close(self):
        if self.a:
            fld_amr_destroy(self.a)
            self.a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
