"""ctypes binding of oracle/cfld.c, the plain C restatement of the FLD substep.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle): loaded by the tests, which pin it to
oracle/fld.py, and by the benchmark's CPU-baseline leg, which times it on the host's
cores; never by the library. The shared object is built by __graft_entry__.build(), or
here on first use when it is missing or older than its source.

The same conventions as oracle/fld.py: arrays in numpy order (z, y, x); h and bc in
(x, y, z) order; bc codes 0 periodic, 1 Neumann, 2 Dirichlet; E_bc maps (axis, side) to
the face array; an opacity law is (kind, kappa0, a_rho, a_T) with kind 0 (constant) or 1
(kappa0 rho^a_rho T^a_T).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cfld.c")
LIB = os.path.join(HERE, "_build", "libcfld.so")
_lib = None


def build(force=False):
    """gcc -O3 with OpenMP when the compiler has it, else without."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    base = ["gcc", "-O3", "-fPIC", "-shared", "-o", LIB, SRC, "-lm"]
    if subprocess.run(base[:4] + ["-fopenmp"] + base[4:], capture_output=True).returncode != 0:
        subprocess.run(base, check=True, capture_output=True)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.c_void_p
        I3 = C.POINTER(C.c_int)
        D3 = C.POINTER(C.c_double)
        L.cfld_threads.restype = C.c_int
        L.cfld_threads.argtypes = [C.c_int]
        L.cfld_diffuse.restype = C.c_int
        L.cfld_diffuse.argtypes = [C.c_int, I3, D3, I3, I3, P, C.c_double, P, P, C.c_int,
                                   C.c_double, C.c_int, C.c_int, C.c_int, D3, I3]
        L.cfld_limiter.restype = None
        L.cfld_limiter.argtypes = [C.c_int, I3, D3, I3, I3, P, C.c_double, C.c_int, C.c_double,
                                   C.c_double, C.c_double, P, P, P, P]
        L.cfld_exchange.restype = None
        L.cfld_exchange.argtypes = [C.c_longlong, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_int, C.c_double, C.c_double,
                                    C.c_double, P, P, P]
        L.cfld_step.restype = C.c_int
        L.cfld_step.argtypes = [C.c_int, I3, D3, I3, I3, P, C.c_double, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_int, C.c_double, C.c_double,
                                C.c_double, P, P, P, C.c_int, C.c_double, C.c_int, C.c_int,
                                C.c_int, D3, I3]
        _lib = L
    return _lib


def threads(n=0):
    """Set the OpenMP thread count (n > 0) and return the count in use (1 without
    OpenMP)."""
    return lib().cfld_threads(int(n))


def _grid(shape, h, bc):
    nd = len(shape)
    n = (C.c_int * 3)(*(list(reversed(shape)) + [1] * (3 - nd)))
    hh = (C.c_double * 3)(*([float(v) for v in h] + [1.0] * (3 - nd)))
    lo = (C.c_int * 3)(*([int(b[0]) for b in bc] + [0] * (3 - nd)))
    hi = (C.c_int * 3)(*([int(b[1]) for b in bc] + [0] * (3 - nd)))
    return nd, n, hh, lo, hi


def _faces(shape, bc, E_bc):
    parts = [np.ascontiguousarray(E_bc[(d, s)], dtype=np.float64).ravel()
             for d in range(len(shape)) for s in (0, 1) if bc[d][s] == 2]
    return np.concatenate(parts) if parts else np.zeros(1)


def _law(op):
    kind, k0, ar, at = op
    if kind not in (0, 1):
        raise ValueError("the C restatement takes the constant and power opacity laws")
    return int(kind), float(k0), float(ar), float(at)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


METHODS = {"vcycle": 0, "pcg": 1}


def diffuse(E, D, h, bc, E_bc, dt, method="vcycle", tol=1e-10, max_it=500, nu=(2, 2)):
    """Backward-Euler diffusion step; returns (E^{n+1}, relative residual, iterations)."""
    nd, n, hh, lo, hi = _grid(E.shape, h, bc)
    x = np.ascontiguousarray(E, dtype=np.float64).copy()
    Dc = np.ascontiguousarray(D, dtype=np.float64)
    fb = _faces(E.shape, bc, E_bc)
    rel, it = C.c_double(), C.c_int()
    st = lib().cfld_diffuse(nd, n, hh, lo, hi, _p(fb), float(dt), _p(Dc), _p(x), METHODS[method],
                            float(tol), int(max_it), int(nu[0]), int(nu[1]), C.byref(rel),
                            C.byref(it))
    if st < 0:
        raise MemoryError("cfld_diffuse")
    return x, rel.value, it.value


def limiter(E, rho, T, h, bc, E_bc, c, op):
    nd, n, hh, lo, hi = _grid(E.shape, h, bc)
    kind, k0, ar, at = _law(op)
    D = np.empty(E.shape)
    Ec, rc, Tc = (np.ascontiguousarray(a, dtype=np.float64) for a in (E, rho, T))
    fb = _faces(E.shape, bc, E_bc)
    lib().cfld_limiter(nd, n, hh, lo, hi, _p(fb), float(c), kind, k0, ar, at, _p(Ec), _p(rc),
                       _p(Tc), _p(D))
    return D


def exchange(rho, T, E, dt, c, a_r, gamma, R_gas, op):
    kind, k0, ar, at = _law(op)
    rc = np.ascontiguousarray(rho, dtype=np.float64)
    Tn = np.ascontiguousarray(T, dtype=np.float64).copy()
    En = np.ascontiguousarray(E, dtype=np.float64).copy()
    lib().cfld_exchange(rc.size, float(dt), float(c), float(a_r), float(gamma), float(R_gas),
                        kind, k0, ar, at, _p(rc), _p(Tn), _p(En))
    return Tn, En


def step(rho, T, E, h, bc, E_bc, dt, c, a_r, gamma, R_gas, op, method="vcycle", tol=1e-10,
         max_it=500, nu=(2, 2)):
    """limiter -> diffuse -> exchange; returns (T', E', relative residual, iterations)."""
    nd, n, hh, lo, hi = _grid(E.shape, h, bc)
    kind, k0, ar, at = _law(op)
    rc = np.ascontiguousarray(rho, dtype=np.float64)
    Tn = np.ascontiguousarray(T, dtype=np.float64).copy()
    En = np.ascontiguousarray(E, dtype=np.float64).copy()
    fb = _faces(E.shape, bc, E_bc)
    rel, it = C.c_double(), C.c_int()
    st = lib().cfld_step(nd, n, hh, lo, hi, _p(fb), float(dt), float(c), float(a_r), float(gamma),
                         float(R_gas), kind, k0, ar, at, _p(rc), _p(Tn), _p(En), METHODS[method],
                         float(tol), int(max_it), int(nu[0]), int(nu[1]), C.byref(rel),
                         C.byref(it))
    if st < 0:
        raise MemoryError("cfld_step")
    return Tn, En, rel.value, it.value
