"""The C-ABI library builds for sm_103a and exports every entry point include/fld.h
declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "fld.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fld_[a-z_0-9]+)\s*\(", txt)))


def test_library_builds_and_exports_all_symbols():
    from paper_2503_02764_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert "fld_step" in names and "fld_diffuse" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2503_02764_gb300 import fld
    for n in declared():
        assert hasattr(fld, n) or n in ("fld_default_opts", "fld_strerror"), n


def test_host_validation_without_gpu():
    # argument checks run on the host before any device work
    from paper_2503_02764_gb300 import fld
    L = fld.lib()
    h = fld.H()
    g = fld.make_grid((8,), (0.1,), ((0, 1),))       # periodic on one side only
    assert L.fld_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(fld.make_opts())) == fld.FLD_ERR_ARG
    g = fld.make_grid((1, 8), (0.1, 0.1), ((0, 0), (0, 0)))   # n < 2 on an active axis
    assert L.fld_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(fld.make_opts())) == fld.FLD_ERR_ARG
    g = fld.make_grid((8,), (0.1,), ((0, 0),))
    assert L.fld_create(ctypes.byref(h), ctypes.byref(g),
                        ctypes.byref(fld.make_opts(nu1=0, nu2=0))) == fld.FLD_ERR_ARG
    assert fld.strerror(fld.FLD_ERR_NOT_CONVERGED).startswith("multigrid")


def test_binding_structs_match_header_layout():
    # every ctypes mirror has the size and field offsets the C compiler gives the header's
    # struct (a wrong layout would pass garbage to the library without any error)
    import shutil
    import subprocess
    import pytest
    from paper_2503_02764_gb300 import build, fld
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = [fld.fld_consts, fld.fld_grid, fld.fld_opacity, fld.fld_opts, fld.fld_stats,
               fld.fld_prof_entry, fld.fld_batch_stat, fld.fld_wave1d_params,
               fld.fld_patch]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fld.h"', "int main(void) {"]
    for s in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s.__name__, s.__name__))
        for name, *_ in s._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));'
                         % (s.__name__, name, s.__name__, name))
    lines.append("return 0; }")
    os.makedirs(build.BUILD, exist_ok=True)
    src = os.path.join(build.BUILD, "abi_layout.c")
    exe = os.path.join(build.BUILD, "abi_layout")
    with open(src, "w") as f:
        f.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                   check=True)
    got = dict(l.split() for l in subprocess.run([exe], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s in structs:
        assert int(got[s.__name__]) == ctypes.sizeof(s), s.__name__
        for name, *_ in s._fields_:
            assert int(got["%s.%s" % (s.__name__, name)]) == getattr(s, name).offset, (s, name)


def test_wave1d_parameter_checks_without_gpu():
    # fld_wave1d_create validates its parameters on the host before any device work
    from paper_2503_02764_gb300 import fld, inputs as I
    L = fld.lib()
    P = I.wave1d(I.WAVE_BACKGROUNDS["strong"], 64, 4, "fast")
    w = fld.H()

    def rc(**change):
        p = fld.make_wave1d_params(P)
        for k, v in change.items():
            setattr(p, k, v)
        return L.fld_wave1d_create(ctypes.byref(w), ctypes.byref(p))

    assert rc(n=7) == fld.FLD_ERR_ARG                      # too few cells
    assert rc(n_driven=61) == fld.FLD_ERR_ARG              # driven region too long
    assert rc(n_driven=-1) == fld.FLD_ERR_ARG
    assert rc(dx=0.0) == fld.FLD_ERR_ARG
    assert rc(gamma=1.0) == fld.FLD_ERR_ARG
    assert rc(E_right=-1.0) == fld.FLD_ERR_ARG
    p = fld.make_wave1d_params(P)
    p.hat[0] = 2.0 * p.W0[0]                               # the drive would make rho < 0
    assert L.fld_wave1d_create(ctypes.byref(w), ctypes.byref(p)) == fld.FLD_ERR_ARG
    assert L.fld_wave1d_create(None, ctypes.byref(p)) == fld.FLD_ERR_ARG


def test_amr_box_checks_without_gpu():
    # fld_amr_create rejects boxes touching one wall without spanning the axis, empty or
    # out-of-range boxes and odd periodic extents on the host, before any device work
    from paper_2503_02764_gb300 import fld
    L = fld.lib()
    g = fld.make_grid((16, 16), (1.0, 1.0), ((1, 1), (1, 1)))
    for lo, hi in (((0, 4), (8, 10)), ((4, 4), (16, 10)), ((4, 4), (4, 10)), ((3, 2), (9, 17))):
        a = fld.H()
        rc = L.fld_amr_create(ctypes.byref(a), ctypes.byref(g),
                              ctypes.byref(fld.make_patch(lo, hi)), None)
        assert rc == fld.FLD_ERR_ARG, (lo, hi)
    g = fld.make_grid((16, 15), (1.0, 1.0), ((0, 0), (1, 1)))      # odd periodic extent
    a = fld.H()
    assert L.fld_amr_create(ctypes.byref(a), ctypes.byref(g),
                            ctypes.byref(fld.make_patch((3, 3), (9, 9))), None) == fld.FLD_ERR_ARG


def test_face_mean_and_diag_checks_without_gpu():
    # the harmonic face mean is refused on the host by MIXED_DF handles, the batched step
    # and the composite grid, constant prolongation by the batched step; unknown
    # face_mean, prolong or diag values by every create call
    from paper_2503_02764_gb300 import fld
    L = fld.lib()
    g = fld.make_grid((16, 16), (1.0, 1.0), ((1, 1), (1, 1)))
    for kw in (dict(precision=fld.PREC_MIXED_DF, face_mean=fld.FACE_HARM),
               dict(face_mean=2), dict(face_mean=-1), dict(diag=4), dict(diag=-1),
               dict(prolong=2), dict(prolong=-1)):
        o = fld.make_opts(**kw)
        h = fld.H()
        assert L.fld_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(o)) == \
            fld.FLD_ERR_ARG, kw
    arr = (fld.fld_grid * 2)(g, g)
    for o in (fld.make_opts(face_mean=fld.FACE_HARM), fld.make_opts(prolong=fld.PROLONG_CONSTANT)):
        b = fld.H()
        assert L.fld_batch_create(ctypes.byref(b), 2, arr, ctypes.byref(o)) == fld.FLD_ERR_ARG
    o = fld.make_opts(face_mean=fld.FACE_HARM)
    a = fld.H()
    assert L.fld_amr_create(ctypes.byref(a), ctypes.byref(g),
                            ctypes.byref(fld.make_patch((3, 3), (9, 9))),
                            ctypes.byref(o)) == fld.FLD_ERR_ARG


def test_normal_build_has_no_bounds_checks():
    # fld_debug_flags answers -1 from the normal build (no device call is made)
    from paper_2503_02764_gb300 import fld
    if os.environ.get("FLD_LIBRARY", "").endswith("_debug.so"):
        return
    assert fld.fld_debug_flags() == -1


def test_size_limits_and_degenerate_grids_without_gpu():
    # the host rejects, before any device work: a grid of 2^31 cells (32-bit indices), a
    # batch member above 2^27 cells, an axis of one cell, a negative or NaN spacing, and
    # a composite box of 2^31 or more fine cells (here the whole box refined: 2^33)
    from paper_2503_02764_gb300 import fld
    L = fld.lib()
    o = fld.make_opts()
    for shape, h in ((((1 << 11), (1 << 10), (1 << 10)), (1.0, 1.0, 1.0)),     # 2^31 cells
                     ((1, 8), (1.0, 1.0)),                                      # n = 1
                     ((8, 8), (1.0, -1.0)),
                     ((8, 8), (float("nan"), 1.0))):
        g = fld.make_grid(shape, h, ((0, 0),) * len(shape))
        hh = fld.H()
        assert L.fld_create(ctypes.byref(hh), ctypes.byref(g), ctypes.byref(o)) == \
            fld.FLD_ERR_ARG, shape
    big = fld.make_grid(((1 << 10), (1 << 9), (1 << 9)), (1.0, 1.0, 1.0), ((0, 0),) * 3)
    arr = (fld.fld_grid * 1)(big)                                               # 2^28 cells
    b = fld.H()
    assert L.fld_batch_create(ctypes.byref(b), 1, arr, ctypes.byref(o)) == fld.FLD_ERR_ARG
    assert L.fld_batch_create(ctypes.byref(b), 0, arr, ctypes.byref(o)) == fld.FLD_ERR_ARG
    g = fld.make_grid(((1 << 10), (1 << 10), (1 << 10)), (1.0, 1.0, 1.0), ((0, 0),) * 3)
    a = fld.H()
    assert L.fld_amr_create(ctypes.byref(a), ctypes.byref(g),
                            ctypes.byref(fld.make_patch((0, 0, 0), (1024, 1024, 1024))),
                            None) == fld.FLD_ERR_ARG                           # 2^33 fine cells
