"""The travelling radiation-damped waves of Sect. 4.3 on the GPU at the paper's
resolutions (fld_wave1d_step with the ARS3 IMEX scheme, 40 wavelengths): the measured
spatial damping of the weakly and strongly radiative fast and slow waves against the
oracle's runs of the same problems (tests/golden/wave_damping.json, written by
oracle/write_wave_damping.py), against Im k of the Appendix-B dispersion relation at the
driving frequency and against the printed damping per length, once the hyperbolic scheme's
own damping (the same grid without radiation) is taken off; the resolution study of the
strongly radiative slow wave (800 to 3200 cells); and the time-step study of the weakly
radiative fast wave, whose error is first order in dt (the gas-radiation exchange there is
stiff by five orders of magnitude per step, and the IMEX scheme's final combination is not
stiffly accurate)."""
import json
import os

import pytest

from oracle import rmhd1d as R
from paper_2503_02764_gb300 import inputs as I
from gpu_util import torch_cuda, library, dev, host

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(__file__)
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_values.json")))
WAVES = json.load(open(os.path.join(HERE, "golden", "wave_damping.json")))["cases"]
OPTS = dict(precision=0, tol=1e-13, max_cycles=200)
_RUNS = {}


def _gpu_damping(c, radiation):
    key = (c["case"], c["kind"], c["n"], c["cfl"], radiation)
    if key in _RUNS:
        return _RUNS[key]
    torch_cuda()
    fld = library()
    P = I.wave1d(GOLD[c["case"]]["background"], c["n"], c["wavelengths"], c["kind"],
                 radiation=radiation)
    orc = R.Wave(P, cfl=c["cfl"], scheme="ars3")
    gpu = fld.Wave1D(P, scheme=1, **OPTS)
    Ud = dev(torch_cuda(), orc.initial())
    t_end = c["t_end"]          # the radiative front's travel time, for both runs
    t, n = 0.0, 0
    while t < t_end * (1.0 - 1e-12):
        dt = min(gpu.max_dt(Ud, c["cfl"]), t_end - t)
        assert gpu.step(Ud, t, dt)["status"] in (0, 3)
        t += dt
        n += 1
    gpu.close()
    k = orc.damping(host(Ud).reshape(8, -1), *c["fit"])
    _RUNS[key] = (k, n)
    return _RUNS[key]


def _error(c):
    """GPU damping (radiative minus the scheme's own) relative to Im k, minus one; the GPU
    runs reproduce the oracle's measured rates and step counts first."""
    k, steps = _gpu_damping(c, True)
    k_num, steps_i = _gpu_damping(c, False)
    assert steps == c["steps"] and steps_i == c["steps_ideal"]
    assert k == pytest.approx(c["k_meas"], rel=1e-6)
    assert k_num == pytest.approx(c["k_num"], rel=1e-6)
    return (k - k_num) / c["im_k"] - 1.0, (k - k_num) / c["printed"] - 1.0


# error bounds on the damping at 80 cells per wavelength and CFL 0.8, from the oracle's
# runs of the same problems with a margin: the strongly radiative waves within 8 %; the
# weakly radiative ones carry the scheme's first-order time error (the study below)
BOUND = {"table3_strong_fast_3200": 0.08, "table3_strong_slow_3200": 0.08,
         "table2_weak_fast_3200": 0.55, "table2_weak_slow_3200": 0.40}


@pytest.mark.parametrize("key", sorted(BOUND))
def test_damping_at_the_papers_resolution(key):
    c = WAVES[key]
    err, err_printed = _error(c)
    assert abs(err) <= BOUND[key], (key, err)
    assert abs(err_printed) <= BOUND[key] + 0.005, (key, err_printed)


def test_resolution_study_strong_slow_wave():
    # the paper's convergence study: the strongly radiative slow wave on 800 to 3200 cells
    # over 40 wavelengths. At 800 cells the scheme's own damping is four times the
    # radiative one, so the difference is noisy; from 1600 cells on the error shrinks
    errs = [abs(_error(WAVES["table3_strong_slow_%d" % n])[0]) for n in (800, 1600, 2400, 3200)]
    assert errs[1] > errs[2] > errs[3], errs
    assert errs[3] < errs[0] and errs[3] <= 0.08, errs


def test_time_step_study_weak_fast_wave():
    # the weakly radiative fast wave on 1600 cells, 12 wavelengths travelled, at CFL 0.8,
    # 0.4 and 0.2: the excess damping over Im k falls by about half per halving of dt
    errs = [_error(WAVES["table2_weak_fast_1600_cfl%g" % c])[0] for c in (0.8, 0.4, 0.2)]
    assert errs[0] > errs[1] > errs[2] > 0, errs
    for a, b in zip(errs, errs[1:]):
        assert 1.6 <= a / b <= 2.8, errs
    assert errs[2] <= 0.25, errs
