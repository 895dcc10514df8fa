"""Writes tests/golden/wave_damping.json: the spatial damping the oracle's 1D radiation-MHD
runs measure for the driven waves of Sect. 4.3.

TEST INFRASTRUCTURE (part of the CPU oracle): run by hand, it calls only oracle/ (and the
seeded input recipes). For each case (background of Table 2 or 3, fast or slow wave,
cells over 40 wavelengths, CFL 0.8, the ARS3 IMEX scheme), the oracle runs the radiative
problem and the same grid without radiation (the hyperbolic scheme's own damping, the same
ARS3 explicit stages with no implicit term) until the radiative front has travelled
`travel` wavelengths (t_end, the same for both runs), and fits the damping over the
wavelengths [1, travel - 3); it also stores Im k from the Appendix-B system at the driving frequency
and the printed damping per length. The resolution study is the strongly radiative slow
wave on 800, 1600, 2400 and 3200 cells. The time-step study is the weakly radiative fast
wave on 1600 cells at CFL 0.8, 0.4 and 0.2: there the stiff gas-radiation exchange makes
the IMEX scheme's error in the damping first order in dt.

    python -m oracle.write_wave_damping        (about ten minutes on eight cores)
    python -m oracle.write_wave_damping --missing    (only the cases the file lacks)
"""
import json
import multiprocessing as mp
import os
import sys
import time

from oracle import dispersion as Disp
from oracle import rmhd1d as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden", "paper_values.json")
OUT = os.path.join(ROOT, "tests", "golden", "wave_damping.json")

CFL = 0.8
NW = 40
CASES = ([("table3_strong", "slow", n, 20, CFL) for n in (800, 1600, 2400, 3200)] +
         [("table2_weak", "slow", 3200, 20, CFL), ("table2_weak", "fast", 3200, 20, CFL),
          ("table3_strong", "fast", 3200, 12, CFL)] +
         [("table2_weak", "fast", 1600, 12, c) for c in (0.8, 0.4, 0.2)])


STUDY = {("table2_weak", "fast", 1600)}      # the time-step study's grid


def key_of(case, kind, n, travel, cfl):
    k = "%s_%s_%d" % (case, kind, n)
    return k + "_cfl%g" % cfl if (case, kind, n) in STUDY else k


def run_case(args):
    from paper_2503_02764_gb300 import inputs as I
    case, kind, n, travel, cfl = args
    gold = json.load(open(GOLD))[case]
    bgd = gold["background"]
    t0 = time.time()
    P = I.wave1d(bgd, n, NW, kind)
    t_end = travel * P.lam / P.phase_speed
    last = travel - 3
    o = R.Wave(P, cfl=cfl, scheme="ars3")
    U, _, steps = o.run(t_end)
    k_meas = o.damping(U, 1, last)
    Pi = I.wave1d(bgd, n, NW, kind, radiation=False)
    oi = R.Wave(Pi, cfl=cfl, scheme="ars3")
    Ui, _, steps_i = oi.run(t_end)
    k_num = oi.damping(Ui, 1, last)
    bg = Disp.background(**{k: v for k, v in bgd.items() if not k.startswith("_")})
    im_k = R.spatial_damping(bg, P.omega, bg["k"]).imag
    return key_of(*args), {
        "case": case, "kind": kind, "n": n, "wavelengths": NW, "cfl": cfl, "scheme": "ars3",
        "travel": travel, "t_end": t_end, "fit": [1, last], "steps": steps,
        "steps_ideal": steps_i,
        "k_meas": k_meas, "k_num": k_num, "im_k": im_k,
        "printed": gold["damping_per_length_" + kind], "seconds": time.time() - t0}


def main():
    res = {}
    todo = CASES
    if "--missing" in sys.argv and os.path.exists(OUT):
        res = json.load(open(OUT))["cases"]
        todo = [c for c in CASES if key_of(*c) not in res]
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(len(todo), os.cpu_count() or 1))) as pool:
        res.update(dict(pool.map(run_case, todo)))
    data = {"written_by": "oracle/write_wave_damping.py",
            "about": "spatial damping (1/cm) measured by the oracle's ARS3 runs of the driven "
                     "waves of Sect. 4.3 (k_meas), the same grids without radiation (k_num, "
                     "the scheme's own damping), Im k of the Appendix-B system at the driving "
                     "frequency and the printed damping per length",
            "cases": res}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")
    print(OUT)


if __name__ == "__main__":
    main()
