"""Writes the fast-mode amplitudes of the 3D linear-mode workload's initial state.

TEST INFRASTRUCTURE (part of the CPU oracle): run by hand, it calls only
oracle.dispersion and writes paper_2503_02764_gb300/linmode_eigen.json, which the input
recipe inputs.linear_mode_3d reads (the recipe module may not import the oracle). The
stored numbers are checked against a fresh computation by tests/test_oracle_dispersion.py.

For each radiation-to-gas pressure ratio of the workload (0.1 and 1): the code-unit
background (rho0 = T0 = R_gas = 1, gamma = 5/3, kappa = c = 1e4, B = 1 at 45 degrees to
k = 2 pi x-hat), the forward fast magnetosonic eigenpair of the Appendix-B system scaled
to a unit relative density amplitude, and from it the complex amplitudes of the gas
temperature (Eq. ideal_gas_law_lin) and of the radiation energy density.

    python -m oracle.write_linmode_eigen
"""
import json
import os

from oracle import dispersion as D

RATIOS = (0.1, 1.0)
OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2503_02764_gb300", "linmode_eigen.json")


def amplitudes(ratio):
    bg = D.code_units_background(ratio)
    w, u = D.fast_mode(bg)
    T1 = D.gas_temperature_amplitude(bg, u)
    return {"a_r": bg["a_r"], "E0": bg["E0"], "omega": [w.real, w.imag],
            "T1": [T1.real, T1.imag], "E1": [u[7].real, u[7].imag],
            "rho1": [u[0].real, u[0].imag]}


def main():
    data = {"written_by": "oracle/write_linmode_eigen.py",
            "about": "fast magnetosonic eigenmode of the Appendix-B system (k = 2 pi, B = 1 at "
                     "45 degrees to k, rho0 = T0 = 1, kappa = c = 1e4): complex amplitudes per "
                     "unit relative density amplitude, keyed by the radiation-to-gas pressure "
                     "ratio",
            "modes": {"%g" % r: amplitudes(r) for r in RATIOS}}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")
    print(OUT)


if __name__ == "__main__":
    main()
