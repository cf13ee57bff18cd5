"""Writes tests/golden/taylor_d3q19.json: the FP64 oracle's steady deformation
of a droplet in the three-dimensional parallel-band shear device at small
capillary number, for the Taylor small-deformation check D = (35/32) Ca
(viscosity ratio 1; Taylor's small-Ca theory is the reference the paper
compares its shear runs with, Sec. 3.1).

Calls only oracle/.  Run from the repository root:
    python tests/golden/make_taylor.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

# Case: D3Q19 shear 128 x 140 x 84, droplet R = 14 (R/H = 0.1, so that the
# confinement by the walls, which raises D like (R/H)^3, stays small; the
# periodic images are 9R and 6R apart), xi = 1 (Cahn number 1/14), tau_f = 2
# (mu = rho0 cs^2 (tau_f - 1/2) = 0.5), Ca = 0.05 through u_w, Reynolds
# number rate R^2 / nu = 0.08.  The small mobility (Gamma = 0.02, M =
# Gamma (tau_g - 1/2) = 0.01) puts the run in the sharp-interface regime of
# Taylor's theory: with a five times larger mobility the diffusive
# relaxation of the interface raises D by about 7% at this resolution.
CASE = dict(nx=128, ny=140, nz=84, R=14.0, A=0.04, kappa=0.04, tau_f=2.0, tau_g=1.0, Gamma=0.02, rho0=1.0, Ca=0.05)
CHECK = 500         # steps between D samples
TOL = 5e-5          # steady when |D - D_prev| < TOL between samples
MAX_STEPS = 12000


def wall_speed(c):
    sigma = (8.0 * c["kappa"] * c["A"] / 9.0) ** 0.5
    mu = c["rho0"] * (c["tau_f"] - 0.5) / 3.0
    rate = c["Ca"] * sigma / (mu * c["R"])   # Ca = mu rate R / sigma
    return rate * c["ny"] / 2.0              # rate = 2 u_w / H, H = ny


def main():
    oracle.build()
    c = CASE
    uw = wall_speed(c)
    o = oracle.Oracle(oracle.D3Q19, oracle.SHEAR, c["nx"], c["ny"], c["nz"], c["tau_f"], c["tau_g"], c["A"],
                      c["kappa"], c["Gamma"], uw, c["rho0"])
    o.init_droplet((c["nx"] - 1) / 2, (c["ny"] - 1) / 2, (c["nz"] - 1) / 2, c["R"])
    w0 = o.observables()["drop_weight"]
    hist, steps, t0 = [], 0, time.time()
    while steps < MAX_STEPS:
        o.step(CHECK)
        steps += CHECK
        ob = o.observables()
        hist.append([steps, ob["D"], ob["theta_deg"], ob["drop_weight"]])
        print(f"{steps:6d} D={ob['D']:.6f} theta={ob['theta_deg']:.2f} W={ob['drop_weight']:.1f} "
              f"({time.time() - t0:.0f} s)", flush=True)
        if len(hist) >= 3 and abs(hist[-1][1] - hist[-2][1]) < TOL:
            break
    # radius of the droplet at the end, from its phi > 0 weight relative to
    # the start (the weight of a sphere scales with R^3)
    r_end = c["R"] * (hist[-1][3] / w0) ** (1.0 / 3.0)
    out = {"what": "FP64 oracle, D3Q19 shear droplet, steady deformation for the Taylor check",
           "case": c, "u_wall": uw, "check_every": CHECK, "steps": steps, "D": hist[-1][1],
           "theta_deg": hist[-1][2], "drop_weight_start": w0, "R_end": r_end,
           "Ca_end": c["Ca"] * r_end / c["R"], "history": hist, "writer": "tests/golden/make_taylor.py"}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "taylor_d3q19.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("D =", out["D"], "Taylor (35/32) Ca =", 35 / 32 * c["Ca"], "with end radius:", 35 / 32 * out["Ca_end"])


if __name__ == "__main__":
    main()
