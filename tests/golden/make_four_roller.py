"""Writes tests/golden/four_roller_d3q19.json: the FP64 oracle's steady
deformation of a droplet at the stagnation point of the three-dimensional
four-roller device (rollers along z, interpolated bounce-back at their
surfaces), for the small-deformation check in planar extensional flow,
D = (35/16) Ca with Ca = mu eps R / sigma (viscosity ratio 1; the paper
compares its four-roller runs with this small-Ca theory, Sec. 3).

Two oracle runs: the droplet-free flow, from which the strain rate eps =
du_x/dx at the centre is measured once the flow is steady, and then a
droplet placed in that flow, stepped until its deformation settles.

Calls only oracle/.  Run from the repository root (about an hour on eight
cores):
    python tests/golden/make_four_roller.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

# Case: D3Q19 four-roller 128 x 128 x 48 (rollers of radius 16 about
# (63.5 +- 32, 63.5 +- 32), periodic in z), droplet R = 10 at the centre
# (the strain rate varies by under 1% over the droplet; the z images are
# 4.8 R apart), xi = 1, tau_f = 2 (mu = 0.5), small mobility as in the
# shear case (Gamma = 0.02), roller surface speed 0.01: Ca near 0.034, a
# quarter of the critical capillary number of planar extension at
# viscosity ratio 1 (at Ca = 0.05 this case deforms 16% beyond the linear
# theory), Reynolds number eps R^2 / nu below 0.05.
CASE = dict(nx=128, ny=128, nz=48, R=10.0, A=0.04, kappa=0.04, tau_f=2.0, tau_g=1.0, Gamma=0.02, rho0=1.0,
            u_wall=0.01, interp=1)
FLOW_STEPS = 4000    # droplet-free run (eps within 0.05% of its value at 16000 steps)
DROP_STEPS = 16000   # droplet run, sampled every SAMPLE steps: D overshoots within
                     # 5000 steps and relaxes over the box's viscous time
                     # (N^2 / nu ~ 3e4 steps), a few percent more
SAMPLE = 1000
AVG = 4              # D: mean of the last AVG samples
FIT = 8              # eps: slope of u_x over x within +-FIT nodes of the centre


def strain_rates(f, c):
    """eps_x = du_x/dx along the centre line in x, eps_y = du_y/dy along the
    centre line in y, least-squares slopes over +-FIT nodes about the
    centre (nodes c - 1 and c straddle it), averaged over z and over the
    two straddling lines."""
    x = np.arange(c - FIT, c + FIT)
    ux = f["ux"][:, c - 1:c + 1, c - FIT:c + FIT].mean(axis=(0, 1))
    uy = f["uy"][:, c - FIT:c + FIT, c - 1:c + 1].mean(axis=(0, 2))
    return float(np.polyfit(x, ux, 1)[0]), float(np.polyfit(x, uy, 1)[0])


def make(c):
    return oracle.Oracle(oracle.D3Q19, oracle.FOUR_ROLLER, c["nx"], c["ny"], c["nz"], c["tau_f"], c["tau_g"],
                         c["A"], c["kappa"], c["Gamma"], c["u_wall"], c["rho0"], interp=c["interp"])


def main():
    oracle.build()
    c = CASE
    shape = (c["nz"], c["ny"], c["nx"])
    t0 = time.time()
    # 1. the droplet-free flow
    o = make(c)
    one, zero = np.ones(shape), np.zeros(shape)
    o.init_fields(one, zero, zero, zero, -one)
    eps_hist = []
    for t in range(0, FLOW_STEPS, 2000):
        o.step(2000)
        ex, ey = strain_rates(o.fields(), c["nx"] // 2)
        eps_hist.append([t + 2000, ex, ey])
        print(f"flow {t + 2000:6d} eps_x={ex:.6e} eps_y={ey:.6e} ({time.time() - t0:.0f} s)", flush=True)
    eps, eps_y = eps_hist[-1][1], eps_hist[-1][2]
    flow = o.fields()
    # 2. a droplet (the oracle's initial profile) in that flow
    d = make(c)
    d.init_droplet((c["nx"] - 1) / 2, (c["ny"] - 1) / 2, (c["nz"] - 1) / 2, c["R"])
    phi = d.fields()["phi"]
    del d
    o.init_fields(flow["rho"], flow["ux"], flow["uy"], flow["uz"], phi)
    w0 = o.observables()["drop_weight"]
    hist = []
    for t in range(0, DROP_STEPS, SAMPLE):
        o.step(SAMPLE)
        ob = o.observables()
        hist.append([t + SAMPLE, ob["D"], ob["theta_deg"], ob["drop_weight"]])
        print(f"drop {t + SAMPLE:6d} D={ob['D']:.6f} theta={ob['theta_deg']:.2f} W={ob['drop_weight']:.1f} "
              f"({time.time() - t0:.0f} s)", flush=True)
    D = float(np.mean([h[1] for h in hist[-AVG:]]))
    sigma = (8.0 * c["kappa"] * c["A"] / 9.0) ** 0.5
    mu = c["rho0"] * (c["tau_f"] - 0.5) / 3.0
    r_end = c["R"] * (hist[-1][3] / w0) ** (1.0 / 3.0)
    ca_end = mu * eps * r_end / sigma
    out = {"what": "FP64 oracle, D3Q19 four-roller droplet, steady deformation in planar extension",
           "case": c, "flow_steps": FLOW_STEPS, "drop_steps": DROP_STEPS, "sample_every": SAMPLE, "avg_last": AVG,
           "fit_half_width": FIT, "eps": eps, "eps_y": eps_y, "eps_history": eps_hist, "D": D,
           "theta_deg": hist[-1][2], "drop_weight_start": w0, "R_end": r_end, "Ca": mu * eps * c["R"] / sigma,
           "Ca_end": ca_end, "taylor_D": 35.0 / 16.0 * ca_end, "history": hist,
           "writer": "tests/golden/make_four_roller.py"}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "four_roller_d3q19.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("D =", D, "(35/16) Ca_end =", out["taylor_D"], "eps =", eps, "eps_y =", eps_y)


if __name__ == "__main__":
    main()
