"""The CUDA path on the four-roller case of tests/golden/make_four_roller.py
(3D four-roller device with interpolated bounce-back at the rollers, droplet
R = 10 at the stagnation point, Ca near 0.034): FP32 storage and arithmetic,
the same two runs (droplet-free flow, then the droplet placed in it),
reproduce the FP64 oracle's strain rate to 1e-4 and steady deformation to
2e-3, and the small-deformation theory D = (35/16) Ca to 10%."""
import importlib.util
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def fre():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    return fre


def test_four_roller_case_fp32(fre):
    spec = importlib.util.spec_from_file_location("make_four_roller", os.path.join(HERE, "make_four_roller.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(HERE, "four_roller_d3q19.json")) as fh:
        g = json.load(fh)
    c = g["case"]
    kw = dict(lattice="d3q19", precision="fp32", device="four_roller", nx=c["nx"], ny=c["ny"], nz=c["nz"],
              tau_f=c["tau_f"], tau_g=c["tau_g"], A=c["A"], kappa=c["kappa"], gamma_mob=c["Gamma"],
              u_wall=c["u_wall"], rho0=c["rho0"], flags=fre.FRE_FLAG_INTERPOLATED_WALLS if c["interp"] else 0)
    shape = (c["nz"], c["ny"], c["nx"])
    n = int(np.prod(shape))
    sim = fre.Simulation(**kw)
    one, zero = np.ones(n), np.zeros(n)
    sim.init_fields(one, zero, zero, zero, -one)
    sim.step(g["flow_steps"])
    flow = sim.fields()
    eps, eps_y = mk.strain_rates(flow, c["nx"] // 2)
    assert abs(eps - g["eps"]) < 1e-4 * g["eps"], (eps, g["eps"])
    d = fre.Simulation(**kw)
    d.init_droplet((c["nx"] - 1) / 2, (c["ny"] - 1) / 2, (c["nz"] - 1) / 2, c["R"])
    phi = d.fields()["phi"]
    d.close()
    sim.init_fields(*[flow[k].ravel() for k in ("rho", "ux", "uy", "uz")], phi.ravel())
    Ds = []
    for _ in range(g["drop_steps"] // g["sample_every"]):
        sim.step(g["sample_every"])
        Ds.append(sim.observables()["D"])
    sim.close()
    D = float(np.mean(Ds[-g["avg_last"]:]))
    assert abs(D - g["D"]) < 2e-3 * g["D"], (D, g["D"])
    assert abs(D - g["taylor_D"]) < 0.10 * g["taylor_D"], (D, g["taylor_D"])
