"""The CUDA path on the Taylor case of tests/golden/make_taylor.py (3D shear,
R = 14, R/H = 0.1, Ca = 0.05): FP32 storage and arithmetic reproduce the FP64
oracle's stored steady deformation to 1e-3 and Taylor's D = (35/32) Ca to 5%."""
import json
import os

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


def test_taylor_case_fp32(fre):
    with open(os.path.join(HERE, "taylor_d3q19.json")) as fh:
        g = json.load(fh)
    c = g["case"]
    sim = fre.Simulation(lattice="d3q19", precision="fp32", device="shear", nx=c["nx"], ny=c["ny"], nz=c["nz"],
                         tau_f=c["tau_f"], tau_g=c["tau_g"], A=c["A"], kappa=c["kappa"], gamma_mob=c["Gamma"],
                         u_wall=g["u_wall"], rho0=c["rho0"])
    sim.init_droplet((c["nx"] - 1) / 2, (c["ny"] - 1) / 2, (c["nz"] - 1) / 2, c["R"])
    sim.step(g["steps"])
    D = sim.observables()["D"]
    sim.close()
    assert abs(D - g["D"]) < 1e-3 * g["D"], (D, g["D"])
    taylor = 35.0 / 32.0 * g["Ca_end"]
    assert abs(D - taylor) < 0.05 * taylor, (D, taylor)
