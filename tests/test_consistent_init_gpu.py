"""The consistent initialisation on the GPU (fre_init_consistent: Sec. 2.3,
populations aligned by collisions before the simulated time starts) against
the oracle's, right after the passes and 200 steps later, on both lattices
and every device: FP64 relative L-inf < 1e-12 on rho, u, phi; FP32 1e-5 on
rho and phi and 1e-4 on u against max(|u|, 0.01), i.e. 1e-6 absolute (the
FP32 bounds of the row and per-node kernels; a droplet at rest has only
spurious currents of ~1e-4, against which FP32 rounding is not small)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DEV = {"shear": 0, "four_roller": 1, "periodic": 2}
CASES = [  # lattice, device, (nx, ny, nz), droplet, overrides
    ("d2q9", "shear", (100, 50, 1), (49.5, 24.5, 0.0, 10.0), dict(u_wall=0.01)),
    ("d2q9", "four_roller", (64, 64, 1), (31.5, 31.5, 0.0, 8.0), dict(u_wall=0.01)),
    ("d3q19", "shear", (40, 24, 20), (19.5, 11.5, 9.5, 6.0), dict(u_wall=0.02, tau_f=0.8)),
    ("d3q19", "periodic", (33, 21, 19), (16.0, 10.0, 9.0, 5.0), dict(tau_g=1.3)),
    ("d3q19", "four_roller", (32, 32, 6), (15.5, 15.5, 2.5, 5.0), dict(u_wall=0.01)),
]
BASE = dict(tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.0, rho0=1.0)


@pytest.fixture(scope="module")
def fre():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    return fre


def errs(a, b, u_floor=1e-300):
    uscale = max(max(np.abs(b[k]).max() for k in ("ux", "uy", "uz")), u_floor)
    return {k: np.abs(a[k] - b[k]).max() / (uscale if k.startswith("u") else np.abs(b[k]).max())
            for k in ("rho", "ux", "uy", "uz", "phi")}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}")
def test_consistent_init_matches_oracle(fre, orc, case, precision, tol):
    lattice, device, (nx, ny, nz), drop, kw = case
    a = dict(BASE, **kw)
    sim = fre.Simulation(lattice=lattice, precision=precision, device=device, nx=nx, ny=ny, nz=nz, **a)
    o = orc.Oracle({"d2q9": 0, "d3q19": 1}[lattice], DEV[device], nx, ny, nz, a["tau_f"], a["tau_g"], a["A"],
                   a["kappa"], a["gamma_mob"], a["u_wall"], a["rho0"])
    for s in (sim, o):
        s.init_droplet(*drop)
        s.init_consistent(60)
    assert sim.steps_taken == 0
    floor = 0.0 if precision == "fp64" else 0.01
    utol = tol if precision == "fp64" else 1e-4
    e0 = errs(sim.fields(), o.fields(), floor)
    for s in (sim, o):
        s.step(200)
    e1 = errs(sim.fields(), o.fields(), floor)
    sim.close()
    for e in (e0, e1):
        assert all(v < (utol if k.startswith("u") else tol) for k, v in e.items()), (e0, e1)


def test_consistent_init_16bit_and_state_rule(fre, orc):
    """FP16-dev storage follows the oracle within its storage tolerance
    (3e-4 on rho and phi after the passes and 100 steps); a stepped
    context refuses the call (FRE_ERR_STATE)."""
    a = dict(BASE, u_wall=0.03, tau_f=2.0, tau_g=2.0, gamma_mob=0.5)
    sim = fre.Simulation(lattice="d3q19", precision="fp16dev", device="shear", nx=64, ny=24, nz=16, **a)
    o = orc.Oracle(1, 0, 64, 24, 16, a["tau_f"], a["tau_g"], a["A"], a["kappa"], a["gamma_mob"], a["u_wall"],
                   a["rho0"])
    for s in (sim, o):
        s.init_droplet(31.5, 11.5, 7.5, 6.0)
        s.init_consistent(60)
        s.step(100)
    e = errs(sim.fields(), o.fields())
    assert e["rho"] < 3e-4 and e["phi"] < 3e-4, e
    with pytest.raises(fre.FreError) as ei:
        sim.init_consistent(5)
    assert ei.value.status == fre.FRE_ERR_STATE
    sim.close()
