"""Accuracy of the storage formats on the 64^3 twin of the 512x256x256
benchmark lattice (same A, kappa, tau, Gamma, wall speed; droplet R = 12
keeps R/H = 48/256): droplet deformation D, droplet volume and Laplace
pressure of FP32, FP16-deviation and BF16-deviation storage against the
FP64 oracle on the same lattice after the same number of steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = 64
STEPS = 2000
PAR = dict(tau_f=2.0, tau_g=2.0, A=0.04, kappa=0.04, gamma_mob=0.5, u_wall=0.03, rho0=1.0)
DROP = ((N - 1) / 2, (N - 1) / 2, (N - 1) / 2, 12.0)
REST = 8  # FRE_FLAG_REST_REFERENCE
# relative error bounds (D, volume, dp) after STEPS steps: FP32 rounding;
# 11 and 8 mantissa bits of the 16-bit stores, which hold f as deviations
# from the Couette equilibrium of the walls (flags 0, the default of the
# shear device) or from the rest equilibrium w_i rho0
# (FRE_FLAG_REST_REFERENCE).  The default FP16 form is held to 1e-3 in D.
# Measured on a GB300: FP32 2.7e-7 / 4.9e-6 / 2.6e-6; Couette reference
# FP16 4.1e-5 / 5.2e-6 / 1.1e-4, BF16 2.3e-4 / 5.8e-6 / 2.5e-4; rest
# reference FP16 3.2e-3 / 4.8e-6 / 2.5e-5, BF16 5.3e-2 / 5.6e-6 / 2.3e-3
# (the rest reference misses 1e-3 in D; the droplet volume is conserved to
# FP32 rounding in every format: the FP32 rest population of g closes
# sum_i g_i on the stored values)
BOUNDS = {("fp32", 0): (1e-6, 1e-5, 1e-4), ("fp16dev", 0): (1e-3, 1e-4, 1e-3), ("bf16dev", 0): (1e-3, 1e-4, 1e-3),
          ("fp16dev", REST): (1e-2, 1e-4, 1e-3), ("bf16dev", REST): (1e-1, 1e-4, 1e-2)}


@pytest.fixture(scope="module")
def fre():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    return fre


@pytest.fixture(scope="module")
def reference(orc):
    o = orc.Oracle(1, 0, N, N, N, PAR["tau_f"], PAR["tau_g"], PAR["A"], PAR["kappa"], PAR["gamma_mob"],
                   PAR["u_wall"], PAR["rho0"])
    o.init_droplet(*DROP)
    o.step(STEPS)
    return o.observables()


@pytest.mark.parametrize("precision,ref", list(BOUNDS))
def test_twin_accuracy(fre, reference, precision, ref):
    sim = fre.Simulation(lattice="d3q19", precision=precision, device="shear", nx=N, ny=N, nz=N, flags=ref, **PAR)
    sim.init_droplet(*DROP)
    sim.step(STEPS)
    ob = sim.observables()
    sim.close()
    refo = reference
    err = {k: abs(ob[k] - refo[k]) / abs(refo[k]) for k in ("D", "volume", "dp")}
    print(f"{precision} ref {ref}: D {ob['D']:.6f} (oracle {refo['D']:.6f}), relative errors {err}")
    bD, bV, bP = BOUNDS[(precision, ref)]
    assert err["D"] < bD and err["volume"] < bV and err["dp"] < bP, err


# Four-roller device (its 16-bit f stores keep the rest reference: no
# moving walls to define a base flow), D3Q19 64 x 64 x 16, droplet R = 8 at
# the centre of the four rollers (radius 8), roller surface speed 0.02;
# errors in D, volume and dp against the FP64 oracle after 1000 steps.
ROLL_N = (64, 64, 16)
ROLL_STEPS = 1000
ROLL_PAR = dict(tau_f=1.5, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=0.5, u_wall=0.02, rho0=1.0)
ROLL_DROP = (31.5, 31.5, 7.5, 8.0)
ROLL_BOUNDS = {"fp32": (1e-5, 1e-5, 1e-4), "fp16dev": (1e-2, 1e-4, 1e-2), "bf16dev": (1e-1, 1e-3, 1e-1)}


@pytest.fixture(scope="module")
def roller_reference(orc):
    nx, ny, nz = ROLL_N
    p = ROLL_PAR
    o = orc.Oracle(1, 1, nx, ny, nz, p["tau_f"], p["tau_g"], p["A"], p["kappa"], p["gamma_mob"], p["u_wall"],
                   p["rho0"])
    o.init_droplet(*ROLL_DROP)
    o.step(ROLL_STEPS)
    return o.observables()


@pytest.mark.parametrize("precision", list(ROLL_BOUNDS))
def test_four_roller_accuracy(fre, roller_reference, precision):
    nx, ny, nz = ROLL_N
    sim = fre.Simulation(lattice="d3q19", precision=precision, device="four_roller", nx=nx, ny=ny, nz=nz,
                         **ROLL_PAR)
    sim.init_droplet(*ROLL_DROP)
    sim.step(ROLL_STEPS)
    ob = sim.observables()
    sim.close()
    refo = roller_reference
    err = {k: abs(ob[k] - refo[k]) / abs(refo[k]) for k in ("D", "volume", "dp")}
    print(f"four-roller {precision}: D {ob['D']:.6f} (oracle {refo['D']:.6f}), relative errors {err}")
    bD, bV, bP = ROLL_BOUNDS[precision]
    assert err["D"] < bD and err["volume"] < bV and err["dp"] < bP, err
