"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 on the GPU: relative L-inf < 1e-12 on rho, u and phi after 500 steps
(max |gpu - oracle| / max |oracle| per field).  FP32 storage and arithmetic:
< 1e-5 after 500 steps.  Sizes span several 256-node blocks with a ragged
tail; every device kind and both lattices are covered.
"""
import numpy as np
import pytest

from paper_2212_01617_gb300 import inputs

pytestmark = pytest.mark.gpu

FIELDS = ("rho", "ux", "uy", "uz", "phi")


@pytest.fixture(scope="module")
def fre():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    return fre


def rel_linf(a, b):
    scale = np.abs(b).max()
    if scale == 0.0:
        return np.abs(a - b).max()
    return np.abs(a - b).max() / scale


def pair(fre, orc, lattice, device, nx, ny, nz, precision="fp64", interp=False, **kw):
    args = dict(tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.0, rho0=1.0)
    args.update(kw)
    flags = fre.FRE_FLAG_INTERPOLATED_WALLS if interp else 0
    sim = fre.Simulation(lattice=lattice, precision=precision, device=device, nx=nx, ny=ny, nz=nz, flags=flags,
                         **args)
    o = orc.Oracle({"d2q9": 0, "d3q19": 1}[lattice], {"shear": 0, "four_roller": 1, "periodic": 2}[device],
                   nx, ny, nz, args["tau_f"], args["tau_g"], args["A"], args["kappa"], args["gamma_mob"],
                   args["u_wall"], args["rho0"], interp=int(interp))
    return sim, o


def compare_fields(sim, o, tol, fields=FIELDS):
    """Relative L-inf per field; the velocity components share one scale,
    max |u| of the oracle (a component that vanishes by symmetry has no
    scale of its own)."""
    a, b = sim.fields(), o.fields()
    uscale = max(np.abs(b[k]).max() for k in ("ux", "uy", "uz"))
    errs = {}
    for k in fields:
        if k in ("ux", "uy", "uz"):
            errs[k] = np.abs(a[k] - b[k]).max() / uscale
        else:
            errs[k] = rel_linf(a[k], b[k])
    bad = {k: v for k, v in errs.items() if not v < tol}
    assert not bad, f"relative L-inf above {tol}: {bad} (all: {errs})"
    return errs


@pytest.mark.parametrize("steps", [0, 1, 500, 2000])
def test_c0_d2q9_fp64_shear_droplet(fre, orc, steps):
    """D2Q9 FP64, 100x50 shear channel, walls at +-0.01, droplet R = 10."""
    sim, o = pair(fre, orc, "d2q9", "shear", 100, 50, 1, u_wall=0.01)
    sim.init_droplet(49.5, 24.5, 0.0, 10.0)
    o.init_droplet(49.5, 24.5, 0.0, 10.0)
    sim.step(steps)
    o.step(steps)
    compare_fields(sim, o, 1e-12, FIELDS + ("mu",))
    fg, gg = sim.populations()
    fo, go = o.populations()
    assert rel_linf(fg, fo) < 1e-12 and rel_linf(gg, go) < 1e-12
    sim.close()


def test_d3q19_fp64_shear_ragged(fre, orc):
    """D3Q19 FP64 shear, 23x17x13 nodes (20 blocks of 256 and a ragged tail)."""
    sim, o = pair(fre, orc, "d3q19", "shear", 23, 17, 13, u_wall=0.02, tau_f=0.8, tau_g=1.3,
                  gamma_mob=0.7)
    sim.init_droplet(11.0, 8.0, 6.0, 5.0)
    o.init_droplet(11.0, 8.0, 6.0, 5.0)
    sim.step(500)
    o.step(500)
    compare_fields(sim, o, 1e-12)
    sim.close()


def test_d2q9_fp64_four_roller(fre, orc):
    """D2Q9 FP64 four-roller device, 64x64, centred droplet."""
    sim, o = pair(fre, orc, "d2q9", "four_roller", 64, 64, 1, u_wall=0.01)
    sim.init_droplet(31.5, 31.5, 0.0, 8.0)
    o.init_droplet(31.5, 31.5, 0.0, 8.0)
    sim.step(500)
    o.step(500)
    compare_fields(sim, o, 1e-12, FIELDS + ("mu",))
    sim.close()


def test_d3q19_fp64_four_roller(fre, orc):
    """D3Q19 FP64 four-roller device (rollers along z), 32x32x6."""
    sim, o = pair(fre, orc, "d3q19", "four_roller", 32, 32, 6, u_wall=0.01)
    sim.init_droplet(15.5, 15.5, 2.5, 5.0)
    o.init_droplet(15.5, 15.5, 2.5, 5.0)
    sim.step(500)
    o.step(500)
    compare_fields(sim, o, 1e-12, FIELDS + ("mu",))
    sim.close()


@pytest.mark.parametrize("lattice,shape", [("d2q9", (64, 64, 1)), ("d3q19", (32, 32, 6))])
def test_fp64_four_roller_interpolated_walls(fre, orc, lattice, shape):
    """FRE_FLAG_INTERPOLATED_WALLS (linear interpolated bounce-back at the
    roller circles), FP64, 500 steps from a centred droplet: 1e-12 against
    the oracle's rule, on the per-node kernels; the interpolation changes
    the flow (the fields differ from half-way bounce-back by far more)."""
    nx, ny, nz = shape
    sim, o = pair(fre, orc, lattice, "four_roller", nx, ny, nz, u_wall=0.01, interp=True)
    assert sim.kernel_path == 0
    c = ((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2 if nz > 1 else 0.0)
    sim.init_droplet(*c, nx / 8)
    o.init_droplet(*c, nx / 8)
    sim.step(500)
    o.step(500)
    compare_fields(sim, o, 1e-12, FIELDS + ("mu",))
    hb, _ = pair(fre, orc, lattice, "four_roller", nx, ny, nz, u_wall=0.01)
    hb.init_droplet(*c, nx / 8)
    hb.step(500)
    a, b = sim.fields(), hb.fields()
    assert np.abs(a["ux"] - b["ux"]).max() > 1e-2 * np.abs(b["ux"]).max()
    sim.close()
    hb.close()


def test_fp32_four_roller_interpolated_walls(fre, orc):
    """The same rule in FP32 storage and arithmetic (D3Q19 32x32x6): 1e-5
    relative L-inf after 500 steps."""
    sim, o = pair(fre, orc, "d3q19", "four_roller", 32, 32, 6, precision="fp32", u_wall=0.01, interp=True)
    sim.init_droplet(15.5, 15.5, 2.5, 5.0)
    o.init_droplet(15.5, 15.5, 2.5, 5.0)
    sim.step(500)
    o.step(500)
    compare_fields(sim, o, 1e-5)
    sim.close()


def test_interpolated_walls_argument_rules(fre):
    """The flag is an argument error off the four-roller device, and batches
    (hence servers) do not take it."""
    p = fre.make_params(lattice="d2q9", precision="fp64", device="shear", nx=16, ny=16, nz=1,
                        flags=fre.FRE_FLAG_INTERPOLATED_WALLS)
    with pytest.raises(fre.FreError):
        fre.fre_create(p)
    with fre.Batch("d2q9", "fp64") as b, pytest.raises(fre.FreError):
        b.add(15.5, 15.5, 0.0, 4.0, device="four_roller", nx=32, ny=32, nz=1,
              flags=fre.FRE_FLAG_INTERPOLATED_WALLS)


@pytest.mark.parametrize("lattice,shape", [("d2q9", (1, 19, 37)), ("d3q19", (7, 9, 11))])
def test_fp64_random_populations_periodic(fre, orc, lattice, shape):
    """Arbitrary (non-equilibrium) seeded populations, periodic box."""
    q = 9 if lattice == "d2q9" else 19
    nz, ny, nx = shape
    f, g = inputs.random_populations(q, shape, seed=7)
    sim, o = pair(fre, orc, lattice, "periodic", nx, ny, nz, tau_f=0.7, tau_g=1.1, A=0.03, kappa=0.05)
    sim.load_populations(f, g)
    o.load_populations(f, g)
    fg, gg = sim.populations()
    assert np.array_equal(fg, f) and np.array_equal(gg, g)  # FP64 round trip is exact
    sim.step(50)
    o.step(50)
    compare_fields(sim, o, 1e-12, FIELDS + ("mu",))
    sim.close()


def test_fp64_observables(fre, orc):
    sim, o = pair(fre, orc, "d2q9", "shear", 100, 50, 1, u_wall=0.01)
    sim.init_droplet(49.5, 24.5, 0.0, 10.0)
    o.init_droplet(49.5, 24.5, 0.0, 10.0)
    sim.step(300)
    o.step(300)
    a, b = sim.observables(), o.observables()
    for k in ("mass", "phi_sum", "volume", "drop_weight", "drop_count", "D", "theta_deg",
              "p_centre", "p_far", "dp", "max_u"):
        assert abs(a[k] - b[k]) <= 1e-10 * max(1.0, abs(b[k])), (k, a[k], b[k])
    assert np.allclose(a["centroid"], b["centroid"], rtol=0, atol=1e-10)
    assert np.allclose(a["I"], b["I"], rtol=1e-10, atol=1e-12)
    assert a["status"] == 0 and a["step"] == 300
    sim.close()


def test_fp32_vs_fp64_oracle_d3q19(fre, orc):
    """FP32 storage and arithmetic: 1e-5 relative L-inf after 500 steps."""
    sim, o = pair(fre, orc, "d3q19", "shear", 40, 24, 20, precision="fp32", u_wall=0.03, tau_f=2.0,
                  tau_g=2.0, gamma_mob=0.5)
    sim.init_droplet(19.5, 11.5, 9.5, 6.0)
    o.init_droplet(19.5, 11.5, 9.5, 6.0)
    sim.step(500)
    o.step(500)
    compare_fields(sim, o, 1e-5)
    sim.close()


@pytest.mark.parametrize("ca", [0.1, 0.42])
def test_c1_d3q19_fp32_vs_fp64_oracle(fre, orc, ca):
    """The 128x64x64 D3Q19 shear case, droplet R = 16, tau = 2, A = kappa =
    0.04: u_w = Ca sigma H / (2 mu R) sets the capillary number, Gamma the
    Peclet number 0.43 (M = rate R xi / (Pe A), Gamma = M / (tau_g - 1/2)).
    FP32 storage and arithmetic (the row kernels) after 500 steps: 1e-5
    relative L-inf on rho, u and phi against the FP64 oracle."""
    sigma = (8 * 0.04 * 0.04 / 9) ** 0.5
    uw = ca * sigma * 64 / (2 * 0.5 * 16)
    gamma = (2 * uw / 64) * 16 / (0.43 * 0.04) / 1.5
    sim, o = pair(fre, orc, "d3q19", "shear", 128, 64, 64, precision="fp32", u_wall=uw, tau_f=2.0,
                  tau_g=2.0, gamma_mob=gamma)
    assert sim.row_kernels
    sim.init_droplet(63.5, 31.5, 31.5, 16.0)
    o.init_droplet(63.5, 31.5, 31.5, 16.0)
    sim.step(500)
    o.step(500)
    compare_fields(sim, o, 1e-5)
    sim.close()


def test_fp32_vs_fp64_oracle_d2q9_c0(fre, orc):
    """FP32 on the 100x50 D2Q9 case.  Plain FP32 populations (up to 4/9) carry
    an absolute rounding of ~3e-8 per value; after 500 steps u is off by
    ~1e-7 absolute, i.e. ~1e-5 of the small wall speed 0.01.  Bound: 3e-5
    relative for u, 1e-5 for rho and phi."""
    sim, o = pair(fre, orc, "d2q9", "shear", 100, 50, 1, precision="fp32", u_wall=0.01)
    sim.init_droplet(49.5, 24.5, 0.0, 10.0)
    o.init_droplet(49.5, 24.5, 0.0, 10.0)
    sim.step(500)
    o.step(500)
    compare_fields(sim, o, 1e-5, ("rho", "phi"))
    compare_fields(sim, o, 3e-5, ("ux", "uy"))
    sim.close()


def test_errors_are_status_codes(fre):
    sim = fre.Simulation(lattice="d2q9", precision="fp32", device="shear", nx=16, ny=8, nz=1)
    with pytest.raises(fre.FreError) as e:
        sim.step(1)  # not initialised
    assert e.value.status == fre.binding.FRE_ERR_STATE
    with pytest.raises(fre.FreError) as e:
        sim.init_droplet(8, 4, 0, -1.0)
    assert e.value.status == fre.binding.FRE_ERR_ARG
    sim.init_droplet(8, 4, 0, 3.0)
    with pytest.raises(fre.FreError):
        sim.step(-1)
    sim.step(2)
    assert sim.steps_taken == 2
    sim.close()
