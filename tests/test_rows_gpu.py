"""The row kernels (x-rows staged in shared memory with 16-byte cp.async
copies; the hot path of the shear and periodic devices in FP32 and 16-bit
storage) against the per-node kernels and the FP64 oracle."""
import numpy as np
import pytest

from paper_2212_01617_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fre():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    return fre


def errs(a, b, u_floor=0.0):
    """Relative L-inf per field; u relative to max |u| of b or u_floor,
    whichever is larger (a resting droplet has only small spurious currents)."""
    uscale = max(max(np.abs(b[k]).max() for k in ("ux", "uy", "uz")), u_floor)
    out = {}
    for k in ("rho", "ux", "uy", "uz", "phi"):
        scale = uscale if k.startswith("u") else np.abs(b[k]).max()
        out[k] = np.abs(a[k] - b[k]).max() / scale
    return out


CASES = [
    # lattice, device, nx, ny, nz, kwargs
    ("d3q19", "shear", 64, 20, 12, dict(u_wall=0.03, tau_f=2.0, tau_g=2.0, gamma_mob=0.5)),
    ("d3q19", "periodic", 96, 12, 10, dict(tau_f=0.8, tau_g=1.2, gamma_mob=0.7)),
    ("d2q9", "shear", 256, 40, 1, dict(u_wall=0.02)),
    ("d2q9", "periodic", 384, 24, 1, dict(tau_f=0.7)),
    # 2 KB FP32 rows: one row per work unit
    ("d3q19", "shear", 512, 6, 4, dict(u_wall=0.02, tau_f=1.2)),
    # odd ny: one row per work unit in every format
    ("d2q9", "shear", 128, 37, 1, dict(u_wall=0.02)),
    # rows of an odd number of half warps (nx a multiple of 32, not of 64):
    # two rows side by side in every pass
    ("d3q19", "shear", 96, 10, 6, dict(u_wall=0.03, tau_f=1.5)),
    ("d2q9", "shear", 160, 20, 1, dict(u_wall=0.02)),
]


def make(fre, lattice, device, nx, ny, nz, precision, flags=0, **kw):
    args = dict(tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.0, rho0=1.0)
    args.update(kw)
    return fre.Simulation(lattice=lattice, precision=precision, device=device, nx=nx, ny=ny, nz=nz,
                          flags=flags, **args)


REST = 8  # FRE_FLAG_REST_REFERENCE


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}")
@pytest.mark.parametrize("precision,ref", [("fp32", 0), ("fp16dev", 0), ("bf16dev", 0), ("fp16dev", REST),
                                           ("bf16dev", REST)])
def test_row_kernels_match_per_node_kernels(fre, orc, case, precision, ref):
    """The row kernels and the per-node kernels compute the same update,
    arranged differently (the row kernels split the collision into parts
    even and odd in c_i and keep 16-bit f as deviations), so their rounding
    differs.  Both are held to the FP64 oracle after 200 steps: FP32 1e-5 on
    rho and phi and 1e-4 on u against max(|u|, 0.01), i.e. 1e-6 absolute
    (populations up to ~0.5 round to ~3e-8 per step in FP32; 200 steps of
    such errors stay below 1e-6 in the velocity moments), FP16 3e-3, BF16
    2e-2 (the 16-bit bounds of the D3Q19 test below), with f stored against
    the Couette equilibrium of the shear walls (ref 0, the default; the
    periodic device has no walls and keeps the rest equilibrium) or the
    rest equilibrium (FRE_FLAG_REST_REFERENCE)."""
    lattice, device, nx, ny, nz, kw = case
    rows = make(fre, lattice, device, nx, ny, nz, precision, flags=ref, **kw)
    gen = make(fre, lattice, device, nx, ny, nz, precision, flags=1 | ref, **kw)
    assert rows.row_kernels and not gen.row_kernels
    a = dict(tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.0, rho0=1.0)
    a.update(kw)
    o = orc.Oracle({"d2q9": 0, "d3q19": 1}[lattice], {"shear": 0, "periodic": 2}[device], nx, ny, nz,
                   a["tau_f"], a["tau_g"], a["A"], a["kappa"], a["gamma_mob"], a["u_wall"], a["rho0"])
    c = ((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, min(nx, ny) / 4)
    for s in (rows, gen, o):
        s.init_droplet(*c)
        s.step(200)
    ref = o.fields()
    tol = {"fp32": 1e-5, "fp16dev": 3e-3, "bf16dev": 2e-2}[precision]
    utol = 1e-4 if precision == "fp32" else tol
    res = {name: errs(sim.fields(), ref, u_floor=0.01) for name, sim in (("rows", rows), ("per-node", gen))}
    for name, e in res.items():
        assert all(v < (utol if k.startswith("u") else tol) for k, v in e.items()), (name, res)
    rows.close()
    gen.close()


def test_row_kernels_random_populations_fp32(fre, orc):
    """Non-equilibrium seeded populations through the row path vs the oracle."""
    shape = (6, 8, 32)
    f, g = inputs.random_populations(19, shape, seed=11)
    sim = make(fre, "d3q19", "periodic", 32, 8, 6, "fp32", tau_f=0.7, tau_g=1.1, A=0.03, kappa=0.05)
    assert sim.row_kernels
    o = orc.Oracle(1, 2, 32, 8, 6, 0.7, 1.1, 0.03, 0.05, 1.0, 0.0, 1.0)
    sim.load_populations(f, g)
    o.load_populations(f, g)
    sim.step(60)
    o.step(60)
    a, b = sim.fields(), o.fields()
    # the random velocities relax towards rest, so u is bounded in absolute
    # terms: FP32 rounding of populations of size ~0.3 is ~2e-8
    for k in ("rho", "phi"):
        assert np.abs(a[k] - b[k]).max() / np.abs(b[k]).max() < 1e-5, k
    for k in ("ux", "uy", "uz"):
        assert np.abs(a[k] - b[k]).max() < 1e-6, k


@pytest.mark.parametrize("precision,ref,tol", [("fp16dev", REST, 3e-3), ("bf16dev", REST, 2e-2),
                                               ("fp16dev", 0, 3e-4), ("bf16dev", 0, 3e-3)])
def test_16bit_storage_vs_fp64_oracle(fre, orc, precision, ref, tol):
    """16-bit deviation storage (FP32 arithmetic) vs the FP64 oracle after 500
    steps of the D3Q19 shear droplet: relative L-inf of rho, u, phi, with f
    stored against the Couette equilibrium (the default) or the rest
    equilibrium."""
    nx, ny, nz = 64, 24, 16
    kw = dict(u_wall=0.03, tau_f=2.0, tau_g=2.0, gamma_mob=0.5)
    sim = make(fre, "d3q19", "shear", nx, ny, nz, precision, flags=ref, **kw)
    assert sim.row_kernels
    o = orc.Oracle(1, 0, nx, ny, nz, 2.0, 2.0, 0.04, 0.04, 0.5, 0.03, 1.0)
    c = ((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, 6.0)
    sim.init_droplet(*c)
    o.init_droplet(*c)
    sim.step(500)
    o.step(500)
    e = errs(sim.fields(), o.fields())
    print(precision, ref, e)
    assert max(e.values()) < tol, e


def test_launch_shapes_in_any_order(fre):
    """Contexts of different row lengths share the kernel instances: a wide
    lattice whose update runs two stages (opt-in set by its launch), then a
    narrow one whose update asks the occupancy calculator about two and
    three stages, then the wide one again.  The shared-memory opt-in of a
    kernel only ever rises, so the third run launches as the first did."""
    kw = dict(u_wall=0.02, tau_f=1.2)
    wide = make(fre, "d3q19", "shear", 256, 8, 4, "fp32", **kw)
    narrow = make(fre, "d3q19", "shear", 64, 8, 4, "fp32", **kw)
    assert wide.row_kernels and narrow.row_kernels
    for s in (wide, narrow, wide):
        if s.steps_taken == 0:
            s.init_droplet(s.params.nx / 2, 3.5, 1.5, 2.0)
        s.step(5)
    for s in (wide, narrow):
        assert np.isfinite(s.fields()["rho"]).all()
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16dev"])
def test_half_warp_rows_take_the_full_row_kernels(fre, precision):
    """A 96-wide lattice (48 consumer threads per row) runs the full-row
    kernels with two rows side by side; an odd ny (no row pairs) falls back
    to the chunked kernels."""
    a = make(fre, "d3q19", "shear", 96, 10, 6, precision, u_wall=0.02)
    b = make(fre, "d3q19", "shear", 96, 9, 6, precision, u_wall=0.02)
    assert a.kernel_path == 2 and b.kernel_path == 1, (a.kernel_path, b.kernel_path)
    a.close()
    b.close()


ROLL_CASES = [
    # lattice, nx, ny, nz: square boxes, a 96-wide one (two rows side by
    # side) and a 192 x 96 box of the serving workload's shape
    ("d3q19", 64, 64, 8),
    ("d3q19", 96, 96, 6),
    ("d3q19", 192, 96, 4),
    ("d2q9", 128, 128, 1),
]


@pytest.mark.parametrize("case", ROLL_CASES, ids=lambda c: f"{c[0]}-{c[1]}x{c[2]}x{c[3]}")
@pytest.mark.parametrize("precision", ["fp32", "fp16dev", "bf16dev"])
@pytest.mark.parametrize("interp", [False, True], ids=["halfway", "interpolated"])
def test_four_roller_row_kernels(fre, orc, case, precision, interp):
    """The four-roller device on the row kernels (roller nodes stored as 0,
    the wall links of each step written into the roller nodes' slots by the
    reflection pass, with half-way bounce-back or, with
    FRE_FLAG_INTERPOLATED_WALLS, the interpolated rule from the link
    fractions; ghost fills between the passes) against the per-node kernels
    and the FP64 oracle after 200 steps, with the bounds of the shear rows
    above."""
    lattice, nx, ny, nz = case
    kw = dict(u_wall=0.01, tau_f=1.2, tau_g=1.0, gamma_mob=0.8)
    iw = fre.FRE_FLAG_INTERPOLATED_WALLS if interp else 0
    rows = make(fre, lattice, "four_roller", nx, ny, nz, precision, flags=iw, **kw)
    gen = make(fre, lattice, "four_roller", nx, ny, nz, precision, flags=1 | iw, **kw)
    assert rows.kernel_path == 2 and gen.kernel_path == 0
    a = dict(tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.0, rho0=1.0)
    a.update(kw)
    o = orc.Oracle({"d2q9": 0, "d3q19": 1}[lattice], 1, nx, ny, nz, a["tau_f"], a["tau_g"], a["A"], a["kappa"],
                   a["gamma_mob"], a["u_wall"], a["rho0"], interp=int(interp))
    c = ((nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2, nx / 10)
    for s in (rows, gen, o):
        s.init_droplet(*c)
        s.step(200)
    ref = o.fields()
    tol = {"fp32": 1e-5, "fp16dev": 3e-3, "bf16dev": 2e-2}[precision]
    utol = 1e-4 if precision == "fp32" else tol
    res = {name: errs(sim.fields(), ref, u_floor=0.01) for name, sim in (("rows", rows), ("per-node", gen))}
    for name, e in res.items():
        assert all(v < (utol if k.startswith("u") else tol) for k, v in e.items()), (name, res)
    rows.close()
    gen.close()
