"""Breakup detection on the GPU (fre_components): the connected components
of the droplet phase phi > 0, labelled by concurrent union-find, against the
oracle's flood fill on the same phi field, bit for bit (an integer result;
the phi > 0 decision is taken on the GPU's own phi, which both sides read).
Seeded fields with many drops of random sizes, some across the periodic
boundary and some touching, on both lattices and every device; then the
serving loop retiring a sheared drop above the critical capillary number as
a breakup at the check where the oracle first sees two drops."""
import numpy as np
import pytest

from paper_2212_01617_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = {"shear": 0, "four_roller": 1, "periodic": 2}


@pytest.fixture(scope="module")
def fre():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    return fre


CASES = [  # lattice, device, (nx, ny, nz), drops, seed
    ("d2q9", "periodic", (203, 121, 1), 40, 1),
    ("d2q9", "shear", (256, 96, 1), 30, 2),
    ("d2q9", "four_roller", (128, 128, 1), 25, 3),
    ("d3q19", "periodic", (47, 39, 35), 60, 4),
    ("d3q19", "shear", (64, 48, 40), 50, 5),
    ("d3q19", "four_roller", (64, 64, 12), 30, 6),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16dev"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{c[1]}")
def test_labels_match_oracle_flood_fill(fre, orc, case, precision):
    lattice, device, (nx, ny, nz), drops, seed = case
    shape = (nz, ny, nx)
    phi0 = inputs.multi_drop_phi(shape, drops, seed=inputs.SEED + 50 + seed,
                                 periodic=(True, device != "shear", True))
    zeros = np.zeros(shape)
    sim = fre.Simulation(lattice=lattice, precision=precision, device=device, nx=nx, ny=ny, nz=nz,
                         tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.01, rho0=1.0)
    sim.init_fields(np.ones(shape), zeros, zeros, zeros if lattice == "d3q19" else None, phi0)
    count, sizes, lab = sim.components(min_size=1, max_sizes=4096, labels=True)
    phi = sim.fields()["phi"]  # the phi the GPU labelled
    o = orc.Oracle({"d2q9": 0, "d3q19": 1}[lattice], DEV[device], nx, ny, nz)
    ocount, olab = o.label_phase(phi)
    assert count == ocount and ocount >= 5
    assert np.array_equal(lab, olab)
    flat = olab.reshape(-1)
    osizes = sorted(np.bincount(flat[flat >= 0])[np.unique(flat[flat >= 0])].tolist(), reverse=True)
    assert sizes == osizes
    # the size filter keeps the components of at least min_size nodes
    m = osizes[len(osizes) // 2]
    c2, s2, _ = sim.components(min_size=m, max_sizes=4096)
    assert c2 == sum(1 for v in osizes if v >= m) and s2 == [v for v in osizes if v >= m]
    sim.close()


def test_one_drop_and_empty_phase(fre):
    with fre.Simulation(lattice="d3q19", precision="fp32", device="shear", nx=64, ny=32, nz=32, tau_f=1.0,
                        tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.01, rho0=1.0) as sim:
        sim.init_droplet(31.5, 15.5, 15.5, 8.0)
        count, sizes, _ = sim.components()
        assert count == 1 and sizes[0] == int(sim.observables()["drop_count"])
        shape = (32, 32, 64)
        z = np.zeros(shape)
        sim.init_fields(np.ones(shape), z, z, z, -np.ones(shape))
        assert sim.components()[0] == 0


BREAK = dict(tau_f=2.0, tau_g=1.0, A=0.01, kappa=0.01, gamma_mob=1.0, rho0=1.0)


def test_serving_retires_a_broken_drop(fre, orc):
    """D2Q9 256 x 64 shear, R = 16, A = kappa = 0.01, tau_f = 2: walls at
    u_w = 0.08 give Ca = mu (2 u_w / H) R / sigma = 4.2, far above the
    critical capillary number of 2D shear (about 0.7, Sec. 3): the drop
    stretches and splits.  With u_w = 0.005 (Ca = 0.27) it settles.  The
    served supercritical request ends as BREAKUP at the first check (every
    500 steps) where the oracle, stepped alike, finds two drops of at least
    0.5% of the initial drop's nodes; the subcritical one does not break."""
    nx, ny, R = 256, 64, 16.0
    drop = ((nx - 1) / 2, (ny - 1) / 2, 0.0, R)
    min_nodes = max(1, int(np.floor(0.005 * np.pi * R * R)))
    o = orc.Oracle(0, 0, nx, ny, 1, BREAK["tau_f"], BREAK["tau_g"], BREAK["A"], BREAK["kappa"],
                   BREAK["gamma_mob"], 0.08, BREAK["rho0"])
    o.init_droplet(*drop)
    o.step(1)
    t_break = None
    for k in range(1, 25):
        o.step(500)
        _, lab = o.label_phase()
        flat = lab.reshape(-1)
        sizes = np.bincount(flat[flat >= 0])
        if np.count_nonzero(sizes >= min_nodes) >= 2:
            t_break = 1 + 500 * k
            break
    assert t_break is not None
    with fre.Server("d2q9", "fp64", chunk_steps=250, check_every=500, tol_D=1e-4, max_steps=12000,
                    breakup_min_frac=0.005) as srv:
        ids = {srv.submit(*drop, lattice="d2q9", device="shear", nx=nx, ny=ny, nz=1, u_wall=uw, **BREAK): uw
               for uw in (0.08, 0.005)}
        res = {}
        for _ in range(2000):
            srv.advance()
            for r in srv.results():
                res[ids[r["id"]]] = r
            if len(res) == 2:
                break
    assert res[0.08]["outcome"] == "breakup" and res[0.08]["steps"] == t_break, (res[0.08], t_break)
    assert res[0.005]["outcome"] in ("converged", "max_steps"), res[0.005]
