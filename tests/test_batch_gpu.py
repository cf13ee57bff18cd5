"""The batch runtime (C ABI fre_batch_*): many independent simulations advanced
by batched launches and CUDA-graph replays.

Every slot of a batch must give what the same case gives on its own: FP64
slots match the FP64 oracle (relative L-inf < 1e-12), FP32 slots match a
single context of the same parameters, and a case run alone or inside a
mixed batch gives the same fields.
"""
import numpy as np
import pytest

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


BASE = dict(tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.0, rho0=1.0)
DEV = {"shear": 0, "four_roller": 1, "periodic": 2}


def errs(a, b, u_floor=1e-300):
    """Relative L-inf per field; u relative to max |u| of b, or to u_floor
    where the flow is slower (a resting droplet has only spurious currents,
    against which FP32 rounding of the populations is not small)."""
    uscale = max(max(np.abs(b[k]).max() for k in ("ux", "uy", "uz")), u_floor)
    out = {}
    for k in ("rho", "ux", "uy", "uz", "phi"):
        scale = uscale if k.startswith("u") else np.abs(b[k]).max()
        out[k] = np.abs(a[k] - b[k]).max() / scale
    return out


# lattice, device, (nx, ny, nz), droplet (cx, cy, cz, R), parameter overrides
MIX_D2Q9 = [
    ("shear", (40, 22, 1), (19.5, 10.5, 0.0, 6.0), dict(u_wall=0.02)),
    ("four_roller", (48, 48, 1), (23.5, 23.5, 0.0, 7.0), dict(u_wall=0.01, tau_f=0.8)),
    ("periodic", (33, 17, 1), (16.0, 8.0, 0.0, 5.0), dict(tau_g=1.3, gamma_mob=0.7)),
    ("shear", (130, 20, 1), (64.5, 9.5, 0.0, 6.0), dict(u_wall=0.015, tau_f=0.7)),
]
MIX_D3Q19 = [
    ("shear", (20, 14, 10), (9.5, 6.5, 4.5, 4.0), dict(u_wall=0.02, tau_f=0.8)),
    ("four_roller", (24, 24, 6), (11.5, 11.5, 2.5, 4.0), dict(u_wall=0.01)),
    ("periodic", (17, 11, 9), (8.0, 5.0, 4.0, 3.5), dict(tau_g=1.2)),
]


def oracle_of(orc, lattice, device, shape, kw):
    a = dict(BASE, **kw)
    nx, ny, nz = shape
    return orc.Oracle({"d2q9": 0, "d3q19": 1}[lattice], DEV[device], nx, ny, nz, a["tau_f"], a["tau_g"],
                      a["A"], a["kappa"], a["gamma_mob"], a["u_wall"], a["rho0"])


@pytest.mark.parametrize("lattice,mix,steps", [("d2q9", MIX_D2Q9, 7), ("d2q9", MIX_D2Q9, 61),
                                               ("d3q19", MIX_D3Q19, 45)])
def test_fp64_mixed_batch_vs_oracle(fre, orc, lattice, mix, steps):
    """A mixed batch (shear, four-roller and periodic slots of different sizes)
    in FP64: every slot equals the oracle.  61 and 45 steps run the autotuner
    (all four candidates take real steps) and graph replays; 7 steps stay on
    the batched kernels with one graph."""
    nz_ok = lattice == "d3q19"
    with fre.Batch(lattice, "fp64") as b:
        slots, oracles = [], []
        for device, shape, drop, kw in mix:
            nx, ny, nz = shape
            assert nz_ok or nz == 1
            slots.append(b.add(*drop, lattice=lattice, device=device, nx=nx, ny=ny, nz=nz, **dict(BASE, **kw)))
            o = oracle_of(orc, lattice, device, shape, kw)
            o.init_droplet(*drop)
            oracles.append(o)
        b.step(steps - 3)
        b.step(3)  # a second call continues on the same graph / odd tail
        for s, o in zip(slots, oracles):
            o.step(steps)
            assert b.steps_taken(s) == steps
            e = errs(b.fields(s), o.fields())
            assert max(e.values()) < 1e-12, (s, e)
        if steps >= 32 + 4:
            t = b.tuning()
            assert t["tuned"] and all(m > 0 for m in t["ms_per_step"]), t


def test_fp32_batch_matches_single_contexts(fre):
    """FP32 slots against one context per case on its own fastest path: the
    difference after 80 steps is FP32 rounding."""
    cases = [("shear", (128, 64, 1), (63.5, 31.5, 0.0, 12.0), dict(u_wall=0.02)),
             ("four_roller", (64, 64, 1), (31.5, 31.5, 0.0, 9.0), dict(u_wall=0.01)),
             ("shear", (96, 48, 1), (47.5, 23.5, 0.0, 8.0), dict(u_wall=0.03, tau_f=0.8)),
             ("periodic", (256, 32, 1), (128.0, 16.0, 0.0, 9.0), dict())]
    with fre.Batch("d2q9", "fp32") as b:
        slots, sims = [], []
        for device, (nx, ny, nz), drop, kw in cases:
            args = dict(BASE, **kw)
            slots.append(b.add(*drop, lattice="d2q9", device=device, nx=nx, ny=ny, nz=nz, **args))
            sim = fre.Simulation(lattice="d2q9", precision="fp32", device=device, nx=nx, ny=ny, nz=nz, **args)
            sim.init_droplet(*drop)
            sims.append(sim)
        b.step(80)
        for s, sim in zip(slots, sims):
            sim.step(80)
            # single contexts may run other kernels (row-staged): FP32
            # rounding order differs; 1e-5 on rho and phi, 3e-5 on u against
            # the wall-speed scale 0.01 (the FP32 bound of the 100x50 case)
            e = errs(b.fields(s), sim.fields(), u_floor=0.01)
            assert all(v < (3e-5 if k.startswith("u") else 1e-5) for k, v in e.items()), (s, e)
            sim.close()


def test_alone_equals_in_mix_fp64(fre):
    """The same case alone in a batch and inside a batch of other cases gives
    the same fields (FP64, 1e-13)."""
    case = ("shear", (40, 22, 1), (19.5, 10.5, 0.0, 6.0), dict(u_wall=0.02))
    device, (nx, ny, nz), drop, kw = case
    args = dict(BASE, **kw)
    with fre.Batch("d2q9", "fp64") as alone:
        s = alone.add(*drop, lattice="d2q9", device=device, nx=nx, ny=ny, nz=nz, **args)
        alone.step(50)
        ref = alone.fields(s)
    with fre.Batch("d2q9", "fp64") as mix:
        for dv, (mx, my, mz), dr, k2 in MIX_D2Q9[1:]:
            mix.add(*dr, lattice="d2q9", device=dv, nx=mx, ny=my, nz=mz, **dict(BASE, **k2))
        s = mix.add(*drop, lattice="d2q9", device=device, nx=nx, ny=ny, nz=nz, **args)
        mix.step(50)
        e = errs(mix.fields(s), ref)
    assert max(e.values()) < 1e-13, e


def test_add_remove_and_budget(fre, orc):
    """Slots join and leave between steps; the remaining slots carry on
    exactly (FP64 vs oracle), the freed slot index is reused, and an add
    over the device-memory budget is refused with FRE_ERR_BUDGET."""
    p0 = dict(BASE, u_wall=0.02)
    one = fre.fre_device_bytes(fre.make_params(lattice="d2q9", precision="fp64", device="shear",
                                               nx=40, ny=22, nz=1, **p0))
    with fre.Batch("d2q9", "fp64", budget_bytes=int(2.5 * one)) as b:
        s0 = b.add(19.5, 10.5, 0.0, 6.0, lattice="d2q9", device="shear", nx=40, ny=22, nz=1, **p0)
        s1 = b.add(19.5, 10.5, 0.0, 6.0, lattice="d2q9", device="shear", nx=40, ny=22, nz=1, **p0)
        assert b.bytes_in_use() == 2 * one
        with pytest.raises(fre.FreError) as ei:
            b.add(19.5, 10.5, 0.0, 6.0, lattice="d2q9", device="shear", nx=40, ny=22, nz=1, **p0)
        assert ei.value.status == fre.FRE_ERR_BUDGET
        o = oracle_of(orc, "d2q9", "shear", (40, 22, 1), dict(u_wall=0.02))
        o.init_droplet(19.5, 10.5, 0.0, 6.0)
        b.step(11)
        b.remove(s0)
        assert b.bytes_in_use() == one and b.slots() == [s1]
        b.step(40)
        s2 = b.add(19.5, 10.5, 0.0, 6.0, lattice="d2q9", device="shear", nx=40, ny=22, nz=1, **p0)
        assert s2 == s0
        b.step(9)
        o.step(60)
        e = errs(b.fields(s1), o.fields())
        assert max(e.values()) < 1e-12, e
        assert b.steps_taken(s1) == 60 and b.steps_taken(s2) == 9


def test_batch_argument_errors(fre):
    with fre.Batch("d2q9", "fp32") as b:
        with pytest.raises(fre.FreError) as ei:
            b.add(1, 1, 0, 1, lattice="d3q19", device="shear", nx=8, ny=8, nz=8)
        assert ei.value.status == fre.FRE_ERR_ARG
        with pytest.raises(fre.FreError):
            b.remove(3)
        b.step(5)  # an empty batch steps nothing
        assert b.slots() == []


# C3-like D2Q9 slots (the benchmarked batch workload's kinds and physics:
# A = kappa = 0.01, tau_f = 2, tau_g = 1, Gamma = 1; shear Ny = Nx/2,
# four-roller Ny = Nx; Ca 0.2 and R/H 0.2 give u_w = Ca sigma / (2 mu R/H))
C3_PHYS = dict(tau_f=2.0, tau_g=1.0, A=0.01, kappa=0.01, gamma_mob=1.0, rho0=1.0)
_SIGMA = (8.0 * 0.01 * 0.01 / 9.0) ** 0.5
_UW = 0.2 * _SIGMA / (2.0 * 0.5 * 0.2)
C3_LIKE = [
    ("shear", (64, 32, 1), (31.5, 15.5, 0.0, 6.4), dict(u_wall=_UW)),
    ("four_roller", (64, 64, 1), (31.5, 31.5, 0.0, 6.4), dict(u_wall=_UW)),
    ("shear", (128, 64, 1), (63.5, 31.5, 0.0, 12.8), dict(u_wall=_UW)),
    ("four_roller", (96, 96, 1), (47.5, 47.5, 0.0, 9.6), dict(u_wall=_UW)),
    ("shear", (160, 80, 1), (79.5, 39.5, 0.0, 16.0), dict(u_wall=_UW)),
]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_fp32_batch_slots_vs_oracle(fre, orc, mode):
    """FP32 slots of a C3-like batch (shear and four-roller D2Q9 cases of
    uneven sizes), each launch mode pinned in turn, against the FP64 oracle
    after 200 steps: 1e-5 relative L-inf on rho and phi, 1e-4 on u against
    max(|u|, 0.01) (the FP32 bounds of the row and per-node kernels)."""
    with fre.Batch("d2q9", "fp32") as b:
        b.set_mode(mode, 64)
        slots, oracles = [], []
        for device, shape, drop, kw in C3_LIKE:
            nx, ny, nz = shape
            args = dict(C3_PHYS, **kw)
            slots.append(b.add(*drop, lattice="d2q9", device=device, nx=nx, ny=ny, nz=nz, **args))
            o = orc.Oracle(0, DEV[device], nx, ny, nz, args["tau_f"], args["tau_g"], args["A"], args["kappa"],
                           args["gamma_mob"], args["u_wall"], args["rho0"])
            o.init_droplet(*drop)
            oracles.append(o)
        b.step(150)
        b.step(50)
        t = b.tuning()
        assert t["mode"] == mode
        for s, o in zip(slots, oracles):
            o.step(200)
            assert b.steps_taken(s) == 200
            e = errs(b.fields(s), o.fields(), u_floor=0.01)
            assert all(v < (1e-4 if k.startswith("u") else 1e-5) for k, v in e.items()), (s, mode, e)
