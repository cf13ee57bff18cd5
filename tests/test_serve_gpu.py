"""The serving loop (C ABI fre_server_*) on the GPU: a request served inside a
mix of others, or after others in a reused context, ends with the same state
as the same case stepped alone for the same number of steps; the stopping
rules and the budget act as declared."""
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


BASE = dict(tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, rho0=1.0)
REQS = [  # device, (nx, ny, nz), droplet, overrides
    ("shear", (40, 22, 1), (19.5, 10.5, 0.0, 6.0), dict(u_wall=0.02)),
    ("four_roller", (48, 48, 1), (23.5, 23.5, 0.0, 7.0), dict(u_wall=0.01)),
    ("shear", (64, 32, 1), (31.5, 15.5, 0.0, 8.0), dict(u_wall=0.01, tau_f=0.8)),
    ("periodic", (33, 17, 1), (16.0, 8.0, 0.0, 5.0), dict()),
    ("shear", (40, 22, 1), (19.5, 10.5, 0.0, 5.0), dict(u_wall=0.03)),
]


def alone(fre, device, shape, drop, kw, steps, precision="fp64"):
    nx, ny, nz = shape
    sim = fre.Simulation(lattice="d2q9", precision=precision, device=device, nx=nx, ny=ny, nz=nz,
                         **dict(BASE, **kw))
    sim.init_droplet(*drop)
    sim.step(steps)
    o = sim.observables()
    sim.close()
    return o


def run(srv, reqs):
    ids = {}
    for k, (device, (nx, ny, nz), drop, kw) in enumerate(reqs):
        ids[srv.submit(*drop, lattice="d2q9", device=device, nx=nx, ny=ny, nz=nz, **dict(BASE, **kw))] = k
    res = {}
    for _ in range(10000):
        srv.advance()
        for r in srv.results():
            res[ids[r["id"]]] = r
        if len(res) == len(reqs):
            break
    return res


@pytest.mark.parametrize("max_running", [0, 1])
def test_server_results_equal_cases_run_alone(fre, max_running):
    """FP64, 5 requests, checks every 60 steps, cap 300 steps, tol_D 1e-3:
    each result's observables equal those of the case stepped alone for the
    same number of steps (relative 1e-11 on D, mass, dp).  max_running = 1
    serves them one at a time, the later ones in reused contexts."""
    with fre.Server("d2q9", "fp64", chunk_steps=25, check_every=60, tol_D=1e-3, max_steps=300,
                    max_running=max_running) as srv:
        res = run(srv, REQS)
        st = srv.stats()
    assert len(res) == len(REQS)
    for k, (device, shape, drop, kw) in enumerate(REQS):
        r = res[k]
        assert r["outcome"] in ("converged", "max_steps", "breakup"), r
        # checks every 60 batch steps after the first step taken on admission
        assert (r["steps"] - 1) % 60 == 0 or r["steps"] == 301
        ref = alone(fre, device, shape, drop, kw, r["steps"])
        for key in ("D", "mass", "dp", "volume"):
            a, b = r["obs"][key], ref[key]
            assert abs(a - b) <= 1e-11 * max(abs(b), 1e-3), (k, key, a, b)
        assert r["t_admit"] >= r["t_submit"] and r["t_done"] >= r["t_admit"]
    if max_running == 1:
        # two requests share the 40x22 shear geometry: the second reuses a context
        assert st["contexts_reused"] >= 1
        assert st["contexts_created"] + st["contexts_reused"] == len(REQS)
    assert st["running"] == 0 and st["bytes_running"] == 0


def test_server_rejects_and_caps(fre):
    p = fre.make_params(lattice="d2q9", precision="fp32", device="shear", nx=40, ny=22, nz=1, **BASE)
    one = fre.fre_device_bytes(p)
    with fre.Server("d2q9", "fp32", budget_bytes=one, chunk_steps=50, check_every=100, tol_D=0.0,
                    max_steps=200) as srv:
        big = srv.submit(31.5, 31.5, 0.0, 8.0, lattice="d2q9", device="shear", nx=64, ny=64, nz=1, **BASE)
        bad = srv.submit(19.5, 10.5, 0.0, -1.0, lattice="d2q9", device="shear", nx=40, ny=22, nz=1, **BASE)
        ok = srv.submit(19.5, 10.5, 0.0, 6.0, lattice="d2q9", device="shear", nx=40, ny=22, nz=1,
                        **dict(BASE, u_wall=0.01))
        out = {r["id"]: r for r in srv.results()}
        assert out[big]["outcome"] == "rejected" and out[bad]["outcome"] == "rejected"
        for _ in range(100):
            srv.advance()
            out.update({r["id"]: r for r in srv.results()})
            if ok in out:
                break
        assert out[ok]["outcome"] == "max_steps" and out[ok]["steps"] == 201
        with pytest.raises(fre.FreError):
            srv.submit(1, 1, 1, 1, lattice="d3q19", device="shear", nx=8, ny=8, nz=8, **BASE)


# D3Q19 requests of the served workload's kinds (shear and four-roller, plus
# a periodic box), small enough for many runs: row-kernel shear lattices
# (nx 64 and 96) and per-node four-roller ones
REQS3 = [
    ("shear", (64, 16, 8), (31.5, 7.5, 3.5, 4.0), dict(u_wall=0.02)),
    ("four_roller", (32, 32, 6), (15.5, 15.5, 2.5, 4.0), dict(u_wall=0.01)),
    ("shear", (96, 12, 6), (47.5, 5.5, 2.5, 3.5), dict(u_wall=0.03, tau_f=0.8)),
    ("periodic", (64, 10, 8), (32.0, 5.0, 4.0, 3.0), dict()),
]
# every request runs exactly 1 + 300 steps: no convergence (tol_D = 0) and
# no breakup within 300 steps of these small, weakly sheared drops
SERVE3 = dict(chunk_steps=50, check_every=100, tol_D=0.0, max_steps=300)


def serve3(fre, precision, mode, reqs):
    with fre.Server("d3q19", precision, **SERVE3) as srv:
        srv.set_batch_mode(mode, 64)
        ids = {}
        for k, (device, (nx, ny, nz), drop, kw) in enumerate(reqs):
            ids[srv.submit(*drop, lattice="d3q19", device=device, nx=nx, ny=ny, nz=nz, **dict(BASE, **kw))] = k
        res = {}
        for _ in range(1000):
            srv.advance()
            for r in srv.results():
                res[ids[r["id"]]] = r
            if len(res) == len(reqs):
                break
        st = srv.stats()
    assert st["batch_mode"] == mode
    return res


@pytest.mark.parametrize("precision", ["fp64", "fp16dev"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_alone_equals_in_mix_every_mode(fre, precision, mode):
    """The served D3Q19 configuration (FP16-dev storage) and FP64, in each
    launch mode of the batch pinned in turn (0 one launch per kernel for all
    slots, 1 each slot's own kernels in turn, 2 the same on four concurrent
    graph branches): a request served inside the mix ends exactly as the
    same request served alone in the same mode (the kernels of a slot do not
    depend on the other slots; bound 1e-14 relative, i.e. equal up to the
    last bit).  Against a context stepped alone on its own kernels: equal
    in modes 1 and 2 (the same kernels); in mode 0 the per-node kernels run
    every slot, which round differently from the row kernels of the shear
    and periodic lattices: 1e-11 relative in FP64, and in FP16-dev 1e-4 on
    D (absolute: D is small here) and 1e-5 relative on the mass and volume
    (11-bit stores of deviations)."""
    mix = serve3(fre, precision, mode, REQS3)
    for k, (device, shape, drop, kw) in enumerate(REQS3):
        r = mix[k]
        assert r["outcome"] == "max_steps" and r["steps"] == 301, r
        one = serve3(fre, precision, mode, [REQS3[k]])[0]
        assert one["steps"] == 301
        for key in ("D", "mass", "dp", "volume", "theta_deg"):
            a, b = r["obs"][key], one["obs"][key]
            assert abs(a - b) <= 1e-14 * max(abs(b), 1e-12), (k, key, a, b)
        nx, ny, nz = shape
        sim = fre.Simulation(lattice="d3q19", precision=precision, device=device, nx=nx, ny=ny, nz=nz,
                             **dict(BASE, **kw))
        sim.init_droplet(*drop)
        sim.step(301)
        ref = sim.observables()
        sim.close()
        # (bound, floor of the scale): |a - b| <= bound * max(|b|, floor)
        if mode in (1, 2):
            tol = {"D": (1e-14, 1e-12), "mass": (1e-14, 1e-12), "volume": (1e-14, 1e-12)}
        elif precision == "fp64":
            tol = {"D": (1e-11, 1e-3), "mass": (1e-11, 1e-12), "volume": (1e-11, 1e-12)}
        else:
            tol = {"D": (1e-4, 1.0), "mass": (1e-5, 1e-12), "volume": (1e-5, 1e-12)}
        for key, (t, floor) in tol.items():
            a, b = r["obs"][key], ref[key]
            assert abs(a - b) <= t * max(abs(b), floor), (k, key, a, b, mode)
