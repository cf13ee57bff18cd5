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
