"""fre_moments_noalloc: the conservation sums and droplet moments for callers
that cannot allocate device memory (their own allocator owns the device, or
an allocation would synchronise where they cannot afford it).

Its results must equal those of fre_observables, which computes the same
quantities with context-owned scratch, within the 1e-10 relative tolerance
the FP64 observables tests use -- on two calls in a row with different data,
since every call shares the library's one static scratch array.  This file
runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_2212_01617_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("mass", "phi_sum", "volume", "drop_weight", "drop_count")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    return torch, fre


def close(a, b, tol=1e-10):
    return abs(a - b) <= tol * max(1.0, abs(b))


@pytest.mark.parametrize("lattice,shape", [("d3q19", (9, 14, 23)), ("d2q9", (1, 40, 71))])
def test_noalloc_moments_match_observables_twice(env, lattice, shape):
    torch, fre = env
    q = 19 if lattice == "d3q19" else 9
    nz, ny, nx = shape
    for seed in (21, 22):  # two calls in a row on different data
        f, g = inputs.random_populations(q, shape, seed=seed)
        with fre.Simulation(lattice=lattice, precision="fp64", device="periodic", nx=nx, ny=ny, nz=nz) as sim:
            sim.load_populations(f, g)
            ref = sim.observables()
        fd = torch.from_numpy(f.reshape(-1).copy()).cuda()
        gd = torch.from_numpy(g.reshape(-1).copy()).cuda()
        out = torch.full((16,), float("nan"), dtype=torch.float64, device="cuda")
        fre.fre_moments_noalloc(lattice, nx, ny, nz, fd.data_ptr(), gd.data_ptr(), out.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        for k, key in enumerate(KEYS):
            assert close(o[k], ref[key]), (seed, key, o[k], ref[key])
        assert np.allclose(o[5:8], ref["centroid"], rtol=0, atol=1e-10)
        assert np.allclose(o[8:14], ref["I"], rtol=1e-10, atol=1e-12)
        assert close(o[14], ref["D"]) and close(o[15], ref["theta_deg"])
        assert ref["drop_count"] > 0  # the droplet moments are exercised


def test_noalloc_rejects_oversized_lattice(env):
    torch, fre = env
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(fre.FreError) as e:
        fre.fre_moments_noalloc("d3q19", 2048, 1024, 1024, out.data_ptr(), out.data_ptr(), out.data_ptr())
    assert e.value.status == fre.binding.FRE_ERR_ARG
    assert "2^30" in fre.fre_last_error()
