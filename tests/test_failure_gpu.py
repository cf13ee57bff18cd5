"""Failure path of the row kernels on the GPU, without a GPU fault.

Every pipeline wait of the row kernels is bounded in time; when it runs out
the kernel sets the context's error word and its warps leave, so a lost copy
or a stuck stage ends as an error status, not a hang.  The test-only flag
FRE_FLAG_TEST_PIPELINE_STALL makes that happen on purpose: the producer
warps issue no copies and the waits give up after 5 ms.  The next
synchronising call must report FRE_ERR_CUDA, and the GPU must stay usable:
a fresh context on the same device then steps and matches the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KW = dict(lattice="d3q19", device="shear", nx=64, ny=16, nz=8, tau_f=1.2, tau_g=1.0, A=0.04, kappa=0.04,
          gamma_mob=1.0, u_wall=0.02, rho0=1.0)
DROP = (31.5, 7.5, 3.5, 4.0)


@pytest.fixture(scope="module")
def fre():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    return fre


@pytest.mark.parametrize("precision", ["fp32", "fp16dev"])
def test_pipeline_wait_timeout_is_reported(fre, orc, precision):
    stall = fre.binding.FRE_FLAG_TEST_PIPELINE_STALL
    bad = fre.Simulation(precision=precision, flags=stall, **KW)
    assert bad.kernel_path == 2  # the row kernels, whose waits are bounded
    bad.init_droplet(*DROP)
    bad.step(3)  # nine kernels, each ends after its consumers' 5 ms waits
    with pytest.raises(fre.FreError) as ei:
        bad.observables()
    assert ei.value.status == fre.FRE_ERR_CUDA
    assert "gave up waiting" in str(ei.value)
    # the error word is read and cleared by the call that reports it
    bad.init_droplet(*DROP)
    assert bad.observables()["status"] == 0
    bad.close()

    # the device is still usable: a fresh context steps normally
    good = fre.Simulation(precision=precision, **KW)
    assert good.kernel_path == 2
    o = orc.Oracle(1, 0, KW["nx"], KW["ny"], KW["nz"], KW["tau_f"], KW["tau_g"], KW["A"], KW["kappa"],
                   KW["gamma_mob"], KW["u_wall"], KW["rho0"])
    good.init_droplet(*DROP)
    o.init_droplet(*DROP)
    good.step(100)
    o.step(100)
    a, b = good.fields(), o.fields()
    tol = 1e-5 if precision == "fp32" else 3e-4
    for k in ("rho", "phi"):
        assert np.abs(a[k] - b[k]).max() / np.abs(b[k]).max() < tol, k
    good.close()
