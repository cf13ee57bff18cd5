"""The C-ABI library builds, loads and exports every entry point that
include/fre.h declares; argument validation runs on the host (no GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fre():
    from paper_2212_01617_gb300 import build
    build.build()
    import paper_2212_01617_gb300 as fre
    fre.load_library()
    return fre


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fre_[a-z0-9_]+)\s*\(", txt))
    return names


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for need in ("fre_create", "fre_init_droplet", "fre_step", "fre_observables", "fre_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(fre):
    import ctypes
    lib = ctypes.CDLL(fre.binding.LIB_PATH)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(fre.EXPORTS) >= declared_symbols()


def test_device_bytes_and_validation(fre):
    p = fre.make_params("d3q19", "fp32", "shear", 512, 256, 256, 1.0, 1.0)
    n = 512 * 256 * 256
    b = fre.fre_device_bytes(p)
    # two buffers of f and g, 19 FP32 populations each, three FP32 fields and
    # the labels and sizes of the component labelling (two ints per node)
    assert b >= 2 * 2 * 19 * 4 * n + 3 * 4 * n + 2 * 4 * n
    assert b < 2 * 2 * 19 * 4 * n + 3 * 4 * n + 2 * 4 * n + (1 << 22)
    p16 = fre.make_params("d3q19", "fp16dev", "shear", 512, 256, 256, 1.0, 1.0)
    b16 = fre.fre_device_bytes(p16)
    assert abs(b16 - (2 * (19 * 2 + 18 * 2 + 4) * n + 3 * 4 * n + 2 * 4 * n)) < (1 << 22)
    bad = [
        fre.make_params("d2q9", "fp64", "shear", 16, 8, 2),          # D2Q9 with nz != 1
        fre.make_params("d2q9", "fp64", "shear", 16, 8, 1, tau_f=0.5),  # tau must be > 1/2
        fre.make_params("d2q9", "fp64", "shear", 16, 8, 1, tau_g=0.4),
        fre.make_params("d2q9", "fp64", "shear", 0, 8, 1),
        fre.make_params("d2q9", 7, "shear", 16, 8, 1),
        fre.make_params("d2q9", "fp64", "four_roller", 4, 4, 1),
    ]
    for p in bad:
        assert fre.fre_device_bytes(p) == 0
        with pytest.raises(fre.FreError) as e:
            fre.fre_create(p, stream=0)
        assert e.value.status == fre.binding.FRE_ERR_ARG
        assert "fre_create" in fre.fre_last_error()


def header_constants():
    """Enumerators (NAME = value) and integer #defines of include/fre.h."""
    txt = open(os.path.join(ROOT, "include", "fre.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for name, val in re.findall(r"\b(FRE_[A-Z0-9_]+)\s*=\s*(\d+)", txt):
        out[name] = int(val)
    for name, val in re.findall(r"#define\s+(FRE_[A-Z0-9_]+)\s+(\d+)u?\b", txt):
        out[name] = int(val)
    return out


def test_binding_constants_match_the_header():
    """Every constant the binding shares with include/fre.h has the header's
    value (status codes, lattices, storage formats, devices, flags)."""
    from paper_2212_01617_gb300 import binding
    hdr = header_constants()
    shared = {n: v for n, v in hdr.items() if hasattr(binding, n)}
    for need in ("FRE_OK", "FRE_ERR_BUDGET", "FRE_D3Q19", "FRE_BF16DEV", "FRE_PERIODIC",
                 "FRE_FLAG_GENERIC_KERNELS", "FRE_FLAG_COUETTE_REFERENCE"):
        assert need in shared, need
    wrong = {n: (v, getattr(binding, n)) for n, v in shared.items() if getattr(binding, n) != v}
    assert not wrong, wrong
