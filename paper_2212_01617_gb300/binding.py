"""Thin ctypes binding of the C ABI in include/fre.h (argument marshalling only).

Every function here has the name of the C entry point it calls; all the
computation runs in the CUDA library libfre.so.  There is no CPU fallback: if
the library is missing or no GPU is visible, the calls raise.

PyTorch supplies the CUDA stream (``torch.cuda.current_stream()``) when it is
importable; the library owns the device memory of each context.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libfre.so")

FRE_OK, FRE_ERR_ARG, FRE_ERR_OOM, FRE_ERR_CUDA, FRE_ERR_UNSTABLE, FRE_ERR_BUDGET, FRE_ERR_STATE = range(7)
FRE_D2Q9, FRE_D3Q19 = 0, 1
FRE_FP64, FRE_FP32, FRE_FP16DEV, FRE_BF16DEV = 0, 1, 2, 3
FRE_SHEAR, FRE_FOUR_ROLLER, FRE_PERIODIC = 0, 1, 2

PRECISIONS = {"fp64": FRE_FP64, "fp32": FRE_FP32, "fp16dev": FRE_FP16DEV, "bf16dev": FRE_BF16DEV}
LATTICES = {"d2q9": FRE_D2Q9, "d3q19": FRE_D3Q19}
DEVICES = {"shear": FRE_SHEAR, "four_roller": FRE_FOUR_ROLLER, "periodic": FRE_PERIODIC}

# every entry point declared in include/fre.h
EXPORTS = ["fre_device_bytes", "fre_create", "fre_init_droplet", "fre_init_fields", "fre_init_consistent",
           "fre_load_populations", "fre_store_populations", "fre_step", "fre_step_timed",
           "fre_copy_fields", "fre_observables", "fre_step_count", "fre_uses_row_kernels",
           "fre_kernel_path", "fre_components", "fre_moments_noalloc",
           "fre_batch_create", "fre_batch_add", "fre_batch_remove", "fre_batch_step",
           "fre_batch_observables", "fre_batch_context", "fre_batch_slots", "fre_batch_bytes_in_use",
           "fre_batch_tuning", "fre_batch_set_mode", "fre_batch_synchronize", "fre_batch_destroy",
           "fre_server_create", "fre_server_submit", "fre_server_advance", "fre_server_results",
           "fre_server_stats", "fre_server_clock", "fre_server_batch", "fre_server_destroy",
           "fre_destroy", "fre_last_error"]
FRE_FLAG_GENERIC_KERNELS = 1
FRE_FLAG_COUETTE_REFERENCE = 4
FRE_FLAG_REST_REFERENCE = 8
FRE_FLAG_TEST_PIPELINE_STALL = 16
FRE_FLAG_INTERPOLATED_WALLS = 32


class FreError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[fre status {status}] {msg}")
        self.status = status


class fre_params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("precision", C.c_int), ("device", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau_f", C.c_double), ("tau_g", C.c_double), ("A", C.c_double),
                ("kappa", C.c_double), ("gamma_mob", C.c_double), ("u_wall", C.c_double),
                ("rho0", C.c_double), ("flags", C.c_uint),
                ("model", C.c_int), ("kappa1", C.c_double), ("kappa2", C.c_double), ("alpha", C.c_double)]


class fre_obs(C.Structure):
    _fields_ = [("mass", C.c_double), ("phi_sum", C.c_double), ("volume", C.c_double),
                ("drop_weight", C.c_double), ("drop_count", C.c_double),
                ("centroid", C.c_double * 3), ("I", C.c_double * 6),
                ("D", C.c_double), ("theta_deg", C.c_double),
                ("p_centre", C.c_double), ("p_far", C.c_double), ("dp", C.c_double),
                ("max_u", C.c_double), ("step", C.c_longlong), ("status", C.c_int)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


SERVE_OUTCOMES = {0: "running", 1: "converged", 2: "breakup", 3: "max_steps", 4: "unstable", 5: "rejected",
                  6: "failed"}


class fre_serve_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("target_nodes", C.c_longlong), ("max_running", C.c_int),
                ("chunk_steps", C.c_int), ("check_every", C.c_int), ("tol_D", C.c_double),
                ("max_steps", C.c_longlong), ("breakup_min_frac", C.c_double)]


class fre_serve_result(C.Structure):
    _fields_ = [("id", C.c_longlong), ("outcome", C.c_int), ("steps", C.c_longlong), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("obs", fre_obs)]

    def as_dict(self) -> dict:
        return {"id": self.id, "outcome": SERVE_OUTCOMES.get(self.outcome, str(self.outcome)),
                "steps": self.steps, "t_submit": self.t_submit, "t_admit": self.t_admit, "t_done": self.t_done,
                "obs": self.obs.as_dict()}


class fre_serve_stats(C.Structure):
    _fields_ = [("running", C.c_int), ("queued", C.c_int), ("bytes_running", C.c_size_t),
                ("bytes_pooled", C.c_size_t), ("running_nodes", C.c_longlong), ("node_updates", C.c_longlong),
                ("steps_advanced", C.c_longlong), ("contexts_created", C.c_longlong),
                ("contexts_reused", C.c_longlong), ("batch_mode", C.c_int), ("batch_bx", C.c_int),
                ("tunes", C.c_longlong), ("captures", C.c_longlong)]


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfre.so and declare the signatures; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FreError(FRE_ERR_STATE, f"CUDA library {path} is not built; run __graft_entry__.build()")
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        L.fre_device_bytes.restype = C.c_size_t
        L.fre_device_bytes.argtypes = [C.POINTER(fre_params)]
        L.fre_create.argtypes = [C.POINTER(fre_params), vp, C.POINTER(vp)]
        L.fre_init_droplet.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_double]
        L.fre_init_fields.argtypes = [vp, dp, dp, dp, dp, dp]
        L.fre_init_consistent.argtypes = [vp, C.c_int]
        L.fre_load_populations.argtypes = [vp, dp, dp]
        L.fre_store_populations.argtypes = [vp, dp, dp]
        L.fre_step.argtypes = [vp, C.c_int]
        L.fre_step_timed.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_longlong)]
        L.fre_copy_fields.argtypes = [vp, dp, dp, dp, dp, dp, dp]
        L.fre_observables.argtypes = [vp, C.POINTER(fre_obs)]
        L.fre_step_count.restype = C.c_longlong
        L.fre_step_count.argtypes = [vp]
        L.fre_uses_row_kernels.restype = C.c_int
        L.fre_uses_row_kernels.argtypes = [vp]
        L.fre_kernel_path.restype = C.c_int
        L.fre_kernel_path.argtypes = [vp]
        L.fre_components.restype = C.c_int
        L.fre_components.argtypes = [vp, C.c_longlong, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.c_int,
                                     C.POINTER(C.c_int)]
        L.fre_moments_noalloc.restype = C.c_int
        L.fre_moments_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp]
        L.fre_destroy.argtypes = [vp]
        L.fre_destroy.restype = None
        L.fre_last_error.restype = C.c_char_p
        L.fre_batch_create.argtypes = [C.c_int, C.c_int, vp, C.c_size_t, C.POINTER(vp)]
        L.fre_batch_add.argtypes = [vp, C.POINTER(fre_params), C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.POINTER(C.c_int)]
        L.fre_batch_remove.argtypes = [vp, C.c_int]
        L.fre_batch_step.argtypes = [vp, C.c_int]
        L.fre_batch_observables.argtypes = [vp, C.c_int, C.POINTER(fre_obs)]
        L.fre_batch_context.restype = vp
        L.fre_batch_context.argtypes = [vp, C.c_int]
        L.fre_batch_slots.restype = C.c_int
        L.fre_batch_slots.argtypes = [vp, C.POINTER(C.c_int), C.c_int]
        L.fre_batch_bytes_in_use.restype = C.c_size_t
        L.fre_batch_bytes_in_use.argtypes = [vp]
        L.fre_batch_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
        L.fre_batch_set_mode.argtypes = [vp, C.c_int, C.c_int]
        L.fre_batch_synchronize.argtypes = [vp]
        L.fre_batch_destroy.argtypes = [vp]
        L.fre_batch_destroy.restype = None
        L.fre_server_create.argtypes = [C.c_int, C.c_int, C.POINTER(fre_serve_config), vp, C.POINTER(vp)]
        L.fre_server_submit.argtypes = [vp, C.POINTER(fre_params), C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.POINTER(C.c_longlong)]
        L.fre_server_advance.argtypes = [vp, C.POINTER(C.c_int)]
        L.fre_server_results.restype = C.c_int
        L.fre_server_results.argtypes = [vp, C.POINTER(fre_serve_result), C.c_int]
        L.fre_server_stats.argtypes = [vp, C.POINTER(fre_serve_stats)]
        L.fre_server_clock.restype = C.c_double
        L.fre_server_clock.argtypes = [vp]
        L.fre_server_batch.restype = vp
        L.fre_server_batch.argtypes = [vp]
        L.fre_server_destroy.restype = None
        L.fre_server_destroy.argtypes = [vp]
        for name in ("fre_server_create", "fre_server_submit", "fre_server_advance", "fre_server_stats"):
            getattr(L, name).restype = C.c_int
        for name in ("fre_batch_create", "fre_batch_add", "fre_batch_remove", "fre_batch_step",
                     "fre_batch_observables", "fre_batch_tuning", "fre_batch_set_mode", "fre_batch_synchronize"):
            getattr(L, name).restype = C.c_int
        for name in ("fre_create", "fre_init_droplet", "fre_init_fields", "fre_init_consistent", "fre_load_populations",
                     "fre_store_populations", "fre_step", "fre_step_timed", "fre_copy_fields",
                     "fre_observables"):
            getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _check(status: int, what: str):
    if status != FRE_OK:
        msg = load_library().fre_last_error().decode(errors="replace")
        raise FreError(status, f"{what}: {msg}")


def _dptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def current_stream_handle():
    """cudaStream_t of torch's current stream (None without torch/CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def make_params(lattice="d2q9", precision="fp64", device="shear", nx=16, ny=8, nz=1,
                tau_f=1.0, tau_g=1.0, A=0.04, kappa=0.04, gamma_mob=1.0, u_wall=0.0,
                rho0=1.0, flags=0, model=0, kappa1=0.0, kappa2=0.0, alpha=0.0) -> fre_params:
    lat = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    dev = DEVICES[device] if isinstance(device, str) else int(device)
    return fre_params(lat, prec, dev, int(nx), int(ny), int(nz), float(tau_f), float(tau_g),
                      float(A), float(kappa), float(gamma_mob), float(u_wall), float(rho0), int(flags),
                      int(model), float(kappa1), float(kappa2), float(alpha))


# --------------------------------------------------- one call per C entry point

def fre_device_bytes(p: fre_params) -> int:
    return int(load_library().fre_device_bytes(C.byref(p)))


def fre_create(p: fre_params, stream=None) -> int:
    h = C.c_void_p()
    s = stream if stream is not None else current_stream_handle()
    _check(load_library().fre_create(C.byref(p), C.c_void_p(s) if s else None, C.byref(h)), "fre_create")
    return h.value


def fre_init_droplet(h, cx, cy, cz, R):
    _check(load_library().fre_init_droplet(h, cx, cy, cz, R), "fre_init_droplet")


def fre_init_fields(h, rho, ux, uy, uz, phi):
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            for a in (rho, ux, uy, uz, phi)]
    _check(load_library().fre_init_fields(h, *[_dptr(a) for a in arrs]), "fre_init_fields")


def fre_init_consistent(h, iterations: int):
    _check(load_library().fre_init_consistent(h, int(iterations)), "fre_init_consistent")


def fre_load_populations(h, f, g):
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    _check(load_library().fre_load_populations(h, _dptr(f), _dptr(g)), "fre_load_populations")


def fre_store_populations(h, f=None, g=None):
    _check(load_library().fre_store_populations(h, _dptr(f), _dptr(g)), "fre_store_populations")


def fre_step(h, nsteps: int):
    _check(load_library().fre_step(h, int(nsteps)), "fre_step")


def fre_step_timed(h, nsteps: int):
    """Returns (ms_phi, ms_mu, ms_update, ms_total, kernel_launches)."""
    ms = np.zeros(4)
    nl = C.c_longlong(0)
    _check(load_library().fre_step_timed(h, int(nsteps), _dptr(ms), C.byref(nl)), "fre_step_timed")
    return float(ms[0]), float(ms[1]), float(ms[2]), float(ms[3]), int(nl.value)


def fre_copy_fields(h, rho=None, ux=None, uy=None, uz=None, phi=None, mu=None):
    _check(load_library().fre_copy_fields(h, *[_dptr(a) for a in (rho, ux, uy, uz, phi, mu)]),
           "fre_copy_fields")


def fre_observables(h, allow_unstable: bool = True) -> dict:
    o = fre_obs()
    s = load_library().fre_observables(h, C.byref(o))
    if not (s == FRE_OK or (allow_unstable and s == FRE_ERR_UNSTABLE)):
        _check(s, "fre_observables")
    return o.as_dict()


def fre_step_count(h) -> int:
    return int(load_library().fre_step_count(h))


def fre_uses_row_kernels(h) -> bool:
    return bool(load_library().fre_uses_row_kernels(h))


def fre_kernel_path(h) -> int:
    return int(load_library().fre_kernel_path(h))


def fre_components(h, min_size=1, max_sizes=16, n=None):
    """Components of the phase phi > 0: (count, sizes largest first, labels
    or None).  Labels are returned when n (the node count) is given."""
    cnt = C.c_int(0)
    sz = np.zeros(max(max_sizes, 1), dtype=np.int64)
    lab = np.zeros(n, dtype=np.int32) if n else None
    _check(load_library().fre_components(h, int(min_size), C.byref(cnt),
                                         sz.ctypes.data_as(C.POINTER(C.c_longlong)), int(max_sizes),
                                         lab.ctypes.data_as(C.POINTER(C.c_int)) if lab is not None else None),
           "fre_components")
    return cnt.value, [int(v) for v in sz[:max_sizes] if v > 0], lab


def fre_moments_noalloc(lattice, nx, ny, nz, f_dev_ptr, g_dev_ptr, out_dev_ptr, stream=None):
    """Device pointers in, device pointer out; queued on `stream`."""
    lat = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    s = stream if stream is not None else current_stream_handle()
    _check(load_library().fre_moments_noalloc(lat, int(nx), int(ny), int(nz), f_dev_ptr, g_dev_ptr,
                                              out_dev_ptr, s), "fre_moments_noalloc")


def fre_destroy(h):
    if h:
        load_library().fre_destroy(h)


def fre_last_error() -> str:
    return load_library().fre_last_error().decode(errors="replace")


# ------------------------------------------------------------ convenience

class Simulation:
    """One context: owns its device memory until close()."""

    def __init__(self, stream=None, **kw):
        self.params = make_params(**kw)
        self.q = 9 if self.params.lattice == FRE_D2Q9 else 19
        self.shape = (self.params.nz, self.params.ny, self.params.nx)
        self.n = self.params.nx * self.params.ny * self.params.nz
        self.h = fre_create(self.params, stream)

    def close(self):
        if getattr(self, "h", None):
            fre_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init_droplet(self, cx, cy, cz, R):
        fre_init_droplet(self.h, cx, cy, cz, R)

    def init_fields(self, rho, ux, uy, uz, phi):
        fre_init_fields(self.h, rho, ux, uy, uz, phi)

    def init_consistent(self, iterations: int):
        fre_init_consistent(self.h, iterations)

    def load_populations(self, f, g):
        fre_load_populations(self.h, f, g)

    def populations(self):
        f = np.zeros(self.q * self.n)
        g = np.zeros(self.q * self.n)
        fre_store_populations(self.h, f, g)
        return f.reshape((self.q,) + self.shape), g.reshape((self.q,) + self.shape)

    def step(self, nsteps: int = 1):
        fre_step(self.h, nsteps)

    def step_timed(self, nsteps: int = 1):
        return fre_step_timed(self.h, nsteps)

    def fields(self) -> dict:
        out = {k: np.zeros(self.n) for k in ("rho", "ux", "uy", "uz", "phi", "mu")}
        fre_copy_fields(self.h, *[out[k] for k in ("rho", "ux", "uy", "uz", "phi", "mu")])
        return {k: v.reshape(self.shape) for k, v in out.items()}

    def observables(self) -> dict:
        return fre_observables(self.h)

    def components(self, min_size=1, max_sizes=16, labels=False):
        """(count, sizes, labels[nz][ny][nx] or None) of the phase phi > 0."""
        cnt, sz, lab = fre_components(self.h, min_size, max_sizes, self.n if labels else None)
        return cnt, sz, (lab.reshape(self.shape) if lab is not None else None)

    @property
    def steps_taken(self) -> int:
        return fre_step_count(self.h)

    @property
    def row_kernels(self) -> bool:
        return fre_uses_row_kernels(self.h)

    @property
    def kernel_path(self) -> int:
        return fre_kernel_path(self.h)


class Batch:
    """Many independent simulations of one lattice and storage format advanced
    together (C ABI fre_batch_*)."""

    def __init__(self, lattice="d2q9", precision="fp32", budget_bytes=150 << 30, stream=None):
        self.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = C.c_void_p()
        st = stream if stream is not None else current_stream_handle()
        _check(load_library().fre_batch_create(self.lattice, self.precision, C.c_void_p(st) if st else None,
                                               int(budget_bytes), C.byref(h)), "fre_batch_create")
        self.h = h.value
        self._shape = {}

    def close(self):
        if getattr(self, "h", None):
            load_library().fre_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def add(self, cx, cy, cz, R, **params) -> int:
        params.setdefault("lattice", self.lattice)
        params.setdefault("precision", self.precision)
        p = make_params(**params)
        slot = C.c_int(-1)
        _check(load_library().fre_batch_add(self.h, C.byref(p), cx, cy, cz, R, C.byref(slot)), "fre_batch_add")
        self._shape[slot.value] = (p.nz, p.ny, p.nx)
        return slot.value

    def remove(self, slot: int):
        _check(load_library().fre_batch_remove(self.h, int(slot)), "fre_batch_remove")
        self._shape.pop(int(slot), None)

    def step(self, nsteps: int = 1):
        _check(load_library().fre_batch_step(self.h, int(nsteps)), "fre_batch_step")

    def observables(self, slot: int, allow_unstable: bool = True) -> dict:
        o = fre_obs()
        s = load_library().fre_batch_observables(self.h, int(slot), C.byref(o))
        if not (s == FRE_OK or (allow_unstable and s == FRE_ERR_UNSTABLE)):
            _check(s, "fre_batch_observables")
        return o.as_dict()

    def context(self, slot: int) -> int:
        return load_library().fre_batch_context(self.h, int(slot))

    def fields(self, slot: int) -> dict:
        shape = self._shape[slot]
        n = int(np.prod(shape))
        out = {k: np.zeros(n) for k in ("rho", "ux", "uy", "uz", "phi", "mu")}
        fre_copy_fields(self.context(slot), *[out[k] for k in ("rho", "ux", "uy", "uz", "phi", "mu")])
        return {k: v.reshape(shape) for k, v in out.items()}

    def populations(self, slot: int):
        shape = self._shape[slot]
        q = 9 if self.lattice == FRE_D2Q9 else 19
        n = int(np.prod(shape))
        f, g = np.zeros(q * n), np.zeros(q * n)
        fre_store_populations(self.context(slot), f, g)
        return f.reshape((q,) + shape), g.reshape((q,) + shape)

    def steps_taken(self, slot: int) -> int:
        return int(load_library().fre_step_count(self.context(slot)))

    def slots(self):
        L = load_library()
        n = L.fre_batch_slots(self.h, None, 0)
        arr = (C.c_int * max(n, 1))()
        L.fre_batch_slots(self.h, arr, n)
        return [arr[i] for i in range(n)]

    def bytes_in_use(self) -> int:
        return int(load_library().fre_batch_bytes_in_use(self.h))

    def tuning(self):
        mode, bx = C.c_int(0), C.c_int(0)
        ms = np.zeros(5)
        s = load_library().fre_batch_tuning(self.h, C.byref(mode), C.byref(bx), _dptr(ms))
        return {"tuned": s == FRE_OK, "mode": mode.value, "bx": bx.value, "ms_per_step": ms.tolist()}

    def set_mode(self, mode: int, bx: int = 64):
        """Pin the launch mode (0 batched, 1 per-slot, 2 concurrent per-slot;
        -1 back to the autotuner)."""
        _check(load_library().fre_batch_set_mode(self.h, int(mode), int(bx)), "fre_batch_set_mode")

    def synchronize(self):
        _check(load_library().fre_batch_synchronize(self.h), "fre_batch_synchronize")


class Server:
    """Serving loop over a batch (C ABI fre_server_*): submit requests,
    call advance() until they finish, collect results()."""

    def __init__(self, lattice="d3q19", precision="fp16dev", budget_bytes=150 << 30, target_nodes=0,
                 max_running=0, chunk_steps=250, check_every=1000, tol_D=1e-4, max_steps=100000,
                 breakup_min_frac=0.005, stream=None):
        self.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg = fre_serve_config(int(budget_bytes), int(target_nodes), int(max_running), int(chunk_steps),
                               int(check_every), float(tol_D), int(max_steps), float(breakup_min_frac))
        h = C.c_void_p()
        st = stream if stream is not None else current_stream_handle()
        _check(load_library().fre_server_create(self.lattice, self.precision, C.byref(cfg),
                                                C.c_void_p(st) if st else None, C.byref(h)), "fre_server_create")
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            load_library().fre_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, cx, cy, cz, R, **params) -> int:
        params.setdefault("lattice", self.lattice)
        params.setdefault("precision", self.precision)
        p = make_params(**params)
        rid = C.c_longlong(0)
        _check(load_library().fre_server_submit(self.h, C.byref(p), cx, cy, cz, R, C.byref(rid)),
               "fre_server_submit")
        return rid.value

    def advance(self) -> int:
        n = C.c_int(0)
        _check(load_library().fre_server_advance(self.h, C.byref(n)), "fre_server_advance")
        return n.value

    def results(self, max_results: int = 256):
        buf = (fre_serve_result * max_results)()
        n = load_library().fre_server_results(self.h, buf, max_results)
        return [buf[i].as_dict() for i in range(max(n, 0))]

    def stats(self) -> dict:
        st = fre_serve_stats()
        _check(load_library().fre_server_stats(self.h, C.byref(st)), "fre_server_stats")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def clock(self) -> float:
        return float(load_library().fre_server_clock(self.h))

    def set_batch_mode(self, mode: int, bx: int = 64):
        """Pin the launch mode of the server's batch (fre_batch_set_mode)."""
        b = load_library().fre_server_batch(self.h)
        _check(load_library().fre_batch_set_mode(b, int(mode), int(bx)), "fre_batch_set_mode")
