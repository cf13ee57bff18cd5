"""ctypes wrapper of the FP64 CPU oracle (oracle/fre_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path
(``paper_2212_01617_gb300``) never imports this package, and this package
imports nothing from it.

The oracle follows the two-lattice free energy LBM of Simonis et al.,
arXiv:2212.01617, Sec. 2.2-2.3 and Algorithm 1, step by step; see the header of
``fre_oracle.c`` for the equations and for the readings of points the paper
leaves open.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fre_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

D2Q9, D3Q19 = 0, 1
SHEAR, FOUR_ROLLER, PERIODIC = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "fre_oracle.h"))
    ):
        cmd = ["gcc", "-O3", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", SRC, "-o", LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("device", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau_f", C.c_double), ("tau_g", C.c_double),
                ("A", C.c_double), ("kappa", C.c_double), ("Gamma", C.c_double),
                ("u_wall", C.c_double), ("rho0", C.c_double),
                ("model", C.c_int), ("kappa1", C.c_double), ("kappa2", C.c_double), ("alpha", C.c_double),
                ("interp", C.c_int)]


class Obs(C.Structure):
    _fields_ = [("mass", C.c_double), ("phi_sum", C.c_double), ("volume", C.c_double),
                ("drop_weight", C.c_double), ("drop_count", C.c_double),
                ("centroid", C.c_double * 3), ("I", C.c_double * 6),
                ("D", C.c_double), ("theta_deg", C.c_double),
                ("p_centre", C.c_double), ("p_far", C.c_double), ("dp", C.c_double),
                ("max_u", C.c_double), ("step", C.c_longlong), ("status", C.c_int)]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            dp = C.POINTER(C.c_double)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(Params)]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_q.argtypes = [C.c_void_p]
            L.orc_nodes.argtypes = [C.c_void_p]
            L.orc_nodes.restype = C.c_longlong
            L.orc_is_solid.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
            L.orc_init_droplet.argtypes = [C.c_void_p] + [C.c_double] * 4
            L.orc_init_fields.argtypes = [C.c_void_p] + [dp] * 5
            L.orc_load_populations.argtypes = [C.c_void_p, dp, dp]
            L.orc_store_populations.argtypes = [C.c_void_p, dp, dp]
            L.orc_step.argtypes = [C.c_void_p, C.c_int]
            L.orc_fields.argtypes = [C.c_void_p] + [dp] * 6
            L.orc_observables.argtypes = [C.c_void_p, C.POINTER(Obs)]
            L.orc_lattice_info.argtypes = [C.c_int, C.POINTER(C.c_int),
                                           C.POINTER(C.c_int), dp]
            L.orc_feq.argtypes = [C.c_int, C.c_double, dp, dp]
            L.orc_geq.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, dp, dp]
            L.orc_guo.argtypes = [C.c_int, C.c_double, dp, dp, dp]
            L.orc_init_consistent.restype = C.c_int
            L.orc_init_consistent.argtypes = [C.c_void_p, C.c_int]
            L.orc_label_phase.restype = C.c_int
            L.orc_label_phase.argtypes = [C.c_void_p, dp, C.POINTER(C.c_int)]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_num_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lattice_info(lattice: int):
    q = C.c_int()
    c = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19)
    lib().orc_lattice_info(lattice, C.byref(q), c.ctypes.data_as(C.POINTER(C.c_int)), _ptr(w))
    return c[: 3 * q.value].reshape(q.value, 3).copy(), w[: q.value].copy()


def feq(lattice: int, rho: float, u) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_feq(lattice, rho, _ptr(np.asarray(u, dtype=np.float64).copy()), _ptr(out))
    return out[: 9 if lattice == D2Q9 else 19]


def geq(lattice: int, phi: float, mu: float, Gamma: float, u) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_geq(lattice, phi, mu, Gamma, _ptr(np.asarray(u, dtype=np.float64).copy()), _ptr(out))
    return out[: 9 if lattice == D2Q9 else 19]


def guo(lattice: int, tau: float, u, F) -> np.ndarray:
    out = np.zeros(19)
    lib().orc_guo(lattice, tau, _ptr(np.asarray(u, dtype=np.float64).copy()),
                  _ptr(np.asarray(F, dtype=np.float64).copy()), _ptr(out))
    return out[: 9 if lattice == D2Q9 else 19]


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def num_threads() -> int:
    return int(lib().orc_num_threads())


class Oracle:
    """One FP64 CPU simulation.  Arrays are [q][nz][ny][nx] / [nz][ny][nx]."""

    def __init__(self, lattice=D2Q9, device=SHEAR, nx=16, ny=8, nz=1, tau_f=1.0,
                 tau_g=1.0, A=0.04, kappa=0.04, Gamma=1.0, u_wall=0.0, rho0=1.0,
                 model=0, kappa1=0.0, kappa2=0.0, alpha=0.0, interp=0):
        """model 0: the reduced functional (A, kappa); model 1: the full
        functional of Eq. functional (kappa1, kappa2, alpha).  interp: the
        four-roller device's interpolated bounce-back at the rollers."""
        self.p = Params(lattice, device, nx, ny, nz, tau_f, tau_g, A, kappa, Gamma,
                        u_wall, rho0, model, kappa1, kappa2, alpha, interp)
        self._h = lib().orc_create(C.byref(self.p))
        if not self._h:
            raise ValueError("oracle: invalid parameters")
        self.q = lib().orc_q(self._h)
        self.shape = (nz, ny, nx)
        self.n = nx * ny * nz

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def solid_mask(self) -> np.ndarray:
        nz, ny, nx = self.shape
        m = np.zeros(self.shape, dtype=bool)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    m[z, y, x] = bool(lib().orc_is_solid(self._h, x, y, z))
        return m

    def init_droplet(self, cx, cy, cz, R):
        if lib().orc_init_droplet(self._h, cx, cy, cz, R) != 0:
            raise ValueError("oracle: init_droplet failed")

    def init_fields(self, rho, ux, uy, uz, phi):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
                for a in (rho, ux, uy, uz, phi)]
        if lib().orc_init_fields(self._h, *[_ptr(a) for a in arrs]) != 0:
            raise ValueError("oracle: init_fields failed")

    def init_consistent(self, iterations: int):
        """Consistent initial populations from the current state (Sec. 2.3,
        Mei et al.): f relaxed with u and F held, g at equilibrium."""
        if lib().orc_init_consistent(self._h, int(iterations)) != 0:
            raise ValueError("oracle: init_consistent failed")

    def load_populations(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        assert f.size == self.q * self.n and g.size == self.q * self.n
        lib().orc_load_populations(self._h, _ptr(f), _ptr(g))

    def populations(self):
        f = np.zeros(self.q * self.n)
        g = np.zeros(self.q * self.n)
        lib().orc_store_populations(self._h, _ptr(f), _ptr(g))
        return f.reshape((self.q,) + self.shape), g.reshape((self.q,) + self.shape)

    def step(self, nsteps: int = 1):
        if lib().orc_step(self._h, int(nsteps)) != 0:
            raise ValueError("oracle: step failed")

    def fields(self) -> dict:
        out = {k: np.zeros(self.n) for k in ("rho", "ux", "uy", "uz", "phi", "mu")}
        lib().orc_fields(self._h, *[_ptr(out[k]) for k in ("rho", "ux", "uy", "uz", "phi", "mu")])
        return {k: v.reshape(self.shape) for k, v in out.items()}

    def observables(self) -> dict:
        o = Obs()
        lib().orc_observables(self._h, C.byref(o))
        return o.as_dict()

    def label_phase(self, phi=None):
        """Components of the phase phi > 0 (phi: [nz][ny][nx], default the
        oracle's own current phi): (count, labels), labels -1 outside the
        phase, else the smallest node index of the component."""
        if phi is None:
            phi = self.fields()["phi"]
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        assert phi.size == self.n
        labels = np.zeros(self.n, dtype=np.int32)
        count = lib().orc_label_phase(self._h, _ptr(phi), labels.ctypes.data_as(C.POINTER(C.c_int)))
        if count < 0:
            raise MemoryError("oracle: label_phase")
        return count, labels.reshape(self.shape)
