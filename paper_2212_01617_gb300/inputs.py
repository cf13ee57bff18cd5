"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

Holds no arithmetic of the method: only random draws (numpy Generator seeded
with an explicit seed) of population arrays, fields and case parameters.
"""
from __future__ import annotations

import numpy as np

SEED = 2212_01617
W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def rng(seed: int = SEED) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_populations(q: int, shape, seed: int = SEED, amp: float = 0.05, phi_amp: float = 0.8):
    """Positive f near rest (w_i (1 + amp*U(-1,1))) and g with phi in (-phi_amp, phi_amp).

    Returns FP64 arrays [q][nz][ny][nx]."""
    r = rng(seed)
    w = W9 if q == 9 else W19
    f = w[:, None, None, None] * (1.0 + amp * r.uniform(-1, 1, (q,) + tuple(shape)))
    g = w[:, None, None, None] * r.uniform(-phi_amp, phi_amp, (q,) + tuple(shape))
    g += w[:, None, None, None] * amp * r.uniform(-1, 1, (q,) + tuple(shape))
    return f, g


def random_fields(shape, seed: int = SEED, u_amp: float = 0.02, drho: float = 0.01):
    """rho ~ 1 +- drho, u ~ U(-u_amp, u_amp), phi ~ smooth random in (-1, 1)."""
    r = rng(seed)
    rho = 1.0 + drho * r.uniform(-1, 1, shape)
    ux, uy, uz = (u_amp * r.uniform(-1, 1, shape) for _ in range(3))
    phi = np.tanh(3.0 * r.uniform(-1, 1, shape))
    return rho, ux, uy, uz, phi


def batch_cases(n: int = 64, seed: int = SEED + 3):
    """Draws of a D2Q9 batch of `n` uneven cases: alternating parallel-band
    shear and four-roller devices, Nx even and uniform in [64, 512], capillary
    number Ca ~ U(0.05, 0.5) and droplet size ratio R/H ~ U(0.1, 0.3).

    Returns a list of dicts (device, nx, ca, r_over_h); the lattice height and
    the wall speed that realises Ca are the caller's."""
    r = rng(seed)
    out = []
    for k in range(n):
        out.append({"device": "shear" if k % 2 == 0 else "four_roller",
                    "nx": 2 * int(r.integers(32, 257)),
                    "ca": float(r.uniform(0.05, 0.5)),
                    "r_over_h": float(r.uniform(0.1, 0.3))})
    return out


SERVE_SIZES = ((64, 64, 64), (96, 96, 96), (128, 64, 64), (192, 96, 96))


def serving_trace(n: int = 400, rate: float = 20.0, seed: int = SEED + 4):
    """A finite Poisson request trace: exponential inter-arrival gaps of mean
    1/rate seconds, lattice size uniform over SERVE_SIZES, device shear or
    four-roller with equal odds, Ca ~ U(0.05, 0.45), R/H ~ U(0.1, 0.3).

    Returns a list of dicts (t_arrival, shape, device, ca, r_over_h) in
    arrival order."""
    r = rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += float(r.exponential(1.0 / rate))
        out.append({"t_arrival": t,
                    "shape": SERVE_SIZES[int(r.integers(0, len(SERVE_SIZES)))],
                    "device": "shear" if r.uniform() < 0.5 else "four_roller",
                    "ca": float(r.uniform(0.05, 0.45)),
                    "r_over_h": float(r.uniform(0.1, 0.3))})
    return out


def multi_drop_phi(shape, n_drops: int, seed: int = SEED + 5, r_min: float = 1.5, r_max: float = 6.0,
                   periodic=(True, True, True)):
    """A phi field [nz][ny][nx] holding n_drops drops of random centres and
    radii (uniform in [r_min, r_max]): phi = the largest of tanh((R_k - d_k)
    / sqrt(2)) over the drops, d_k the distance to drop k's centre, taken
    with the periodic wrap along the axes flagged in `periodic` (z, y, x)."""
    r = rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = -np.ones(shape)
    for _ in range(n_drops):
        c = (r.uniform(0, nz), r.uniform(0, ny), r.uniform(0, nx))
        R = r.uniform(r_min, r_max)
        d2 = np.zeros(shape)
        for coord, n, cc, per in ((z, nz, c[0], periodic[0]), (y, ny, c[1], periodic[1]), (x, nx, c[2], periodic[2])):
            if n == 1:
                continue
            dd = np.abs(coord - cc)
            if per:
                dd = np.minimum(dd, n - dd)
            d2 += dd * dd
        phi = np.maximum(phi, np.tanh((R - np.sqrt(d2)) / np.sqrt(2.0)))
    return phi
