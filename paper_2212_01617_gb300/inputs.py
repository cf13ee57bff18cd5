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
