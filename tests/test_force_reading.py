"""Evidence for the lattice form of the interfacial force (Eq. F without the
rho term, F = -phi grad(mu)).

Written on a lattice, the literal product -phi grad_h(mu) and the product-rule
form mu grad_h(phi) - grad_h(phi mu) are the same force in the continuum but
not on the grid.  This is an independent numpy D2Q9 two-lattice step (it
shares nothing with the oracle or the CUDA library): a resting flat
interface pair, periodic in x and y, with a 1e-10 velocity in the staggered
mode k = (pi, 0) (u_x alternating in sign from node to node).  Under the
literal form that mode grows exponentially; under the product-rule form,
the one the oracle and the kernels use, it decays.  Both runs are otherwise
identical (A = kappa = 0.04, Gamma = 1, tau_g = 1)."""
import numpy as np
import pytest

CS2 = 1.0 / 3.0
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _nb(a, i):
    """a(x + c_i) on the periodic grid a[y, x]."""
    return np.roll(a, (-C[i, 1], -C[i, 0]), axis=(0, 1))


def _lap(a):
    return (2 / CS2) * sum(W[i] * (_nb(a, i) - a) for i in range(1, 9))


def _grad(a):
    return [(1 / CS2) * sum(W[i] * C[i, k] * _nb(a, i) for i in range(1, 9)) for k in range(2)]


def _feq(rho, ux, uy):
    usq = ux * ux + uy * uy
    out = []
    for i in range(9):
        cu = C[i, 0] * ux + C[i, 1] * uy
        out.append(W[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq))
    return np.array(out)


def _geq(phi, mu, ux, uy, gamma):
    usq = ux * ux + uy * uy
    out = []
    for i in range(9):
        cu = C[i, 0] * ux + C[i, 1] * uy
        out.append(W[i] * (3 * gamma * mu + phi * (3 * cu + 4.5 * cu * cu - 1.5 * usq)))
    out = np.array(out)
    out[0] = phi - out[1:].sum(0)
    return out


def staggered_amplitude(form, tau_f, steps=2000, eps=1e-10, nx=64, ny=4, A=0.04, kappa=0.04, gamma=1.0,
                        tau_g=1.0):
    """|k = (pi, 0) component of u_x| every 500 steps."""
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    phi = np.tanh((x - nx / 4) / np.sqrt(2)) - np.tanh((x - 3 * nx / 4) / np.sqrt(2)) - 1
    stag = (-1.0) ** np.arange(nx)
    rho = np.ones((ny, nx))
    ux, uy = eps * (-1.0) ** x, np.zeros((ny, nx))
    mu = A * (phi ** 3 - phi) - kappa * _lap(phi)
    f, g = _feq(rho, ux, uy), _geq(phi, mu, ux, uy, gamma)
    out = []
    for t in range(steps + 1):
        rho, phi = f.sum(0), g.sum(0)
        mu = A * (phi ** 3 - phi) - kappa * _lap(phi)
        if form == "literal":
            gm = _grad(mu)
            F = [-phi * gm[0], -phi * gm[1]]
        else:
            gp, gq = _grad(phi), _grad(phi * mu)
            F = [mu * gp[0] - gq[0], mu * gp[1] - gq[1]]
        jx = sum(C[i, 0] * f[i] for i in range(9))
        jy = sum(C[i, 1] * f[i] for i in range(9))
        ux, uy = (jx + 0.5 * F[0]) / rho, (jy + 0.5 * F[1]) / rho
        if t % 500 == 0:
            out.append(abs((ux.mean(0) * stag).mean()))
        k = 1 - 0.5 / tau_f
        uF = ux * F[0] + uy * F[1]
        S = np.array([k * W[i] * (3 * (C[i, 0] * F[0] + C[i, 1] * F[1] - uF)
                                  + 9 * (C[i, 0] * ux + C[i, 1] * uy) * (C[i, 0] * F[0] + C[i, 1] * F[1]))
                      for i in range(9)])
        f = f - (f - _feq(rho, ux, uy)) / tau_f + S
        g = g - (g - _geq(phi, mu, ux, uy, gamma)) / tau_g
        for i in range(9):
            f[i] = np.roll(f[i], (C[i, 1], C[i, 0]), axis=(0, 1))
            g[i] = np.roll(g[i], (C[i, 1], C[i, 0]), axis=(0, 1))
    return np.array(out)


@pytest.mark.parametrize("tau_f", [0.8, 1.0, 1.5])
def test_literal_force_grows_the_staggered_mode(tau_f):
    lit = staggered_amplitude("literal", tau_f)
    prod = staggered_amplitude("product", tau_f)
    # literal: grows at every checkpoint, by more than 50x over 2000 steps
    assert np.all(np.diff(lit) > 0) and lit[-1] > 50 * lit[0], lit
    # product rule: the same seed decays
    assert np.all(np.diff(prod) < 0) and prod[-1] < 0.1 * prod[0], prod
