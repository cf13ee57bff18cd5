"""Pins of the oracle's droplet-component labelling (breakup detection,
Sec. 3: a drop that breaks up leaves separate drops).

The oracle labels the phase phi > 0 of the fluid nodes into connected
components, two nodes being connected when a lattice velocity links them
(D2Q9: 8 neighbours, D3Q19: 18), with the device's periodic wrap, and gives
each node the smallest node index of its component.  It is pinned against
scipy.ndimage.label with the matching structuring element (away from the
periodic boundary), against translation covariance on the torus (which
exercises every wrap), and against hand-built cases whose counts are known.
"""
import numpy as np
import pytest

ndimage = pytest.importorskip("scipy.ndimage")


def canonical(labels):
    """Partition of the phase as labels = smallest flat index of the set."""
    flat = labels.reshape(-1)
    out = np.full(flat.shape, -1, dtype=np.int64)
    for v in np.unique(flat[flat >= 0]):
        idx = np.flatnonzero(flat == v)
        out[idx] = idx.min()
    return out.reshape(labels.shape)


def structure(lattice):
    """Neighbourhood of the lattice velocities: D2Q9 the 3x3 square, D3Q19 the
    3x3x3 cube without its 8 corners."""
    return ndimage.generate_binary_structure(2, 2) if lattice == 0 else ndimage.generate_binary_structure(3, 2)


def random_phase(rng, shape, frac):
    return np.where(rng.uniform(size=shape) < frac, 1.0, -1.0)


@pytest.mark.parametrize("lattice,shape", [(0, (1, 30, 41)), (1, (17, 13, 19))])
@pytest.mark.parametrize("frac", [0.2, 0.45])
def test_matches_scipy_away_from_the_boundary(orc, lattice, shape, frac):
    rng = np.random.default_rng(31)
    phi = random_phase(rng, shape, frac)
    # a frame of -1 keeps every component away from the periodic boundary
    phi[..., :1, :] = phi[..., -1:, :] = -1.0
    phi[..., :, :1] = phi[..., :, -1:] = -1.0
    if lattice == 1:
        phi[:1] = phi[-1:] = -1.0
    o = orc.Oracle(lattice, orc.PERIODIC, shape[2], shape[1], shape[0])
    count, lab = o.label_phase(phi)
    ref, nref = ndimage.label(phi[0] > 0 if lattice == 0 else phi > 0, structure=structure(lattice))
    ref = ref.reshape(shape) - 1  # -1 outside, 0.. inside
    assert count == nref
    assert np.array_equal(lab, canonical(ref))


@pytest.mark.parametrize("lattice,shape", [(0, (1, 24, 29)), (1, (11, 9, 14))])
def test_translation_covariance_on_the_torus(orc, lattice, shape):
    """Rolling the field periodically rolls the partition: every wrap of
    x, y (and z) is exercised by the components that cross the boundary."""
    rng = np.random.default_rng(32)
    phi = random_phase(rng, shape, 0.35)
    o = orc.Oracle(lattice, orc.PERIODIC, shape[2], shape[1], shape[0])
    count, lab = o.label_phase(phi)
    for shift in [(0, 5, 7), (0, -3, 11)] + ([(4, 2, -6)] if lattice == 1 else []):
        c2, lab2 = o.label_phase(np.roll(phi, shift, axis=(0, 1, 2)))
        assert c2 == count
        assert np.array_equal(canonical(lab2), canonical(np.roll(lab, shift, axis=(0, 1, 2))))
    # not vacuous: some component crosses the boundary, and the labels are
    # the smallest index of each component
    flat = lab.reshape(-1)
    assert any(len(np.unique(flat[flat == v])) and np.any(lab[..., 0, :] == v) and np.any(lab[..., -1, :] == v)
               for v in np.unique(flat[flat >= 0]))
    for v in np.unique(flat[flat >= 0]):
        assert np.flatnonzero(flat == v).min() == v


def test_known_counts(orc):
    nx = ny = nz = 16
    o = orc.Oracle(1, orc.PERIODIC, nx, ny, nz)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]

    def ball(cx, cy, cz, r):
        return (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= r * r

    phi = np.where(ball(4, 4, 4, 2.5) | ball(11, 11, 11, 2.5), 1.0, -1.0)
    assert o.label_phase(phi)[0] == 2
    # two single nodes touching along an edge direction (1, 1, 0) are linked
    # by a D3Q19 velocity; touching only at a corner (1, 1, 1) they are not
    phi = -np.ones((nz, ny, nx))
    phi[5, 5, 5] = phi[5, 6, 6] = 1.0
    assert o.label_phase(phi)[0] == 1
    phi = -np.ones((nz, ny, nx))
    phi[5, 5, 5] = phi[6, 6, 6] = 1.0
    assert o.label_phase(phi)[0] == 2
    # a slab across the whole box in x and z wraps into one component
    phi = np.where((y >= 6) & (y <= 8), 1.0, -1.0)
    assert o.label_phase(phi)[0] == 1


def test_shear_walls_do_not_wrap_and_rollers_are_not_phase(orc):
    nx, ny = 24, 16
    sh = orc.Oracle(0, orc.SHEAR, nx, ny, 1)
    pe = orc.Oracle(0, orc.PERIODIC, nx, ny, 1)
    phi = -np.ones((1, ny, nx))
    phi[0, 0, 10:13] = phi[0, ny - 1, 10:13] = 1.0  # touching rows at both walls
    assert sh.label_phase(phi)[0] == 2 and pe.label_phase(phi)[0] == 1
    # four-roller box entirely in the phase: the rollers' solid nodes are
    # excluded and the fluid around them is one component
    fr = orc.Oracle(0, orc.FOUR_ROLLER, 32, 32, 1)
    solid = fr.solid_mask()
    count, lab = fr.label_phase(np.ones((1, 32, 32)))
    assert count == 1 and np.all(lab[solid] == -1) and np.all(lab[~solid] == 0)
