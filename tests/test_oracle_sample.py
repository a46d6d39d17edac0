"""Pins for the oracle's trilinear resampling (step (a), Section 2.1).

Checked against: exact lattice reads at integer displacements, exact
reproduction of affine intensity fields, scipy's trilinear interpolation with
zero padding ('grid-constant'), and central finite differences of J with
respect to u."""
import numpy as np
import pytest
from scipy import ndimage

pytestmark = pytest.mark.filterwarnings("ignore")


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_integer_displacement_reads_lattice(oracle_mod):
    rng = _rng(1)
    M = rng.random((5, 6, 7))
    u = rng.integers(-2, 3, (3, 5, 6, 7)).astype(float)
    J, _ = oracle_mod.sample(M, u)
    for z in range(5):
        for y in range(6):
            for x in range(7):
                qx, qy, qz = x + u[0, z, y, x], y + u[1, z, y, x], z + u[2, z, y, x]
                inside = 0 <= qx < 7 and 0 <= qy < 6 and 0 <= qz < 5
                want = M[int(qz), int(qy), int(qx)] if inside else 0.0
                assert J[z, y, x] == want


def test_affine_field_reproduced_exactly(oracle_mod):
    rng = _rng(2)
    n = 9
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float)] * 3, indexing="ij")
    a, b, c, d = 0.3, -0.7, 1.1, 0.25
    M = a * xx + b * yy + c * zz + d
    u = rng.uniform(-1.0, 1.0, (3, n, n, n))
    J, dJ = oracle_mod.sample(M, u)
    inner = (slice(2, n - 2),) * 3
    want = a * (xx + u[0]) + b * (yy + u[1]) + c * (zz + u[2]) + d
    np.testing.assert_allclose(J[inner], want[inner], rtol=0, atol=1e-12)
    np.testing.assert_allclose(dJ[0][inner], a, atol=1e-12)
    np.testing.assert_allclose(dJ[1][inner], b, atol=1e-12)
    np.testing.assert_allclose(dJ[2][inner], c, atol=1e-12)


def test_matches_scipy_trilinear_zero_padding(oracle_mod):
    rng = _rng(3)
    shape = (6, 7, 8)
    M = rng.random(shape)
    u = rng.uniform(-2.5, 2.5, (3,) + shape)
    J, _ = oracle_mod.sample(M, u)
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float) for n in shape],
                             indexing="ij")
    coords = np.stack([zz + u[2], yy + u[1], xx + u[0]])
    want = ndimage.map_coordinates(M, coords, order=1, mode="grid-constant",
                                   cval=0.0)
    np.testing.assert_allclose(J, want, rtol=0, atol=1e-12)


def test_gradient_matches_finite_difference(oracle_mod):
    rng = _rng(4)
    shape = (5, 6, 7)
    M = rng.random(shape)
    base = rng.integers(-1, 2, (3,) + shape).astype(float)
    u = base + rng.uniform(0.1, 0.9, (3,) + shape)   # away from cell edges
    _, dJ = oracle_mod.sample(M, u)
    h = 1e-6
    for i in range(3):
        up, um = u.copy(), u.copy()
        up[i] += h
        um[i] -= h
        fd = (oracle_mod.sample(M, up)[0] - oracle_mod.sample(M, um)[0]) / (2 * h)
        np.testing.assert_allclose(dJ[i], fd, rtol=0, atol=1e-8)


def test_far_outside_is_zero(oracle_mod):
    M = np.ones((4, 4, 4))
    u = np.full((3, 4, 4, 4), 50.0)
    J, dJ = oracle_mod.sample(M, u)
    assert not J.any() and not dJ.any()
