"""Pins for the oracle's coarse-to-fine pyramid (Section 2.1: the warp is
carried from the coarser level to the finer one).  Closed forms: constants
and linear ramps are reproduced away from the border; fields are rescaled by
the factor ratio."""
import numpy as np
import pytest


def test_level_dims(oracle_mod):
    assert oracle_mod.level_dims((160, 192, 224), 4) == (40, 48, 56)
    assert oracle_mod.level_dims((67, 65, 64), 2) == (33, 32, 32)
    assert oracle_mod.level_dims((3, 1, 2), 4) == (1, 1, 1)


@pytest.mark.parametrize("f", [2, 4])
def test_downsample_linear_ramp_interior(oracle_mod, f):
    n = 48
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float)] * 3, indexing="ij")
    X = 0.01 * xx - 0.02 * yy + 0.005 * zz + 0.3
    Y = oracle_mod.downsample(X, f)
    m = n // f
    R = int(np.ceil(3 * 0.5 * f))
    lo = -(-R // f) + 1
    hi = m - lo
    q = f * np.arange(m) + 0.5 * (f - 1)
    qz, qy, qx = np.meshgrid(q, q, q, indexing="ij")
    want = 0.01 * qx - 0.02 * qy + 0.005 * qz + 0.3
    sl = (slice(lo, hi),) * 3
    np.testing.assert_allclose(Y[sl], want[sl], atol=1e-12)


def test_resample_field_constant_and_linear(oracle_mod):
    a = (5, 6, 7)
    Ua = np.stack([np.full(a, 1.0), np.full(a, -0.5), np.full(a, 0.25)])
    b = oracle_mod.level_dims((10, 12, 14), 1)
    Ub = oracle_mod.resample_field(Ua, 2, (10, 12, 14), 1)
    np.testing.assert_allclose(Ub[0], 2.0, atol=1e-15)
    np.testing.assert_allclose(Ub[1], -1.0, atol=1e-15)
    np.testing.assert_allclose(Ub[2], 0.5, atol=1e-15)
    # a field linear in the level-a coordinate is reproduced inside
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float) for n in a],
                             indexing="ij")
    Ua = np.stack([0.1 * xx, 0.2 * yy, -0.1 * zz])
    Ub = oracle_mod.resample_field(Ua, 2, (10, 12, 14), 1)
    q = [(np.arange(n) - 0.5) / 2.0 for n in (10, 12, 14)]
    qz, qy, qx = np.meshgrid(*q, indexing="ij")
    inner = (slice(1, 9), slice(1, 11), slice(1, 13))
    np.testing.assert_allclose(Ub[0][inner], 2 * 0.1 * qx[inner], atol=1e-14)
    np.testing.assert_allclose(Ub[1][inner], 2 * 0.2 * qy[inner], atol=1e-14)
    np.testing.assert_allclose(Ub[2][inner], -2 * 0.1 * qz[inner], atol=1e-14)


def test_multilevel_register_lowers_loss(oracle_mod):
    import synth
    F, M, _ = synth.blob_pair((24, 24, 24), seed=5, max_disp=2.0)
    P = oracle_mod.params(lambda0=0.006, step=1.0)
    u, log, evals = oracle_mod.register(F, M, P, [4, 2, 1], [10, 10, 5])
    L0 = oracle_mod.loss(F, M, np.zeros_like(u), P)
    L1 = oracle_mod.loss(F, M, u, P)
    assert L1 < 0.9 * L0
    assert evals >= 25 + 3


@pytest.mark.parametrize("f", [2, 4])
def test_downsample_matches_scipy(oracle_mod, f):
    """Every level voxel, borders included, against SciPy: the zero-padded
    Gaussian of sigma f/2 truncated at ceil(3 sigma) taps (scipy's radius
    int(3 sigma + 0.5) is the same for these sigmas), then trilinear reads
    with zero padding at the fine coordinate f p + (f - 1)/2."""
    from scipy import ndimage
    rng = np.random.default_rng(7)
    X = rng.random((20, 22, 24))
    Y = oracle_mod.downsample(X, f)
    B = ndimage.gaussian_filter(X, 0.5 * f, mode="constant", cval=0.0,
                                truncate=3.0)
    dims = oracle_mod.level_dims(X.shape, f)
    q = [f * np.arange(m) + 0.5 * (f - 1) for m in dims]
    coords = np.stack(np.meshgrid(*q, indexing="ij"))
    want = ndimage.map_coordinates(B, coords, order=1, mode="constant",
                                   cval=0.0)
    assert Y.shape == want.shape
    np.testing.assert_allclose(Y, want, rtol=0, atol=1e-13)
