"""Pins for the oracle's factored LM step, compositive update and smoothing.

Eq. tile1 against an explicit damped 3x3 solve (Appendix A, Sherman-Morrison);
its Gauss-Newton and gradient-descent limits (Section 2.2, classical LM);
Eq. compositive against scipy's clamp-to-edge trilinear interpolation and
closed forms; Gaussian taps and filters against brute-force convolution."""
import numpy as np
import pytest
from scipy import ndimage


def _field(rng, shape, lo=-1.0, hi=1.0):
    return rng.uniform(lo, hi, (3,) + shape)


@pytest.mark.parametrize("lam", [1e-6, 1e-3, 0.006, 1.0, 1e3])
def test_step_equals_explicit_damped_solve(oracle_mod, lam):
    rng = np.random.default_rng(0)
    shape = (3, 4, 5)
    g = rng.normal(0, 1, (3,) + shape)
    u = np.zeros((3,) + shape)
    gmax = np.sqrt((g ** 2).sum(0)).max()
    r = 0.37
    P = oracle_mod.params(step=1.0)
    _, du = oracle_mod.trial(u, g, gmax, r, lam, P)
    gh = g / gmax
    for z in range(shape[0]):
        for y in range(shape[1]):
            for x in range(shape[2]):
                v = gh[:, z, y, x]
                A = np.outer(v, v) + lam * np.eye(3)
                want = np.linalg.solve(A, -r * v)
                # LAPACK's solve loses ~cond(A) = (|v|^2 + lam) / lam digits
                rtol = max(1e-11, 1e-15 * (1.0 + 1.0 / lam))
                np.testing.assert_allclose(du[:, z, y, x], want, rtol=rtol,
                                           atol=1e-14)


def test_step_limits(oracle_mod):
    rng = np.random.default_rng(1)
    shape = (2, 3, 4)
    g = rng.normal(0, 1, (3,) + shape)
    gmax = np.sqrt((g ** 2).sum(0)).max()
    gh = g / gmax
    n2 = (gh ** 2).sum(0)
    r = 0.5
    P = oracle_mod.params(step=1.0)
    u = np.zeros((3,) + shape)
    _, du_gn = oracle_mod.trial(u, g, gmax, r, 1e-12, P)
    np.testing.assert_allclose(du_gn, -r * gh / n2, rtol=1e-9)
    _, du_gd = oracle_mod.trial(u, g, gmax, r, 1e9, P)
    np.testing.assert_allclose(du_gd, -r * gh / 1e9, rtol=1e-8)


def test_zero_gradient_gives_zero_step(oracle_mod):
    shape = (3, 3, 3)
    u = np.random.default_rng(2).uniform(-1, 1, (3,) + shape)
    P = oracle_mod.params()
    out, du = oracle_mod.trial(u, np.zeros_like(u), 0.0, 0.5, 0.1, P)
    assert not du.any()
    np.testing.assert_array_equal(out, u)


def test_compose_closed_forms(oracle_mod):
    rng = np.random.default_rng(3)
    shape = (5, 6, 7)
    u, v = _field(rng, shape), _field(rng, shape)
    np.testing.assert_array_equal(oracle_mod.compose(u, np.zeros_like(u)), u)
    np.testing.assert_allclose(oracle_mod.compose(np.zeros_like(u), v), v,
                               atol=0)
    s = np.array([0.3, -1.2, 2.5])[:, None, None, None] * np.ones((3,) + shape)
    t = np.array([-0.7, 0.45, 1.6])[:, None, None, None] * np.ones((3,) + shape)
    np.testing.assert_allclose(oracle_mod.compose(s, t), s + t, atol=1e-14)


def test_compose_matches_scipy_clamped_trilinear(oracle_mod):
    rng = np.random.default_rng(4)
    shape = (5, 6, 7)
    u, v = _field(rng, shape), _field(rng, shape, -2.0, 2.0)
    out = oracle_mod.compose(u, v)
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float) for n in shape],
                             indexing="ij")
    coords = np.stack([zz + v[2], yy + v[1], xx + v[0]])
    for i in range(3):
        want = v[i] + ndimage.map_coordinates(u[i], coords, order=1,
                                              mode="nearest")
        np.testing.assert_allclose(out[i], want, atol=1e-12)


@pytest.mark.parametrize("sigma", [0.5, 1.0, 1.7, 2.0])
def test_gauss_taps(oracle_mod, sigma):
    t = oracle_mod.gauss_taps(sigma)
    R = int(np.ceil(3 * sigma))
    assert t.size == 2 * R + 1
    assert t.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(t, t[::-1], atol=0)
    j = np.arange(-R, R + 1)
    np.testing.assert_allclose(t / t[R], np.exp(-j * j / (2 * sigma ** 2)),
                               rtol=1e-14)


def test_gauss_zero_sigma_is_identity(oracle_mod):
    X = np.random.default_rng(5).random((4, 5, 6))
    np.testing.assert_array_equal(oracle_mod.smooth(X, 0.0), X)


def test_smooth_matches_brute_force_3d(oracle_mod):
    rng = np.random.default_rng(6)
    X = rng.random((7, 8, 9))
    t = oracle_mod.gauss_taps(1.0)
    k3 = t[:, None, None] * t[None, :, None] * t[None, None, :]
    want = ndimage.convolve(X, k3, mode="constant", cval=0.0)
    np.testing.assert_allclose(oracle_mod.smooth(X, 1.0), want, atol=1e-14)
    # edge-clamped variant used for displacement fields
    want_c = X
    for ax in range(3):
        want_c = ndimage.correlate1d(want_c, t, axis=ax, mode="nearest")
    np.testing.assert_allclose(oracle_mod.smooth(X, 1.0, clamp=True), want_c,
                               atol=1e-14)


def test_smooth_preserves_constant_interior(oracle_mod):
    X = np.full((12, 12, 12), 0.7)
    Y = oracle_mod.smooth(X, 1.0)
    np.testing.assert_allclose(Y[3:9, 3:9, 3:9], 0.7, atol=1e-15)
    np.testing.assert_allclose(oracle_mod.smooth(X, 1.0, clamp=True), 0.7,
                               atol=1e-15)


def test_warp_smoothing_applied_after_compose(oracle_mod):
    rng = np.random.default_rng(7)
    shape = (6, 6, 6)
    u = _field(rng, shape)
    g = rng.normal(0, 1, (3,) + shape)
    gmax = np.sqrt((g ** 2).sum(0)).max()
    P0 = oracle_mod.params(sigma_warp=0.0)
    P1 = oracle_mod.params(sigma_warp=1.0)
    raw, _ = oracle_mod.trial(u, g, gmax, 0.3, 0.1, P0)
    sm, _ = oracle_mod.trial(u, g, gmax, 0.3, 0.1, P1)
    np.testing.assert_allclose(sm, oracle_mod.smooth(raw, 1.0, clamp=True),
                               atol=1e-14)
