"""Pins for the oracle's pooled-curvature step, Eq. tilen (Section 2.2; tile
side k swept in Section 3).

Readings under test: non-overlapping k^3 tiles aligned at the grid origin
(the last tile of an axis cut at the volume edge) and the mean of
ghat ghat^T over a tile.  Pinned against:
  - k = 1: the closed form of Eq. tile1 (Sherman-Morrison, Appendix A);
  - tiles whose voxels share one ghat: the mean is that rank-1 matrix, so
    every voxel again takes the Eq. tile1 step;
  - brute force: per-tile numpy outer-product means and numpy's LAPACK
    solve, on ragged shapes;
  - a tile covering the whole volume: H is the global second moment;
  - the Gauss-Newton and gradient-descent limits of the damped system;
  - the trial field: Eq. compositive applied to step * du.
"""
import numpy as np
import pytest


def _ghat(rng, shape):
    g = rng.normal(0, 1, (3,) + shape)
    return g / np.sqrt((g ** 2).sum(0)).max()


def _brute(gh, k, r, lam):
    """Per tile: mean of outer products; per voxel: LAPACK solve."""
    _, nz, ny, nx = gh.shape
    du = np.empty_like(gh)
    for tz in range(0, nz, k):
        for ty in range(0, ny, k):
            for tx in range(0, nx, k):
                blk = gh[:, tz:tz + k, ty:ty + k, tx:tx + k].reshape(3, -1)
                H = blk @ blk.T / blk.shape[1]
                A = H + lam * np.eye(3)
                sol = np.linalg.solve(A, -r * blk)
                du[:, tz:tz + k, ty:ty + k, tx:tx + k] = sol.reshape(
                    (3,) + gh[:, tz:tz + k, ty:ty + k, tx:tx + k].shape[1:])
    return du


@pytest.mark.parametrize("lam", [1e-4, 0.006, 1.0])
def test_k1_is_eq_tile1(oracle_mod, lam):
    gh = _ghat(np.random.default_rng(0), (4, 5, 6))
    r = 0.42
    du = oracle_mod.tile_du(gh, 1, r, lam)
    want = -r * gh / ((gh ** 2).sum(0) + lam)
    np.testing.assert_allclose(du, want, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("k", [2, 3])
def test_constant_tiles_reduce_to_eq_tile1(oracle_mod, k):
    rng = np.random.default_rng(1)
    shape = (2 * k, 3 * k, 2 * k)
    base = _ghat(rng, (2, 3, 2))
    gh = np.repeat(np.repeat(np.repeat(base, k, 1), k, 2), k, 3)
    r, lam = 0.3, 0.01
    du = oracle_mod.tile_du(gh, k, r, lam)
    want = -r * gh / ((gh ** 2).sum(0) + lam)
    np.testing.assert_allclose(du, want, rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("k,shape", [(2, (5, 7, 4)), (3, (7, 5, 8)),
                                     (4, (4, 9, 6)), (10, (11, 3, 12))])
@pytest.mark.parametrize("lam", [1e-3, 0.5])
def test_matches_brute_force(oracle_mod, k, shape, lam):
    gh = _ghat(np.random.default_rng(2 + k), shape)
    r = 0.61
    du = oracle_mod.tile_du(gh, k, r, lam)
    want = _brute(gh, k, r, lam)
    # both solves lose ~cond(A) <= (1 + lam) / lam digits of 1e-16
    rtol = max(1e-11, 1e-15 * (1.0 + 1.0 / lam))
    np.testing.assert_allclose(du, want, rtol=rtol, atol=1e-14)


def test_single_tile_uses_global_second_moment(oracle_mod):
    gh = _ghat(np.random.default_rng(5), (3, 4, 5))
    r, lam = 0.25, 0.02
    du = oracle_mod.tile_du(gh, 8, r, lam)
    flat = gh.reshape(3, -1)
    H = flat @ flat.T / flat.shape[1]
    want = np.linalg.solve(H + lam * np.eye(3), -r * flat).reshape(gh.shape)
    np.testing.assert_allclose(du, want, rtol=1e-10, atol=1e-15)


def test_damping_limits(oracle_mod):
    gh = _ghat(np.random.default_rng(6), (4, 4, 4))
    r = 0.5
    # gradient descent: du -> -r ghat / lam, up to |H| / lam ~ 1e-9 of the
    # step's scale r / lam
    lam = 1e9
    np.testing.assert_allclose(oracle_mod.tile_du(gh, 2, r, lam),
                               -r * gh / lam, rtol=1e-8, atol=1e-8 * r / lam)
    # Gauss-Newton on a full-rank tile: H du = -r ghat
    du = oracle_mod.tile_du(gh, 4, r, 0.0)
    flat = gh.reshape(3, -1)
    H = flat @ flat.T / flat.shape[1]
    np.testing.assert_allclose(H @ du.reshape(3, -1), -r * flat, rtol=1e-9,
                               atol=1e-12)


def test_zero_gradient_gives_zero_step(oracle_mod):
    du = oracle_mod.tile_du(np.zeros((3, 3, 4, 5)), 2, 0.5, 0.01)
    assert not du.any()


def test_trial_uses_tile_step(oracle_mod):
    rng = np.random.default_rng(7)
    shape = (5, 6, 7)
    g = rng.normal(0, 1, (3,) + shape)
    gmax = np.sqrt((g ** 2).sum(0)).max()
    u = 0.3 * rng.uniform(-1, 1, (3,) + shape)
    r, lam, step = 0.4, 0.05, 0.7
    P = oracle_mod.params(step=step, tile=3)
    out, du = oracle_mod.trial(u, g, gmax, r, lam, P)
    np.testing.assert_allclose(du, oracle_mod.tile_du(g / gmax, 3, r, lam),
                               rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(out, oracle_mod.compose(u, step * du),
                               rtol=1e-12, atol=1e-15)
    # tile = 1 keeps Eq. tile1
    _, du1 = oracle_mod.trial(u, g, gmax, r, lam, oracle_mod.params(step=step))
    gh = g / gmax
    np.testing.assert_allclose(du1, -r * gh / ((gh ** 2).sum(0) + lam),
                               rtol=1e-12)
