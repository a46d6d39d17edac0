"""Pins for the oracle's LNCC statistics and loss gradient (step (b),
Section 2.2 squared-loss form, and Appendix A's use of the loss gradient as
the Jacobian).

Checked against: a brute-force window loop, scipy's uniform_filter, numpy's
biased covariance on interior windows, invariants (affine intensity maps
give cc = 1, cc <= 1 by Cauchy-Schwarz), and central finite differences of
the loss with respect to J and to u."""
import numpy as np
import pytest
from scipy import ndimage


def test_box_matches_brute_force_and_scipy(oracle_mod):
    rng = np.random.default_rng(0)
    X = rng.random((6, 7, 8))
    for k in (3, 5):
        S = oracle_mod.box(X, k)
        w = k // 2
        P = np.pad(X, w)
        brute = np.zeros_like(X)
        for z in range(6):
            for y in range(7):
                for x in range(8):
                    brute[z, y, x] = P[z:z + k, y:y + k, x:x + k].sum() / k ** 3
        np.testing.assert_allclose(S, brute, rtol=0, atol=1e-14)
        lib = ndimage.uniform_filter(X, size=k, mode="constant", cval=0.0)
        np.testing.assert_allclose(S, lib, rtol=0, atol=1e-13)


def test_box_of_constant_is_inside_fraction(oracle_mod):
    X = np.full((5, 5, 5), 2.0)
    S = oracle_mod.box(X, 5)
    # corner voxel: 3 x 3 x 3 of the 125 window cells are inside
    assert S[0, 0, 0] == pytest.approx(2.0 * 27 / 125, abs=1e-15)
    assert S[2, 2, 2] == pytest.approx(2.0, abs=1e-15)


def test_interior_cc_matches_numpy_covariance(oracle_mod):
    rng = np.random.default_rng(1)
    F = rng.random((9, 9, 9))
    J = 0.5 * F + 0.3 * rng.random((9, 9, 9))
    eps = 1e-5
    cc, _, _, _ = oracle_mod.lncc_terms(F, J, 5, eps, eps)
    for (z, y, x) in [(2, 2, 2), (4, 5, 3), (6, 6, 6), (3, 4, 5)]:
        wf = F[z - 2:z + 3, y - 2:y + 3, x - 2:x + 3].ravel()
        wj = J[z - 2:z + 3, y - 2:y + 3, x - 2:x + 3].ravel()
        cov = np.cov(np.stack([wf, wj]), bias=True)
        want = (cov[0, 1] ** 2 + eps) / (cov[0, 0] * cov[1, 1] + eps)
        assert cc[z, y, x] == pytest.approx(want, rel=1e-12)


def test_affine_intensity_map_gives_unit_cc(oracle_mod):
    rng = np.random.default_rng(2)
    F = rng.random((8, 8, 8))
    cc, _, _, _ = oracle_mod.lncc_terms(F, 2.5 * F, 5, 1e-5, 1e-5)
    np.testing.assert_allclose(cc, 1.0, rtol=0, atol=1e-12)
    cc, _, _, _ = oracle_mod.lncc_terms(F, -0.5 * F + 0.2, 5, 1e-5, 1e-5)
    inner = (slice(2, 6),) * 3   # zero padding breaks the offset at borders
    np.testing.assert_allclose(cc[inner], 1.0, rtol=0, atol=1e-12)


def test_cc_bounded_by_one(oracle_mod):
    rng = np.random.default_rng(3)
    F, J = rng.random((7, 7, 7)), rng.random((7, 7, 7))
    cc, _, _, _ = oracle_mod.lncc_terms(F, J, 5, 1e-5, 1e-5)
    assert cc.max() <= 1.0 + 1e-12
    assert cc.min() >= 0.0


def _loss_at_identity(oracle_mod, F, M, P):
    return oracle_mod.loss(F, M, np.zeros((3,) + F.shape), P)


@pytest.mark.parametrize("k", [3, 5])
def test_dLdJ_matches_finite_difference(oracle_mod, k):
    # at u = 0, J = M exactly, so d L / d M(y) = d L / d J(y)
    rng = np.random.default_rng(4)
    shape = (6, 7, 8)
    F = rng.random(shape)
    M = 0.6 * F + 0.4 * rng.random(shape)
    P = oracle_mod.params(win=k, sigma_grad=0.0)
    ev = oracle_mod.evaluate(F, M, np.zeros((3,) + shape), P)
    h = 1e-5
    picks = [(0, 0, 0), (2, 3, 4), (5, 6, 7), (1, 6, 2), (3, 0, 7)]
    for idx in picks:
        Mp, Mm = M.copy(), M.copy()
        Mp[idx] += h
        Mm[idx] -= h
        fd = (_loss_at_identity(oracle_mod, F, Mp, P)
              - _loss_at_identity(oracle_mod, F, Mm, P)) / (2 * h)
        assert ev["dLdJ"][idx] == pytest.approx(fd, rel=1e-6, abs=1e-13)


def test_loss_gradient_wrt_u_matches_finite_difference(oracle_mod):
    rng = np.random.default_rng(5)
    shape = (6, 7, 8)
    F = ndimage.gaussian_filter(rng.random(shape), 1.0)
    M = ndimage.gaussian_filter(rng.random(shape), 1.0)
    u = (rng.integers(-1, 2, (3,) + shape)
         + rng.uniform(0.2, 0.8, (3,) + shape)).astype(float)
    P = oracle_mod.params(sigma_grad=0.0)
    ev = oracle_mod.evaluate(F, M, u, P)
    h = 1e-6
    for idx in [(1, 2, 3), (4, 5, 6), (0, 6, 0), (5, 0, 7)]:
        for i in range(3):
            up, um = u.copy(), u.copy()
            up[(i,) + idx] += h
            um[(i,) + idx] -= h
            fd = (oracle_mod.loss(F, M, up, P) - oracle_mod.loss(F, M, um, P)) / (2 * h)
            assert ev["graw"][(i,) + idx] == pytest.approx(fd, rel=1e-5, abs=1e-12)


def test_smoothed_gradient_is_smoothed_raw_gradient(oracle_mod):
    rng = np.random.default_rng(6)
    shape = (6, 7, 8)
    F, M = rng.random(shape), rng.random(shape)
    u = rng.uniform(-1, 1, (3,) + shape)
    P = oracle_mod.params(sigma_grad=1.0)
    ev = oracle_mod.evaluate(F, M, u, P)
    t = oracle_mod.gauss_taps(1.0)
    k3 = t[:, None, None] * t[None, :, None] * t[None, None, :]
    for i in range(3):
        want = ndimage.convolve(ev["graw"][i], k3, mode="constant", cval=0.0)
        np.testing.assert_allclose(ev["g"][i], want, rtol=1e-12, atol=1e-20)
    nrm = np.sqrt((ev["g"] ** 2).sum(0)).max()
    assert ev["gmax"] == pytest.approx(nrm, rel=1e-15)


def test_clamp_slope_keeps_b_continuous(oracle_mod):
    # Reading: max(C, 0) only guards against rounding, so b is the same
    # expression on both sides of C = 0 and a constant J window gives the
    # limit of nearly constant windows.
    rng = np.random.default_rng(7)
    F = rng.random((7, 7, 7))
    J0 = np.full((7, 7, 7), 0.625)
    J1 = J0 + 1e-9 * rng.standard_normal((7, 7, 7))
    _, _, b0, _ = oracle_mod.lncc_terms(F, J0, 5, 1e-5, 1e-5)
    _, _, b1, _ = oracle_mod.lncc_terms(F, J1, 5, 1e-5, 1e-5)
    inner = (slice(2, 5),) * 3
    np.testing.assert_allclose(b0[inner], b1[inner], rtol=1e-6)
    assert np.all(b0[inner] < 0)
