"""Pins for the oracle's mutual-information loss (Section 2.2: the
squared-loss form (log2 B - MI)^2 with B Parzen bins).

Readings under test: cubic B-spline Parzen windows over B bins, both images
binned over the joint range of F, M and 0, MI in bits, r = log2 B - MI.
Pinned against:
  - independence: F varying along x only and J along y only on a full grid
    give p_ij = p_i q_j exactly, so MI = 0 and r = log2 B;
  - a brute-force numpy histogram (its own B-spline weights) and MI;
  - symmetry MI(F, J) = MI(J, F) and 0 <= MI <= log2 B;
  - dMI/dJ and dL/du against central finite differences;
  - the smoothed gradient and the LM iteration reducing r.
"""
import numpy as np
import pytest
from scipy import ndimage


def _bspline3(x):
    a = np.abs(x)
    return np.where(a < 1, 2 / 3 - a ** 2 + 0.5 * a ** 3,
                    np.where(a < 2, (2 - a) ** 3 / 6, 0.0))


def _brute_mi(F, J, B, lo, hi):
    t_f = 1 + (B - 3) * (F.ravel() - lo) / (hi - lo)
    t_j = 1 + (B - 3) * (J.ravel() - lo) / (hi - lo)
    A = _bspline3(t_f[:, None] - np.arange(B)[None, :])
    W = _bspline3(t_j[:, None] - np.arange(B)[None, :])
    np.testing.assert_allclose(A.sum(1), 1.0, rtol=1e-13)   # partition of unity
    p = A.T @ W / F.size
    pi, qj = p.sum(1), p.sum(0)
    nz = p > 0
    return float((p[nz] * np.log2(p[nz] / np.outer(pi, qj)[nz])).sum())


def _pair(seed, shape=(7, 8, 9)):
    rng = np.random.default_rng(seed)
    return (ndimage.gaussian_filter(rng.random(shape), 1.0),
            ndimage.gaussian_filter(rng.random(shape), 1.0))


@pytest.mark.parametrize("B", [8, 32])
def test_independent_images_have_zero_mi(oracle_mod, B):
    shape = (5, 6, 7)
    x = np.linspace(0.1, 0.9, shape[2])
    y = np.linspace(0.2, 0.7, shape[1]) ** 2
    F = np.broadcast_to(x[None, None, :], shape).copy()
    M = np.broadcast_to(y[None, :, None], shape).copy()
    lo, hi = oracle_mod.mi_range(F, M)
    mi, _ = oracle_mod.mi(F, M, B, lo, hi)
    assert abs(mi) < 1e-12
    P = oracle_mod.params(loss=oracle_mod.MI, bins=B)
    L = oracle_mod.loss(F, M, np.zeros((3,) + shape), P)
    assert L == pytest.approx(np.log2(B), abs=1e-12)


@pytest.mark.parametrize("B", [8, 16, 64])
def test_matches_brute_force_histogram(oracle_mod, B):
    F, M = _pair(1)
    lo, hi = oracle_mod.mi_range(F, M)
    assert lo == 0.0 and hi == max(F.max(), M.max())
    mi, _ = oracle_mod.mi(F, M, B, lo, hi)
    assert mi == pytest.approx(_brute_mi(F, M, B, lo, hi), rel=1e-12)


def test_symmetry_and_bounds(oracle_mod):
    F, M = _pair(2)
    lo, hi = oracle_mod.mi_range(F, M)
    a, _ = oracle_mod.mi(F, M, 16, lo, hi)
    b, _ = oracle_mod.mi(M, F, 16, lo, hi)
    assert a == pytest.approx(b, rel=1e-13)
    self_mi, _ = oracle_mod.mi(F, F, 16, lo, hi)
    assert 0 <= a < self_mi <= np.log2(16)


def test_dmi_dj_matches_finite_difference(oracle_mod):
    F, M = _pair(3)
    lo, hi = -0.1, 1.2          # fixed binning range for the difference
    _, d = oracle_mod.mi(F, M, 16, lo, hi)
    h = 1e-6
    for idx in [(0, 0, 0), (3, 4, 5), (6, 7, 8), (2, 1, 6)]:
        Jp, Jm = M.copy(), M.copy()
        Jp[idx] += h
        Jm[idx] -= h
        fd = (oracle_mod.mi(F, Jp, 16, lo, hi)[0]
              - oracle_mod.mi(F, Jm, 16, lo, hi)[0]) / (2 * h)
        assert d[idx] == pytest.approx(fd, rel=1e-5, abs=1e-12)


def test_loss_gradient_wrt_u_matches_finite_difference(oracle_mod):
    rng = np.random.default_rng(4)
    F, M = _pair(4, (6, 7, 8))
    u = (rng.integers(-1, 2, (3,) + F.shape)
         + rng.uniform(0.2, 0.8, (3,) + F.shape)).astype(float)
    P = oracle_mod.params(loss=oracle_mod.MI, bins=12, sigma_grad=0.0)
    ev = oracle_mod.evaluate(F, M, u, P)
    h = 1e-6
    for idx in [(1, 2, 3), (4, 5, 6), (0, 6, 0)]:
        for i in range(3):
            up, um = u.copy(), u.copy()
            up[(i,) + idx] += h
            um[(i,) + idx] -= h
            fd = (oracle_mod.loss(F, M, up, P)
                  - oracle_mod.loss(F, M, um, P)) / (2 * h)
            assert ev["graw"][(i,) + idx] == pytest.approx(fd, rel=1e-4,
                                                          abs=1e-11)


def test_smoothed_gradient_and_lm_iteration(oracle_mod):
    import synth
    F, M, _ = synth.blob_pair((16, 16, 16), seed=3, max_disp=1.5)
    # r = log2 B - MI stays of order 1 at the optimum, so the LM step
    # -r ghat / (|ghat|^2 + lambda) is up to r / (2 sqrt(lambda)) voxels:
    # lambda0 = 1 and step 0.25 keep it below half a voxel
    P = oracle_mod.params(loss=oracle_mod.MI, bins=16, lambda0=1.0,
                          step=0.25)
    u0 = np.zeros((3,) + F.shape)
    ev = oracle_mod.evaluate(F, M, u0, P)
    for i in range(3):
        np.testing.assert_allclose(ev["g"][i],
                                   oracle_mod.smooth(ev["graw"][i], 1.0),
                                   rtol=1e-12, atol=1e-18)
    st = oracle_mod.State(F, M, u0, P)
    L0 = st.L
    for _ in range(6):
        oracle_mod.lm_step(st)
    assert st.L < L0
