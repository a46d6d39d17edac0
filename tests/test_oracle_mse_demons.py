"""Pins for the oracle's MSE loss (Section 2.2) and its Demons special case
(Section 2.3, Eq. demons).

MSE: the closed form at the identity, the gradient against central
finite differences of the loss, and the smoothing of the raw gradient.
Demons: Eq. demons against an explicit damped 3x3 solve of
(n n^T + alpha^2 r^2 I) du = r n (the Sherman-Morrison derivation of the
paper), the bound |du| <= 1 / (2 alpha) (AM-GM), zero residual and zero
image gradient, the trial field as Eq. compositive of step * g, and the
iteration keeping every step with lambda untouched.
"""
import numpy as np
import pytest
from scipy import ndimage


def _pair(seed=0, shape=(8, 9, 10)):
    rng = np.random.default_rng(seed)
    F = ndimage.gaussian_filter(rng.random(shape), 1.0)
    M = ndimage.gaussian_filter(rng.random(shape), 1.0)
    return F, M


def _cell_field(rng, shape):
    # displacements inside cells (no corner crossings under +-1e-6)
    return (rng.integers(-1, 2, (3,) + shape)
            + rng.uniform(0.2, 0.8, (3,) + shape)).astype(float)


def test_mse_at_identity_is_the_mean_square(oracle_mod):
    F, M = _pair(1)
    P = oracle_mod.params(loss=oracle_mod.MSE)
    ev = oracle_mod.evaluate(F, M, np.zeros((3,) + F.shape), P)
    assert ev["L"] == pytest.approx(np.mean((F - M) ** 2), rel=1e-13)
    np.testing.assert_allclose(ev["cc"], (F - M) ** 2, rtol=1e-13)
    np.testing.assert_allclose(ev["dLdJ"], -2 * (F - M) / F.size, rtol=1e-13)


def test_mse_gradient_matches_finite_difference(oracle_mod):
    rng = np.random.default_rng(2)
    F, M = _pair(2, (6, 7, 8))
    u = _cell_field(rng, F.shape)
    P = oracle_mod.params(loss=oracle_mod.MSE, sigma_grad=0.0)
    ev = oracle_mod.evaluate(F, M, u, P)
    h = 1e-6
    for idx in [(1, 2, 3), (4, 5, 6), (0, 6, 0), (5, 0, 7)]:
        for i in range(3):
            up, um = u.copy(), u.copy()
            up[(i,) + idx] += h
            um[(i,) + idx] -= h
            fd = (oracle_mod.loss(F, M, up, P)
                  - oracle_mod.loss(F, M, um, P)) / (2 * h)
            assert ev["graw"][(i,) + idx] == pytest.approx(fd, rel=1e-5,
                                                          abs=1e-12)


def test_mse_smoothed_gradient(oracle_mod):
    rng = np.random.default_rng(3)
    F, M = _pair(3)
    u = rng.uniform(-1, 1, (3,) + F.shape)
    P = oracle_mod.params(loss=oracle_mod.MSE, sigma_grad=1.0)
    ev = oracle_mod.evaluate(F, M, u, P)
    for i in range(3):
        np.testing.assert_allclose(ev["g"][i],
                                   oracle_mod.smooth(ev["graw"][i], 1.0),
                                   rtol=1e-12, atol=1e-18)
    n = np.sqrt((ev["g"] ** 2).sum(0)).max()
    assert ev["gmax"] == pytest.approx(n, rel=1e-14)


@pytest.mark.parametrize("alpha", [0.25, 1.0, 3.0])
def test_demons_force_is_the_damped_solve(oracle_mod, alpha):
    rng = np.random.default_rng(4)
    F, M = _pair(4)
    u = rng.uniform(-1.5, 1.5, (3,) + F.shape)
    du = oracle_mod.demons_force(F, M, u, alpha)
    J, dJ = oracle_mod.sample(M, u)
    r = F - J
    for idx in [(0, 0, 0), (3, 4, 5), (7, 8, 9), (2, 6, 1), (5, 1, 8)]:
        n = dJ[(slice(None),) + idx]
        rr = r[idx]
        A = np.outer(n, n) + alpha ** 2 * rr ** 2 * np.eye(3)
        want = np.linalg.solve(A, rr * n)
        np.testing.assert_allclose(du[(slice(None),) + idx], want,
                                   rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("alpha", [0.5, 1.0, 2.0])
def test_demons_step_length_bound(oracle_mod, alpha):
    rng = np.random.default_rng(5)
    F, M = _pair(5, (10, 10, 10))
    M = 3.0 * M     # larger residuals than gradients in places
    du = oracle_mod.demons_force(F, M, rng.uniform(-2, 2, (3,) + F.shape),
                                 alpha)
    norm = np.sqrt((du ** 2).sum(0))
    assert norm.max() <= 1.0 / (2 * alpha) * (1 + 1e-12)
    assert norm.max() > 0.5 / (2 * alpha)   # the bound is approached


def test_demons_zero_residual_or_gradient(oracle_mod):
    F, _ = _pair(6)
    z = np.zeros((3,) + F.shape)
    assert not oracle_mod.demons_force(F, F, z, 1.0).any()
    # constant moving image: n = 0 inside, the update vanishes there
    C = np.full(F.shape, 0.3)
    du = oracle_mod.demons_force(F, C, z, 1.0)
    assert not du[:, 1:-1, 1:-1, 1:-1].any()


def test_demons_iteration_keeps_every_step(oracle_mod):
    rng = np.random.default_rng(7)
    F, M = _pair(7, (10, 11, 12))
    P = oracle_mod.params(method=oracle_mod.DEMONS, loss=oracle_mod.MSE,
                          alpha=1.0, step=1.0, sigma_grad=1.0,
                          lambda0=0.25)
    u0 = 0.3 * rng.uniform(-1, 1, (3,) + F.shape)
    st = oracle_mod.State(F, M, u0, P)
    ev0 = oracle_mod.demons_evaluate(F, M, u0, P)
    assert st.L == pytest.approx(ev0["L"], rel=1e-15)
    g0 = st.g.copy()
    for _ in range(3):
        u_prev, g_prev = st.u.copy(), st.g.copy()
        info = oracle_mod.lm_step(st)
        assert info["accepted"] == 1 and info["evals"] == 1
        assert st.lam == 0.25
        np.testing.assert_allclose(st.u, oracle_mod.compose(u_prev, g_prev),
                                   rtol=1e-12, atol=1e-15)
    # the smoothed update is Eq. demons smoothed by sigma_grad
    want = np.stack([oracle_mod.smooth(c, 1.0) for c in
                     oracle_mod.demons_force(F, M, u0, 1.0)])
    np.testing.assert_allclose(g0, want, rtol=1e-12, atol=1e-18)


def test_demons_reduces_mse_on_a_blob_pair(oracle_mod):
    import synth
    F, M, _ = synth.blob_pair((16, 16, 16), seed=1, max_disp=1.5)
    P = oracle_mod.params(method=oracle_mod.DEMONS, loss=oracle_mod.MSE,
                          alpha=1.0, step=1.0, sigma_grad=1.0)
    st = oracle_mod.State(F, M, np.zeros((3,) + F.shape), P)
    L0 = st.L
    for _ in range(10):
        oracle_mod.lm_step(st)
    assert st.L < 0.5 * L0


def test_mse_lm_reduces_loss_and_follows_the_damping_rule(oracle_mod):
    import synth
    F, M, _ = synth.blob_pair((16, 16, 16), seed=2, max_disp=1.5)
    P = oracle_mod.params(loss=oracle_mod.MSE, lambda0=0.1, step=1.0)
    st = oracle_mod.State(F, M, np.zeros((3,) + F.shape), P)
    L0 = st.L
    for _ in range(8):
        Lt, lam = st.L, st.lam
        oracle_mod.lm_step(st)
        assert st.lam == pytest.approx(lam * (1.5 if st.L > Lt else 0.975),
                                       rel=1e-15)
    assert st.L < 0.8 * L0
