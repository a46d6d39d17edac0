"""End-to-end pins for the oracle: identity invariants and recovery of a
known translation (the behaviour the method must have, Section 2)."""
import numpy as np
import pytest


def test_identity_is_stationary(oracle_mod):
    import synth
    F, _, _ = synth.blob_pair((16, 16, 16), seed=1)
    u = np.zeros((3,) + F.shape)
    P = oracle_mod.params()
    ev = oracle_mod.evaluate(F, F, u, P)
    assert ev["L"] == 0.0                     # cc == 1 at every voxel
    # d cc / d J vanishes analytically (2b = -a, c = 0); only rounding is left
    assert np.abs(ev["graw"]).max() < 1e-15
    st = oracle_mod.State(F, F, u, P)
    info = oracle_mod.lm_step(st)
    assert info["accepted"] == 1
    assert np.abs(st.u).max() == 0.0          # r = 0 gives a zero step
    assert st.L == 0.0


def test_translation_recovered(oracle_mod):
    # textured phantom, M(p) = F(p + t): the field should converge to -t
    from scipy import ndimage
    import synth
    rng = np.random.default_rng(3)
    n = 24
    F = ndimage.gaussian_filter(rng.standard_normal((n, n, n)), 2.0)
    F = (F - F.min()) / (F.max() - F.min())
    t = (2, -1, 1)
    shift = np.stack([np.full((n, n, n), float(c)) for c in t])
    M = synth._warp_image(F, shift)
    P = oracle_mod.params(lambda0=0.006, step=1.0, sigma_warp=1.0,
                          lambda_max=0.1)
    st = oracle_mod.State(F, M, np.zeros((3, n, n, n)), P)
    L0 = st.L
    for _ in range(200):
        oracle_mod.lm_step(st)
    c = st.u[:, 8:16, 8:16, 8:16].reshape(3, -1)
    err_mean = np.abs(c.mean(1) + np.array(t)).max()
    err_max = np.abs(c + np.array(t)[:, None]).max()
    assert st.L < 0.2 * L0
    assert err_mean < 0.1, c.mean(1)
    assert err_max < 0.3
