"""Pins of the U-Net oracle (oracle/unet.py) against facts other than
itself: SciPy's n-D correlation, the adjoint (dot-product) identity, central
finite differences of the training loss, Adam's closed form under a
constant gradient, and torch's float32 -> bfloat16 conversion."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet as U


def _rng(s):
    return np.random.default_rng(s)


def test_conv3d_matches_scipy_correlate():
    r = _rng(1)
    x = r.standard_normal((3, 5, 6, 7))
    w = r.standard_normal((2, 3, 3, 3, 3))
    b = r.standard_normal(2)
    y = U.conv3d(x, w, b)
    for o in range(2):
        ref = sum(ndimage.correlate(x[i], w[o, i], mode="constant", cval=0.0)
                  for i in range(3)) + b[o]
        np.testing.assert_allclose(y[o], ref, rtol=1e-12, atol=1e-12)


def test_conv3d_backward_adjoint_and_weight_linearity():
    r = _rng(2)
    x = r.standard_normal((4, 4, 5, 6))
    w = r.standard_normal((3, 4, 3, 3, 3))
    dy = r.standard_normal((3, 4, 5, 6))
    dx, dw, db = U.conv3d_backward(x, w, dy)
    # <conv(x), dy> = <x, dx> (the data gradient is the adjoint)
    np.testing.assert_allclose(np.sum(U.conv3d(x, w) * dy), np.sum(x * dx),
                               rtol=1e-12)
    # the output is linear in w: <conv(x, e), dy> = dw . e for any e
    e = r.standard_normal(w.shape)
    np.testing.assert_allclose(np.sum(U.conv3d(x, e) * dy), np.sum(dw * e),
                               rtol=1e-12)
    np.testing.assert_allclose(db, dy.sum(axis=(1, 2, 3)), rtol=1e-12)


def test_pool_up_adjoints_and_leaky_relu():
    r = _rng(3)
    x = r.standard_normal((2, 4, 6, 8))
    y = r.standard_normal((2, 2, 3, 4))
    np.testing.assert_allclose(np.sum(U.pool(x) * y),
                               np.sum(x * U.pool_backward(y)), rtol=1e-12)
    np.testing.assert_allclose(np.sum(U.up(y) * x),
                               np.sum(y * U.up_backward(x)), rtol=1e-12)
    assert U.pool(np.ones((1, 4, 4, 4))).tolist() == np.ones((1, 2, 2, 2)).tolist()
    z = np.array([-2.0, -0.5, 0.0, 0.5, 3.0])
    np.testing.assert_array_equal(U.leaky_relu(z), [-0.4, -0.1, 0.0, 0.5, 3.0])
    np.testing.assert_array_equal(U.leaky_relu_backward(z, np.ones(5)),
                                  [0.2, 0.2, 0.2, 1.0, 1.0])


def _small_params(seed):
    """Oracle-shaped random parameters with non-zero biases."""
    r = _rng(seed)
    ps = []
    for cin, cout, _ in U.LAYERS:
        w = r.standard_normal((cout, cin, 3, 3, 3)) * np.sqrt(1.0 / (27 * cin))
        ps.append((w, 0.1 * r.standard_normal(cout)))
    return ps


def test_network_shapes_and_zero_weights():
    F = _rng(4).random((8, 8, 16))
    M = _rng(5).random((8, 8, 16))
    ps = _small_params(6)
    out = U.forward(ps, F, M)
    assert out.shape == (3, 4, 4, 8)
    # all-zero weights: the output is the head's bias everywhere
    zs = [(np.zeros_like(w), b) for w, b in ps]
    out0 = U.forward(zs, F, M)
    for c in range(3):
        np.testing.assert_allclose(out0[c], ps[-1][1][c], rtol=0, atol=0)


@pytest.mark.parametrize("layer", [0, 5, 8, 10, 12])
def test_network_gradient_matches_finite_differences(layer):
    F = _rng(7).random((8, 8, 8))
    M = _rng(8).random((8, 8, 8))
    tgt = _rng(9).standard_normal((3, 4, 4, 4))
    ps = _small_params(10)
    out, tape = U.forward(ps, F, M, keep=True)
    L, dout = U.mse(out, tgt)
    grads = U.backward(ps, tape, dout)
    r = _rng(11 + layer)
    w, b = ps[layer]
    h = 1e-5
    for _ in range(4):
        idx = tuple(int(r.integers(0, n)) for n in w.shape)
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        pp = list(ps)
        pp[layer] = (wp, b)
        Lp = U.mse(U.forward(pp, F, M), tgt)[0]
        pp[layer] = (wm, b)
        Lm = U.mse(U.forward(pp, F, M), tgt)[0]
        fd = (Lp - Lm) / (2 * h)
        an = grads[layer][0][idx]
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (idx, fd, an)
    j = int(r.integers(0, b.shape[0]))
    bp, bm = b.copy(), b.copy()
    bp[j] += h
    bm[j] -= h
    pp = list(ps)
    pp[layer] = (w, bp)
    Lp = U.mse(U.forward(pp, F, M), tgt)[0]
    pp[layer] = (w, bm)
    Lm = U.mse(U.forward(pp, F, M), tgt)[0]
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - grads[layer][1][j]) <= 1e-6 * max(abs(fd), 1e-3)


def test_adam_constant_gradient_closed_form():
    # with a constant gradient g, m_hat = g and v_hat = g^2 at every step,
    # so each step moves p by -lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3])
    p0 = np.array([1.0, 2.0, 3.0])
    p, m, v = p0.copy(), np.zeros(3), np.zeros(3)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 8):
        p, m, v = U.adam(p, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + eps),
                                   rtol=1e-12, atol=1e-15)


def test_train_step_lowers_the_loss():
    F = _rng(12).random((8, 8, 8))
    M = _rng(13).random((8, 8, 8))
    tgt = 0.5 * _rng(14).standard_normal((3, 4, 4, 4))
    ps = _small_params(15)
    st = [(np.zeros_like(w), np.zeros_like(w), np.zeros_like(b),
           np.zeros_like(b)) for w, b in ps]
    L0 = U.mse(U.forward(ps, F, M), tgt)[0]
    for t in range(1, 6):
        _, ps, st = U.train_step(ps, st, [(F, M, tgt)], 1e-3, t)
    assert U.mse(U.forward(ps, F, M), tgt)[0] < L0


def test_bf16_round_matches_torch():
    # bf16_round against torch's own float32 -> bfloat16 conversion (round
    # to nearest even), exact ties with even and odd kept bits included
    torch = pytest.importorskip("torch")
    r = _rng(20)
    x = (r.standard_normal(4000) * 10.0 ** r.integers(-30, 30, 4000)).astype(np.float32)
    hi = r.integers(0, 0x7F7F, 2000).astype(np.uint32) << 16
    ties = (hi | np.uint32(0x8000)).view(np.float32)
    x = np.concatenate([x, ties, -ties, np.float32([0.0, -0.0, 1.0, 3.0e38])])
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy().astype(np.float64)
    got = U.bf16_round(x)
    assert np.array_equal(got, ref)
    assert np.array_equal(U.bf16_round(got), got)   # idempotent
