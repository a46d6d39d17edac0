"""FP64 CPU oracle for the learned warm start: a small 3-D U-Net that maps a
fixed/moving pair to a half-resolution displacement, its MSE training loss,
reverse-mode gradients and the Adam update.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU legs are the only callers; the CUDA product path never
imports this module, and this module never imports the product.

The paper has no network (the warm start is an addition on top of the LM
optimizer), so the architecture here is the project's own definition, written
out independently of the CUDA side:

  input  x0 = (F, M)                              2 ch, D x H x W
  e0 = a(c1(a(c0(x0))))                           16 ch, full res
  e1 = a(c3(a(c2(pool(e0)))))                     32 ch, 1/2
  e2 = a(c5(a(c4(pool(e1)))))                     64 ch, 1/4
  e3 = a(c7(a(c6(pool(e2)))))                    128 ch, 1/8
  d2 = a(c9(a(c8([up(e3), e2]))))                 64 ch, 1/4
  d1 = a(c11(a(c10([up(d2), e1]))))               32 ch, 1/2
  out = c12(d1)                                    3 ch, 1/2 (no activation)

c_i: 3x3x3 cross-correlation with zero padding 1 and a bias; a: leaky ReLU
with slope 0.2; pool: 2x2x2 average; up: 2x2x2 nearest-neighbour copy;
[a, b]: channel concatenation.  The output is the displacement at half
resolution in half-resolution voxels, channel order (x, y, z) like the
optimizer's fields.  The training loss is the mean squared error to a target
field; Adam (Kingma & Ba) updates FP32 master weights.

Arrays are float64 numpy arrays with shape (C, D, H, W) (x fastest); conv
weights are (Cout, Cin, 3, 3, 3) indexed [o, i, kz, ky, kx], biases (Cout,).
Every function is the plain definition: explicit sums over the 27 taps, no
blocking or fusion.  bf16_round() gives the bfloat16 value of a number, for
comparisons with tensors a network stores in that format.
"""
from __future__ import annotations

import numpy as np

SLOPE = 0.2
# (cin, cout, leaky ReLU after it) of c0 .. c12
LAYERS = [(2, 16, True), (16, 16, True),
          (16, 32, True), (32, 32, True),
          (32, 64, True), (64, 64, True),
          (64, 128, True), (128, 128, True),
          (192, 64, True), (64, 64, True),
          (96, 32, True), (32, 32, True),
          (32, 3, False)]


def bf16_round(x):
    """x rounded to the nearest bfloat16 (ties to even), via FP32, returned
    as float64 (finite inputs)."""
    f = np.ascontiguousarray(np.asarray(x, np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3d(x, w, b=None):
    """y[o, p] = b[o] + sum_{i, t} w[o, i, t] x[i, p + t - 1], zero outside."""
    ci, D, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    y = np.zeros((w.shape[0], D, H, W))
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                y += np.einsum("oi,idhw->odhw", w[:, :, kz, ky, kx],
                               xp[:, kz:kz + D, ky:ky + H, kx:kx + W])
    if b is not None:
        y += b[:, None, None, None]
    return y


def conv3d_backward(x, w, dy):
    """Gradients of sum(dy * conv3d(x, w, b)) with respect to x, w and b."""
    ci, D, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                dxp[:, kz:kz + D, ky:ky + H, kx:kx + W] += np.einsum(
                    "oi,odhw->idhw", w[:, :, kz, ky, kx], dy)
                dw[:, :, kz, ky, kx] = np.einsum(
                    "odhw,idhw->oi", dy, xp[:, kz:kz + D, ky:ky + H, kx:kx + W])
    return dxp[:, 1:-1, 1:-1, 1:-1], dw, dy.sum(axis=(1, 2, 3))


def leaky_relu(x):
    return np.where(x > 0, x, SLOPE * x)


def leaky_relu_backward(x, dy):
    """dy * a'(x), with a'(0) taken as the slope (x = pre-activation)."""
    return dy * np.where(x > 0, 1.0, SLOPE)


def pool(x):
    c, D, H, W = x.shape
    return x.reshape(c, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 1), 2, 2), 2, 3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def up_backward(dy):
    c, D, H, W = dy.shape
    return dy.reshape(c, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


def forward(params, F, M, keep=False):
    """Network output (3, D/2, H/2, W/2) for images F, M (D, H, W divisible
    by 8).  params: list of (w, b) for c0 .. c12.  With keep=True also
    returns the tape needed by backward()."""
    tape = {}

    def conv(name, i, x):
        w, b = params[i]
        z = conv3d(x, w, b)
        tape[name] = (i, x, z)
        return leaky_relu(z) if LAYERS[i][2] else z

    x0 = np.stack([np.asarray(F, np.float64), np.asarray(M, np.float64)])
    e0 = conv("c1", 1, conv("c0", 0, x0))
    e1 = conv("c3", 3, conv("c2", 2, pool(e0)))
    e2 = conv("c5", 5, conv("c4", 4, pool(e1)))
    e3 = conv("c7", 7, conv("c6", 6, pool(e2)))
    d2 = conv("c9", 9, conv("c8", 8, np.concatenate([up(e3), e2])))
    d1 = conv("c11", 11, conv("c10", 10, np.concatenate([up(d2), e1])))
    out = conv("c12", 12, d1)
    return (out, tape) if keep else out


def backward(params, tape, dout):
    """Gradients [(dw, db)] of sum(dout * forward(...)) for c0 .. c12."""
    grads = [None] * len(LAYERS)

    def conv_back(name, dy):
        i, x, z = tape[name]
        if LAYERS[i][2]:
            dy = leaky_relu_backward(z, dy)
        dx, dw, db = conv3d_backward(x, params[i][0], dy)
        grads[i] = (dw, db)
        return dx

    dd1 = conv_back("c12", dout)
    dd1 = conv_back("c10", conv_back("c11", dd1))      # wrt [up(d2), e1]
    n2 = LAYERS[9][1]                                   # channels of d2
    dd2 = up_backward(dd1[:n2])
    de1 = dd1[n2:]
    dd2 = conv_back("c8", conv_back("c9", dd2))        # wrt [up(e3), e2]
    n3 = LAYERS[7][1]                                   # channels of e3
    de3 = up_backward(dd2[:n3])
    de2 = dd2[n3:]
    dp2 = conv_back("c6", conv_back("c7", de3))
    de2 = de2 + pool_backward(dp2)
    dp1 = conv_back("c4", conv_back("c5", de2))
    de1 = de1 + pool_backward(dp1)
    dp0 = conv_back("c2", conv_back("c3", de1))
    de0 = pool_backward(dp0)
    conv_back("c0", conv_back("c1", de0))
    return grads


def mse(pred, target):
    """Mean squared error and its gradient with respect to pred."""
    d = np.asarray(pred, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step at step count t >= 1; returns (p, m, v) updated."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def train_step(params, state, batch, lr, t):
    """One Adam step on the mean of the per-pair MSE losses of a batch of
    (F, M, target) triples.  state: list of (mw, vw, mb, vb) per layer.
    Returns (mean loss, new params, new state)."""
    acc = None
    total = 0.0
    for F, M, tgt in batch:
        out, tape = forward(params, F, M, keep=True)
        L, dout = mse(out, tgt)
        total += L
        g = backward(params, tape, dout / len(batch))
        acc = g if acc is None else [(a[0] + b[0], a[1] + b[1])
                                     for a, b in zip(acc, g)]
    new_p, new_s = [], []
    for (w, b), (dw, db), (mw, vw, mb, vb) in zip(params, acc, state):
        w2, mw, vw = adam(w, dw, mw, vw, t, lr)
        b2, mb, vb = adam(b, db, mb, vb, t, lr)
        new_p.append((w2, b2))
        new_s.append((mw, vw, mb, vb))
    return total / len(batch), new_p, new_s
