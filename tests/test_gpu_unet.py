"""GPU parity of the learned warm start against the FP64 oracle
(oracle/unet.py).

Operands are bfloat16 on the GPU, so the oracle receives the same
bfloat16-rounded inputs and weights (promoted exactly to FP64).  Bars:

* one convolution with an FP32 output: only the FP32 accumulation order
  differs, |error| <= 2e-5 * max|y| (K <= 27 * 128 terms, each product exact
  in FP32);
* the data gradient, stored as bfloat16: one rounding, |error| <= 2^-8 of
  the largest magnitude plus the accumulation error;
* weight and bias gradients (FP32 accumulators): <= 1e-4 relative to the
  largest entry;
* the whole network, whose hidden activations and activation gradients
  are stored as bfloat16 (relative rounding 2^-9 each): relative L2 error
  <= 3e-2 on the output (12 roundings on the way, 12 * 2^-9 = 2.3%) and
  <= 0.15 on every layer's weight and bias gradient.  A layer's gradient
  is a sum of products of an activation (up to 12 roundings) and an
  activation gradient (up to 13 more), so each factor carries up to
  25 * 2^-9 = 4.9% and the product about 10%; at the 1/4 and 1/8 levels
  the sums run over only 64 and 8 voxels (16^3 input), so nothing averages
  out.  Measured: 0.1% (head) to 9% (c5).  A wrong index, tap orientation
  or transpose gives errors of order 1.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19371_gb300 import build, lmreg
    build.build()
    lmreg.load()
    return lmreg


def _bf(a):
    """numpy float -> (torch bfloat16 CUDA tensor, float64 copy of it)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)
    return t.cuda(), t.float().numpy().astype(np.float64)


def _to_cl(x):
    """(C, D, H, W) -> (D, H, W, C)"""
    return np.ascontiguousarray(np.moveaxis(x, 0, -1))


def _w_internal(w):
    """(cout, cin, 3, 3, 3) -> (cout, 27, cin) with tap = 9 kz + 3 ky + kx"""
    co, ci = w.shape[:2]
    return np.ascontiguousarray(w.reshape(co, ci, 27).transpose(0, 2, 1))


# the odd shapes take the gathering kernel; the rest (channels a multiple
# of 16, x-y planes that tile into runs of 128 voxels) the TMA-fed one:
# W = 16 / 32 / 64 (several rows per tile), 128 (one row) and 256 (half a
# row), every one with a zero-padded border on all six faces
@pytest.mark.parametrize("shape,cin,cout", [((5, 6, 7), 16, 16),
                                            ((5, 6, 7), 2, 32),
                                            ((9, 10, 11), 32, 64),
                                            ((4, 8, 12), 64, 128),
                                            ((6, 6, 6), 192, 64),
                                            ((4, 8, 16), 16, 32),
                                            ((3, 4, 32), 32, 64),
                                            ((2, 2, 64), 64, 16),
                                            ((3, 2, 128), 16, 16),
                                            ((2, 3, 256), 32, 96),
                                            ((3, 8, 16), 192, 64),
                                            ((2, 8, 16), 96, 192),
                                            ((2, 8, 16), 128, 128)])
def test_conv3d_forward_matches_oracle(P, oracle_mod, shape, cin, cout):
    import torch
    from oracle import unet as U
    r = np.random.default_rng(cin * 7 + cout)
    x = r.standard_normal((cin,) + shape)
    w = r.standard_normal((cout, cin, 3, 3, 3)) / np.sqrt(27 * cin)
    b = r.standard_normal(cout)
    xt, x64 = _bf(_to_cl(x))
    wt, w64 = _bf(_w_internal(w))
    bt = torch.from_numpy(b.astype(np.float32)).cuda()
    for act in (0, 1):
        y = torch.empty(shape + (cout,), device="cuda")
        P.lm_conv3d_forward(xt, wt, bt, act, y)
        torch.cuda.synchronize()
        w_or = w64.reshape(cout, 27, cin).transpose(0, 2, 1).reshape(cout, cin, 3, 3, 3)
        ref = U.conv3d(np.moveaxis(x64, -1, 0), w_or, b.astype(np.float32))
        if act:
            ref = U.leaky_relu(ref)
        got = np.moveaxis(y.cpu().numpy().astype(np.float64), -1, 0)
        err = np.abs(got - ref).max()
        assert err <= 2e-5 * np.abs(ref).max(), (act, err)


@pytest.mark.parametrize("shape,cin,cout", [((5, 6, 7), 16, 16),
                                            ((5, 6, 7), 2, 16),
                                            ((9, 10, 11), 32, 64),
                                            ((6, 6, 6), 192, 64),
                                            ((8, 8, 8), 96, 32),
                                            ((4, 8, 16), 32, 16),
                                            ((3, 4, 32), 64, 32)])
def test_conv3d_backward_matches_oracle(P, oracle_mod, shape, cin, cout):
    import torch
    from oracle import unet as U
    r = np.random.default_rng(cin * 11 + cout)
    x = r.standard_normal((cin,) + shape)
    w = r.standard_normal((cout, cin, 3, 3, 3)) / np.sqrt(27 * cin)
    dy = r.standard_normal((cout,) + shape)
    xt, x64 = _bf(_to_cl(x))
    wt, w64 = _bf(_w_internal(w))
    dyt, dy64 = _bf(_to_cl(dy))
    dx = torch.empty(shape + (cin,), device="cuda", dtype=torch.bfloat16) \
        if cin != 2 else None
    dw = torch.zeros((cout, 27, cin), device="cuda")
    db = torch.zeros(cout, device="cuda")
    P.lm_conv3d_backward(xt, wt, dyt, dx, dw, db)
    torch.cuda.synchronize()
    w_or = w64.reshape(cout, 27, cin).transpose(0, 2, 1).reshape(cout, cin, 3, 3, 3)
    rdx, rdw, rdb = U.conv3d_backward(np.moveaxis(x64, -1, 0), w_or,
                                      np.moveaxis(dy64, -1, 0))
    gdw = dw.cpu().numpy().astype(np.float64).transpose(0, 2, 1).reshape(rdw.shape)
    assert np.abs(gdw - rdw).max() <= 1e-4 * np.abs(rdw).max()
    assert np.abs(db.cpu().numpy() - rdb).max() <= 1e-4 * np.abs(rdb).max()
    if dx is not None:
        gdx = np.moveaxis(dx.float().cpu().numpy().astype(np.float64), -1, 0)
        assert np.abs(gdx - rdx).max() <= 2 ** -8 * np.abs(rdx).max() + 1e-6


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _net_case(seed, shape=(16, 16, 16)):
    import synth
    from oracle import unet as U
    shapes = [(ci, co) for ci, co, _ in U.LAYERS]
    init = synth.unet_init(shapes, seed=seed, last_scale=1.0)
    # the GPU keeps bfloat16 weights: give the oracle the same values
    import torch
    params = [(torch.from_numpy(w).to(torch.bfloat16).float().numpy().astype(np.float64),
               b.astype(np.float64)) for w, b in init]
    r = np.random.default_rng(seed + 1)
    F = r.random(shape).astype(np.float32)
    M = r.random(shape).astype(np.float32)
    tgt = (0.5 * r.standard_normal((3,) + tuple(n // 2 for n in shape))).astype(np.float32)
    return init, params, F, M, tgt


def test_unet_forward_matches_oracle(P, oracle_mod):
    import torch
    from oracle import unet as U
    init, params, F, M, _ = _net_case(3)
    net = P.lm_unet_create(F.shape, init)
    Ft, F64 = _bf(F)
    Mt, M64 = _bf(M)
    u = torch.empty((3,) + tuple(n // 2 for n in F.shape), device="cuda")
    P.lm_unet_forward(net, Ft, Mt, u)
    torch.cuda.synchronize()
    ref = U.forward(params, F64, M64)
    assert _rel(u.cpu().numpy().astype(np.float64), ref) <= 3e-2
    # FP32 images give the same network input after rounding
    u2 = torch.empty_like(u)
    P.lm_unet_forward(net, torch.from_numpy(F).cuda(), torch.from_numpy(M).cuda(), u2)
    torch.cuda.synchronize()
    assert torch.equal(u, u2)


def test_unet_gradients_match_oracle(P, oracle_mod):
    import torch
    from oracle import unet as U
    init, params, F, M, tgt = _net_case(5)
    net = P.lm_unet_create(F.shape, init)
    Ft, F64 = _bf(F)
    Mt, M64 = _bf(M)
    tt = torch.from_numpy(tgt).cuda()
    L = P.lm_unet_train_step(net, [Ft], [Mt], [tt], lr=0.0)
    grads = P.lm_unet_get_grads(net)
    out, tape = U.forward(params, F64, M64, keep=True)
    Lr, dout = U.mse(out, tgt.astype(np.float64))
    rg = U.backward(params, tape, dout)
    assert abs(L - Lr) <= 2e-2 * Lr
    errs = [(_rel(gw.astype(np.float64), rw), _rel(gb.astype(np.float64), rb))
            for (gw, gb), (rw, rb) in zip(grads, rg)]
    print("relative L2 gradient errors (w, b) per layer:",
          [(round(a, 4), round(b, 4)) for a, b in errs])
    for i, (ew, eb) in enumerate(errs):
        assert ew <= 0.15 and eb <= 0.15, (i, ew, eb)
    # the head sees a single rounding (of the loss gradient): tight there
    assert errs[-1][0] <= 1e-2 and errs[-1][1] <= 1e-2
    # lr = 0 leaves the weights as they were
    w_now = P.lm_unet_get_weights(net)
    for (a, _), (b, _) in zip(w_now, init):
        assert np.array_equal(a, b)


def test_unet_adam_step_matches_oracle(P, oracle_mod):
    """One Adam step: the oracle applies it to the GPU's own gradients, so
    the comparison isolates the update (FP32 vs FP64 arithmetic)."""
    import torch
    from oracle import unet as U
    init, _, F, M, tgt = _net_case(7)
    net = P.lm_unet_create(F.shape, init)
    Ft, _ = _bf(F)
    Mt, _ = _bf(M)
    lr = 1e-3
    P.lm_unet_train_step(net, [Ft], [Mt], [torch.from_numpy(tgt).cuda()], lr=lr)
    g = P.lm_unet_get_grads(net)
    w1 = P.lm_unet_get_weights(net)
    for (w0, b0), (gw, gb), (wa, ba) in zip(init, g, w1):
        for p0, gg, pa in ((w0, gw, wa), (b0, gb, ba)):
            p0 = p0.astype(np.float64)
            ref, _, _ = U.adam(p0, gg.astype(np.float64), np.zeros_like(p0),
                               np.zeros_like(p0), 1, lr)
            assert np.abs(pa - ref).max() <= 1e-6 + 1e-6 * np.abs(ref).max()


def test_unet_training_lowers_the_loss(P):
    import torch
    init, _, F, M, tgt = _net_case(9)
    net = P.lm_unet_create(F.shape, init)
    Ft, _ = _bf(F)
    Mt, _ = _bf(M)
    tt = torch.from_numpy(tgt).cuda()
    losses = [P.lm_unet_train_step(net, [Ft], [Mt], [tt], lr=5e-4)
              for _ in range(30)]
    print("losses:", losses[::5])
    assert losses[-1] < 0.7 * losses[0], losses[::5]


# 128^3 16 -> 16: four one-row tiles per CTA sharing their x taps' loads;
# 64^3 96 -> 32: one two-row tile per CTA; 320x64x64 32 -> 32: four
# two-row tiles per CTA; 128^3 2 -> 16: the gathering kernel
@pytest.mark.parametrize("shape,cin,cout", [((128, 128, 128), 16, 16),
                                            ((64, 64, 64), 96, 32),
                                            ((320, 64, 64), 32, 32),
                                            ((128, 128, 128), 2, 16)])
def test_conv3d_forward_full_size_sampled(P, oracle_mod, shape, cin, cout):
    """The network's largest layer shapes (128^3 and 64^3 levels): sampled
    outputs against the oracle's convolution of each sample's 3x3x3
    neighbourhood."""
    import torch
    from oracle import unet as U
    D, H, W = shape
    r = np.random.default_rng(D + H + cin)
    xt = torch.randn(shape + (cin,), generator=torch.Generator().manual_seed(5)).to(torch.bfloat16)
    w = r.standard_normal((cout, cin, 3, 3, 3)) / np.sqrt(27 * cin)
    wt, w64 = _bf(_w_internal(w))
    b = r.standard_normal(cout).astype(np.float32)
    y = torch.empty(shape + (cout,), device="cuda")
    P.lm_conv3d_forward(xt.cuda(), wt, torch.from_numpy(b).cuda(), 1, y)
    torch.cuda.synchronize()
    x64 = xt.float().numpy().astype(np.float64)
    xp = np.pad(x64, ((1, 1), (1, 1), (1, 1), (0, 0)))
    w_or = w64.reshape(cout, 27, cin).transpose(0, 2, 1).reshape(cout, cin, 3, 3, 3)
    yg = y.cpu().numpy()
    pts = np.stack([r.integers(0, n, 300) for n in shape], axis=1)
    pts[:20] = ([[0, 0, 0], [D - 1, H - 1, W - 1], [0, H - 1, 5]] * 6 +
                [[1, 0, W - 1]] * 2)
    for z, yy, x in pts:
        patch = np.moveaxis(xp[z:z + 3, yy:yy + 3, x:x + 3], -1, 0)   # (cin, 3, 3, 3)
        ref = U.leaky_relu(U.conv3d(patch, w_or, b.astype(np.float64))[:, 1, 1, 1])
        assert np.abs(yg[z, yy, x] - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())


def test_unet_full_size_properties(P):
    """128^3 input: with every convolution weight zero the output is the
    head's bias everywhere (exactly); with real weights the forward is
    finite and deterministic."""
    import torch
    import synth
    from oracle import unet as U
    shapes = [(ci, co) for ci, co, _ in U.LAYERS]
    init = synth.unet_init(shapes, seed=11)
    zero = [(np.zeros_like(w), b) for w, b in init]
    zero[-1] = (zero[-1][0], np.array([0.25, -1.5, 3.0], np.float32))
    F = torch.rand((128, 128, 128), generator=torch.Generator().manual_seed(1)).cuda()
    M = torch.rand((128, 128, 128), generator=torch.Generator().manual_seed(2)).cuda()
    u = torch.empty((3, 64, 64, 64), device="cuda")
    net0 = P.lm_unet_create((128, 128, 128), zero)
    P.lm_unet_forward(net0, F, M, u)
    torch.cuda.synchronize()
    for c, v in enumerate([0.25, -1.5, 3.0]):
        assert bool((u[c] == v).all())
    net = P.lm_unet_create((128, 128, 128), init)
    u1, u2 = torch.empty_like(u), torch.empty_like(u)
    P.lm_unet_forward(net, F, M, u1)
    P.lm_unet_forward(net, F, M, u2)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(u1).all()) and torch.equal(u1, u2)
