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


def _ulp_bf16(v):
    """Spacing of bfloat16 numbers at |v| (8 significant bits)."""
    a = np.maximum(np.abs(v), 1e-30)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


def _near_bf16(got, ref, name, floor=1e-5, frac=0.05):
    """got and ref (bfloat16 values) at most one bfloat16 spacing apart (plus
    an absolute floor for values that cancel to near zero), and equal for
    all but a small fraction: only the FP32 accumulation order differs, and
    it flips a rounding only where the exact value lies near a midpoint."""
    d = np.abs(got - ref)
    tol = _ulp_bf16(np.maximum(np.abs(ref), np.abs(got))) + floor * np.abs(ref).max()
    assert (d <= tol).all(), (name, float(d.max()), float((d - tol).max()))
    moved = float(np.mean(d > 0))
    assert moved <= frac, (name, moved)
    return moved


@pytest.mark.parametrize("seed", [5, 6])
def test_unet_layers_match_oracle_on_their_own_inputs(P, oracle_mod, seed):
    """Layer-local parity of the whole network: every stage is recomputed by
    the oracle from the tensors the network itself stored for that stage's
    inputs (lm_unet_get_tensor), so no rounding is carried from layer to
    layer and each stage is held to its own bar: a convolution's bfloat16
    output within one bfloat16 spacing of the FP64 result rounded the same
    way, pooling and concatenation exact, weight and bias gradients at the
    1e-4 bar of a single convolution, the activation masks and the skip and
    pooled-gradient sums between the layers bit for bit."""
    import torch
    from oracle import unet as U
    init, params, F, M, tgt = _net_case(seed)
    net = P.lm_unet_create(F.shape, init)
    Ft, _ = _bf(F)
    Mt, _ = _bf(M)
    tt = torch.from_numpy(tgt).cuda()
    L = P.lm_unet_train_step(net, [Ft], [Mt], [tt], lr=0.0)
    grads = P.lm_unet_get_grads(net)
    T = {n: np.moveaxis(P.lm_unet_get_tensor(net, n), -1, 0).astype(np.float64)
         for n in P.UNET_TENSORS}
    bf = U.bf16_round
    cout = [co for _, co, _ in U.LAYERS]
    moved = {}
    # forward: each hidden convolution on its own stored input
    convs = [("x0", "e0a", 0), ("e0a", "e0", 1), ("p0", "e1a", 2), ("e1a", "e1", 3),
             ("p1", "e2a", 4), ("e2a", "e2", 5), ("p2", "e3a", 6), ("e3a", "e3", 7),
             ("cat2", "d2a", 8), ("d2a", "d2", 9), ("cat1", "d1a", 10),
             ("d1a", "d1", 11)]
    for xin, yout, i in convs:
        w, b = params[i]
        ref = bf(U.leaky_relu(U.conv3d(T[xin], w, b)))
        moved[yout] = _near_bf16(T[yout], ref, yout)
    # the head (FP32 output, channels 3..15 are padding)
    ref = U.conv3d(T["d1"], *params[12])
    assert np.abs(T["out"][:3] - ref).max() <= 2e-5 * np.abs(ref).max()
    assert not T["out"][3:].any()
    # the input pair, pooling (FP32 mean of 8, rounded) and concatenation
    assert np.array_equal(T["x0"][0], U.bf16_round(F))
    assert np.array_equal(T["x0"][1], U.bf16_round(M))
    for src, dst in (("e0", "p0"), ("e1", "p1"), ("e2", "p2")):
        moved[dst] = _near_bf16(T[dst], bf(U.pool(T[src])), dst, floor=0.0, frac=1e-3)
    assert np.array_equal(T["cat2"][:128], U.up(T["e3"]))
    assert np.array_equal(T["cat2"][128:], T["e2"])
    assert np.array_equal(T["cat1"][:64], U.up(T["d2"]))
    assert np.array_equal(T["cat1"][64:], T["e1"])
    # the loss gradient at the head: 2 (out - tgt) / N, rounded
    n_out = 3 * tgt[0].size
    dz = bf(np.float32(2.0) * (T["out"][:3].astype(np.float32) - tgt) *
            np.float32(1.0 / n_out))
    assert np.abs(T["dy12"][:3] - dz).max() <= _ulp_bf16(np.abs(dz).max())
    assert not T["dy12"][3:].any()
    # weight and bias gradients from the layer's own input and output
    # gradient (the layers whose gradient survives the reverse pass)
    back = [(0, "x0", "dy0"), (1, "e0a", "dy1"), (2, "p0", "dy2"), (3, "e1a", "dy3"),
            (4, "p1", "dy4"), (5, "e2a", "dy5"), (6, "p2", "dy6"), (12, "d1", "dy12")]
    for i, xin, dyn in back:
        dx, dw, db = U.conv3d_backward(T[xin], params[i][0], T[dyn][:cout[i]])
        gw, gb = grads[i]
        assert np.abs(gw - dw).max() <= 1e-4 * np.abs(dw).max(), (i, "w")
        assert np.abs(gb - db).max() <= 1e-4 * np.abs(db).max(), (i, "b")
        if dyn in ("dy2", "dy4", "dy6"):   # their data gradients survive too
            dxn = "dx" + dyn[2:]
            moved[dxn] = _near_bf16(T[dxn], bf(dx), dxn)
    # between the layers, bit for bit in FP32 then bfloat16 as the network
    # does it: the activation mask (slope 0.2f where the stored output is not
    # positive) of the pooled gradient, alone (c1) or added to the skip
    # connection's gradient (c3, c5)
    s32 = np.float32(U.SLOPE)

    def mask(y, g):
        g32 = g.astype(np.float32)
        return bf(np.where(y > 0, g32, s32 * g32))

    g1 = np.float32(0.125) * U.up(T["dx2"]).astype(np.float32)
    assert np.array_equal(T["dy1"], mask(T["e0"], bf(g1)))
    for dyn, y, dxp, skip in (("dy3", "e1", "dx4", T["dx10"][64:]),
                              ("dy5", "e2", "dx6", T["dx8"][128:])):
        g = np.float32(0.125) * U.up(T[dxp]).astype(np.float32) + skip.astype(np.float32)
        assert np.array_equal(T[dyn], mask(T[y], bf(g))), dyn
    print("fraction of bfloat16 values one spacing off:",
          {k: round(v, 4) for k, v in moved.items()}, "loss", L)


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
