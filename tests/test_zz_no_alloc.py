"""lm_eval_noalloc: the evaluation entry point that allocates nothing.

It is meant for callers that cannot allocate device memory while they
evaluate (inside another framework's allocator, or in loops where
cudaMalloc's device synchronisation is not allowed); its scratch is a static
device array in the library.  The tests call it through the C ABI twice in a
row, on two different fields, and check each result against the FP64 oracle
and against lm_eval on a context, with the parity tests' tolerances; they
cover LNCC, MSE and Demons, FP32 and BF16 images, a ragged shape whose rows
are padded in the scratch, gradient smoothing off and wide, and a volume at
the size limit.  They also check that a call leaves the device's free memory
unchanged and that host pointers are refused before any launch.  This file is
collected last so that a run stopping at the first failure has run every
other test before.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_L = 1e-5     # relative loss
TOL_G = 1e-4     # gradient, relative to gmax


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19371_gb300 import build, lmreg
    build.build()
    return lmreg


def _oracle_params(oracle, p):
    return oracle.params(win=p.win, eps_nr=float(np.float32(p.eps_nr)),
                         eps_dr=float(np.float32(p.eps_dr)),
                         sigma_grad=float(p.sigma_grad), sigma_warp=0.0,
                         step=float(p.step), lambda0=p.lambda0,
                         mu_inc=p.mu_inc, mu_dec=p.mu_dec,
                         lambda_max=p.lambda_max, reject=0, tau=p.tau,
                         max_retries=p.max_retries, tile=1, loss=p.loss,
                         method=p.method, alpha=float(np.float32(p.alpha)),
                         bins=p.bins)


def _call(P, Ft, Mt, u, g, loss, gmax, params, dt):
    vf = P.Volume(*Ft.shape, dt, Ft.data_ptr())
    vm = P.Volume(*Mt.shape, dt, Mt.data_ptr())
    return P.load().lm_eval_noalloc(
        ctypes.byref(vf), ctypes.byref(vm), ctypes.byref(params),
        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(loss.data_ptr()) if loss is not None else None,
        ctypes.c_void_p(gmax.data_ptr()) if gmax is not None else None,
        ctypes.c_void_p(0))


def _images(F, M, dtype):
    import torch
    Ft = torch.from_numpy(F).cuda()
    Mt = torch.from_numpy(M).cuda()
    if dtype == "bf16":
        Ft, Mt = Ft.to(torch.bfloat16), Mt.to(torch.bfloat16)
    return Ft, Mt, Ft.float().cpu().numpy().astype(np.float64), \
        Mt.float().cpu().numpy().astype(np.float64)


CASES = [
    # (loss, dtype, shape, sigma_grad)
    ("lncc", "f32", (40, 36, 44), 1.0),
    ("mse", "f32", (40, 36, 44), 1.0),
    ("demons", "f32", (40, 36, 44), 1.0),
    ("lncc", "bf16", (40, 36, 44), 1.0),
    ("lncc", "f32", (17, 19, 23), 0.0),     # rows of 23 padded to 24
    ("mse", "bf16", (17, 19, 23), 2.0),
    ("demons", "bf16", (17, 19, 23), 1.0),
]


@pytest.mark.parametrize("loss,dtype,shape,sg", CASES)
def test_noalloc_matches_oracle_and_lm_eval_on_two_calls(lib, oracle_mod,
                                                         loss, dtype, shape,
                                                         sg):
    import torch
    import synth
    P = lib
    F, M, _ = synth.blob_pair(shape, seed=21)
    Ft, Mt, Fo, Mo = _images(F, M, dtype)
    dt = P.LM_BF16 if dtype == "bf16" else P.LM_F32
    kw = dict(sigma_grad=sg)
    if loss == "mse":
        kw["loss"] = P.LM_LOSS_MSE
    elif loss == "demons":
        kw.update(loss=P.LM_LOSS_MSE, method=P.LM_METHOD_DEMONS)
    params = P.lm_default_params(**kw)
    Po = _oracle_params(oracle_mod, params)
    ctx = P.lm_init(Ft, Mt, params)
    for seed in (31, 32):
        u0 = synth.random_field(shape, seed=seed, scale=1.6)
        u = torch.from_numpy(u0).cuda()
        g_ref = torch.empty_like(u)
        L_ref, gmax_ref = P.lm_eval(ctx, u, g_ref)
        g = torch.full_like(u, float("nan"))
        lo = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        gm = torch.zeros((1,), dtype=torch.float32, device="cuda")
        assert _call(P, Ft, Mt, u, g, lo, gm, params, dt) == P.LM_OK, \
            P.lm_last_error()
        torch.cuda.synchronize()
        L, gmax = float(lo.item()), float(gm.item())
        # against the FP64 oracle on the same inputs
        ev = oracle_mod.evaluate(Fo, Mo, u0.astype(np.float64), Po)
        assert abs(L - ev["L"]) <= TOL_L * ev["L"], (L, ev["L"])
        gg = g.cpu().numpy().astype(np.float64)
        err = np.abs(gg - ev["g"]).max()
        assert err <= TOL_G * ev["gmax"], (err, ev["gmax"])
        assert abs(gmax - ev["gmax"]) <= 1e-4 * ev["gmax"]
        # and against the context path
        assert abs(L - L_ref) <= TOL_L * L_ref, (L, L_ref)
        err = float((g - g_ref).abs().max())
        assert err <= TOL_G * gmax_ref, (err, gmax_ref)
    P.lm_destroy(ctx)


def test_noalloc_allocates_nothing(lib):
    """After a first call (which loads the library's kernels and looks up the
    static array), calls leave the device's free memory unchanged."""
    import torch
    import synth
    P = lib
    shape = (24, 28, 30)
    F, M, _ = synth.blob_pair(shape, seed=22)
    Ft, Mt = torch.from_numpy(F).cuda(), torch.from_numpy(M).cuda()
    u = torch.from_numpy(synth.random_field(shape, seed=33, scale=1.2)).cuda()
    g = torch.empty_like(u)
    lo = torch.empty((1,), dtype=torch.float64, device="cuda")
    gm = torch.empty((1,), dtype=torch.float32, device="cuda")
    params = P.lm_default_params()
    assert _call(P, Ft, Mt, u, g, lo, gm, params, P.LM_F32) == P.LM_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _call(P, Ft, Mt, u, g, lo, gm, params, P.LM_F32) == P.LM_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_at_the_size_limit_through_the_binding(lib, oracle_mod):
    """64 x 64 x 127 voxels: rows padded to 128 fill LM_NOALLOC_MAX_VOXELS
    exactly.  Called through the Python binding."""
    import torch
    import synth
    P = lib
    shape = (64, 64, 127)
    assert 64 * 64 * 128 == P.LM_NOALLOC_MAX_VOXELS
    F, M, _ = synth.blob_pair(shape, seed=23)
    Ft, Mt = torch.from_numpy(F).cuda(), torch.from_numpy(M).cuda()
    u0 = synth.random_field(shape, seed=34, scale=1.4)
    u = torch.from_numpy(u0).cuda()
    g = torch.empty_like(u)
    lo = torch.empty((1,), dtype=torch.float64, device="cuda")
    gm = torch.empty((1,), dtype=torch.float32, device="cuda")
    params = P.lm_default_params()
    P.lm_eval_noalloc(Ft, Mt, u, g, lo, gm, params)
    torch.cuda.synchronize()
    ev = oracle_mod.evaluate(F.astype(np.float64), M.astype(np.float64),
                             u0.astype(np.float64),
                             _oracle_params(oracle_mod, params))
    assert abs(float(lo.item()) - ev["L"]) <= TOL_L * ev["L"]
    err = np.abs(g.cpu().numpy().astype(np.float64) - ev["g"]).max()
    assert err <= TOL_G * ev["gmax"], (err, ev["gmax"])
    # one more column of padding is past the limit
    big = torch.zeros((64, 64, 129), device="cuda")
    ub = torch.zeros((3, 64, 64, 129), device="cuda")
    with pytest.raises(P.LMError) as e:
        P.lm_eval_noalloc(big, big, ub, ub.clone(), lo, gm, params)
    assert e.value.code == P.LM_EINVAL


def test_noalloc_refuses_host_pointers_and_wrong_outputs(lib):
    """A host pointer among the outputs is refused on the host, before any
    launch; the binding refuses a float32 loss or a CPU gmax."""
    import torch
    P = lib
    shape = (8, 8, 8)
    Ft = torch.rand(shape, device="cuda")
    u = torch.zeros((3,) + shape, device="cuda")
    g = torch.zeros_like(u)
    host_loss = np.zeros(1, np.float64)
    vf = P.Volume(*shape, P.LM_F32, Ft.data_ptr())
    params = P.lm_default_params()
    rc = P.load().lm_eval_noalloc(
        ctypes.byref(vf), ctypes.byref(vf), ctypes.byref(params),
        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(host_loss.ctypes.data), None, None)
    assert rc == P.LM_EINVAL and "device pointer" in P.lm_last_error()
    host_u = np.zeros((3,) + shape, np.float32)
    rc = P.load().lm_eval_noalloc(
        ctypes.byref(vf), ctypes.byref(vf), ctypes.byref(params),
        ctypes.c_void_p(host_u.ctypes.data), ctypes.c_void_p(g.data_ptr()),
        None, None, None)
    assert rc == P.LM_EINVAL and "device pointer" in P.lm_last_error()
    with pytest.raises(ValueError):
        P.lm_eval_noalloc(Ft, Ft, u, g,
                          torch.zeros(1, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        P.lm_eval_noalloc(Ft, Ft, u, g, None, torch.zeros(1))


def test_noalloc_rejects_volumes_above_the_limit(lib):
    import torch
    P = lib
    small = torch.zeros(8, device="cuda")
    D = P.LM_NOALLOC_MAX_VOXELS // (128 * 128) + 1
    vf = P.Volume(D, 128, 128, P.LM_F32, small.data_ptr())
    params = P.lm_default_params()
    rc = P.load().lm_eval_noalloc(ctypes.byref(vf), ctypes.byref(vf),
                                  ctypes.byref(params),
                                  ctypes.c_void_p(small.data_ptr()),
                                  ctypes.c_void_p(small.data_ptr()), None,
                                  None, None)
    assert rc == P.LM_EINVAL
    assert "LM_NOALLOC_MAX_VOXELS" in P.lm_last_error()


def test_noalloc_refuses_the_mi_loss(lib):
    """The MI loss needs per-pair histogram buffers, which only lm_init
    allocates."""
    import torch
    P = lib
    small = torch.zeros(4 * 4 * 4 * 3, device="cuda")
    vf = P.Volume(4, 4, 4, P.LM_F32, small.data_ptr())
    params = P.lm_default_params(loss=P.LM_LOSS_MI)
    rc = P.load().lm_eval_noalloc(ctypes.byref(vf), ctypes.byref(vf),
                                  ctypes.byref(params),
                                  ctypes.c_void_p(small.data_ptr()),
                                  ctypes.c_void_p(small.data_ptr()),
                                  None, None, ctypes.c_void_p(0))
    assert rc == P.LM_EUNSUPPORTED and "MI" in P.lm_last_error()
