"""lm_eval_noalloc: the evaluation entry point that allocates nothing.

It is meant for callers that cannot allocate device memory while they
evaluate (inside another framework's allocator, or in loops where
cudaMalloc's device synchronisation is not allowed); its scratch is a static
device array in the library.  The test calls it through the C ABI twice in a
row, on two different fields, and checks each result against lm_eval on a
context, with the parity tests' tolerances.  This file is collected last so
that a run stopping at the first failure has run every other test before.
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


def _call(P, Ft, Mt, u, g, loss, gmax, params):
    vf = P.Volume(*Ft.shape, P.LM_F32, Ft.data_ptr())
    vm = P.Volume(*Mt.shape, P.LM_F32, Mt.data_ptr())
    rc = P.load().lm_eval_noalloc(
        ctypes.byref(vf), ctypes.byref(vm), ctypes.byref(params),
        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(gmax.data_ptr()),
        ctypes.c_void_p(0))
    return rc


@pytest.mark.parametrize("loss", ["lncc", "mse"])
def test_noalloc_matches_lm_eval_on_two_calls(lib, loss):
    import torch
    import synth
    P = lib
    shape = (40, 36, 44)
    F, M, _ = synth.blob_pair(shape, seed=21)
    Ft = torch.from_numpy(F).cuda()
    Mt = torch.from_numpy(M).cuda()
    params = P.lm_default_params(
        loss=P.LM_LOSS_MSE if loss == "mse" else P.LM_LOSS_LNCC)
    ctx = P.lm_init(Ft, Mt, params)
    for seed in (31, 32):
        u = torch.from_numpy(synth.random_field(shape, seed=seed, scale=1.6)).cuda()
        g_ref = torch.empty_like(u)
        L_ref, gmax_ref = P.lm_eval(ctx, u, g_ref)
        g = torch.full_like(u, float("nan"))
        loss = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        gmax = torch.zeros((1,), dtype=torch.float32, device="cuda")
        assert _call(P, Ft, Mt, u, g, loss, gmax, params) == P.LM_OK, \
            P.lm_last_error()
        torch.cuda.synchronize()
        L = float(loss.item())
        assert abs(L - L_ref) <= TOL_L * L_ref, (L, L_ref)
        err = float((g - g_ref).abs().max())
        assert err <= TOL_G * gmax_ref, (err, gmax_ref)
        assert abs(float(gmax.item()) - gmax_ref) <= 1e-4 * gmax_ref
    P.lm_destroy(ctx)


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
