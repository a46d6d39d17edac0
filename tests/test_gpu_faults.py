"""Failure detection without a device fault: host-side injection.

LM_FAULT_ALLOC=n fails the n-th device allocation of a context as if
cudaMalloc had; LM_FAULT_TIMEOUT=1 makes the gradient-smoothing kernel wait
on a barrier that no copy completes, so that its bounded wait runs out.  No
test here faults, traps or hangs the device: the injected wait is bounded in
time, nothing is in flight while it runs, and each test ends by using the
same device and process again.
"""
import time

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


def _pair(shape=(24, 20, 28), seed=21):
    import torch
    import synth
    F, M, _ = synth.blob_pair(shape, seed=seed)
    return torch.from_numpy(F).cuda(), torch.from_numpy(M).cuda()


@pytest.mark.parametrize("n", [1, 6, 12, 18])
def test_injected_allocation_failure(P, monkeypatch, n):
    import torch
    F, M = _pair()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("LM_FAULT_ALLOC", str(n))
    for _ in range(3):
        with pytest.raises(P.LMError) as e:
            P.lm_init(F, M, P.lm_default_params())
        assert e.value.code == P.LM_ENOMEM
        assert "LM_FAULT_ALLOC" in str(e.value)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # what the failed creates had allocated was given back
    assert free1 >= free0 - (64 << 20), (free0, free1)
    monkeypatch.delenv("LM_FAULT_ALLOC")
    ctx = P.lm_init(F, M, P.lm_default_params())
    L, gmax = P.lm_eval(ctx, torch.zeros((3,) + tuple(F.shape), device="cuda"))
    assert np.isfinite(L) and gmax > 0


def test_injected_wait_timeout_is_reported(P, monkeypatch):
    import torch
    F, M = _pair()
    u = torch.zeros((3,) + tuple(F.shape), device="cuda")
    ref = P.lm_init(F, M, P.lm_default_params())
    L_ref, g_ref = P.lm_eval(ref, u)
    P.lm_destroy(ref)

    monkeypatch.setenv("LM_FAULT_TIMEOUT", "1")
    ctx = P.lm_init(F, M, P.lm_default_params())
    monkeypatch.delenv("LM_FAULT_TIMEOUT")
    t0 = time.perf_counter()
    with pytest.raises(P.LMError) as e:
        P.lm_eval(ctx, u)
    assert e.value.code == P.LM_ETIMEOUT
    # one launch of waits bounded by half a second each, all in one wave
    assert time.perf_counter() - t0 < 30.0
    # the reset evaluation runs out too; the state reports it
    P.lm_reset(ctx, u)
    with pytest.raises(P.LMError) as e:
        P.lm_iterate(ctx, u, 1)
    assert e.value.code == P.LM_ETIMEOUT
    P.lm_destroy(ctx)

    # the device and the process are usable: a fresh context evaluates the
    # same pair to the same result
    ctx = P.lm_init(F, M, P.lm_default_params())
    L, gmax = P.lm_eval(ctx, u)
    assert L == L_ref and gmax == g_ref
    assert torch.isfinite(F.sum()).item()
