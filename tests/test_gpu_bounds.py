"""Bounds checks in place of a memory sanitizer.

The same workload runs twice, each in a process of its own: once on the
release library, once on the debug-bounds build (liblmreg_dbg.so,
-DLM_DEBUG_BOUNDS), whose device buffers sit between guard bands of 0xFF
bytes.  The caller's buffers (F, M, u, g) are guarded the same way by the
worker itself, with a NaN sentinel.  The bar:
  - no guard band changes (no kernel writes outside a buffer);
  - every result is bitwise the release library's (a kernel reading outside
    a buffer would read NaN or -1 in the debug build and change it);
on tiny, ragged and odd shapes, both image types, every loss and method,
the warp-smoothing path, rejection, the pyramid and a batch.
"""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GUARD = 4096                 # sentinel elements on each side of a buffer
SENT_F32 = 0x7FC0DEAD        # NaN payloads that no kernel writes
SENT_BF16 = 0x7FC1


def _guarded(shape, dtype):
    import torch
    n = int(np.prod(shape))
    if dtype == torch.bfloat16:
        big = torch.full((n + 2 * GUARD,), SENT_BF16, dtype=torch.int16,
                         device="cuda").view(torch.bfloat16)
    else:
        big = torch.full((n + 2 * GUARD,), SENT_F32, dtype=torch.int32,
                         device="cuda").view(torch.float32)
    return big, big[GUARD:GUARD + n].view(shape)


def _bands_intact(big):
    import torch
    bits = big.view(torch.int16 if big.dtype == torch.bfloat16 else torch.int32)
    s = SENT_BF16 if big.dtype == torch.bfloat16 else SENT_F32
    return bool((bits[:GUARD] == s).all()) and bool((bits[-GUARD:] == s).all())


def _digest(t):
    return hashlib.sha256(t.detach().cpu().contiguous().numpy().tobytes()
                          ).hexdigest()[:16]


CASES = [
    # name, shape, dtype, params, ops
    ("tiny", (1, 1, 1), "f32", {}, "eval reset iter"),
    ("odd", (5, 7, 3), "f32", {}, "eval reset iter"),
    ("ragged_tile3", (13, 17, 29), "f32", {"tile": 3}, "eval reset iter"),
    ("bf16_win7", (9, 70, 33), "bf16", {"win": 7}, "eval reset iter"),
    ("mse", (19, 23, 37), "f32", {"loss": 1}, "eval reset iter"),
    ("mi", (19, 23, 37), "f32", {"loss": 2, "bins": 24, "lambda0": 1.0,
                                 "step": 0.25}, "eval reset iter"),
    ("demons", (13, 17, 29), "f32", {"method": 1, "loss": 1, "sigma_warp": 1.0},
     "eval reset iter"),
    ("warp_reject", (24, 20, 28), "f32", {"sigma_warp": 1.0, "reject": 1,
                                          "lambda0": 0.3}, "eval reset iter"),
    ("pyramid", (24, 20, 28), "f32", {}, "register"),
]


def _worker(debug):
    import torch
    sys.path.insert(0, ROOT)
    import synth
    from paper_2603_19371_gb300 import lmreg as P
    out = {}
    for name, shape, dt, kw, ops in CASES:
        dtype = torch.bfloat16 if dt == "bf16" else torch.float32
        F, M, _ = synth.blob_pair(shape, seed=31)
        bF, tF = _guarded(shape, dtype)
        bM, tM = _guarded(shape, dtype)
        tF.copy_(torch.from_numpy(F))
        tM.copy_(torch.from_numpy(M))
        bu, u = _guarded((3,) + shape, torch.float32)
        bg, g = _guarded((3,) + shape, torch.float32)
        u.zero_()
        ctx = P.lm_init(tF, tM, P.lm_default_params(**kw))
        rec = []
        for op in ops.split():
            if op == "eval":
                L, gm = P.lm_eval(ctx, u, g)
                rec += [float(L).hex(), float(gm).hex(), _digest(g)]
            elif op == "reset":
                P.lm_reset(ctx, u)
            elif op == "iter":
                info = P.lm_iterate(ctx, u, 3)
                rec += [float(info.loss).hex(), float(info.lambda_).hex(),
                        _digest(u)]
            elif op == "register":
                rep = P.lm_register(ctx, [(4, 2), (2, 2), (1, 2)], u)
                rec += [float(rep.final_loss).hex(), _digest(u)]
            if debug:
                P.lm_debug_check(ctx)
        torch.cuda.synchronize()
        for b in (bF, bM, bu, bg):
            assert _bands_intact(b), f"{name}: a caller buffer's band changed"
        P.lm_destroy(ctx)
        out[name] = rec
    # a batch of two pairs of different shapes
    shapes = [(13, 17, 29), (6, 9, 11)]
    Fs, Ms, us, bands = [], [], [], []
    for i, s in enumerate(shapes):
        F, M, _ = synth.blob_pair(s, seed=40 + i)
        bF, tF = _guarded(s, torch.float32)
        bM, tM = _guarded(s, torch.float32)
        tF.copy_(torch.from_numpy(F))
        tM.copy_(torch.from_numpy(M))
        bu, u = _guarded((3,) + s, torch.float32)
        u.zero_()
        Fs.append(tF), Ms.append(tM), us.append(u)
        bands += [bF, bM, bu]
    b = P.lm_batch_init(Fs, Ms, P.lm_default_params())
    P.lm_batch_reset(b, us)
    infos = P.lm_batch_iterate(b, us, 3)
    if debug:
        P.lm_batch_debug_check(b)
    torch.cuda.synchronize()
    assert all(_bands_intact(x) for x in bands), "batch: a band changed"
    out["batch"] = [float(i.loss).hex() for i in infos] + [_digest(u) for u in us]
    P.lm_batch_destroy(b)
    if not debug:
        # the release library has no guard bands to check
        ctx = P.lm_init(Fs[0], Ms[0], P.lm_default_params())
        with pytest.raises(P.LMError) as e:
            P.lm_debug_check(ctx)
        assert e.value.code == P.LM_EUNSUPPORTED
    print("RESULT " + json.dumps(out))


def _run(lib):
    env = dict(os.environ, PYTHONPATH=ROOT)
    if lib:
        env["LMREG_LIBRARY"] = lib
    else:
        env.pop("LMREG_LIBRARY", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__),
                        "debug" if lib else "release"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.mark.gpu
def test_debug_bounds_build_matches_release_bitwise():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19371_gb300 import build
    build.build()
    dbg = build.build(debug_bounds=True)
    rel = _run(None)
    deb = _run(dbg)
    assert set(rel) == set(deb)
    for k in rel:
        assert rel[k] == deb[k], (k, rel[k], deb[k])


if __name__ == "__main__":
    _worker(sys.argv[1] == "debug")
