"""GPU parity of the batched path: several pairs of uneven shapes share each
kernel launch; every pair must match the FP64 oracle exactly as a single
pair does (same bars as test_gpu_parity)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_U = 1e-4
TOL_L = 1e-5
TOL_G = 1e-4

SHAPES = [(20, 24, 28), (32, 32, 32), (13, 17, 29), (40, 36, 44)]


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_19371_gb300 import build, lmreg
    build.build()
    lmreg.load()
    return lmreg


def _oracle_params(oracle, p):
    return oracle.params(win=p.win, eps_nr=float(np.float32(p.eps_nr)),
                         eps_dr=float(np.float32(p.eps_dr)),
                         sigma_grad=float(p.sigma_grad),
                         sigma_warp=float(p.sigma_warp), step=float(p.step),
                         lambda0=p.lambda0, mu_inc=p.mu_inc, mu_dec=p.mu_dec,
                         lambda_max=p.lambda_max, reject=p.reject, tau=p.tau,
                         max_retries=p.max_retries)


def _pairs(seed0=40, dtype=None):
    import torch
    import synth
    Fs, Ms = [], []
    for i, sh in enumerate(SHAPES):
        F, M, _ = synth.blob_pair(sh, seed=seed0 + i)
        Ft, Mt = torch.from_numpy(F).cuda(), torch.from_numpy(M).cuda()
        if dtype is not None:
            Ft, Mt = Ft.to(dtype), Mt.to(dtype)
        Fs.append(Ft)
        Ms.append(Mt)
    return Fs, Ms


@pytest.mark.parametrize("bf16", [False, True])
def test_batch_eval_matches_oracle(P, oracle_mod, bf16):
    import torch
    import synth
    Fs, Ms = _pairs(dtype=torch.bfloat16 if bf16 else None)
    params = P.lm_default_params()
    b = P.lm_batch_init(Fs, Ms, params)
    us = [torch.from_numpy(synth.random_field(sh, seed=7 + i, scale=1.6)).cuda()
          for i, sh in enumerate(SHAPES)]
    gs = [torch.empty_like(u) for u in us]
    L, gm = P.lm_batch_eval(b, us, gs)
    Po = _oracle_params(oracle_mod, params)
    for i in range(len(SHAPES)):
        ev = oracle_mod.evaluate(Fs[i].float().cpu().numpy(),
                                 Ms[i].float().cpu().numpy(),
                                 us[i].cpu().numpy().astype(np.float64), Po)
        assert abs(L[i] - ev["L"]) <= TOL_L * ev["L"], (i, L[i], ev["L"])
        err = np.abs(gs[i].cpu().numpy() - ev["g"]).max()
        assert err <= TOL_G * ev["gmax"], (i, err, ev["gmax"])


def test_batch_iterations_teacher_forced(P, oracle_mod):
    import torch
    Fs, Ms = _pairs(seed0=50)
    params = P.lm_default_params(lambda0=0.02, step=1.0)
    Po = _oracle_params(oracle_mod, params)
    b = P.lm_batch_init(Fs, Ms, params)
    us = [torch.zeros((3,) + sh, device="cuda") for sh in SHAPES]
    P.lm_batch_reset(b, us)
    infos = P.lm_batch_iterate(b, us, 0)
    L = [x.loss for x in infos]
    Lp = [0.0] * len(SHAPES)
    hp = [0] * len(SHAPES)
    lam = [x.lambda_ for x in infos]
    Fo = [F.cpu().numpy().astype(np.float64) for F in Fs]
    Mo = [M.cpu().numpy().astype(np.float64) for M in Ms]
    for t in range(4):
        ut = [u.cpu().numpy().astype(np.float64) for u in us]
        expect = []
        for i in range(len(SHAPES)):
            ev = oracle_mod.evaluate(Fo[i], Mo[i], ut[i], Po)
            assert abs(L[i] - ev["L"]) <= TOL_L * ev["L"], (t, i)
            u1, _ = oracle_mod.trial(ut[i], ev["g"], ev["gmax"], ev["L"],
                                     lam[i], Po)
            L1 = oracle_mod.loss(Fo[i], Mo[i], u1, Po)
            act, lam_o = oracle_mod.decide(L1, ev["L"], Lp[i], hp[i], lam[i],
                                           0, Po)
            expect.append((u1, L1, lam_o, ev["L"]))
        infos = P.lm_batch_iterate(b, us, 1)
        for i, x in enumerate(infos):
            u1, L1, lam_o, L0 = expect[i]
            assert abs(x.loss_first - L1) <= TOL_L * L1, (t, i)
            tie = abs(L1 - L0) < 1e-6 * L0
            assert x.accepted == 1
            if not tie:
                assert x.lambda_ == pytest.approx(lam_o, rel=1e-12)
            err = np.abs(us[i].cpu().numpy().astype(np.float64) - u1).max()
            assert err <= TOL_U, (t, i, err)
            Lp[i], hp[i], L[i], lam[i] = L0, 1, x.loss, x.lambda_


def test_batch_register_lowers_every_loss(P):
    import torch
    Fs, Ms = _pairs(seed0=60)
    params = P.lm_default_params(lambda0=0.006, step=1.0)
    b = P.lm_batch_init(Fs, Ms, params)
    us = [torch.zeros((3,) + sh, device="cuda") for sh in SHAPES]
    L0, _ = P.lm_batch_eval(b, us)
    reps = P.lm_batch_register(b, [(2, 10), (1, 10)], us)
    L1, _ = P.lm_batch_eval(b, us)
    for i, r in enumerate(reps):
        assert r.level_iters[0] == 10 and r.level_iters[1] == 10
        assert L1[i] < L0[i]
        assert r.final_loss == pytest.approx(L1[i], rel=1e-6)
    # the one-shot form gives the same fields
    us2 = [torch.zeros((3,) + sh, device="cuda") for sh in SHAPES]
    P.lm_register_batch(Fs, Ms, us2, [(2, 10), (1, 10)], params)
    for a, c in zip(us, us2):
        assert float((a - c).abs().max()) < 1e-4


def test_batch_rejects_mixed_dtypes(P):
    import torch
    Fs, Ms = _pairs(seed0=70)
    Fs[1] = Fs[1].to(torch.bfloat16)
    Ms[1] = Ms[1].to(torch.bfloat16)
    with pytest.raises(P.LMError) as e:
        P.lm_batch_init(Fs, Ms, P.lm_default_params())
    assert e.value.code == P.LM_EINVAL


def test_batch_targets_stop_pairs(P):
    """A pair whose loss reaches its target stops; the others go on."""
    import torch
    Fs, Ms = _pairs(seed0=80)
    params = P.lm_default_params(lambda0=0.02, step=1.0)
    b = P.lm_batch_init(Fs, Ms, params)
    us = [torch.zeros((3,) + sh, device="cuda") for sh in SHAPES]
    P.lm_batch_reset(b, us)
    P.lm_batch_iterate(b, us, 2)
    inf, nan = float("inf"), float("nan")
    P.lm_batch_set_targets(b, [inf] + [nan] * (len(SHAPES) - 1))
    infos = P.lm_batch_iterate(b, us, 1)       # pair 0 stops after this one
    assert infos[0].stopped == 1
    assert all(x.stopped == 0 for x in infos[1:])
    snap = [u.clone() for u in us]
    L_stop = infos[0].loss
    infos = P.lm_batch_iterate(b, us, 4)
    assert infos[0].stopped == 1 and infos[0].loss == L_stop
    assert torch.equal(us[0], snap[0])
    for i in range(1, len(SHAPES)):
        assert infos[i].stopped == 0
        assert not torch.equal(us[i], snap[i])
    # clearing the targets keeps the stop; a reset lifts it
    P.lm_batch_set_targets(b, None)
    assert P.lm_batch_iterate(b, us, 1)[0].stopped == 1
    P.lm_batch_reset(b, us)
    infos = P.lm_batch_iterate(b, us, 1)
    assert infos[0].stopped == 0
    assert not torch.equal(us[0], snap[0])


def test_batch_autotune_keeps_results(P, oracle_mod):
    """The autotuned work split changes timing, not results: evaluations
    still match the oracle and iterations still run."""
    import torch
    import synth
    Fs, Ms = _pairs(seed0=90)
    params = P.lm_default_params()
    b = P.lm_batch_init(Fs, Ms, params)
    us = [torch.from_numpy(synth.random_field(sh, seed=20 + i, scale=1.3)).cuda()
          for i, sh in enumerate(SHAPES)]
    t, w1, w2, ms = P.lm_batch_autotune(b, us, reps=2)
    assert t in (0, 1) and w1 in (1, 2, 4, 8) and w2 in (2, 3, 4, 8, 16)
    assert ms > 0
    gs = [torch.empty_like(u) for u in us]
    L, _ = P.lm_batch_eval(b, us, gs)
    Po = _oracle_params(oracle_mod, params)
    for i in range(len(SHAPES)):
        ev = oracle_mod.evaluate(Fs[i].cpu().numpy(), Ms[i].cpu().numpy(),
                                 us[i].cpu().numpy().astype(np.float64), Po)
        assert abs(L[i] - ev["L"]) <= TOL_L * ev["L"]
        assert np.abs(gs[i].cpu().numpy() - ev["g"]).max() <= TOL_G * ev["gmax"]
    P.lm_batch_reset(b, us)
    infos = P.lm_batch_iterate(b, us, 3)
    assert all(np.isfinite(x.loss) for x in infos)


@pytest.mark.parametrize("mode", ["lncc", "tile2", "mse", "demons"])
def test_batch_equals_single_pair_bitwise(P, mode):
    """The loss is an exact integer sum, so neither the batch's work split
    nor the autotuner's choice changes any result: a batch and one context
    per pair end on bitwise-equal fields after the same iterations (LNCC
    with Eq. tile1 and Eq. tilen, MSE, Demons)."""
    import torch
    Fs, Ms = _pairs(seed0=100)
    params = P.lm_default_params(lambda0=0.02, step=1.0, **{
        "lncc": {}, "tile2": dict(tile=2), "mse": dict(loss=P.LM_LOSS_MSE),
        "demons": dict(loss=P.LM_LOSS_MSE,
                       method=P.LM_METHOD_DEMONS)}[mode])
    b = P.lm_batch_init(Fs, Ms, params)
    ub = [torch.zeros((3,) + sh, device="cuda") for sh in SHAPES]
    P.lm_batch_autotune(b, ub, reps=1)
    P.lm_batch_reset(b, ub)
    ib = P.lm_batch_iterate(b, ub, 8)
    for i, sh in enumerate(SHAPES):
        ctx = P.lm_init(Fs[i], Ms[i], params)
        u = torch.zeros((3,) + sh, device="cuda")
        P.lm_reset(ctx, u)
        info = P.lm_iterate(ctx, u, 8)
        assert info.loss == ib[i].loss and info.lambda_ == ib[i].lambda_
        assert torch.equal(u, ub[i]), i


def test_batch_rejection_loop_matches_single_pairs(P):
    """Eq. rejection in a batch: each graph replay runs every pair's own
    next attempt (the retry of a rejected trial or its next iteration),
    pairs that have finished their iterations sit the replays out, and each
    pair ends bitwise where a context of its own stepping through lm_step
    (every attempt launched) ends."""
    import torch
    Fs, Ms = _pairs(seed0=120)
    params = P.lm_default_params(lambda0=1e-3, step=3.0, reject=1, tau=1.0,
                                 lambda_max=1.0, max_retries=3)
    b = P.lm_batch_init(Fs, Ms, params)
    ub = [torch.zeros((3,) + sh, device="cuda") for sh in SHAPES]
    P.lm_batch_reset(b, ub)
    ib = P.lm_batch_iterate(b, ub, 6)
    retried = False
    for i, sh in enumerate(SHAPES):
        ctx = P.lm_init(Fs[i], Ms[i], params)
        u = torch.zeros((3,) + sh, device="cuda")
        P.lm_reset(ctx, u)
        for _ in range(6):
            info = P.lm_step(ctx, u)
        retried = retried or any(r["retries"] > 0 for r in P.lm_get_log(ctx))
        assert info.loss == ib[i].loss and info.lambda_ == ib[i].lambda_
        assert info.retries == ib[i].retries
        assert torch.equal(u, ub[i]), i
        P.lm_destroy(ctx)
    assert retried
    P.lm_batch_destroy(b)
