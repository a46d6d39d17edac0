"""Helpers shared by the GPU parity tests: device tensors from numpy, the
oracle's parameter block from the library's, and the teacher-forced
iteration check (both sides step from the GPU's FP32 state; per iteration
max |u_gpu - u_oracle| <= 1e-4 voxel, relative loss <= 1e-5, the same
accept / reject decision and damping, near-ties reported)."""
import numpy as np
import pytest

TOL_U = 1e-4        # voxels
TOL_L = 1e-5        # relative
TOL_G = 1e-4        # relative to gmax


def _t(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def _oracle_params(oracle, p):
    return oracle.params(win=p.win, eps_nr=float(np.float32(p.eps_nr)),
                         eps_dr=float(np.float32(p.eps_dr)),
                         sigma_grad=float(p.sigma_grad),
                         sigma_warp=float(p.sigma_warp), step=float(p.step),
                         lambda0=p.lambda0, mu_inc=p.mu_inc, mu_dec=p.mu_dec,
                         lambda_max=p.lambda_max, reject=p.reject, tau=p.tau,
                         max_retries=p.max_retries, tile=p.tile,
                         loss=p.loss, method=p.method,
                         alpha=float(np.float32(p.alpha)), bins=p.bins)


def _images(F, M, dtype):
    """Device images and the exact values the oracle must see."""
    import torch
    if dtype == "bf16":
        Ft, Mt = _t(F, torch.bfloat16), _t(M, torch.bfloat16)
        return Ft, Mt, Ft.float().cpu().numpy(), Mt.float().cpu().numpy()
    return _t(F), _t(M), F.astype(np.float64), M.astype(np.float64)


def _worst(err):
    idx = np.unravel_index(int(np.argmax(err)), err.shape)
    return f"max err {float(err[idx]):.3e} at {tuple(int(i) for i in idx)}"


def _teacher_forced(P, oracle_mod, F, M, params, iters, dtype="f32",
                    u0=None, use_iterate=False, tol_u=TOL_U, images=None,
                    u0_dev=None, keep=False):
    """Run the GPU iteration and check every step against the oracle.

    images: (Ft, Mt, Fo, Mo) to use instead of F, M (the device images and
    the values the oracle sees); u0_dev: the initial field as a device
    tensor; keep: return (decisions, u) with the final device field."""
    import torch
    Ft, Mt, Fo, Mo = _images(F, M, dtype) if images is None else images
    Po = _oracle_params(oracle_mod, params)
    ctx = P.lm_init(Ft, Mt, params)
    shape = tuple(Ft.shape)
    if u0_dev is not None:
        u = u0_dev
    else:
        u = torch.zeros((3,) + shape, device="cuda") if u0 is None else _t(u0)
    P.lm_reset(ctx, u)
    near_ties = 0
    decisions = []
    for t in range(iters):
        st = P.lm_get_state(ctx)
        ut = u.cpu().numpy().astype(np.float64)
        ev = oracle_mod.evaluate(Fo, Mo, ut, Po)
        assert abs(st.loss - ev["L"]) <= TOL_L * ev["L"] + 1e-12, (t, st.loss,
                                                                  ev["L"])
        u1, _ = oracle_mod.trial(ut, ev["g"], ev["gmax"], ev["L"], st.lambda_,
                                 Po)
        L1 = oracle_mod.loss(Fo, Mo, u1, Po)
        act, lam_o = oracle_mod.decide(L1, ev["L"], st.loss_prev, st.has_prev,
                                       st.lambda_, 0, Po)
        if Po.method == oracle_mod.DEMONS:   # every step kept, lambda unused
            act, lam_o = oracle_mod.ACCEPT, st.lambda_
        info = (P.lm_iterate(ctx, u, 1) if use_iterate
                else P.lm_step(ctx, u))
        assert abs(info.loss_first - L1) <= TOL_L * L1 + 1e-12, (t, info.loss_first, L1)
        # decision of the first trial
        margin = abs((L1 - ev["L"]) - (Po.tau * abs(ev["L"] - st.loss_prev)
                                        if (Po.reject and st.has_prev) else 0.0))
        tie = margin < 1e-6 * ev["L"]
        first_rejected = info.retries > 0 or info.accepted == 0
        if tie:
            near_ties += 1
        else:
            assert first_rejected == (act != oracle_mod.ACCEPT), t
        if info.retries == 0 and info.accepted == 1 and not tie:
            assert info.lambda_ == pytest.approx(lam_o, rel=1e-12), t
            err = np.abs(u.cpu().numpy().astype(np.float64) - u1)
            assert err.max() <= tol_u, (t, _worst(err), st.lambda_, ev["L"])
        decisions.append((info.accepted, info.retries))
    P.lm_destroy(ctx)
    # near-ties are listed, not hidden (their decision is not compared)
    print(f"teacher-forced {iters} iterations: {near_ties} near-ties")
    assert near_ties <= max(1, iters // 10), near_ties
    return (decisions, u) if keep else decisions
