"""Pins for the oracle's damping / rejection control (Eq. lambda-update,
Eq. rejection) and for the LM iteration built on it."""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden",
                      "damping_traces.json")


def _golden_cases():
    with open(GOLDEN) as f:
        doc = json.load(f)
    for s in doc["sets"]:
        for i, c in enumerate(s["cases"]):
            yield pytest.param(s["params"], c, id=f"{s['name'][:24]}-{i}")


@pytest.mark.parametrize("params,case", list(_golden_cases()))
def test_decide_scripted_traces(oracle_mod, params, case):
    kw = {k: (math.inf if v == "inf" else v) for k, v in params.items()}
    P = oracle_mod.params(**kw)
    act, lam = oracle_mod.decide(*case["in"], P)
    names = {0: "ACCEPT", 1: "RETRY", 2: "DISCARD"}
    assert names[act] == case["action"], case["why"]
    assert lam == pytest.approx(case["lambda"], rel=1e-15), case["why"]


def _pair(seed=0, n=10):
    rng = np.random.default_rng(seed)
    from scipy import ndimage
    F = ndimage.gaussian_filter(rng.random((n, n, n)), 1.0)
    M = ndimage.gaussian_filter(rng.random((n, n, n)), 1.0)
    return F, M


def test_step_without_rejection_always_accepts(oracle_mod):
    F, M = _pair(1)
    P = oracle_mod.params(lambda0=0.5)
    st = oracle_mod.State(F, M, np.zeros((3,) + F.shape), P)
    for _ in range(4):
        L0, lam0 = st.L, st.lam
        info = oracle_mod.lm_step(st)
        assert info["accepted"] == 1 and info["evals"] == 1
        np.testing.assert_array_equal(st.u, info["u_first"])
        assert st.L == info["L_first"]
        assert st.L_prev == L0 and st.has_prev == 1
        want = lam0 * (1.5 if st.L > L0 else 0.975)
        assert st.lam == pytest.approx(want, rel=1e-15)


def test_step_rejection_invariants(oracle_mod):
    F, M = _pair(2)
    rng = np.random.default_rng(3)
    u0 = rng.uniform(-1.5, 1.5, (3,) + F.shape)
    P = oracle_mod.params(lambda0=1e-4, step=4.0, reject=1, tau=1.0,
                          lambda_max=1.0, max_retries=3)
    st = oracle_mod.State(F, M, u0, P)
    saw_retry = False
    for _ in range(6):
        u_before, L_before, lam_before = st.u.copy(), st.L, st.lam
        Lp_before, hp_before = st.L_prev, st.has_prev
        info = oracle_mod.lm_step(st)
        assert info["evals"] == info["retries"] + 1
        saw_retry |= info["retries"] > 0
        if info["accepted"]:
            if hp_before:
                assert st.L - L_before <= P.tau * abs(L_before - Lp_before)
            else:
                assert st.L <= L_before
        else:
            assert info["retries"] == P.max_retries
            np.testing.assert_array_equal(st.u, u_before)
            assert st.L == L_before and st.L_prev == Lp_before
            want = min(lam_before * 1.5 ** (P.max_retries + 1), 1.0)
            assert st.lam == pytest.approx(want, rel=1e-12)
    assert saw_retry


def test_register_single_level_equals_manual_steps(oracle_mod):
    F, M = _pair(4, 8)
    P = oracle_mod.params(lambda0=0.3)
    u, log, evals = oracle_mod.register(F, M, P, [1], [3])
    st = oracle_mod.State(F, M, np.zeros((3,) + F.shape), P)
    losses = []
    for _ in range(3):
        oracle_mod.lm_step(st)
        losses.append(st.L)
    np.testing.assert_array_equal(u, st.u)
    np.testing.assert_array_equal(log, losses)
    assert evals == 4
