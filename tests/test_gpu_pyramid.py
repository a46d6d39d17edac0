"""GPU parity of the coarse-to-fine pyramid (Section 2.1) at the per-iteration
bars: every level image against the oracle's downsampling, the loss each
level starts from, one step per level through lm_register, and the
160x192x224 Voronoi schedule (levels 4 / 2 / 1) teacher-forced on a few
iterations of every level, each level starting from the GPU's carried field.

Bars: max |u_gpu - u_oracle| <= 1e-4 voxel (of the level), relative loss
<= 1e-5, the same accept / reject decision and damping.
"""
import numpy as np
import pytest

from parity_helpers import (TOL_L, TOL_U, _oracle_params, _t,
                            _teacher_forced, _worst)

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


@pytest.mark.parametrize("shape", [(40, 44, 48), (25, 21, 29), (5, 6, 7),
                                   (3, 9, 2)])
@pytest.mark.parametrize("f", [2, 4])
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_downsample_matches_oracle(P, oracle_mod, shape, f, dtype):
    """Every level voxel against the oracle's blur-and-sample (C16)."""
    import torch
    rng = np.random.default_rng(sum(shape) + f)
    X = rng.random(shape).astype(np.float32)
    Xt = _t(X)
    if dtype == "bf16":
        Xt = Xt.to(torch.bfloat16)
    Xo = Xt.float().cpu().numpy().astype(np.float64)
    Y = P.lm_downsample(Xt, f)
    torch.cuda.synchronize()
    ref = oracle_mod.downsample(Xo, f)
    assert tuple(Y.shape) == ref.shape == oracle_mod.level_dims(shape, f)
    got = Y.float().cpu().numpy().astype(np.float64)
    err = np.abs(got - ref)
    if dtype == "f32":
        # FP32 blur (three passes of at most 13 taps) and trilinear read
        assert err.max() <= 2e-6 * max(1.0, np.abs(ref).max()), _worst(err)
    else:
        # one BF16 rounding of the FP32 level value (8 significant bits)
        assert (err <= 2.0 ** -8 * np.abs(ref) + 2e-6).all(), _worst(err)


def _levels_oracle(oracle_mod, F, M, u0, factors):
    """Per level the oracle's level images and the carried start field."""
    out = []
    cur, cf = u0, 1
    for f in factors:
        Fl = F if f == 1 else oracle_mod.downsample(F, f)
        Ml = M if f == 1 else oracle_mod.downsample(M, f)
        ul = cur if f == cf else oracle_mod.resample_field(cur, cf, Fl.shape, f)
        out.append((Fl, Ml, ul))
        cur, cf = ul, f
    return out


@pytest.mark.parametrize("kind", ["lncc", "mse", "lncc_bf16"])
def test_register_level_start_losses(P, oracle_mod, kind):
    """Schedule (4, 0), (2, 0), (1, 0) from a non-zero field: each level's
    loss is the loss of the level images at the carried field, which pins
    the downsampled images and the field resampling through the loss; the
    field comes back through the chain 1 -> 4 -> 2 -> 1."""
    import torch
    import synth
    shape = (40, 44, 48)
    F, M, _ = synth.blob_pair(shape, seed=17, max_disp=2.0)
    kw = dict(lambda0=0.006, step=1.0)
    if kind == "mse":
        kw["loss"] = P.LM_LOSS_MSE
    params = P.lm_default_params(**kw)
    Ft, Mt = _t(F), _t(M)
    if kind == "lncc_bf16":
        Ft, Mt = Ft.to(torch.bfloat16), Mt.to(torch.bfloat16)
    Fo = Ft.float().cpu().numpy().astype(np.float64)
    Mo = Mt.float().cpu().numpy().astype(np.float64)
    u0 = synth.random_field(shape, seed=8, scale=1.5)
    ctx = P.lm_init(Ft, Mt, params)
    u = _t(u0)
    rep = P.lm_register(ctx, [(4, 0), (2, 0), (1, 0)], u)
    Po = _oracle_params(oracle_mod, params)
    levels = _levels_oracle(oracle_mod, Fo, Mo, u0.astype(np.float64),
                            [4, 2, 1])
    if kind == "lncc_bf16":
        # BF16 storage holds every level image in BF16 too: the oracle gets
        # the level images rounded as the library stores them
        def bf(X):
            return torch.from_numpy(X).to(torch.bfloat16).double().numpy()
        levels = [(bf(Fl), bf(Ml), ul) if Fl.shape != Fo.shape
                  else (Fl, Ml, ul) for Fl, Ml, ul in levels]
    for l, (Fl, Ml, ul) in enumerate(levels):
        assert tuple(rep.level_dims[l]) == Fl.shape
        L = oracle_mod.loss(Fl, Ml, ul, Po)
        assert abs(rep.level_loss[l] - L) <= TOL_L * L, (l, rep.level_loss[l],
                                                          L)
        assert rep.level_iters[l] == 0
    err = np.abs(u.cpu().numpy().astype(np.float64) - levels[-1][2])
    assert err.max() <= TOL_U, _worst(err)
    P.lm_destroy(ctx)


@pytest.mark.parametrize("kind", ["lncc", "mse"])
def test_register_one_step_per_level(P, oracle_mod, kind):
    """Schedule (4, 1), (2, 1), (1, 1) from zero through lm_register against
    the oracle's coarse-to-fine run: the loss at the end of every level and
    the final field."""
    import torch
    import synth
    shape = (40, 44, 48)
    F, M, _ = synth.blob_pair(shape, seed=19, max_disp=2.0)
    kw = dict(lambda0=0.006, step=1.0)
    if kind == "mse":
        kw["loss"] = P.LM_LOSS_MSE
    params = P.lm_default_params(**kw)
    ctx = P.lm_init(_t(F), _t(M), params)
    u = torch.zeros((3,) + shape, device="cuda")
    rep = P.lm_register(ctx, [(4, 1), (2, 1), (1, 1)], u)
    uo, log, evals = oracle_mod.register(
        F.astype(np.float64), M.astype(np.float64),
        _oracle_params(oracle_mod, params), [4, 2, 1], [1, 1, 1])
    assert evals == sum(rep.level_evals[:3])
    for l in range(3):
        assert abs(rep.level_loss[l] - log[l]) <= TOL_L * log[l], (
            l, rep.level_loss[l], log[l])
    err = np.abs(u.cpu().numpy().astype(np.float64) - uo)
    assert err.max() <= TOL_U, _worst(err)
    P.lm_destroy(ctx)


def _level_images(P, oracle_mod, F, M, f):
    """Device level images as lm_register builds them and the oracle's own
    level images (each side downsamples independently)."""
    import torch
    Ft, Mt = _t(F), _t(M)
    if f == 1:
        return Ft, Mt, F.astype(np.float64), M.astype(np.float64)
    Fl, Ml = P.lm_downsample(Ft, f), P.lm_downsample(Mt, f)
    torch.cuda.synchronize()
    return (Fl, Ml, oracle_mod.downsample(F.astype(np.float64), f),
            oracle_mod.downsample(M.astype(np.float64), f))


def _schedule_teacher_forced(P, oracle_mod, F, M, params, plan):
    """plan: [(factor, iterations)].  Each level's context runs on the GPU's
    level images; its first field is the GPU's field of the previous level
    carried by lm_field_resample (zero at the first level); every iteration
    is checked against the oracle stepping from the GPU's state on the
    oracle's own level images."""
    import torch
    cur, cf = None, None
    for f, n in plan:
        Ft, Mt, Fo, Mo = _level_images(P, oracle_mod, F, M, f)
        lshape = tuple(Ft.shape)
        if cur is None:
            u = torch.zeros((3,) + lshape, device="cuda")
        elif cf == f:
            u = cur
        else:
            u = torch.empty((3,) + lshape, device="cuda")
            P.lm_field_resample(cur, cf, u, f)
            torch.cuda.synchronize()
        dec, u = _teacher_forced(P, oracle_mod, None, None, params, n,
                                 images=(Ft, Mt, Fo, Mo), u0_dev=u,
                                 keep=True)
        assert all(a == 1 for a, _ in dec) or params.reject
        cur, cf = u, f


def test_blob_schedule_teacher_forced(P, oracle_mod):
    """A 48 x 40 x 56 blob pair on levels 4 / 2 / 1, six iterations each."""
    import synth
    F, M, _ = synth.blob_pair((48, 40, 56), seed=23, max_disp=3.0)
    params = P.lm_default_params(lambda0=0.006, step=1.0)
    _schedule_teacher_forced(P, oracle_mod, F, M, params,
                             [(4, 6), (2, 6), (1, 6)])


def test_voronoi_schedule_teacher_forced_full_size(P, oracle_mod):
    """The 160x192x224 Voronoi workload (k = 5, levels 4 / 2 / 1, the
    default damping): five iterations at 40x48x56, four at 80x96x112 and
    two at full resolution, every one teacher-forced."""
    import synth
    F, M, _ = synth.voronoi_pair((160, 192, 224), seed=0)
    params = P.lm_default_params()
    _schedule_teacher_forced(P, oracle_mod, F, M, params,
                             [(4, 5), (2, 4), (1, 2)])
