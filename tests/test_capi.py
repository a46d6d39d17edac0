"""C ABI checks that need no GPU: the library loads, exports every symbol
declared in include/*.h, and validates arguments on the host before any
CUDA call."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h)
           for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2603_19371_gb300 import build, lmreg
    build.build()
    return lmreg.load()


def _declared():
    names = set()
    for h in HEADERS:
        with open(h) as f:
            names |= set(re.findall(r"LM_API\s+[\w\s\*]*?\b(lm_\w+)\s*\(",
                                    f.read()))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("lm_init", "lm_step", "lm_register", "lm_destroy",
              "lm_strerror", "lm_state_save", "lm_state_load",
              "lm_register_batch", "lm_unet_create", "lm_unet_forward",
              "lm_unet_train_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2603_19371_gb300 import lmreg
    assert sorted(lmreg.EXPORTED) == _declared()


def test_default_params_match_the_paper(lib):
    from paper_2603_19371_gb300 import lmreg
    p = lmreg.lm_default_params()
    # Section 3: lambda0 = 0.006, mu+ = 1.5, mu- = 0.975; Section 3.4: tau 1,
    # 10 retries, rejection off by default
    assert p.lambda0 == pytest.approx(0.006)
    assert p.mu_inc == 1.5 and p.mu_dec == pytest.approx(0.975)
    assert p.reject == 0 and p.tau == 1.0 and p.max_retries == 10
    assert math.isinf(p.lambda_max) and p.win == 5
    # Section 3: tile_size 1 (the pointwise step of Eq. tile1)
    assert p.tile == 1
    assert p.loss == lmreg.LM_LOSS_LNCC and p.method == lmreg.LM_METHOD_LM
    assert p.alpha == 1.0 and p.bins == 32
    with pytest.raises(KeyError):
        lmreg.lm_default_params(tile_size=2)


def test_strerror(lib):
    from paper_2603_19371_gb300 import lmreg
    assert lmreg.lm_strerror(0) == "ok"
    assert "invalid" in lmreg.lm_strerror(-1)
    assert lmreg.lm_strerror(-99) == "unknown error"


def _init(lib, fixed, moving, params=None):
    from paper_2603_19371_gb300 import lmreg
    h = ctypes.c_void_p()
    p = ctypes.byref(params) if params is not None else None
    rc = lib.lm_init(ctypes.byref(h), ctypes.byref(fixed),
                     ctypes.byref(moving), p, None)
    return rc, lmreg.lm_last_error()


def test_init_rejects_bad_arguments_on_host(lib):
    from paper_2603_19371_gb300 import lmreg
    V = lmreg.Volume
    ok = V(4, 4, 4, lmreg.LM_F32, 0x1000)
    rc, msg = _init(lib, V(0, 4, 4, lmreg.LM_F32, 0x1000), ok)
    assert rc == lmreg.LM_EINVAL and "dimension" in msg
    rc, msg = _init(lib, ok, V(4, 4, 5, lmreg.LM_F32, 0x1000))
    assert rc == lmreg.LM_EINVAL and "shapes differ" in msg
    rc, msg = _init(lib, ok, V(4, 4, 4, lmreg.LM_BF16, 0x1000))
    assert rc == lmreg.LM_EINVAL and "dtypes differ" in msg
    rc, msg = _init(lib, V(4, 4, 4, 7, 0x1000), ok)
    assert rc == lmreg.LM_EINVAL and "dtype" in msg
    rc, msg = _init(lib, V(4, 4, 4, lmreg.LM_F32, 0), ok)
    assert rc == lmreg.LM_EINVAL and "NULL" in msg
    for field, val, word in [("win", 4, "win"), ("win", 11, "win"),
                             ("mu_inc", 1.0, "mu_inc"),
                             ("mu_dec", 1.0, "mu_dec"),
                             ("lambda0", 0.0, "lambda0"),
                             ("sigma_grad", 3.0, "sigma"),
                             ("step", float("nan"), "step"),
                             ("max_retries", 99, "max_retries"),
                             ("lambda_max", 1e-9, "lambda_max"),
                             ("tile", 0, "tile"), ("tile", 17, "tile"),
                             ("loss", 3, "loss"), ("method", 5, "method"),
                             ("alpha", 0.0, "alpha"), ("bins", 3, "bins"),
                             ("bins", 65, "bins")]:
        p = lmreg.lm_default_params()
        setattr(p, field, val)
        rc, msg = _init(lib, ok, ok, p)
        assert rc == lmreg.LM_EINVAL and word in msg, (field, msg)


def test_null_arguments(lib):
    from paper_2603_19371_gb300 import lmreg
    assert lib.lm_default_params(None) == lmreg.LM_EINVAL
    assert lib.lm_step(None, None, None) == lmreg.LM_EINVAL
    assert lib.lm_register(None, None, None, None) == lmreg.LM_EINVAL
    n = ctypes.c_int(-1)
    assert lib.lm_get_log(None, None, 0, ctypes.byref(n)) == lmreg.LM_EINVAL
    assert lib.lm_debug_check(None) == lmreg.LM_EINVAL
    assert lib.lm_batch_debug_check(None) == lmreg.LM_EINVAL
    lib.lm_destroy(None)


def test_failure_codes_have_messages(lib):
    from paper_2603_19371_gb300 import lmreg
    assert "timed out" in lmreg.lm_strerror(lmreg.LM_ETIMEOUT)
    assert "outside" in lmreg.lm_strerror(lmreg.LM_EBOUNDS)
    assert "finite" in lmreg.lm_strerror(lmreg.LM_ENONFINITE)
    with open(os.path.join(ROOT, "include", "lmreg.h")) as f:
        h = f.read()
    assert re.search(r"#define LM_EBOUNDS\s+-8\b", h)
    assert re.search(r"#define LM_LOG_CAP 8192\b", h)


def test_unet_shapes_match_the_oracle(lib):
    from oracle import unet as U
    from paper_2603_19371_gb300 import lmreg
    shapes, n = lmreg.lm_unet_shapes()
    assert shapes == [(ci, co) for ci, co, _ in U.LAYERS]
    assert n == sum(27 * ci * co + co for ci, co, _ in U.LAYERS)


def test_unet_create_validates_sizes_on_the_host(lib):
    from paper_2603_19371_gb300 import lmreg
    h = ctypes.c_void_p()
    w = (ctypes.c_float * 4)()
    # not a multiple of 8
    assert lib.lm_unet_create(ctypes.byref(h), 12, 16, 16, w, None) == lmreg.LM_EINVAL
    # no weights
    assert lib.lm_unet_create(ctypes.byref(h), 16, 16, 16, None, None) == lmreg.LM_EINVAL
    assert not h.value
    # unsupported convolution shapes fail before any CUDA call
    assert lib.lm_conv3d_forward(4, 4, 4, 3, 16, w, w, None, 0, w, None) == lmreg.LM_EINVAL
    assert lib.lm_conv3d_forward(4, 4, 4, 16, 8, w, w, None, 0, w, None) == lmreg.LM_EINVAL
    # tensor inspection without a network
    assert lib.lm_unet_get_tensor(None, 0, None, None, None) == lmreg.LM_EINVAL


def test_unet_tensor_names_follow_the_header(lib):
    """The binding's tensor names are the header's LM_UNET_* enum, in order."""
    from paper_2603_19371_gb300 import lmreg
    with open(os.path.join(ROOT, "include", "lmunet.h")) as f:
        h = f.read()
    body = h[h.index("LM_UNET_X0"):h.index("LM_UNET_NTENSORS")]
    names = re.findall(r"LM_UNET_(\w+)", body)
    assert [n.lower() for n in names] == list(lmreg.UNET_TENSORS)


def test_noalloc_validates_on_the_host(lib):
    """lm_eval_noalloc checks its parameters with lm_init's rules and refuses
    pointers that are not device memory before any launch (on a machine
    without a GPU no pointer is device memory)."""
    from paper_2603_19371_gb300 import lmreg
    V = lmreg.Volume
    buf = (ctypes.c_float * 64)()
    addr = ctypes.addressof(buf)
    vol = V(4, 4, 4, lmreg.LM_F32, addr)
    p = lmreg.lm_default_params()
    p.eps_nr = float("inf")
    rc = lib.lm_eval_noalloc(ctypes.byref(vol), ctypes.byref(vol),
                             ctypes.byref(p), ctypes.c_void_p(addr),
                             ctypes.c_void_p(addr), None, None, None)
    assert rc == lmreg.LM_EINVAL and "eps" in lmreg.lm_last_error()
    rc = lib.lm_eval_noalloc(ctypes.byref(vol), ctypes.byref(vol), None,
                             ctypes.c_void_p(addr), ctypes.c_void_p(addr),
                             None, None, None)
    assert rc == lmreg.LM_EINVAL
    assert "device pointer" in lmreg.lm_last_error()
