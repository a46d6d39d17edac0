"""Python binding of the C ABI in include/lmreg.h (argument marshalling only).

Every computation runs in liblmreg.so's CUDA kernels; this module only turns
torch tensors into device pointers and C structs into Python values.  If the
library is missing the import of a function raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# LMREG_LIBRARY selects another build of the same ABI (the debug-bounds
# liblmreg_dbg.so); it is read once, at import
LIB_PATH = os.environ.get("LMREG_LIBRARY") or os.path.join(HERE, "liblmreg.so")

LM_OK, LM_EINVAL, LM_ENOMEM, LM_ECUDA = 0, -1, -2, -3
LM_ENONFINITE, LM_ETIMEOUT, LM_EUNSUPPORTED, LM_ESTATE = -4, -5, -6, -7
LM_EBOUNDS = -8
LM_F32, LM_BF16 = 0, 1
LM_LOSS_LNCC, LM_LOSS_MSE, LM_LOSS_MI = 0, 1, 2
LM_METHOD_LM, LM_METHOD_DEMONS = 0, 1
LM_MAX_LEVELS = 4
LM_NOALLOC_MAX_VOXELS = 1 << 19
LM_E1_TILE_32X16, LM_E1_TILE_32X32 = 0, 1


class LMError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__(f"{fn} failed ({code}: {msg})")
        self.code = code


class Volume(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("dtype", ctypes.c_int), ("data", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("win", ctypes.c_int), ("eps_nr", ctypes.c_float),
                ("eps_dr", ctypes.c_float), ("sigma_grad", ctypes.c_float),
                ("sigma_warp", ctypes.c_float), ("step", ctypes.c_float),
                ("lambda0", ctypes.c_double), ("mu_inc", ctypes.c_double),
                ("mu_dec", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("reject", ctypes.c_int), ("tau", ctypes.c_double),
                ("max_retries", ctypes.c_int), ("tile", ctypes.c_int),
                ("loss", ctypes.c_int), ("method", ctypes.c_int),
                ("alpha", ctypes.c_float), ("bins", ctypes.c_int)]


class Schedule(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int),
                ("factor", ctypes.c_int * LM_MAX_LEVELS),
                ("iters", ctypes.c_int * LM_MAX_LEVELS)]


class StepInfo(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_double), ("loss_first", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("gmax", ctypes.c_float),
                ("accepted", ctypes.c_int), ("retries", ctypes.c_int),
                ("evals", ctypes.c_int), ("stopped", ctypes.c_int)]


class State(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_double), ("loss_prev", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("gmax", ctypes.c_float),
                ("has_prev", ctypes.c_int), ("iter", ctypes.c_int),
                ("evals", ctypes.c_int), ("kernel_launches", ctypes.c_longlong)]


class LogEntry(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("gmax", ctypes.c_float), ("accepted", ctypes.c_int),
                ("retries", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int),
                ("level_dims", (ctypes.c_int * 3) * LM_MAX_LEVELS),
                ("level_iters", ctypes.c_int * LM_MAX_LEVELS),
                ("level_evals", ctypes.c_int * LM_MAX_LEVELS),
                ("level_accepted", ctypes.c_int * LM_MAX_LEVELS),
                ("level_loss", ctypes.c_double * LM_MAX_LEVELS),
                ("final_loss", ctypes.c_double),
                ("voxel_evals", ctypes.c_longlong),
                ("wall_ms", ctypes.c_double)]


_lib = None


def load():
    """Load liblmreg.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build()"
                          " (the CUDA library has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    V, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "lm_default_params": [ctypes.POINTER(Params)],
        "lm_init": [ctypes.POINTER(V), ctypes.POINTER(Volume),
                    ctypes.POINTER(Volume), ctypes.POINTER(Params), V],
        "lm_eval": [V, V, ctypes.POINTER(D), V, ctypes.POINTER(ctypes.c_float)],
        "lm_reset": [V, V],
        "lm_step": [V, V, ctypes.POINTER(StepInfo)],
        "lm_iterate": [V, V, I, ctypes.POINTER(StepInfo)],
        "lm_get_state": [V, ctypes.POINTER(State)],
        "lm_set_state": [V, ctypes.POINTER(State)],
        "lm_register": [V, ctypes.POINTER(Schedule), V,
                        ctypes.POINTER(Report)],
        "lm_state_save": [V, V, ctypes.POINTER(ctypes.c_size_t)],
        "lm_state_load": [V, V, ctypes.c_size_t],
        "lm_time_passes": [V, V, I, ctypes.POINTER(D), ctypes.POINTER(D)],
        "lm_eval_noalloc": [ctypes.POINTER(Volume), ctypes.POINTER(Volume),
                            ctypes.POINTER(Params), V, V, V, V, V],
        "lm_batch_init": [ctypes.POINTER(V), I, ctypes.POINTER(Volume),
                          ctypes.POINTER(Volume), ctypes.POINTER(Params), V],
        "lm_batch_eval": [V, ctypes.POINTER(V), ctypes.POINTER(V),
                          ctypes.POINTER(D), ctypes.POINTER(ctypes.c_float)],
        "lm_batch_reset": [V, ctypes.POINTER(V)],
        "lm_batch_iterate": [V, ctypes.POINTER(V), I,
                             ctypes.POINTER(StepInfo)],
        "lm_batch_set_targets": [V, ctypes.POINTER(D)],
        "lm_field_resample": [V, I, I, I, I, V, I, I, I, I, V],
        "lm_downsample": [ctypes.POINTER(Volume), I, V, V, ctypes.POINTER(I),
                          V],
        "lm_batch_autotune": [V, ctypes.POINTER(V), I, ctypes.POINTER(I),
                              ctypes.POINTER(I), ctypes.POINTER(I),
                              ctypes.POINTER(D)],
        "lm_autotune": [V, V, I, ctypes.POINTER(I), ctypes.POINTER(I),
                        ctypes.POINTER(I), ctypes.POINTER(D)],
        "lm_batch_register": [V, ctypes.POINTER(Schedule), ctypes.POINTER(V),
                              ctypes.POINTER(Report)],
        "lm_register_batch": [I, ctypes.POINTER(Volume), ctypes.POINTER(Volume),
                              ctypes.POINTER(V), ctypes.POINTER(Params),
                              ctypes.POINTER(Schedule), V,
                              ctypes.POINTER(Report)],
        "lm_unet_shapes": [ctypes.POINTER(I), ctypes.POINTER(I),
                           ctypes.POINTER(ctypes.c_longlong)],
        "lm_unet_create": [ctypes.POINTER(V), I, I, I, V, V],
        "lm_unet_forward": [V, ctypes.POINTER(Volume), ctypes.POINTER(Volume), V],
        "lm_unet_train_step": [V, I, ctypes.POINTER(Volume),
                               ctypes.POINTER(Volume), ctypes.POINTER(V),
                               ctypes.c_float, ctypes.POINTER(D)],
        "lm_unet_get_weights": [V, V],
        "lm_unet_get_grads": [V, V],
        "lm_unet_get_tensor": [V, I, V, ctypes.POINTER(I), ctypes.POINTER(I)],
        "lm_conv3d_forward": [I, I, I, I, I, V, V, V, I, V, V],
        "lm_conv3d_backward": [I, I, I, I, I, V, V, V, V, V, V, V],
        "lm_debug_check": [V],
        "lm_get_log": [V, V, I, ctypes.POINTER(I)],
        "lm_batch_debug_check": [V],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = I
    lib.lm_destroy.argtypes = [V]
    lib.lm_destroy.restype = None
    lib.lm_batch_destroy.argtypes = [V]
    lib.lm_batch_destroy.restype = None
    lib.lm_unet_destroy.argtypes = [V]
    lib.lm_unet_destroy.restype = None
    lib.lm_strerror.argtypes = [I]
    lib.lm_strerror.restype = ctypes.c_char_p
    lib.lm_last_error.argtypes = []
    lib.lm_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(rc, fn):
    if rc != LM_OK:
        lib = load()
        msg = lib.lm_last_error().decode() or lib.lm_strerror(rc).decode()
        raise LMError(rc, fn, msg)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _volume(t):
    import torch
    if not t.is_cuda or not t.is_contiguous() or t.dim() != 3:
        raise ValueError("images must be contiguous 3-D CUDA tensors")
    if t.dtype == torch.float32:
        dt = LM_F32
    elif t.dtype == torch.bfloat16:
        dt = LM_BF16
    else:
        raise ValueError("images must be float32 or bfloat16")
    D, H, W = t.shape
    return Volume(D, H, W, dt, t.data_ptr())


def _field_ptr(u, shape=None):
    import torch
    if (not u.is_cuda or u.dtype != torch.float32 or not u.is_contiguous()
            or u.dim() != 4 or u.shape[0] != 3):
        raise ValueError("fields must be contiguous float32 CUDA tensors of "
                         "shape (3, D, H, W)")
    if shape is not None and tuple(u.shape[1:]) != tuple(shape):
        raise ValueError(f"field shape {tuple(u.shape)} does not match the "
                         f"images {tuple(shape)}")
    return ctypes.c_void_p(u.data_ptr())


class Context:
    """Owns an lm_ctx handle and keeps its images alive."""

    def __init__(self, handle, fixed, moving, stream):
        self.handle = handle
        self.fixed, self.moving = fixed, moving
        self.shape = tuple(fixed.shape)
        self.stream = stream

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.lm_destroy(h)


def lm_default_params(**overrides) -> Params:
    p = Params()
    _check(load().lm_default_params(ctypes.byref(p)), "lm_default_params")
    names = {f[0] for f in Params._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise KeyError(f"lm_params has no field {k!r}")
        setattr(p, k, math.inf if v is None and k == "lambda_max" else v)
    return p


def lm_init(fixed, moving, params: Params | None = None, stream=None):
    lib = load()
    vf, vm = _volume(fixed), _volume(moving)
    h = ctypes.c_void_p()
    p = ctypes.byref(params) if params is not None else None
    _check(lib.lm_init(ctypes.byref(h), ctypes.byref(vf), ctypes.byref(vm), p,
                       _stream_handle(stream)), "lm_init")
    return Context(h, fixed, moving, stream)


def lm_destroy(ctx: Context):
    h, ctx.handle = ctx.handle, None
    if h:
        load().lm_destroy(h)


def lm_get_log(ctx: Context):
    """The iteration log since the last lm_reset, oldest first: a list of
    dicts (loss, lambda, gmax, accepted, retries)."""
    n = ctypes.c_int()
    _check(load().lm_get_log(ctx.handle, None, 0, ctypes.byref(n)),
           "lm_get_log")
    buf = (LogEntry * max(n.value, 1))()
    _check(load().lm_get_log(ctx.handle, buf, n.value, ctypes.byref(n)),
           "lm_get_log")
    return [{"loss": e.loss, "lambda": e.lambda_, "gmax": e.gmax,
             "accepted": e.accepted, "retries": e.retries}
            for e in buf[:n.value]]


def lm_log_jsonl(ctx: Context, path):
    """Appends the iteration log to a JSON-lines file, one record a line."""
    import json
    with open(path, "a") as f:
        for i, r in enumerate(lm_get_log(ctx)):
            f.write(json.dumps(dict(r, iteration=i)) + "\n")


def lm_debug_check(ctx: Context):
    """Debug-bounds build: raises LMError (LM_EBOUNDS) if a kernel wrote
    into a guard band of the context's buffers."""
    _check(load().lm_debug_check(ctx.handle), "lm_debug_check")


def lm_eval(ctx: Context, u, g_out=None):
    """Returns (loss, gmax); fills g_out (3, D, H, W) when given."""
    L = ctypes.c_double()
    gm = ctypes.c_float()
    gp = _field_ptr(g_out, ctx.shape) if g_out is not None else None
    _check(load().lm_eval(ctx.handle, _field_ptr(u, ctx.shape),
                          ctypes.byref(L), gp, ctypes.byref(gm)), "lm_eval")
    return L.value, gm.value


def lm_reset(ctx: Context, u):
    _check(load().lm_reset(ctx.handle, _field_ptr(u, ctx.shape)), "lm_reset")


def lm_step(ctx: Context, u, info=True):
    si = StepInfo() if info else None
    _check(load().lm_step(ctx.handle, _field_ptr(u, ctx.shape),
                          ctypes.byref(si) if si is not None else None),
           "lm_step")
    return si


def lm_iterate(ctx: Context, u, n, info=True):
    si = StepInfo() if info else None
    _check(load().lm_iterate(ctx.handle, _field_ptr(u, ctx.shape), int(n),
                             ctypes.byref(si) if si is not None else None),
           "lm_iterate")
    return si


def lm_get_state(ctx: Context) -> State:
    s = State()
    _check(load().lm_get_state(ctx.handle, ctypes.byref(s)), "lm_get_state")
    return s


def lm_set_state(ctx: Context, s: State):
    _check(load().lm_set_state(ctx.handle, ctypes.byref(s)), "lm_set_state")


def lm_register(ctx: Context, levels, u) -> Report:
    """levels: sequence of (factor, iters)."""
    s = _schedule(levels)
    r = Report()
    _check(load().lm_register(ctx.handle, ctypes.byref(s),
                              _field_ptr(u, ctx.shape), ctypes.byref(r)),
           "lm_register")
    return r


def lm_state_save(ctx: Context) -> bytes:
    n = ctypes.c_size_t()
    _check(load().lm_state_save(ctx.handle, None, ctypes.byref(n)),
           "lm_state_save")
    buf = ctypes.create_string_buffer(n.value)
    _check(load().lm_state_save(ctx.handle, buf, ctypes.byref(n)),
           "lm_state_save")
    return buf.raw[:n.value]


def lm_state_load(ctx: Context, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    _check(load().lm_state_load(ctx.handle, buf, len(data)), "lm_state_load")


def lm_time_passes(ctx: Context, u, n):
    """Mean ms per launch of (pass 1 evaluation, pass 2 trial)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().lm_time_passes(ctx.handle, _field_ptr(u, ctx.shape), int(n),
                                 ctypes.byref(a), ctypes.byref(b)),
           "lm_time_passes")
    return a.value, b.value


class Batch:
    """Owns an lm_batch handle and keeps its images alive."""

    def __init__(self, handle, fixed, moving, stream):
        self.handle = handle
        self.fixed, self.moving = list(fixed), list(moving)
        self.shapes = [tuple(f.shape) for f in fixed]
        self.stream = stream

    def __len__(self):
        return len(self.shapes)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.lm_batch_destroy(h)


def _ptr_array(ts, shapes=None):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _field_ptr(t, shapes[i] if shapes else None).value
    return arr


def _schedule(levels):
    s = Schedule()
    s.nlevels = len(levels)
    for i, (f, it) in enumerate(levels):
        s.factor[i] = int(f)
        s.iters[i] = int(it)
    return s


def lm_batch_init(fixed, moving, params: Params | None = None, stream=None):
    vf = (Volume * len(fixed))(*[_volume(t) for t in fixed])
    vm = (Volume * len(moving))(*[_volume(t) for t in moving])
    h = ctypes.c_void_p()
    p = ctypes.byref(params) if params is not None else None
    _check(load().lm_batch_init(ctypes.byref(h), len(fixed), vf, vm, p,
                                _stream_handle(stream)), "lm_batch_init")
    return Batch(h, fixed, moving, stream)


def lm_batch_destroy(b: Batch):
    h, b.handle = b.handle, None
    if h:
        load().lm_batch_destroy(h)


def lm_batch_debug_check(b: Batch):
    _check(load().lm_batch_debug_check(b.handle), "lm_batch_debug_check")


def lm_batch_eval(b: Batch, us, g_outs=None):
    """Returns (losses, gmaxes) lists; fills g_outs when given."""
    n = len(b)
    L = (ctypes.c_double * n)()
    gm = (ctypes.c_float * n)()
    gp = _ptr_array(g_outs, b.shapes) if g_outs is not None else None
    _check(load().lm_batch_eval(b.handle, _ptr_array(us, b.shapes), gp, L, gm),
           "lm_batch_eval")
    return list(L), list(gm)


def lm_batch_reset(b: Batch, us):
    _check(load().lm_batch_reset(b.handle, _ptr_array(us, b.shapes)),
           "lm_batch_reset")


def lm_batch_iterate(b: Batch, us, n, info=True):
    infos = (StepInfo * len(b))() if info else None
    _check(load().lm_batch_iterate(b.handle, _ptr_array(us, b.shapes), int(n),
                                   infos), "lm_batch_iterate")
    return list(infos) if info else None


def lm_batch_set_targets(b: Batch, targets=None):
    """Per-pair stopping losses (None clears; NaN entries mean no target)."""
    arr = None
    if targets is not None:
        arr = (ctypes.c_double * len(b))(*[float(t) for t in targets])
    _check(load().lm_batch_set_targets(b.handle, arr), "lm_batch_set_targets")


def lm_batch_autotune(b: Batch, us, reps=3):
    """Pick the fastest moment-kernel tile and evaluation work split for
    this batch; returns (e1_tile, e1_waves, e2_waves, ms per evaluation)."""
    t, w1, w2 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    _check(load().lm_batch_autotune(b.handle, _ptr_array(us, b.shapes), int(reps),
                                    ctypes.byref(t), ctypes.byref(w1),
                                    ctypes.byref(w2), ctypes.byref(ms)),
           "lm_batch_autotune")
    return t.value, w1.value, w2.value, ms.value


def lm_autotune(ctx: Context, u, reps=3):
    """As lm_batch_autotune for a single-pair context at field u."""
    t, w1, w2 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    _check(load().lm_autotune(ctx.handle, _field_ptr(u, ctx.shape), int(reps),
                              ctypes.byref(t), ctypes.byref(w1),
                              ctypes.byref(w2), ctypes.byref(ms)),
           "lm_autotune")
    return t.value, w1.value, w2.value, ms.value


def lm_field_resample(src, fa, dst, fb, stream=None):
    """dst (3, Db, Hb, Wb) of pyramid factor fb from src (3, Da, Ha, Wa) of
    factor fa, as between lm_register's levels."""
    _, Da, Ha, Wa = src.shape
    _, Db, Hb, Wb = dst.shape
    _check(load().lm_field_resample(_field_ptr(src), Da, Ha, Wa, int(fa),
                                    _field_ptr(dst), Db, Hb, Wb, int(fb),
                                    _stream_handle(stream)), "lm_field_resample")


def lm_downsample(src, factor, stream=None):
    """Pyramid level of factor 2 or 4 of a 3-D CUDA image (as lm_register
    builds it); returns a new tensor of the image's dtype."""
    import torch
    v = _volume(src)
    dims = (ctypes.c_int * 3)()
    D, H, W = src.shape
    Dl, Hl, Wl = (max(1, n // int(factor)) for n in (D, H, W))
    dst = torch.empty((Dl, Hl, Wl), dtype=src.dtype, device=src.device)
    tmp = torch.empty((2 * D * H * W,), dtype=torch.float32,
                      device=src.device)
    _check(load().lm_downsample(ctypes.byref(v), int(factor),
                                ctypes.c_void_p(dst.data_ptr()),
                                ctypes.c_void_p(tmp.data_ptr()), dims,
                                _stream_handle(stream)), "lm_downsample")
    assert tuple(dims) == (Dl, Hl, Wl)
    return dst


def lm_batch_register(b: Batch, levels, us):
    s = _schedule(levels)
    reps = (Report * len(b))()
    _check(load().lm_batch_register(b.handle, ctypes.byref(s),
                                    _ptr_array(us, b.shapes), reps),
           "lm_batch_register")
    return list(reps)


def lm_register_batch(fixed, moving, us, levels, params: Params | None = None,
                      stream=None):
    vf = (Volume * len(fixed))(*[_volume(t) for t in fixed])
    vm = (Volume * len(moving))(*[_volume(t) for t in moving])
    s = _schedule(levels)
    reps = (Report * len(fixed))()
    p = ctypes.byref(params) if params is not None else None
    _check(load().lm_register_batch(len(fixed), vf, vm,
                                    _ptr_array(us, [f.shape for f in fixed]),
                                    p, ctypes.byref(s),
                                    _stream_handle(stream), reps),
           "lm_register_batch")
    return list(reps)


def lm_eval_noalloc(fixed, moving, u, g_out, loss_out=None, gmax_out=None,
                    params: Params | None = None, stream=None):
    """Evaluation without allocation (static scratch, at most
    LM_NOALLOC_MAX_VOXELS voxels); outputs are device tensors: g_out a
    (3, D, H, W) float32 field, loss_out a float64 and gmax_out a float32
    CUDA tensor of at least one element (the kernel writes element 0)."""
    import torch
    vf, vm = _volume(fixed), _volume(moving)
    if tuple(moving.shape) != tuple(fixed.shape):
        raise ValueError("fixed and moving differ in shape")
    p = ctypes.byref(params) if params is not None else None

    def scalar_ptr(t, dtype, name):
        if t is None:
            return None
        if not t.is_cuda or t.dtype != dtype or t.numel() < 1:
            raise ValueError(f"{name} must be a CUDA {dtype} tensor with at "
                             "least one element")
        return ctypes.c_void_p(t.data_ptr())

    lp = scalar_ptr(loss_out, torch.float64, "loss_out")
    gp = scalar_ptr(gmax_out, torch.float32, "gmax_out")
    _check(load().lm_eval_noalloc(ctypes.byref(vf), ctypes.byref(vm), p,
                                  _field_ptr(u, fixed.shape),
                                  _field_ptr(g_out, fixed.shape), lp, gp,
                                  _stream_handle(stream)), "lm_eval_noalloc")


def lm_strerror(code: int) -> str:
    return load().lm_strerror(int(code)).decode()


def lm_last_error() -> str:
    return load().lm_last_error().decode()


#: every function declared in include/lmreg.h
EXPORTED = ("lm_default_params", "lm_init", "lm_destroy", "lm_eval",
            "lm_reset", "lm_step", "lm_iterate", "lm_get_state",
            "lm_set_state", "lm_register", "lm_state_save", "lm_state_load",
            "lm_time_passes", "lm_batch_init", "lm_batch_destroy",
            "lm_batch_eval", "lm_batch_reset", "lm_batch_iterate",
            "lm_batch_set_targets", "lm_field_resample", "lm_batch_autotune",
            "lm_downsample", "lm_autotune",
            "lm_batch_register", "lm_register_batch", "lm_eval_noalloc",
            "lm_strerror", "lm_last_error", "lm_debug_check", "lm_get_log",
            "lm_batch_debug_check",
            "lm_unet_shapes", "lm_unet_create", "lm_unet_destroy",
            "lm_unet_forward", "lm_unet_train_step", "lm_unet_get_weights",
            "lm_unet_get_grads", "lm_unet_get_tensor", "lm_conv3d_forward",
            "lm_conv3d_backward")


# ---------------------------------------------------------------------------
# Learned warm start (include/lmunet.h)
# ---------------------------------------------------------------------------
LM_UNET_LAYERS = 13


def lm_unet_shapes():
    """([(cin, cout)] of the 13 convolutions, packed parameter count)."""
    cin = (ctypes.c_int * LM_UNET_LAYERS)()
    cout = (ctypes.c_int * LM_UNET_LAYERS)()
    n = ctypes.c_longlong()
    _check(load().lm_unet_shapes(cin, cout, ctypes.byref(n)), "lm_unet_shapes")
    return [(cin[i], cout[i]) for i in range(LM_UNET_LAYERS)], n.value


def pack_weights(params):
    """[(w (cout, cin, 3, 3, 3), b (cout,))] -> packed float32 host array."""
    import numpy as np
    parts = []
    for w, b in params:
        parts.append(np.asarray(w, np.float32).reshape(-1))
        parts.append(np.asarray(b, np.float32).reshape(-1))
    return np.ascontiguousarray(np.concatenate(parts))


def unpack_weights(flat):
    import numpy as np
    shapes, _ = lm_unet_shapes()
    out, k = [], 0
    for cin, cout in shapes:
        nw = cout * cin * 27
        w = np.asarray(flat[k:k + nw]).reshape(cout, cin, 3, 3, 3)
        k += nw
        out.append((w, np.asarray(flat[k:k + cout])))
        k += cout
    return out


class UNet:
    """Owns an lm_unet handle."""

    def __init__(self, handle, shape, stream):
        self.handle = handle
        self.shape = tuple(shape)
        self.stream = stream

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.lm_unet_destroy(h)


def lm_unet_create(shape, params, stream=None):
    import numpy as np
    flat = pack_weights(params)
    _, n = lm_unet_shapes()
    if flat.size != n:
        raise ValueError(f"expected {n} packed parameters, got {flat.size}")
    h = ctypes.c_void_p()
    D, H, W = shape
    _check(load().lm_unet_create(ctypes.byref(h), int(D), int(H), int(W),
                                 flat.ctypes.data_as(ctypes.c_void_p),
                                 _stream_handle(stream)), "lm_unet_create")
    return UNet(h, shape, stream)


def lm_unet_destroy(net: UNet):
    h, net.handle = net.handle, None
    if h:
        load().lm_unet_destroy(h)


def lm_unet_forward(net: UNet, fixed, moving, u_half):
    vf, vm = _volume(fixed), _volume(moving)
    _check(load().lm_unet_forward(net.handle, ctypes.byref(vf), ctypes.byref(vm),
                                  _field_ptr(u_half)), "lm_unet_forward")


def lm_unet_train_step(net: UNet, fixed, moving, targets, lr, loss=True):
    n = len(fixed)
    vf = (Volume * n)(*[_volume(t) for t in fixed])
    vm = (Volume * n)(*[_volume(t) for t in moving])
    tp = _ptr_array(targets)
    L = ctypes.c_double() if loss else None
    _check(load().lm_unet_train_step(net.handle, n, vf, vm, tp,
                                     ctypes.c_float(lr),
                                     ctypes.byref(L) if L is not None else None),
           "lm_unet_train_step")
    return L.value if L is not None else None


def lm_unet_get_weights(net: UNet):
    import numpy as np
    _, n = lm_unet_shapes()
    out = np.empty(n, np.float32)
    _check(load().lm_unet_get_weights(net.handle,
                                      out.ctypes.data_as(ctypes.c_void_p)),
           "lm_unet_get_weights")
    return unpack_weights(out)


def lm_unet_get_grads(net: UNet):
    import numpy as np
    _, n = lm_unet_shapes()
    out = np.empty(n, np.float32)
    _check(load().lm_unet_get_grads(net.handle,
                                    out.ctypes.data_as(ctypes.c_void_p)),
           "lm_unet_get_grads")
    return unpack_weights(out)


# lm_unet_get_tensor names (include/lmunet.h), in enum order
UNET_TENSORS = ("x0", "e0a", "e0", "p0", "e1a", "e1", "p1", "e2a", "e2", "p2",
                "e3a", "e3", "cat2", "d2a", "d2", "cat1", "d1a", "d1", "out",
                "dy0", "dy1", "dy2", "dy3", "dy4", "dy5", "dy6", "dy12",
                "dx2", "dx4", "dx6", "dx8", "dx10")


def lm_unet_get_tensor(net: UNet, name: str):
    """A stored tensor of the network's last pass as float32
    (D >> l, H >> l, W >> l, C), channels last."""
    import numpy as np
    which = UNET_TENSORS.index(name)
    lvl, ch = ctypes.c_int(), ctypes.c_int()
    lib = load()
    _check(lib.lm_unet_get_tensor(net.handle, which, None, ctypes.byref(lvl),
                                  ctypes.byref(ch)), "lm_unet_get_tensor")
    D, H, W = (n >> lvl.value for n in net.shape)
    out = np.empty((D, H, W, ch.value), np.float32)
    _check(lib.lm_unet_get_tensor(net.handle, which,
                                  out.ctypes.data_as(ctypes.c_void_p), None,
                                  None), "lm_unet_get_tensor")
    return out


def lm_conv3d_forward(x, w, bias, act, y, stream=None):
    """x bf16 (D, H, W, cin), w bf16 (cout, 27, cin), bias f32 (cout,) or
    None, y f32 (D, H, W, cout) (all CUDA tensors)."""
    D, H, W, cin = x.shape
    cout = w.shape[0]
    _check(load().lm_conv3d_forward(
        D, H, W, cin, cout, ctypes.c_void_p(x.data_ptr()),
        ctypes.c_void_p(w.data_ptr()),
        ctypes.c_void_p(bias.data_ptr()) if bias is not None else None,
        int(act), ctypes.c_void_p(y.data_ptr()), _stream_handle(stream)),
        "lm_conv3d_forward")


def lm_conv3d_backward(x, w, dy, dx, dw, db, stream=None):
    D, H, W, cin = x.shape
    cout = w.shape[0]
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(load().lm_conv3d_backward(D, H, W, cin, cout, p(x), p(w), p(dy),
                                     p(dx), p(dw), p(db),
                                     _stream_handle(stream)),
           "lm_conv3d_backward")
