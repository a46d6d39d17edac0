"""FP64 CPU oracle for the factored Levenberg-Marquardt LNCC iteration.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA product path
never imports this package, and this package never imports the product.

Thin ctypes wrapper over ``lmoracle.c`` (plain C, FP64).  Arrays are numpy
float64, C-contiguous: scalar volumes have shape (nz, ny, nx) (x fastest) and
vector fields shape (3, nz, ny, nx) with component 0 = x.  Each function cites
the passage of the paper it follows; readings of points the paper leaves open
are documented in ``lmoracle.c``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lmoracle.c")
_LIB_PATH = os.path.join(_HERE, "liblmoracle.so")
_lock = threading.Lock()
_lib = None

ACCEPT, RETRY, DISCARD = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile lmoracle.c into liblmoracle.so beside it (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Mirror of ``or_params`` in lmoracle.c."""
    _fields_ = [
        ("win", ctypes.c_int),
        ("eps_nr", ctypes.c_double),
        ("eps_dr", ctypes.c_double),
        ("sigma_grad", ctypes.c_double),
        ("sigma_warp", ctypes.c_double),
        ("step", ctypes.c_double),
        ("lambda0", ctypes.c_double),
        ("mu_inc", ctypes.c_double),
        ("mu_dec", ctypes.c_double),
        ("lambda_max", ctypes.c_double),
        ("reject", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("max_retries", ctypes.c_int),
        ("tile", ctypes.c_int),
        ("loss", ctypes.c_int),
        ("method", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("bins", ctypes.c_int),
    ]


# Section 3 (experiments): lambda0 = 0.006, mu+ = 1.5, mu- = 0.975, tile 1;
# Section 3.4 (rejection): tau = 1 with cap 1 when rejection is on.
DEFAULTS = dict(win=5, eps_nr=1e-5, eps_dr=1e-5, sigma_grad=1.0,
                sigma_warp=0.0, step=0.5, lambda0=0.006, mu_inc=1.5,
                mu_dec=0.975, lambda_max=math.inf, reject=0, tau=1.0,
                max_retries=10, tile=1, loss=0, method=0, alpha=1.0,
                bins=32)

LNCC, MSE, MI = 0, 1, 2   # Section 2.2 squared-loss forms
LM, DEMONS = 0, 1         # Section 2.2 optimiser / Section 2.3 special case


def params(**kw) -> Params:
    d = dict(DEFAULTS)
    for k in kw:
        if k not in d:
            raise KeyError(k)
    d.update(kw)
    return Params(**d)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(ctypes.c_double)
        I = ctypes.c_int
        D = ctypes.c_double
        PP = ctypes.POINTER(Params)
        PI = ctypes.POINTER(ctypes.c_int)
        lib.or_sample.argtypes = [I, I, I, P, P, P, P]
        lib.or_box.argtypes = [I, I, I, I, P, P]
        lib.or_lncc_terms.argtypes = [I, I, I, I, D, D, P, P, P, P, P, P]
        lib.or_gauss_radius.argtypes = [D]
        lib.or_gauss_radius.restype = I
        lib.or_gauss_taps.argtypes = [D, P]
        lib.or_gauss_taps.restype = I
        lib.or_smooth.argtypes = [I, I, I, D, P, P]
        lib.or_smooth_field.argtypes = [I, I, I, D, P, P]
        lib.or_eval.argtypes = [I, I, I, P, P, P, PP, P, P, P, P, P, P]
        lib.or_compose.argtypes = [I, I, I, P, P, P]
        lib.or_trial.argtypes = [I, I, I, P, P, D, D, D, PP, P, P]
        lib.or_tile_du.argtypes = [I, I, I, I, P, D, D, P]
        lib.or_demons_force.argtypes = [I, I, I, P, P, P, D, P]
        lib.or_mi_range.argtypes = [I, I, I, P, P, P, P]
        lib.or_mi.argtypes = [I, I, I, I, D, D, P, P, P, P]
        lib.or_demons_eval.argtypes = [I, I, I, P, P, P, PP, P, P, P]
        lib.or_decide.argtypes = [D, D, D, I, D, I, PP, P]
        lib.or_decide.restype = I
        lib.or_lm_step.argtypes = [I, I, I, P, P, PP, P, P, P, P, P, PI, P,
                                   P, P, PI, PI, PI]
        lib.or_level_dims.argtypes = [I, I, I, I, PI, PI, PI]
        lib.or_downsample.argtypes = [I, I, I, I, P, P]
        lib.or_resample_field.argtypes = [I, I, I, I, P, I, I, I, I, P]
        lib.or_register.argtypes = [I, I, I, P, P, PP, I, PI, PI, P, P, PI]
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dims(vol):
    nz, ny, nx = vol.shape[-3:]
    return nx, ny, nz


# --------------------------------------------------------------------------
# Step (a): trilinear resampling (Section 2.1).
# --------------------------------------------------------------------------
def sample(M, u):
    """J = M(p + u(p)) with zero padding, and dJ/du (3, nz, ny, nx)."""
    M, u = _f64(M), _f64(u)
    nx, ny, nz = _dims(M)
    J = np.empty_like(M)
    dJ = np.empty((3,) + M.shape)
    _load().or_sample(nx, ny, nz, _ptr(M), _ptr(u), _ptr(J), _ptr(dJ))
    return J, dJ


def box(X, k):
    """k^3 window mean with zero padding and fixed divisor k^3."""
    X = _f64(X)
    nx, ny, nz = _dims(X)
    S = np.empty_like(X)
    _load().or_box(nx, ny, nz, int(k), _ptr(X), _ptr(S))
    return S


def lncc_terms(F, J, k=5, eps_nr=1e-5, eps_dr=1e-5):
    """Per-voxel cc and the backward coefficients (a, b, c) (Section 2.2)."""
    F, J = _f64(F), _f64(J)
    nx, ny, nz = _dims(F)
    out = [np.empty_like(F) for _ in range(4)]
    _load().or_lncc_terms(nx, ny, nz, int(k), eps_nr, eps_dr, _ptr(F),
                          _ptr(J), *[_ptr(o) for o in out])
    return tuple(out)


def gauss_taps(sigma):
    lib = _load()
    R = lib.or_gauss_radius(float(sigma))
    t = np.empty(2 * R + 1)
    lib.or_gauss_taps(float(sigma), _ptr(t))
    return t


def smooth(X, sigma, clamp=False):
    """Separable Gaussian of a scalar volume or of each component of a
    (3, ...) field; zero padding, or edge clamping when ``clamp``."""
    X = _f64(X)
    if X.ndim == 4:
        return np.stack([smooth(X[i], sigma, clamp)
                         for i in range(X.shape[0])])
    nx, ny, nz = _dims(X)
    Y = np.empty_like(X)
    fn = _load().or_smooth_field if clamp else _load().or_smooth
    fn(nx, ny, nz, float(sigma), _ptr(X), _ptr(Y))
    return Y


def mi_range(F, M):
    """Joint intensity range [lo, hi] of F, M and 0 (the MI binning)."""
    F, M = _f64(F), _f64(M)
    nx, ny, nz = _dims(F)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _load().or_mi_range(nx, ny, nz, _ptr(F), _ptr(M), ctypes.byref(lo),
                        ctypes.byref(hi))
    return lo.value, hi.value


def mi(F, J, bins, lo, hi):
    """Parzen-window (cubic B-spline) mutual information in bits of the
    pair (F, J) and dMI/dJ per voxel (Section 2.2, MI loss)."""
    F, J = _f64(F), _f64(J)
    nx, ny, nz = _dims(F)
    out = ctypes.c_double()
    d = np.empty_like(F)
    _load().or_mi(nx, ny, nz, int(bins), float(lo), float(hi), _ptr(F),
                  _ptr(J), ctypes.byref(out), _ptr(d))
    return out.value, d


def demons_force(F, M, u, alpha):
    """Update of Eq. demons (Section 2.3): r n / (|n|^2 + alpha^2 r^2) with
    r = F - M(p + u) and n the gradient of M at p + u."""
    F, M, u = _f64(F), _f64(M), _f64(u)
    nx, ny, nz = _dims(F)
    du = np.empty_like(u)
    _load().or_demons_force(nx, ny, nz, _ptr(F), _ptr(M), _ptr(u),
                            float(alpha), _ptr(du))
    return du


def demons_evaluate(F, M, u, P: Params):
    """Demons evaluation: L = MSE and g = G_sigma_grad * (Eq. demons)."""
    F, M, u = _f64(F), _f64(M), _f64(u)
    nx, ny, nz = _dims(F)
    L = ctypes.c_double()
    gmax = ctypes.c_double()
    g = np.empty((3,) + F.shape)
    _load().or_demons_eval(nx, ny, nz, _ptr(F), _ptr(M), _ptr(u),
                           ctypes.byref(P), ctypes.byref(L), _ptr(g),
                           ctypes.byref(gmax))
    return dict(L=L.value, g=g, gmax=gmax.value)


def evaluate(F, M, u, P: Params):
    """One loss/gradient evaluation, steps (a)-(c).

    Returns dict with L (= r = 1 - LNCC, the MSE for P.loss = MSE, or
    log2(B) - MI for P.loss = MI), dLdJ, graw, g (smoothed), gmax, cc
    (per-voxel cc, (F - J)^2 for MSE, 0 for MI).
    For P.method = DEMONS, L is the MSE and g the smoothed update of
    Eq. demons (no dLdJ, graw, cc).
    """
    if P.method == DEMONS:
        return demons_evaluate(F, M, u, P)
    F, M, u = _f64(F), _f64(M), _f64(u)
    nx, ny, nz = _dims(F)
    L = ctypes.c_double()
    gmax = ctypes.c_double()
    dLdJ = np.empty_like(F)
    graw = np.empty((3,) + F.shape)
    g = np.empty((3,) + F.shape)
    cc = np.empty_like(F)
    _load().or_eval(nx, ny, nz, _ptr(F), _ptr(M), _ptr(u), ctypes.byref(P),
                    ctypes.byref(L), _ptr(dLdJ), _ptr(graw), _ptr(g),
                    ctypes.byref(gmax), _ptr(cc))
    return dict(L=L.value, dLdJ=dLdJ, graw=graw, g=g, gmax=gmax.value, cc=cc)


def loss(F, M, u, P: Params) -> float:
    if P.method == DEMONS:
        return demons_evaluate(F, M, u, P)["L"]
    F, M, u = _f64(F), _f64(M), _f64(u)
    nx, ny, nz = _dims(F)
    L = ctypes.c_double()
    _load().or_eval(nx, ny, nz, _ptr(F), _ptr(M), _ptr(u), ctypes.byref(P),
                    ctypes.byref(L), None, None, None, None, None)
    return L.value


def compose(u, v):
    """v + u o (Id + v), Eq. compositive; u read with clamp-to-edge."""
    u, v = _f64(u), _f64(v)
    nx, ny, nz = _dims(u)
    out = np.empty_like(u)
    _load().or_compose(nx, ny, nz, _ptr(u), _ptr(v), _ptr(out))
    return out


def tile_du(ghat, k, r, lam):
    """Step of the pooled curvature, Eq. tilen: per non-overlapping k^3 tile
    the mean of ghat ghat^T, then du = -(H + lam I)^-1 r ghat per voxel
    (k = 1 is Eq. tile1)."""
    ghat = _f64(ghat)
    nx, ny, nz = _dims(ghat)
    du = np.empty_like(ghat)
    _load().or_tile_du(nx, ny, nz, int(k), _ptr(ghat), float(r), float(lam),
                       _ptr(du))
    return du


def trial(u, g, gmax, r, lam, P: Params):
    """Trial field from Eq. tile1 (Eq. tilen when P.tile > 1) + Eq.
    compositive; returns (u', du)."""
    u, g = _f64(u), _f64(g)
    nx, ny, nz = _dims(u)
    out = np.empty_like(u)
    du = np.empty_like(u)
    _load().or_trial(nx, ny, nz, _ptr(u), _ptr(g), float(gmax), float(r),
                     float(lam), ctypes.byref(P), _ptr(out), _ptr(du))
    return out, du


def decide(L_trial, L_t, L_prev, has_prev, lam, retries, P: Params):
    """Damping/rejection rule (Eq. lambda-update, Eq. rejection)."""
    out = ctypes.c_double()
    act = _load().or_decide(float(L_trial), float(L_t), float(L_prev),
                            int(has_prev), float(lam), int(retries),
                            ctypes.byref(P), ctypes.byref(out))
    return act, out.value


class State:
    """Optimizer state of one LM run: field, gradient, scalars."""

    def __init__(self, F, M, u, P: Params):
        self.F, self.M = _f64(F), _f64(M)
        self.u = _f64(u).copy()
        ev = evaluate(self.F, self.M, self.u, P)
        self.g = ev["g"]
        self.gmax = ev["gmax"]
        self.L = ev["L"]
        self.L_prev = 0.0
        self.has_prev = 0
        self.lam = P.lambda0
        self.P = P


def lm_step(st: State):
    """One LM iteration (Section 2.2 and 3.3); updates st in place.

    Returns dict(accepted, retries, evals, u_first, L_first).
    """
    nx, ny, nz = _dims(st.F)
    g = np.ascontiguousarray(st.g)
    gm = ctypes.c_double(st.gmax)
    L = ctypes.c_double(st.L)
    Lp = ctypes.c_double(st.L_prev)
    hp = ctypes.c_int(st.has_prev)
    lam = ctypes.c_double(st.lam)
    u_first = np.empty_like(st.u)
    L_first = ctypes.c_double()
    acc, ret, ev = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _load().or_lm_step(nx, ny, nz, _ptr(st.F), _ptr(st.M), ctypes.byref(st.P),
                       _ptr(st.u), _ptr(g), ctypes.byref(gm), ctypes.byref(L),
                       ctypes.byref(Lp), ctypes.byref(hp), ctypes.byref(lam),
                       _ptr(u_first), ctypes.byref(L_first),
                       ctypes.byref(acc), ctypes.byref(ret), ctypes.byref(ev))
    st.g, st.gmax, st.L, st.L_prev = g, gm.value, L.value, Lp.value
    st.has_prev, st.lam = hp.value, lam.value
    return dict(accepted=acc.value, retries=ret.value, evals=ev.value,
                u_first=u_first, L_first=L_first.value)


def level_dims(shape, f):
    nz, ny, nx = shape
    ox, oy, oz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _load().or_level_dims(nx, ny, nz, int(f), ctypes.byref(ox),
                          ctypes.byref(oy), ctypes.byref(oz))
    return oz.value, oy.value, ox.value


def downsample(X, f):
    """Anti-aliased pyramid level of factor f (Section 2.1 pyramid)."""
    X = _f64(X)
    nx, ny, nz = _dims(X)
    Y = np.empty(level_dims(X.shape, f))
    _load().or_downsample(nx, ny, nz, int(f), _ptr(X), _ptr(Y))
    return Y


def resample_field(Ua, fa, shape_b, fb):
    """Carry a field from a level of factor fa to one of factor fb."""
    Ua = _f64(Ua)
    ax, ay, az = _dims(Ua)
    bz, by, bx = shape_b
    Ub = np.empty((3, bz, by, bx))
    _load().or_resample_field(ax, ay, az, int(fa), _ptr(Ua), bx, by, bz,
                              int(fb), _ptr(Ub))
    return Ub


def register(F, M, P: Params, factors, iters, u0=None):
    """Coarse-to-fine registration; returns (u, loss_log, evals)."""
    F, M = _f64(F), _f64(M)
    nx, ny, nz = _dims(F)
    u = np.zeros((3,) + F.shape) if u0 is None else _f64(u0).copy()
    n = len(factors)
    fa = (ctypes.c_int * n)(*factors)
    it = (ctypes.c_int * n)(*iters)
    log = np.empty(int(sum(iters)))
    ev = ctypes.c_int()
    _load().or_register(nx, ny, nz, _ptr(F), _ptr(M), ctypes.byref(P), n,
                        fa, it, _ptr(u), _ptr(log), ctypes.byref(ev))
    return u, log, ev.value
