"""Seeded synthetic registration pairs shared by the tests, the smoke check
and the benchmark.

This module generates INPUTS only: it holds none of the registration
method's arithmetic (no LNCC, no LM step, no compositive update of the
optimizer).  Resampling and smoothing here are scipy.ndimage library calls
used to build phantoms and ground-truth warps, not the method's own steps.

Arrays: images float32 (nz, ny, nx), x fastest; fields float32
(3, nz, ny, nx) with component 0 along x, in voxel units, and a field u
names the sample point p + u(p).

Recipes (the paper's datasets are not available; these stand in for them):
  * ``blob_pair``     -- sum of 20 random 3-D Gaussian blobs (sigma 2-5 vox,
    amplitude U[0.2, 1]) plus N(0, 0.01) noise; the moving image is the fixed
    one warped by the exponential of a stationary velocity field (N(0, 1)
    noise, Gaussian sigma 4, scaled to max displacement 3 vox, 6 squarings).
  * ``voronoi_pair``  -- brain-MRI-shaped piecewise-constant phantom: 30-label
    Voronoi partition with label intensities U[0, 1], a smooth multiplicative
    bias field in [0.8, 1.2], N(0, 0.02) noise, clipped to [0, 1]; SVF warp
    with sigma 8 and max displacement 8 vox.
  * ``lung_pair``     -- lung-CT-shaped phantom at 448x448x384 (W x H x D):
    HU -1000 (air) outside an ellipsoidal body, tissue U[-100, 100] inside
    (smoothed at sigma 1 and rescaled to that range), 200 vessel-like tubes
    (random smoothed splines, radius 1-3 vox, values U[200, 400] HU);
    clipped to [-1000, 400] and mapped to [0, 1]; SVF warp with sigma 10
    and max displacement 15 vox.  The cross-modal variant remaps the moving
    image by the monotone cubic 3m^2 - 2m^3 and adds N(0, 0.02).
  * ``translation_pair`` -- moving(p) = fixed(p + t) for an integer t.
  * ``uneven_shapes`` -- per-pair shapes drawn uniformly per axis between
    64^3 and 160x192x224.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np
from scipy import ndimage

_VERSION = "synth-v1"


def _cache_path(key: str):
    root = os.environ.get("LMREG_SYNTH_CACHE", "/tmp/lmreg_synth_cache")
    try:
        os.makedirs(root, exist_ok=True)
    except OSError:
        return None
    h = hashlib.sha1((_VERSION + key).encode()).hexdigest()[:20]
    return os.path.join(root, h + ".npz")


def _cached(key, fn, cache=True):
    path = _cache_path(key) if cache else None
    if path and os.path.exists(path):
        try:
            with np.load(path) as z:
                return tuple(z[f"a{i}"] for i in range(len(z.files)))
        except Exception:
            pass
    out = fn()
    if path:
        tmp = f"{path}.{os.getpid()}.tmp.npz"
        try:
            np.savez(tmp, **{f"a{i}": a for i, a in enumerate(out)})
            os.replace(tmp, path)
        except OSError:
            pass
    return out


def _grid(shape):
    return np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape],
                       indexing="ij")


def _warp_image(img, u, cval=0.0):
    """img(p + u(p)) by scipy trilinear interpolation, zero outside."""
    zz, yy, xx = _grid(img.shape)
    coords = np.stack([zz + u[2], yy + u[1], xx + u[0]])
    return ndimage.map_coordinates(img, coords, order=1, mode="constant",
                                   cval=cval)


def _warp_field(f, u):
    """Each component of f read at p + u(p), clamp to edge."""
    zz, yy, xx = _grid(f.shape[1:])
    coords = np.stack([zz + u[2], yy + u[1], xx + u[0]])
    return np.stack([ndimage.map_coordinates(f[i], coords, order=1,
                                             mode="nearest")
                     for i in range(3)])


def svf_field(shape, rng, sigma, max_disp, squarings=6, coarse=1,
              coarse_exp=False):
    """Exponential of a smooth random stationary velocity field.

    v ~ N(0, 1) per component, Gaussian-smoothed (sigma voxels), scaled so
    max |v| = max_disp, then exp(v) by scaling and squaring.  ``coarse`` > 1
    draws v on a grid ``coarse`` times smaller and upsamples it (a cheaper
    route to the same band-limited field for large volumes); with
    ``coarse_exp`` the squarings run on that grid too (in its units) and
    the resulting displacement is upsampled and rescaled.
    """
    shape = tuple(int(n) for n in shape)
    if coarse > 1 and coarse_exp:
        cs = tuple(max(4, -(-n // coarse)) for n in shape)
        v = np.stack([ndimage.gaussian_filter(rng.standard_normal(cs),
                                              sigma / coarse)
                      for _ in range(3)])
        nrm = np.sqrt((v ** 2).sum(0)).max()
        v *= (max_disp / coarse) / max(nrm, 1e-12)
        u = v / (2.0 ** squarings)
        for _ in range(squarings):
            u = u + _warp_field(u, u)
        zoom = [n / c for n, c in zip(shape, cs)]
        out = np.empty((3,) + shape, dtype=np.float32)
        for i in range(3):
            # component i is along axis 2 - i: rescale by that axis' zoom
            out[i] = ndimage.zoom(u[i], zoom, order=1)[
                :shape[0], :shape[1], :shape[2]] * zoom[2 - i]
        return out
    if coarse > 1:
        cs = tuple(max(4, -(-n // coarse)) for n in shape)
        v = np.stack([ndimage.gaussian_filter(rng.standard_normal(cs),
                                              sigma / coarse)
                      for _ in range(3)])
        zoom = [n / c for n, c in zip(shape, cs)]
        v = np.stack([ndimage.zoom(v[i], zoom, order=1) for i in range(3)])
        v = v[:, :shape[0], :shape[1], :shape[2]]
    else:
        v = np.stack([ndimage.gaussian_filter(rng.standard_normal(shape),
                                              sigma)
                      for _ in range(3)])
    nrm = np.sqrt((v ** 2).sum(0)).max()
    v *= max_disp / max(nrm, 1e-12)
    u = v / (2.0 ** squarings)
    for _ in range(squarings):
        u = u + _warp_field(u, u)
    return u


def blob_image(shape, rng, n_blobs=20, sigma=(2.0, 5.0), amp=(0.2, 1.0),
               noise=0.01):
    shape = tuple(int(n) for n in shape)
    zz, yy, xx = _grid(shape)
    img = np.zeros(shape)
    for _ in range(n_blobs):
        c = rng.uniform(0, 1, 3) * (np.array(shape) - 1)
        s = rng.uniform(*sigma)
        a = rng.uniform(*amp)
        d2 = (zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2
        img += a * np.exp(-d2 / (2 * s * s))
    img += rng.normal(0.0, noise, shape)
    return img


def blob_pair(shape=(32, 32, 32), seed=0, svf_sigma=4.0, max_disp=3.0):
    """(F, M, u_true) float32 for the 32^3 Gaussian-blob workload."""
    def make():
        rng = np.random.default_rng(seed)
        F = blob_image(shape, rng)
        u = svf_field(shape, rng, svf_sigma, max_disp)
        M = _warp_image(F, u)
        return (F.astype(np.float32), M.astype(np.float32),
                u.astype(np.float32))
    return _cached(f"blob{tuple(shape)}:{seed}:{svf_sigma}:{max_disp}", make)


def voronoi_image(shape, rng, n_labels=30, bias=0.2, noise=0.02):
    shape = tuple(int(n) for n in shape)
    seeds = rng.uniform(0, 1, (n_labels, 3)) * (np.array(shape) - 1)
    inten = rng.uniform(0, 1, n_labels)
    lab = np.empty(shape, dtype=np.int32)
    yy, xx = np.meshgrid(np.arange(shape[1]), np.arange(shape[2]),
                         indexing="ij")
    for z in range(shape[0]):
        d = ((z - seeds[:, 0, None, None]) ** 2
             + (yy[None] - seeds[:, 1, None, None]) ** 2
             + (xx[None] - seeds[:, 2, None, None]) ** 2)
        lab[z] = np.argmin(d, axis=0)
    img = inten[lab]
    cs = tuple(max(4, n // 8) for n in shape)
    b = ndimage.gaussian_filter(rng.standard_normal(cs), 2.0)
    b = ndimage.zoom(b, [n / c for n, c in zip(shape, cs)], order=1)
    b = b[:shape[0], :shape[1], :shape[2]]
    b = (b - b.min()) / max(b.max() - b.min(), 1e-12) * 2 - 1
    img = img * (1.0 + bias * b)
    img = img + rng.normal(0.0, noise, shape)
    return np.clip(img, 0.0, 1.0)


def voronoi_pair(shape=(160, 192, 224), seed=0, svf_sigma=8.0, max_disp=8.0,
                 coarse_exp=False, cache=True):
    """(F, M, u_true) float32 for the brain-MRI-shaped Voronoi workload
    (coarse_exp: the warp's squarings on the 4x coarser grid, see
    svf_field; with cache=False nothing is written to the disk cache: data
    sets of thousands of pairs)."""
    def make():
        rng = np.random.default_rng(seed)
        F = voronoi_image(shape, rng)
        coarse = 4 if np.prod(shape) > 64 ** 3 else 1
        u = svf_field(shape, rng, svf_sigma, max_disp, coarse=coarse,
                      coarse_exp=coarse_exp and coarse > 1)
        M = _warp_image(F, u)
        return (F.astype(np.float32), M.astype(np.float32),
                u.astype(np.float32))
    key = f"voronoi{tuple(shape)}:{seed}:{svf_sigma}:{max_disp}"
    return _cached(key + (":cexp" if coarse_exp else ""), make, cache)


def _spline_points(rng, lo, hi, n_ctrl=5, step=0.5):
    """Points every ``step`` voxels along a smooth random curve through
    n_ctrl control points drawn inside the box [lo, hi] (Catmull-Rom)."""
    P = rng.uniform(lo, hi, (n_ctrl, 3))
    P = np.vstack([2 * P[0] - P[1], P, 2 * P[-1] - P[-2]])
    pts = []
    for i in range(1, n_ctrl):
        p0, p1, p2, p3 = P[i - 1], P[i], P[i + 1], P[i + 2]
        n = max(2, int(np.linalg.norm(p2 - p1) / step))
        t = np.linspace(0, 1, n, endpoint=False)[:, None]
        pts.append(0.5 * (2 * p1 + (-p0 + p2) * t
                          + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t ** 2
                          + (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 3))
    return np.vstack(pts)


def lung_image(shape, rng, n_tubes=200):
    """Lung-CT-shaped phantom in [0, 1] (HU clipped to [-1000, 400])."""
    shape = tuple(int(n) for n in shape)
    c = (np.array(shape) - 1) / 2.0
    ax = 0.45 * np.array(shape)               # body semi-axes
    zz = ((np.arange(shape[0]) - c[0]) / ax[0]) ** 2
    yy = ((np.arange(shape[1]) - c[1]) / ax[1]) ** 2
    xx = ((np.arange(shape[2]) - c[2]) / ax[2]) ** 2
    body = (zz[:, None, None] + yy[None, :, None] + xx[None, None, :]) <= 1.0
    t = ndimage.gaussian_filter(rng.random(shape, dtype=np.float32), 1.0)
    t = (t - t.min()) / max(float(t.max() - t.min()), 1e-12) * 200 - 100
    hu = np.where(body, t, np.float32(-1000.0)).astype(np.float32)
    del t
    lo, hi = c - 0.8 * ax / np.sqrt(3), c + 0.8 * ax / np.sqrt(3)
    for _ in range(n_tubes):
        pts = _spline_points(rng, lo, hi)
        r = rng.uniform(1.0, 3.0)
        val = rng.uniform(200.0, 400.0)
        R = int(np.ceil(r))
        o = np.arange(-R, R + 1)
        off = np.stack(np.meshgrid(o, o, o, indexing="ij"), -1).reshape(-1, 3)
        off = off[(off ** 2).sum(1) <= r * r]
        vox = np.unique((np.rint(pts)[:, None, :] + off[None]).reshape(-1, 3)
                        .astype(np.int64), axis=0)
        ok = np.all((vox >= 0) & (vox < np.array(shape)), axis=1)
        vox = vox[ok]
        hu[vox[:, 0], vox[:, 1], vox[:, 2]] = np.maximum(
            hu[vox[:, 0], vox[:, 1], vox[:, 2]], val)
    return (np.clip(hu, -1000.0, 400.0) + 1000.0) / 1400.0


def lung_pair(shape=(384, 448, 448), seed=0, svf_sigma=10.0, max_disp=15.0,
              cross_modal=False):
    """(F, M, u_true) float32 for the lung-CT-shaped workload (shape is
    (D, H, W): 448 x 448 in-plane, 384 slices)."""
    def make():
        rng = np.random.default_rng(seed)
        F = lung_image(shape, rng)
        u = svf_field(shape, rng, svf_sigma, max_disp, coarse=4,
                      coarse_exp=True)
        M = _warp_image(F, u)
        if cross_modal:
            M = 3 * M ** 2 - 2 * M ** 3 + rng.normal(0.0, 0.02, M.shape)
        return (F.astype(np.float32), M.astype(np.float32),
                u.astype(np.float32))
    return _cached(f"lung{tuple(shape)}:{seed}:{svf_sigma}:{max_disp}:"
                   f"{int(cross_modal)}", make)


def translation_pair(shape=(32, 32, 32), seed=0, t=(2, -1, 1)):
    """F = blob image, M(p) = F(p + t) (t in (x, y, z) voxels, integers)."""
    rng = np.random.default_rng(seed)
    F = blob_image(shape, rng)
    u = np.zeros((3,) + tuple(shape))
    for i in range(3):
        u[i] = t[i]
    M = _warp_image(F, u)
    return F.astype(np.float32), M.astype(np.float32)


def random_field(shape, seed, scale=1.0):
    """Smooth random field with non-integer values (test states)."""
    rng = np.random.default_rng(seed)
    u = np.stack([ndimage.gaussian_filter(rng.standard_normal(shape), 1.5)
                  for _ in range(3)])
    u *= scale / max(np.abs(u).max(), 1e-12)
    return u.astype(np.float32)


def uneven_shapes(n=64, seed=0, lo=(64, 64, 64), hi=(160, 192, 224)):
    """Per-pair (nz, ny, nx) drawn uniformly per axis in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return [tuple(int(rng.integers(lo[i], hi[i] + 1)) for i in range(3))
            for _ in range(n)]


def unet_init(shapes, seed=0, last_scale=0.1):
    """Initial network weights: for each (cin, cout) a (cout, cin, 3, 3, 3)
    array drawn uniformly with the He/Kaiming bound for a leaky ReLU of
    slope 0.2 (fan-in 27 cin) and a zero bias; the last layer is scaled by
    ``last_scale`` so that the untrained output is near zero.  float32."""
    rng = np.random.default_rng(seed)
    out = []
    for n, (cin, cout) in enumerate(shapes):
        fan_in = 27 * cin
        bound = np.sqrt(3.0 * 2.0 / ((1.0 + 0.04) * fan_in))
        if n == len(shapes) - 1:
            bound *= last_scale
        w = rng.uniform(-bound, bound, (cout, cin, 3, 3, 3))
        out.append((w.astype(np.float32), np.zeros(cout, np.float32)))
    return out
