"""Naive local Laplacian filtering in float64 (oracle; test infrastructure only).

Sec. II-C of the paper: for every level l below the top and every pixel p
of that level, take g = G_l[I]_p, remap the input about g
(r_g(I) = I + f(I - g)), build the Laplacian pyramid of the remapped image
and keep its coefficient at (l, p) as L_l[O]_p; the top level is G_top[I]
(Eq. (14) text); then collapse (Eq. (4)).  Eq. (13) states the same
coefficient as G_l[r] - up(G_{l+1}[r]) at p.

The remapped image is built either over the whole image (``window=False``;
brute force, for small images) or over an exact dependency window
(``window=True``): the rectangle, aligned to 2^(l+1) level-0 pixels and
clipped at the true image borders, that holds every level-0 pixel the
coefficient at (l, p) depends on.  That is the level-0 radius
6 * 2^l - 2 around 2^l p: 2^(l+1) - 2 for G_l at p, plus 2^(l+1) from the
two coarse neighbours the upsampling reads, plus 2^(l+2) - 2 for G_{l+1}
at those neighbours.  The alignment keeps every level of the window on the
global sampling grid and the clipping keeps the true reflect-101 borders, so
the windowed value equals the whole-image value; a test checks this.

``f`` is any vectorised callable d -> f(d): the exact remap detail, its
Fourier approximation f_K, or a linear f for the closed-form check.
``remap_fn`` (optional) replaces the whole remap by any vectorised
(i, g) -> r(i, g), for remaps that are not a function of i - g alone.
"""

import numpy as np

from .pyramid import gaussian_pyramid, reduce, expand, collapse, coarse_size

_MAX_BATCH_ELEMS = 1 << 22


def _laplacian_at(windows, g, f, level, ly, lx, s=None, remap_fn=None):
    """Coefficient L_level[w + s f(w - g)] at local level positions (ly, lx), batched.

    ``s`` (one value per coefficient, default 1) scales the remap detail: the
    pixel-by-pixel parameter of Sec. III-B.  With ``remap_fn`` the remapped
    window is remap_fn(w, g) instead."""
    if remap_fn is not None:
        r = remap_fn(windows, g[:, None, None])
    else:
        d = f(windows - g[:, None, None])
        r = windows + (d if s is None else s[:, None, None] * d)
    for _ in range(level):
        r = reduce(r)
    coarse = reduce(r)
    lap = r - expand(coarse, r.shape[-2:])
    return lap[np.arange(len(g)), ly, lx]


def _window_1d(p, level, n, margin):
    """Aligned, clipped window [lo, hi) on one axis for level-``level`` positions p."""
    align = 2 ** (level + 1)
    centre = p * 2 ** level
    lo = np.maximum(0, ((centre - margin) // align) * align)
    hi = np.minimum(n, -((-(centre + margin + 1)) // align) * align)
    return lo, hi


def _level_coefficients(img, gl, level, f, window, scale=None, remap_fn=None):
    """L_level[O] for every pixel of one level (level < top); ``scale``: per-pixel
    detail scale at this level (same shape as gl) or None."""
    h0, w0 = img.shape
    hl, wl = gl.shape
    py, px = np.meshgrid(np.arange(hl), np.arange(wl), indexing="ij")
    py, px = py.ravel(), px.ravel()
    g = gl[py, px]
    sc = None if scale is None else np.asarray(scale, dtype=np.float64)[py, px]
    out = np.empty(hl * wl)
    if window:
        margin = 6 * 2 ** level - 2
        y0, y1 = _window_1d(py, level, h0, margin)
        x0, x1 = _window_1d(px, level, w0, margin)
    else:
        y0, y1 = np.zeros_like(py), np.full_like(py, h0)
        x0, x1 = np.zeros_like(px), np.full_like(px, w0)
    shapes = np.stack([y1 - y0, x1 - x0], axis=1)
    for hh, ww in np.unique(shapes, axis=0):
        sel = np.nonzero((shapes[:, 0] == hh) & (shapes[:, 1] == ww))[0]
        step = max(1, _MAX_BATCH_ELEMS // int(hh * ww))
        for s in range(0, len(sel), step):
            idx = sel[s:s + step]
            rows = y0[idx, None] + np.arange(hh)[None, :]
            cols = x0[idx, None] + np.arange(ww)[None, :]
            win = img[rows[:, :, None], cols[:, None, :]]
            ly = py[idx] - y0[idx] // 2 ** level
            lx = px[idx] - x0[idx] // 2 ** level
            out[idx] = _laplacian_at(win, g[idx], f, level, ly, lx, None if sc is None else sc[idx],
                                     remap_fn)
    return out.reshape(hl, wl)


def naive_llf(img, levels, f, window=True, scale=None, remap_fn=None):
    """Naive LLF of a plane (H, W) or planar channels (C, H, W); float64.

    ``scale``: optional list of per-level arrays (level l shaped like G_l);
    the coefficient at (l, p) then remaps with r = I + scale[l]_p f(I - g),
    i.e. a pixel-by-pixel remap parameter (Sec. III-B).  ``remap_fn``:
    optional (i, g) -> r(i, g) used instead of I + f(I - g)."""
    img = np.asarray(img, dtype=np.float64)
    if img.ndim == 3:
        return np.stack([naive_llf(ch, levels, f, window, scale, remap_fn) for ch in img])
    g = gaussian_pyramid(img, levels)
    lap_o = [_level_coefficients(img, g[l], l, f, window, None if scale is None else scale[l], remap_fn)
             for l in range(levels - 1)]
    lap_o.append(g[-1])
    return collapse(lap_o)


def naive_llf_adaptive(img, levels, gain, sigma_r, window=True):
    """Parameter-adaptive naive LLF (Sec. III-B): the gain m of the remap
    becomes m_p.  ``gain`` is the level-0 map (H, W); at level l the gain is
    G_l[gain]_p (reading: the Gaussian pyramid of the map, which keeps a
    constant map constant), and the coefficient at (l, p) remaps with
    f(d) = (G_l[gain]_p - 1) d exp(-d^2 / (2 sigma_r^2))."""
    gm = gaussian_pyramid(np.asarray(gain, dtype=np.float64), levels)
    unit = lambda d: d * np.exp(-d * d / (2.0 * sigma_r * sigma_r))
    return naive_llf(img, levels, unit, window, [x - 1.0 for x in gm])


__all__ = ["naive_llf", "naive_llf_adaptive", "coarse_size"]
