"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on natural photographs (512 x 512 grayscale test images
and colour photographs, Sec. IV) that are not available here.  These
generators stand in for them with images that have the same ingredients a
local Laplacian filter reacts to: flat regions separated by step edges
(large |i - g|, which the remap must leave alone) and fine texture plus
noise (small |i - g|, which the remap enhances or smooths).

Recipe (every draw from ``numpy.random.default_rng(seed)``, in this order):

* background level ~ U[0.1, 0.9];
* ``polygons`` random simple polygons painted in order (later on top): a
  centre uniform over the image, 3-8 vertices at sorted uniform angles,
  radii log-uniform in [0.03, 0.3] * min(H, W), a constant level
  ~ U[0.1, 0.9], hard step edges (no anti-aliasing);
* per region (background and each polygon) a 2-D sinusoid texture of
  amplitude 0.05, period ~ U[4, 32] px, orientation ~ U[0, pi),
  phase ~ U[0, 2 pi);
* additive Gaussian noise, sigma = 0.02; clamp to [0, 1];
* colour images share the polygon geometry; each channel draws its own
  levels, textures and noise.

This module holds input generation only and none of the filter's
arithmetic; both the CUDA path's tests and the oracle consume its output.
"""

import math

import numpy as np


def _polygon_mask(h, w, cx, cy, angles, radii):
    """Even-odd rule rasterisation of one polygon over its bounding box."""
    vx = cx + radii * np.cos(angles)
    vy = cy + radii * np.sin(angles)
    x0, x1 = max(int(math.floor(vx.min())), 0), min(int(math.ceil(vx.max())) + 1, w)
    y0, y1 = max(int(math.floor(vy.min())), 0), min(int(math.ceil(vy.max())) + 1, h)
    if x0 >= x1 or y0 >= y1:
        return None
    ys, xs = np.mgrid[y0:y1, x0:x1]
    px, py = xs + 0.5, ys + 0.5
    inside = np.zeros(px.shape, dtype=bool)
    n = len(vx)
    for e in range(n):
        ax, ay, bx, by = vx[e], vy[e], vx[(e + 1) % n], vy[(e + 1) % n]
        crosses = (ay > py) != (by > py)
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = ax + (py - ay) * (bx - ax) / (by - ay)
        inside ^= crosses & (px < xint)
    return (y0, y1, x0, x1), inside


def polygon_labels(h, w, polygons, rng):
    """Region label per pixel: 0 = background, j = j-th polygon (topmost wins)."""
    labels = np.zeros((h, w), dtype=np.int32)
    s = min(h, w)
    for j in range(1, polygons + 1):
        nv = int(rng.integers(3, 9))
        cx, cy = rng.uniform(0, w), rng.uniform(0, h)
        angles = np.sort(rng.uniform(0, 2 * np.pi, nv))
        radii = np.exp(rng.uniform(np.log(0.03), np.log(0.3), nv)) * s
        hit = _polygon_mask(h, w, cx, cy, angles, radii)
        if hit is None:
            continue
        (y0, y1, x0, x1), inside = hit
        labels[y0:y1, x0:x1][inside] = j
    return labels


def synth_image(h, w, channels=1, polygons=6, seed=0):
    """Planar float32 image (channels, h, w) in [0, 1] following the recipe above."""
    rng = np.random.default_rng(seed)
    background = [rng.uniform(0.1, 0.9) for _ in range(channels)]
    labels = polygon_labels(h, w, polygons, rng)
    nreg = polygons + 1
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    out = np.empty((channels, h, w), dtype=np.float32)
    for c in range(channels):
        level = rng.uniform(0.1, 0.9, nreg)
        level[0] = background[c]
        period = rng.uniform(4.0, 32.0, nreg)
        theta = rng.uniform(0.0, np.pi, nreg)
        phase = rng.uniform(0.0, 2 * np.pi, nreg)
        kx = (2 * np.pi / period * np.cos(theta))[labels]
        ky = (2 * np.pi / period * np.sin(theta))[labels]
        img = level[labels] + 0.05 * np.sin(kx * xs + ky * ys + phase[labels])
        img += rng.normal(0.0, 0.02, (h, w))
        out[c] = np.clip(img, 0.0, 1.0)
    return out


# Fixed workloads.  Sizes and parameters follow the filter's headline
# configurations: a small grayscale check image and a 4K RGB frame.
SMALL_GRAY = dict(H=256, W=256, C=1, polygons=6, seed=1,
                  levels=5, K=4, m=3.0, sigma_r=0.1, T=2.0)
UHD_RGB = dict(H=2160, W=3840, C=3, polygons=40, seed=2,
               levels=8, K=8, m=3.0, sigma_r=0.2, T=2.0)


def workload_image(cfg):
    return synth_image(cfg["H"], cfg["W"], cfg["C"], cfg["polygons"], cfg["seed"])


def auto_levels(h, w, cap=8):
    """Pyramid depth for images of arbitrary size: the top side stays >= 8 px."""
    s = min(h, w)
    return max(1, min(cap, 1 + int(math.floor(math.log2(max(s, 1) / 8.0))))) if s >= 8 else 1


def batch_workload(n=64, seed=4):
    """Mixed-size batch: sides log-uniform in [256, 4096], aspect in [0.5, 2].

    Each item is a dict with the image and its own filter parameters
    (K in {4, 8}, sigma_r ~ U[0.05, 0.4], m ~ U[0.5, 4], T = 2).
    """
    rng = np.random.default_rng(seed)
    items = []
    for i in range(n):
        w = int(round(math.exp(rng.uniform(math.log(256), math.log(4096)))))
        a = math.exp(rng.uniform(math.log(0.5), math.log(2.0)))
        h = int(min(max(round(w * a), 256), 4096))
        c = 3 if rng.uniform() < 0.5 else 1
        p = int(min(max(round(40 * h * w / (3840 * 2160)), 6), 40))
        k = int(rng.choice([4, 8]))
        sigma = float(rng.uniform(0.05, 0.4))
        m = float(rng.uniform(0.5, 4.0))
        img_seed = int(rng.integers(0, 2 ** 31 - 1))
        items.append(dict(H=h, W=w, C=c, polygons=p, seed=img_seed,
                          levels=auto_levels(h, w), K=k, m=m, sigma_r=sigma, T=2.0))
    return items


def request_stream(rate, duration, seed=5, max_side=8192, min_side=512):
    """Poisson arrivals of filter requests (arrival time in s, parameters).

    Sides log-uniform in [min_side, max_side], aspect in [0.5, 2],
    C in {1, 3}, K in {4, 8, 16}, sigma_r ~ U[0.05, 0.4], m ~ U[0.5, 4], T = 2.
    """
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        w = int(round(math.exp(rng.uniform(math.log(min_side), math.log(max_side)))))
        a = math.exp(rng.uniform(math.log(0.5), math.log(2.0)))
        h = int(min(max(round(w * a), min_side), max_side))
        c = 3 if rng.uniform() < 0.5 else 1
        out.append(dict(t=t, H=h, W=w, C=c,
                        polygons=int(min(max(round(40 * h * w / (3840 * 2160)), 6), 40)),
                        seed=int(rng.integers(0, 2 ** 31 - 1)),
                        levels=auto_levels(h, w), K=int(rng.choice([4, 8, 16])),
                        m=float(rng.uniform(0.5, 4.0)),
                        sigma_r=float(rng.uniform(0.05, 0.4)), T=2.0))


def variance_gain_map(img, m_lo=1.0, m_hi=3.0, radius=3, var_ref=None):
    """Per-pixel gain map for pixel-adaptive enhancement, as in the paper's
    experiment: the degree of enhancement follows the variance of the pixels
    in a local window, and low variance gets a small enhancement.

    ``img``: (H, W) or (C, H, W); the variance is taken over a
    (2 radius + 1)^2 box of the channel mean (edges replicated).  The gain is
    m_lo + (m_hi - m_lo) * min(var / var_ref, 1), with var_ref the 90th
    percentile of the variance unless given.  Returns (H, W) float32.
    """
    x = np.asarray(img, dtype=np.float64)
    if x.ndim == 3:
        x = x.mean(axis=0)
    k = 2 * radius + 1
    pad = np.pad(x, radius, mode="edge")
    s1 = np.zeros_like(x)
    s2 = np.zeros_like(x)
    h, w = x.shape
    for dy in range(k):
        for dx in range(k):
            v = pad[dy:dy + h, dx:dx + w]
            s1 += v
            s2 += v * v
    mean = s1 / (k * k)
    var = np.maximum(s2 / (k * k) - mean * mean, 0.0)
    ref = float(np.percentile(var, 90)) if var_ref is None else float(var_ref)
    t = np.minimum(var / max(ref, 1e-12), 1.0)
    return (m_lo + (m_hi - m_lo) * t).astype(np.float32)
