"""Fast local Laplacian filtering in float64 (oracle; test infrastructure only).

Sec. II-D of the paper (the fast LLF of Aubry et al. that it compares
against), step by step:

1. build the guide Gaussian pyramid G_l[I] for every level;
2. sample the intensities at equal intervals tau: g_j = lo + tau j,
   j = 0 .. S-1;
3. remap the input about every sample, R_j = r(I, g_j), and build the
   Laplacian pyramid L_l[R_j] of each;
4. at every level l below the top and pixel p, take g = G_l[I]_p, find the
   samples that bracket it, g = (1 - a) g_j + a g_{j+1} with 0 <= a <= 1,
   and interpolate: L_l[O]_p = (1 - a) L_l[R_j]_p + a L_l[R_{j+1}]_p;
   the top level is G_top[I], as in LLF;
5. collapse (Eq. (4)).

The S remapped pyramids and the guide pyramid are the |I| + 1 pyramids the
paper counts for fast LLF.

Readings where the paper is silent:

* the samples cover [lo, hi] = [0, 1] (the documented input range), so
  tau = 1 / (S - 1) and S >= 2;
* j = floor((g - lo) / tau) is clamped to 0 .. S-2, so g = hi uses the last
  pair with a = 1; a guide value outside [lo, hi] (not produced by inputs in
  [0, 1], whose Gaussian pyramid stays in [0, 1]) extrapolates linearly;
* the remap is the package's r(i, g) = i + f(i - g) with the exact
  f(d) = (m - 1) d exp(-d^2 / (2 sigma_r^2)), or any vectorised f given.
"""

import numpy as np

from .pyramid import gaussian_pyramid, laplacian_pyramid, collapse
from .remap import remap_detail


def fast_samples(S, lo=0.0, hi=1.0):
    """The S sampled intensities g_j = lo + tau j and the interval tau."""
    if S < 2:
        raise ValueError("fast LLF needs S >= 2 samples")
    tau = (hi - lo) / (S - 1)
    return lo + tau * np.arange(S), tau


def fast_bracket(g, S, lo=0.0, hi=1.0):
    """(j, a) with g = (1 - a) g_j + a g_{j+1}, j clamped to 0 .. S-2 (step 4)."""
    _, tau = fast_samples(S, lo, hi)
    t = (np.asarray(g, dtype=np.float64) - lo) / tau
    j = np.clip(np.floor(t), 0, S - 2)
    return j.astype(np.int64), t - j


def fast_llf(img, levels, S, m, sigma_r, f=None, lo=0.0, hi=1.0):
    """Fast LLF of a plane (H, W) or of planar channels (C, H, W); float64.

    ``f``: remap detail d -> f(d) (default: the exact Gaussian detail with
    m and sigma_r)."""
    img = np.asarray(img, dtype=np.float64)
    if img.ndim == 3:
        return np.stack([fast_llf(ch, levels, S, m, sigma_r, f, lo, hi) for ch in img])
    if f is None:
        f = lambda d: remap_detail(d, m, sigma_r)
    g = gaussian_pyramid(img, levels)                       # step 1
    samples, _ = fast_samples(S, lo, hi)                    # step 2
    brackets = [fast_bracket(g[l], S, lo, hi) for l in range(levels - 1)]
    out = [np.zeros_like(g[l]) for l in range(levels - 1)]
    for j, gj in enumerate(samples):
        lap_r = laplacian_pyramid(img + f(img - gj), levels)    # step 3: L_l[R_j]
        for l in range(levels - 1):                         # step 4
            jl, a = brackets[l]
            out[l] += np.where(jl == j, 1.0 - a, 0.0) * lap_r[l]
            out[l] += np.where(jl + 1 == j, a, 0.0) * lap_r[l]
    out.append(g[-1])                                       # L_top[O] = G_top[I]
    return collapse(out)                                    # step 5


__all__ = ["fast_llf", "fast_samples", "fast_bracket"]
