"""Gaussian and Laplacian pyramids in float64 (oracle; test infrastructure only).

Sec. II-A of the paper.  Eq. (1): each Gaussian level is the previous level
blurred with the 5-tap binomial kernel (standard deviation about 1) and
downsampled by two; G_0[I] = I.  Eq. (2): each Laplacian level is a Gaussian
level minus the next, coarser level upsampled with the same kernel; the top
Laplacian level is the top Gaussian level.  Eq. (4): the image is the sum of
its Laplacian levels, each brought back to full size.

Readings of points the paper leaves open (each is a numbered reading in the
design notes):

* Border: reflect-101 ("dcb|abcd|cba"), applied at every level and at the
  size of the array being filtered.
* Odd sizes: the coarse size is ceil(n/2); coarse sample j is fine sample 2j.
* Upsampling: zero insertion at the fine size (coarse j -> fine 2j, zeros at
  odd positions), then the same 5-tap kernel times 2 per axis, with
  reflect-101 at the fine size.  The result is cropped to the fine size.
* Level count: ``levels`` counts every level including level 0, so the top
  level is ``levels - 1``.
* Size-1 axes: reflect-101 has no period when n = 1, so the literal zero
  insertion would double the gain there; an axis whose fine size is 1 is
  upsampled as the identity (its single sample is the coarse sample).

All functions act on the last two axes, so a leading batch axis is allowed.
"""

import numpy as np

# 5-tap binomial kernel [1, 4, 6, 4, 1] / 16 (Sec. II-A, after Eq. (1)).
BINOMIAL5 = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def reflect101(i, n):
    """Map integer indices onto [0, n) by the reflect-101 border rule.

    The reflect-101 extension of a length-n sequence is periodic with period
    2(n-1) and mirrors about 0 and n-1 without repeating the edge sample.
    For n == 1 every index maps to 0.
    """
    i = np.asarray(i)
    if n == 1:
        return np.zeros_like(i)
    period = 2 * (n - 1)
    i = np.mod(i, period)
    return np.where(i >= n, period - i, i)


def coarse_size(n):
    """Size of the next coarser level: ceil(n/2)."""
    return (n + 1) // 2


def level_shapes(h, w, levels):
    """(height, width) of every pyramid level 0..levels-1."""
    shapes = [(h, w)]
    for _ in range(levels - 1):
        h, w = coarse_size(h), coarse_size(w)
        shapes.append((h, w))
    return shapes


def reduce(x):
    """One REDUCE step of Eq. (1): blur with the binomial kernel, keep even samples.

    out[..., j, i] = sum_{a,b} k[a] k[b] x[..., refl(2j+a-2), refl(2i+b-2)]
    """
    x = np.asarray(x, dtype=np.float64)
    h, w = x.shape[-2:]
    rows = 2 * np.arange(coarse_size(h))
    y = sum(BINOMIAL5[t] * x[..., reflect101(rows + t - 2, h), :]
            for t in range(5))
    cols = 2 * np.arange(coarse_size(w))
    return sum(BINOMIAL5[t] * y[..., :, reflect101(cols + t - 2, w)]
               for t in range(5))


def expand(x, shape):
    """Upsample a coarse level to the fine ``shape`` (the up-arrow of Eq. (2)).

    Zero insertion (coarse j -> fine 2j), then correlation with 2*k per axis
    under reflect-101 at the fine size.
    """
    x = np.asarray(x, dtype=np.float64)
    h, w = shape
    if x.shape[-2:] != (coarse_size(h), coarse_size(w)):
        raise ValueError(f"coarse shape {x.shape[-2:]} does not match fine {shape}")
    up = np.zeros(x.shape[:-2] + (h, w))
    up[..., 0::2, 0::2] = x
    k2 = 2.0 * BINOMIAL5
    rows = np.arange(h)
    y = up if h == 1 else sum(k2[t] * up[..., reflect101(rows + t - 2, h), :]
                              for t in range(5))
    if w == 1:
        return y
    cols = np.arange(w)
    return sum(k2[t] * y[..., :, reflect101(cols + t - 2, w)] for t in range(5))


def gaussian_pyramid(img, levels):
    """[G_0, ..., G_{levels-1}] with G_0 = img (Eq. (1))."""
    g = [np.asarray(img, dtype=np.float64)]
    for _ in range(levels - 1):
        g.append(reduce(g[-1]))
    return g


def laplacian_from_gaussian(g):
    """Eq. (2): L_l = G_l - expand(G_{l+1}); the top level is G_top."""
    lap = [g[l] - expand(g[l + 1], g[l].shape[-2:]) for l in range(len(g) - 1)]
    lap.append(g[-1])
    return lap


def laplacian_pyramid(img, levels):
    return laplacian_from_gaussian(gaussian_pyramid(img, levels))


def collapse(lap):
    """Eq. (4): sum the Laplacian levels from the top down, expanding each partial sum."""
    out = lap[-1]
    for l in range(len(lap) - 2, -1, -1):
        out = lap[l] + expand(out, lap[l].shape[-2:])
    return out


def reduce_matrix(n):
    """Dense 1-D REDUCE operator (ceil(n/2) x n) built from the definition.

    Used by the tests to check the 2-D REDUCE against R_h X R_w^T.
    """
    m = coarse_size(n)
    r = np.zeros((m, n))
    for j in range(m):
        for t in range(5):
            r[j, int(reflect101(2 * j + t - 2, n))] += BINOMIAL5[t]
    return r


def expand_matrix(n):
    """Dense 1-D EXPAND operator (n x ceil(n/2)) built from the definition."""
    m = coarse_size(n)
    u = np.zeros((n, m))
    if n == 1:
        u[0, 0] = 1.0
        return u
    for p in range(n):
        for t in range(5):
            q = int(reflect101(p + t - 2, n))
            if q % 2 == 0:
                u[p, q // 2] += 2.0 * BINOMIAL5[t]
    return u
