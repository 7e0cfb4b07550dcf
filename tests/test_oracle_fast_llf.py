"""Pins of the fast LLF oracle (Sec. II-D) against facts fixed independently of it.

* Linearity: fast LLF is naive LLF run with the remap interpolated in its
  reference value, r~(i, g) = sum_j hat_j(g) r(i, g_j) (hat functions on the
  sample grid, written here without the oracle's floor/clamp), because the
  Laplacian pyramid is linear and the hat weights sum to one.  The naive
  oracle is pinned on its own (test_oracle_llf.py), so this fixes the
  remapped pyramids, the bracketing, the interpolation and the collapse.
* m = 1: f = 0 and every remapped image is I: the output is the input.
* A constant image stays constant.
* A linear detail f(d) = c d makes L_l[R_j] = (1 + c) L_l[I] for every
  sample: the output is the Laplacian enhancement (Eq. (3)) for any S.
* Sampling error: against naive LLF with the exact remap, the error is at
  most (levels - 1) tau^2 sup|f''| / 4 (linear interpolation in g of
  L_l[r(I, g)]_p, whose second g-derivative is L_l[f''(I - g)]_p with
  |L_l| <= 2, summed over the convex collapse), and it falls with S.
"""

import numpy as np
import pytest

import oracle as o


def _img(h, w, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:h, 0:w]
    base = 0.5 + 0.3 * np.sin(x / 3.0 + seed) * np.cos(y / 4.0)
    return np.clip(base + 0.05 * rng.standard_normal((h, w)), 0.0, 1.0)


def _hat_remap(samples, m, sigma):
    tau = samples[1] - samples[0]

    def r(i, g):
        out = np.zeros(np.broadcast(i, g).shape)
        for gj in samples:
            w = np.maximum(0.0, 1.0 - np.abs(g - gj) / tau)
            out = out + w * o.remap(i, gj, m, sigma)
        return out
    return r


@pytest.mark.parametrize("h,w,levels,S,m,sigma", [
    (23, 31, 3, 5, 3.0, 0.2),
    (40, 33, 4, 9, 0.5, 0.3),
    (17, 48, 4, 2, 4.0, 0.1),
    (32, 32, 5, 16, 2.0, 0.15),
])
def test_equals_naive_llf_with_the_interpolated_remap(h, w, levels, S, m, sigma):
    img = _img(h, w, h + w)
    samples, _ = o.fast_samples(S)
    fast = o.fast_llf(img, levels, S, m, sigma)
    naive = o.naive_llf(img, levels, None, window=False, remap_fn=_hat_remap(samples, m, sigma))
    assert np.max(np.abs(fast - naive)) <= 1e-12


def test_identity_constant_and_channels():
    img = _img(30, 26, 3)
    assert np.max(np.abs(o.fast_llf(img, 4, 8, 1.0, 0.2) - img)) <= 1e-13
    c = np.full((21, 19), 0.37)
    assert np.max(np.abs(o.fast_llf(c, 4, 6, 3.0, 0.2) - 0.37)) <= 1e-13
    rgb = np.stack([img, img[::-1], 1.0 - img])
    out = o.fast_llf(rgb, 4, 8, 3.0, 0.2)
    for ch in range(3):
        np.testing.assert_allclose(out[ch], o.fast_llf(rgb[ch], 4, 8, 3.0, 0.2), rtol=0, atol=0)


@pytest.mark.parametrize("S", [2, 3, 7])
def test_linear_detail_is_laplacian_enhancement(S):
    img = _img(27, 35, 5)
    c, levels = 0.7, 4
    out = o.fast_llf(img, levels, S, 0.0, 1.0, f=lambda d: c * d)
    lap = o.laplacian_pyramid(img, levels)
    ref = o.collapse([(1.0 + c) * x for x in lap[:-1]] + [lap[-1]])
    assert np.max(np.abs(out - ref)) <= 1e-12


def test_bracketing():
    j, a = o.fast_bracket(np.array([0.0, 0.1, 0.5, 0.999, 1.0]), 5)
    np.testing.assert_array_equal(j, [0, 0, 2, 3, 3])
    np.testing.assert_allclose(a, [0.0, 0.4, 0.0, 0.996, 1.0], atol=1e-12)
    with pytest.raises(ValueError):
        o.fast_samples(1)


def test_sampling_error_bound_and_decay():
    img = _img(48, 40, 9)
    levels, m, sigma = 4, 3.0, 0.2
    naive = o.naive_llf(img, levels, lambda d: o.remap_detail(d, m, sigma), window=False)
    d = np.linspace(-1.0, 1.0, 200001)
    f2 = (m - 1.0) * (d ** 3 / sigma ** 4 - 3.0 * d / sigma ** 2) * np.exp(-d * d / (2 * sigma * sigma))
    sup_f2 = float(np.max(np.abs(f2)))
    errs = []
    for S in (4, 8, 16, 32):
        tau = 1.0 / (S - 1)
        err = float(np.max(np.abs(o.fast_llf(img, levels, S, m, sigma) - naive)))
        assert err <= (levels - 1) * tau * tau * sup_f2 / 4.0
        errs.append(err)
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_windowed_naive_with_the_interpolated_remap():
    # the exact dependency windows of naive LLF hold for a remap of (i, g) too
    img = _img(44, 52, 12)
    levels, S, m, sigma = 4, 7, 3.0, 0.2
    samples, _ = o.fast_samples(S)
    r = _hat_remap(samples, m, sigma)
    whole = o.naive_llf(img, levels, None, window=False, remap_fn=r)
    windowed = o.naive_llf(img, levels, None, window=True, remap_fn=r)
    assert np.max(np.abs(windowed - whole)) <= 1e-12
    assert np.max(np.abs(o.fast_llf(img, levels, S, m, sigma) - windowed)) <= 1e-12
