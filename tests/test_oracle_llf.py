"""Pins for the Fourier LLF oracle (Eq. (14)) and the naive LLF oracle (Sec. II-C).

Fourier LLF with coefficients a_k is exactly naive LLF run with the
truncated remap f_K (the pyramid is linear), so the two oracles -- which
share only the pinned pyramid primitives -- check each other at roundoff.
"""

import numpy as np
import pytest

import oracle as o
from paper_2206_04681_gb300.synth import synth_image


def _img(h, w, seed):
    return synth_image(h, w, 1, polygons=3, seed=seed)[0].astype(np.float64)


@pytest.mark.parametrize("h,w,levels,K", [(8, 8, 2, 2), (21, 17, 3, 4), (40, 33, 4, 8),
                                          (64, 64, 5, 6), (13, 50, 4, 16)])
def test_fourier_equals_naive_with_truncated_remap(h, w, levels, K):
    img = _img(h, w, h * w)
    a = o.coeffs_quadrature(3.0, 0.2, 2.0, K)
    fk = lambda d: o.fourier_detail(d, a, 2.0)
    out_f = o.fourier_llf(img, levels, a, 2.0)
    out_n = o.naive_llf(img, levels, fk, window=False)
    np.testing.assert_allclose(out_f, out_n, rtol=0, atol=1e-12)


def test_windowed_naive_equals_whole_image():
    # Windows are strictly smaller than the image at levels 0..2 here.
    img = _img(96, 80, 5)
    f = lambda d: o.remap_detail(d, 3.0, 0.1)
    full = o.naive_llf(img, 4, f, window=False)
    win = o.naive_llf(img, 4, f, window=True)
    np.testing.assert_allclose(win, full, rtol=0, atol=1e-13)


@pytest.mark.parametrize("m", [1.0])
def test_identity_remap_returns_input(m):
    img = _img(37, 45, 2)
    a = o.coeffs_quadrature(m, 0.2, 2.0, 8)
    np.testing.assert_allclose(o.fourier_llf(img, 5, a, 2.0), img, atol=1e-13)
    f = lambda d: o.remap_detail(d, m, 0.2)
    np.testing.assert_allclose(o.naive_llf(img, 5, f), img, atol=1e-13)


@pytest.mark.parametrize("m,sigma,K", [(3.0, 0.2, 8), (0.5, 0.4, 4), (4.0, 0.05, 16)])
def test_constant_image_unchanged(m, sigma, K):
    img = np.full((19, 26), 0.42)
    a = o.coeffs_quadrature(m, sigma, 2.0, K)
    np.testing.assert_allclose(o.fourier_llf(img, 4, a, 2.0), 0.42, atol=1e-13)
    f = lambda d: o.remap_detail(d, m, sigma)
    np.testing.assert_allclose(o.naive_llf(img, 4, f), 0.42, atol=1e-13)


def test_level0_fourier_term_cancels():
    # r(I, I_p) = I (Eq. (14) text): the S~_0 / C~_0 part of L_0[O] vanishes.
    img = _img(33, 31, 9)
    a = o.coeffs_quadrature(3.0, 0.2, 2.0, 8)
    _, term0 = o.fourier_llf_levels(img, 4, a, 2.0)
    assert np.max(np.abs(term0)) < 1e-15


@pytest.mark.parametrize("c", [0.5, 2.0, -0.7])
def test_linear_remap_is_laplacian_enhancement(c):
    # With f(d) = c d, every L_l[r_g(I)]_p = (1 + c) L_l[I]_p because the
    # Laplacian of a constant is zero, so naive LLF reduces to Eq. (3) with
    # r(i, 0) = (1 + c) i on every level below the top.
    img = _img(45, 38, 4)
    levels = 4
    lap = o.laplacian_pyramid(img, levels)
    expect = o.collapse([(1 + c) * l for l in lap[:-1]] + [lap[-1]])
    got = o.naive_llf(img, levels, lambda d: c * d, window=True)
    np.testing.assert_allclose(got, expect, atol=1e-13)


def test_fourier_error_bounded_by_series_error_and_falls_with_K():
    # |O_Fourier - O_naive| <= 2 (L - 1) sup_D |f_K - f|: REDUCE and EXPAND
    # are convex combinations, so |L_l[u]| <= 2 sup|u| and the collapse adds
    # one such term per level below the top.
    img = _img(48, 40, 11)
    levels, m, sigma = 4, 3.0, 0.1
    f = lambda d: o.remap_detail(d, m, sigma)
    naive = o.naive_llf(img, levels, f)
    d = np.linspace(img.min() - img.max(), img.max() - img.min(), 8001)
    errs = []
    for K in (4, 8, 16):
        a = o.coeffs_quadrature(m, sigma, 2.0, K)
        err = np.max(np.abs(o.fourier_llf(img, levels, a, 2.0) - naive))
        sup = np.max(np.abs(o.fourier_detail(d, a, 2.0) - f(d)))
        assert err <= 2 * (levels - 1) * sup + 1e-12
        errs.append(err)
    assert errs[0] > errs[1] > errs[2]


def test_channels_filtered_independently():
    img = synth_image(20, 24, 3, polygons=3, seed=8).astype(np.float64)
    a = o.coeffs_quadrature(3.0, 0.2, 2.0, 4)
    out = o.fourier_llf(img, 3, a, 2.0)
    for c in range(3):
        np.testing.assert_array_equal(out[c], o.fourier_llf(img[c], 3, a, 2.0))


def test_enhancement_increases_local_contrast():
    # m > 1 amplifies the small-amplitude texture: the mean absolute finest
    # Laplacian coefficient grows.
    img = _img(64, 64, 12)
    a = o.coeffs_quadrature(3.0, 0.2, 2.0, 8)
    out = o.fourier_llf(img, 4, a, 2.0)
    before = np.mean(np.abs(o.laplacian_pyramid(img, 2)[0]))
    after = np.mean(np.abs(o.laplacian_pyramid(out, 2)[0]))
    assert after > 1.3 * before


# ---- pixel-by-pixel enhancement (Sec. III-B) ----------------------------------------
def _gain_map(h, w, seed, lo=0.5, hi=4.0):
    """A smooth, non-constant gain map in [lo, hi] (values of the paper's m range)."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:h, 0:w]
    a, b, ph = rng.uniform(0.05, 0.3), rng.uniform(0.05, 0.3), rng.uniform(0, 6.3)
    return lo + (hi - lo) * 0.5 * (1 + np.sin(a * y + ph) * np.cos(b * x))


@pytest.mark.parametrize("h,w,levels,K", [(16, 16, 3, 3), (21, 17, 3, 4), (40, 33, 4, 8),
                                          (13, 50, 4, 6)])
def test_adaptive_fourier_equals_adaptive_naive_with_truncated_remap(h, w, levels, K):
    # Per pixel the remap detail is (m_p - 1) times the unit detail, whose
    # K-term series has coefficients c_k: the adaptive Fourier LLF must equal
    # the per-pixel naive LLF run with that truncated series, at roundoff.
    img = _img(h, w, 7 * h + w)
    gain = _gain_map(h, w, h * w)
    c = o.coeffs_quadrature(2.0, 0.2, 2.0, K)        # m - 1 = 1: the unit detail
    unit_k = lambda d: o.fourier_detail(d, c, 2.0)
    gm = o.gaussian_pyramid(gain, levels)
    out_f = o.fourier_llf_adaptive(img, levels, c, 2.0, gain)
    out_n = o.naive_llf(img, levels, unit_k, window=False, scale=[x - 1.0 for x in gm])
    np.testing.assert_allclose(out_f, out_n, rtol=0, atol=1e-12)


@pytest.mark.parametrize("m", [0.5, 3.0])
def test_adaptive_with_constant_gain_is_the_fixed_filter(m):
    img = _img(37, 29, 11)
    gain = np.full(img.shape, m)
    c = o.coeffs_quadrature(2.0, 0.15, 2.0, 8)
    a = o.coeffs_quadrature(m, 0.15, 2.0, 8)
    np.testing.assert_allclose(o.fourier_llf_adaptive(img, 5, c, 2.0, gain),
                               o.fourier_llf(img, 5, a, 2.0), rtol=0, atol=1e-12)
    f = lambda d: o.remap_detail(d, m, 0.15)
    np.testing.assert_allclose(o.naive_llf_adaptive(img, 4, gain, 0.15, window=False),
                               o.naive_llf(img, 4, f, window=False), rtol=0, atol=1e-13)


def test_adaptive_unit_gain_returns_input_and_windowed_naive_matches():
    img = _img(48, 40, 3)
    c = o.coeffs_quadrature(2.0, 0.2, 2.0, 6)
    out = o.fourier_llf_adaptive(img, 5, c, 2.0, np.ones_like(img))
    np.testing.assert_allclose(out, img, rtol=0, atol=1e-13)
    gain = _gain_map(48, 40, 5)
    full = o.naive_llf_adaptive(img, 4, gain, 0.1, window=False)
    win = o.naive_llf_adaptive(img, 4, gain, 0.1, window=True)
    np.testing.assert_allclose(win, full, rtol=0, atol=1e-13)


# ---- colour by luma (Sec. IV: LLF on Y of YUV, U and V kept) -------------------------
def test_yuv_round_trip_and_luma_of_gray():
    rng = np.random.default_rng(0)
    rgb = rng.uniform(0, 1, (3, 9, 7))
    np.testing.assert_allclose(o.yuv_to_rgb(o.rgb_to_yuv(rgb)), rgb, rtol=0, atol=1e-14)
    gray = np.repeat(rng.uniform(0, 1, (1, 5, 6)), 3, axis=0)
    yuv = o.rgb_to_yuv(gray)
    np.testing.assert_allclose(yuv[0], gray[0], rtol=0, atol=1e-15)   # weights sum to 1
    np.testing.assert_allclose(yuv[1:], 0.0, rtol=0, atol=1e-15)


def test_luma_mode_of_a_gray_image_filters_each_channel_alike():
    img = _img(40, 36, 2)
    a = o.coeffs_quadrature(3.0, 0.2, 2.0, 6)
    out = o.fourier_llf_luma(np.stack([img] * 3), 5, a, 2.0)
    ref = o.fourier_llf(img, 5, a, 2.0)
    for c in range(3):
        np.testing.assert_allclose(out[c], ref, rtol=0, atol=1e-13)


def test_luma_mode_adds_the_luma_change_to_every_channel():
    # U and V kept => every channel moves by Y' - Y (the form the library uses)
    rgb = synth_image(33, 45, 3, polygons=4, seed=6).astype(np.float64)
    a = o.coeffs_quadrature(2.5, 0.15, 2.0, 8)
    out = o.fourier_llf_luma(rgb, 5, a, 2.0)
    y = sum(w * c for w, c in zip(o.LUMA_BT601, rgb))
    dy = o.fourier_llf(y, 5, a, 2.0) - y
    np.testing.assert_allclose(out, rgb + dy[None], rtol=0, atol=1e-13)
    np.testing.assert_allclose(o.fourier_llf_luma(rgb, 5, a * 0.0, 2.0), rgb, rtol=0, atol=1e-13)
