"""Pins for the oracle's pyramid primitives (Eqs. (1), (2), (4)).

Each check is independent of the oracle's own code: a library routine
(scipy.ndimage.correlate1d with the 'mirror' border, which is reflect-101),
a hand-written dense matrix, or an invariant of the definition.
"""

import numpy as np
import pytest
from scipy import ndimage

import oracle as o

K5 = np.array([1, 4, 6, 4, 1]) / 16.0


def scipy_reduce(x):
    y = ndimage.correlate1d(x, K5, axis=0, mode="mirror")
    y = ndimage.correlate1d(y, K5, axis=1, mode="mirror")
    return y[0::2, 0::2]


def scipy_expand(x, shape):
    up = np.zeros(shape)
    up[0::2, 0::2] = x
    y = ndimage.correlate1d(up, 2 * K5, axis=0, mode="mirror")
    return ndimage.correlate1d(y, 2 * K5, axis=1, mode="mirror")


@pytest.mark.parametrize("h,w", [(3, 3), (4, 7), (8, 5), (9, 9), (16, 11), (31, 64)])
def test_reduce_expand_match_scipy_mirror(h, w):
    rng = np.random.default_rng(h * 100 + w)
    x = rng.standard_normal((h, w))
    np.testing.assert_allclose(o.reduce(x), scipy_reduce(x), rtol=0, atol=1e-14)
    c = rng.standard_normal(((h + 1) // 2, (w + 1) // 2))
    np.testing.assert_allclose(o.expand(c, (h, w)), scipy_expand(c, (h, w)),
                               rtol=0, atol=1e-14)


def test_reflect101_small_sizes():
    # dcb|abcd|cba on n = 4; n = 2 alternates; n = 1 is constant.
    np.testing.assert_array_equal(o.reflect101(np.arange(-3, 7), 4),
                                  [3, 2, 1, 0, 1, 2, 3, 2, 1, 0])
    np.testing.assert_array_equal(o.reflect101(np.arange(-2, 4), 2), [0, 1, 0, 1, 0, 1])
    np.testing.assert_array_equal(o.reflect101(np.arange(-2, 3), 1), [0] * 5)


def _hand_reduce_matrix(n):
    # Row j of REDUCE on an interior point: weights 1,4,6,4,1 at 2j-2..2j+2;
    # out-of-range taps folded back by the mirror written out by hand.
    m = (n + 1) // 2
    r = np.zeros((m, n))
    for j in range(m):
        for t, wgt in zip(range(-2, 3), K5):
            i = 2 * j + t
            while i < 0 or i > n - 1:
                i = -i if i < 0 else 2 * (n - 1) - i
            if n == 1:
                i = 0
            r[j, i] += wgt
    return r


@pytest.mark.parametrize("n", range(3, 12))
def test_dense_operator_matrices(n):
    rng = np.random.default_rng(n)
    r = _hand_reduce_matrix(n)
    np.testing.assert_allclose(o.reduce_matrix(n), r, atol=1e-15)
    # 2-D REDUCE is R_h X R_w^T.
    x = rng.standard_normal((n, n + 2))
    np.testing.assert_allclose(o.reduce(x), r @ x @ _hand_reduce_matrix(n + 2).T, atol=1e-14)
    # EXPAND rows sum to one (constant preserving) and match the 2-D operator.
    u = o.expand_matrix(n)
    np.testing.assert_allclose(u.sum(axis=1), 1.0, atol=1e-15)
    c = rng.standard_normal(((n + 1) // 2, (n + 3) // 2))
    np.testing.assert_allclose(o.expand(c, (n, n + 2)), u @ c @ o.expand_matrix(n + 2).T,
                               atol=1e-14)


@pytest.mark.parametrize("h,w", [(1, 1), (1, 5), (2, 2), (3, 8), (17, 9)])
def test_constant_preserved(h, w):
    x = np.full((h, w), 0.37)
    np.testing.assert_allclose(o.reduce(x), 0.37, atol=1e-15)
    np.testing.assert_allclose(o.expand(o.reduce(x), (h, w)), 0.37, atol=1e-15)


def test_level_shapes_odd():
    assert o.level_shapes(2160, 3840, 8)[-1] == (17, 30)
    assert o.level_shapes(5, 9, 4) == [(5, 9), (3, 5), (2, 3), (1, 2)]


@pytest.mark.parametrize("h,w,levels", [(1, 1, 1), (7, 5, 3), (33, 64, 6), (64, 48, 8)])
def test_perfect_reconstruction(h, w, levels):
    # collapse(laplacian(I)) == I: Eq. (2) telescopes under Eq. (4).
    x = np.random.default_rng(h + w).random((h, w))
    np.testing.assert_allclose(o.collapse(o.laplacian_pyramid(x, levels)), x, atol=1e-13)


def test_batched_axes_match_unbatched():
    x = np.random.default_rng(3).random((4, 13, 10))
    np.testing.assert_allclose(o.reduce(x)[2], o.reduce(x[2]), atol=0)
    c = o.reduce(x)
    np.testing.assert_allclose(o.expand(c, (13, 10))[1], o.expand(c[1], (13, 10)), atol=0)
