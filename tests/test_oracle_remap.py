"""Pins for the remap function, its Fourier coefficients and Eq. (12)."""

import math
import os

import numpy as np
import pytest

import oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("m,sigma,T", [(3.0, 0.1, 2.0), (3.0, 0.2, 2.0), (0.5, 0.4, 2.0),
                                       (4.0, 0.05, 2.0), (7.0, 15.0, 256.0)])
def test_quadrature_matches_closed_form_within_tail(m, sigma, T):
    # Eqs. (9)-(11) integrate over the whole line; the period integral differs
    # only by the Gaussian tail outside [-T/2, T/2].
    K = 16
    q = o.coeffs_quadrature(m, sigma, T, K)
    cf = o.coeffs_closed_form(m, sigma, T, K)
    bound = o.coeff_tail_bound(m, sigma, T)
    assert np.max(np.abs(q - cf)) <= bound + 1e-14 * max(1.0, np.max(np.abs(cf)))


def test_quadrature_is_an_orthogonal_projection():
    # The sine basis is orthogonal on one period: projecting sin(omega_j x)
    # returns the unit vector e_j.
    T, K = 2.0, 12
    for j in (1, 5, 12):
        om = 2 * math.pi * j / T
        a = o.coeffs_quadrature(0, 1, T, K, detail=lambda x: np.sin(om * x))
        expect = np.zeros(K)
        expect[j - 1] = 1.0
        np.testing.assert_allclose(a, expect, atol=1e-13)


def test_quadrature_converged():
    a1 = o.coeffs_quadrature(3.0, 0.2, 2.0, 64)
    a2 = o.coeffs_quadrature(3.0, 0.2, 2.0, 64, panels=1024, nodes=24)
    np.testing.assert_allclose(a1, a2, atol=1e-15)


def test_identity_remap_has_zero_coefficients():
    assert np.all(o.coeffs_quadrature(1.0, 0.2, 2.0, 8) == 0.0)
    np.testing.assert_array_equal(o.remap(np.array([0.1, 0.7]), 0.3, 1.0, 0.2), [0.1, 0.7])


def test_remap_enhances_small_details():
    # m > 1 pushes i away from g for |i - g| << sigma_r; far intensities stay.
    g = 0.5
    assert o.remap(0.52, g, 3.0, 0.1) > 0.53
    assert o.remap(0.48, g, 3.0, 0.1) < 0.47
    assert abs(o.remap(0.95, g, 3.0, 0.1) - 0.95) < 1e-3
    assert abs(o.remap(0.52, g, 0.5, 0.1) - g) < 0.02 - 1e-3


def test_series_converges_for_narrow_remap():
    # sup |f_K - f| over |d| <= 1 falls with K when sigma_r <= 0.2 (T = 2).
    d = np.linspace(-1, 1, 4001)
    f = o.remap_detail(d, 3.0, 0.1)
    errs = []
    for K in (4, 8, 16):
        a = o.coeffs_quadrature(3.0, 0.1, 2.0, K)
        errs.append(np.max(np.abs(o.fourier_detail(d, a, 2.0) - f)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_optimal_period_matches_paper():
    # Sec. IV: sigma_r = 30 (0-255 range) gives T = 405.9 as the minimiser of Eq. (12).
    rows = [l.split() for l in open(os.path.join(GOLDEN, "period_sigma30.txt"))
            if l.strip() and not l.startswith("#")]
    for sigma, K, R, T in rows:
        t = o.optimal_period(float(sigma), int(K), float(R))
        assert abs(t - float(T)) / float(T) < 2e-3
        # and it is a local minimum of E_K(T)
        e = o.period_error(t, float(sigma), int(K), float(R))
        assert e <= o.period_error(t * 0.99, float(sigma), int(K), float(R))
        assert e <= o.period_error(t * 1.01, float(sigma), int(K), float(R))
