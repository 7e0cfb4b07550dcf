"""Remap function and its Fourier sine series (oracle; test infrastructure only).

Sec. II-E and III-A of the paper.

Reading of the remap (the paper's Eq. (5) and Eq. (11) disagree in sign; the
reading below agrees with Eq. (11) and with "m > 0 enhances"): the remapped
intensity is

    r_g(i) = i + f(i - g),   f(d) = (m - 1) * d * exp(-d^2 / (2 sigma_r^2)),

so m = 1 is the identity, m > 1 enhances detail and m < 1 smooths it.  This
is the paper's detail term (i - g) w_r(i - g) with the paper's multiplier
m_paper = m - 1.

Fourier sine series over the period T (Eqs. (9)-(11)):

    f(d) ~= f_K(d) = sum_{k=1..K} a_k sin(omega_k d),   omega_k = 2 pi k / T.

``coeffs_quadrature`` integrates f over one period (the default);
``coeffs_closed_form`` is the paper's closed form
a_k = m_paper * 2 sigma_r^2 alpha_k omega_k with
alpha_k = sigma_r sqrt(2 pi) / T * exp(-(omega_k sigma_r)^2 / 2), which is the
integral over the whole real line.  They differ by at most
``coeff_tail_bound``.
"""

import math

import numpy as np


def remap_detail(d, m, sigma_r):
    """f(d) = (m - 1) d exp(-d^2 / (2 sigma_r^2))."""
    d = np.asarray(d, dtype=np.float64)
    return (m - 1.0) * d * np.exp(-d * d / (2.0 * sigma_r * sigma_r))


def remap(i, g, m, sigma_r):
    """r_g(i) = i + f(i - g)."""
    i = np.asarray(i, dtype=np.float64)
    return i + remap_detail(i - g, m, sigma_r)


def omegas(T, K):
    """omega_k = 2 pi k / T for k = 1..K (Eq. (9))."""
    return 2.0 * np.pi * np.arange(1, K + 1) / T


def coeffs_quadrature(m, sigma_r, T, K, panels=512, nodes=16, detail=None):
    """a_k = (2/T) * integral_{-T/2}^{T/2} f(x) sin(omega_k x) dx, k = 1..K.

    Composite Gauss-Legendre quadrature (``panels`` equal panels of
    ``nodes`` nodes) in float64.  ``detail`` overrides f (a callable d -> f(d)).
    """
    x, w = np.polynomial.legendre.leggauss(nodes)
    edges = np.linspace(-T / 2.0, T / 2.0, panels + 1)
    lo, hi = edges[:-1], edges[1:]
    half = (hi - lo) / 2.0
    xs = (half[:, None] * x[None, :] + ((lo + hi) / 2.0)[:, None]).ravel()
    ws = (half[:, None] * w[None, :]).ravel()
    fx = remap_detail(xs, m, sigma_r) if detail is None else np.asarray(detail(xs))
    return np.array([(2.0 / T) * np.sum(ws * fx * np.sin(om * xs))
                     for om in omegas(T, K)])


def coeffs_closed_form(m, sigma_r, T, K):
    """Eqs. (9)-(11): a_k = (m - 1) * 2 sigma_r^2 alpha_k omega_k."""
    om = omegas(T, K)
    alpha = sigma_r * math.sqrt(2.0 * math.pi) / T * np.exp(-0.5 * (om * sigma_r) ** 2)
    return (m - 1.0) * 2.0 * sigma_r * sigma_r * alpha * om


def coeff_tail_bound(m, sigma_r, T):
    """Bound on |quadrature - closed form| for every k.

    The closed form integrates over the whole line; the part outside
    [-T/2, T/2] is at most (2/T) * 2 * |m-1| * int_{T/2}^inf x exp(-x^2/2s^2) dx.
    """
    return 4.0 / T * abs(m - 1.0) * sigma_r ** 2 * math.exp(-T * T / (8.0 * sigma_r ** 2))


def fourier_detail(d, a, T):
    """f_K(d) = sum_k a_k sin(omega_k d)."""
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    for ak, om in zip(a, omegas(T, len(a))):
        out = out + ak * np.sin(om * d)
    return out


def period_error(T, sigma, K, R):
    """E_K(T) of Eq. (12): erfc(pi sigma (2K+1) / T) + erfc((T - R) / sigma)."""
    return math.erfc(math.pi * sigma * (2 * K + 1) / T) + math.erfc((T - R) / sigma)


def optimal_period(sigma, K, R, tol=1e-10):
    """argmin_T E_K(T) (Eq. (12)) by a dense scan then golden-section refinement.

    The first term grows with T and the second falls, so the minimum lies
    above R; the scan covers (R, R + 40 sigma + pi sigma (2K+1)].
    """
    lo, hi = R + 1e-9 * max(1.0, R), R + 40.0 * sigma + math.pi * sigma * (2 * K + 1)
    grid = np.linspace(lo, hi, 4001)
    vals = np.array([period_error(t, sigma, K, R) for t in grid])
    j = int(np.argmin(vals))
    a, b = grid[max(j - 1, 0)], grid[min(j + 1, len(grid) - 1)]
    g = (math.sqrt(5.0) - 1.0) / 2.0
    c, d = b - g * (b - a), a + g * (b - a)
    while b - a > tol * max(1.0, abs(b)):
        if period_error(c, sigma, K, R) < period_error(d, sigma, K, R):
            b, d = d, c
            c = b - g * (b - a)
        else:
            a, c = c, d
            d = a + g * (b - a)
    return 0.5 * (a + b)
