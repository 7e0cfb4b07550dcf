"""Fourier local Laplacian filtering in float64 (oracle; test infrastructure only).

Sec. III-A of the paper.  The output local Laplacian pyramid is defined by
Eq. (13): at level l and pixel p, the Laplacian coefficient of the image
remapped about g = G_l[I]_p.  Substituting the sine series of the remap
detail (Eq. (11)) makes every term separable into a per-pixel coefficient
and a pyramid of the input only, which is Eq. (14).  In this package's
parametrisation (r_g(i) = i + f(i - g), f ~= sum_k a_k sin(omega_k d)):

    L_l[O]_p = L_l[I]_p
             + sum_k a_k [ cos(omega_k g) L_l[sin(omega_k I)]_p
                         - sin(omega_k g) L_l[cos(omega_k I)]_p ],   l < top
    L_top[O] = G_top[I],

where L_l[sin(omega_k I)] = S~_{l,k} - up(S~_{l+1,k}) with
S~_{l,k} = G_l[sin(omega_k I)] and C~_{l,k} = G_l[cos(omega_k I)] (the
Gaussian Fourier pyramids of Fig. 1), and the output is the collapse of
Eq. (4).  At l = 0 the paper drops the S~_0 / C~_0 terms because
r(I, I_p) = I makes them cancel; this oracle keeps them and evaluates the
general form at every level (the cancellation is checked by a test).
"""

import numpy as np

from .pyramid import gaussian_pyramid, laplacian_from_gaussian, collapse
from .remap import omegas


def fourier_llf_levels(img, levels, a, T):
    """Return (output Laplacian pyramid, level-0 Fourier term) for one plane.

    ``img``: 2-D float array.  ``a``: Fourier sine coefficients a_1..a_K.
    The second value is the part of L_0[O] - L_0[I] that comes from the
    level-0 pyramids S~_0, C~_0 (zero up to rounding by r(I, I_p) = I).
    """
    img = np.asarray(img, dtype=np.float64)
    g = gaussian_pyramid(img, levels)
    lap_i = laplacian_from_gaussian(g)
    out = [lap_i[l].copy() for l in range(levels - 1)]
    level0_term = np.zeros_like(img)
    for ak, om in zip(a, omegas(T, len(a))):
        c_pyr = gaussian_pyramid(np.cos(om * img), levels)   # C~_{l,k}
        s_pyr = gaussian_pyramid(np.sin(om * img), levels)   # S~_{l,k}
        lap_c = laplacian_from_gaussian(c_pyr)
        lap_s = laplacian_from_gaussian(s_pyr)
        for l in range(levels - 1):
            cg, sg = np.cos(om * g[l]), np.sin(om * g[l])     # per-pixel coefficients
            out[l] += ak * (cg * lap_s[l] - sg * lap_c[l])
        level0_term += ak * (np.cos(om * img) * s_pyr[0] - np.sin(om * img) * c_pyr[0])
    out.append(g[-1])                                         # L_top[O] = G_top[I]
    return out, level0_term


def fourier_llf(img, levels, a, T):
    """Fourier LLF of a plane (H, W) or of planar channels (C, H, W).

    Each channel is filtered independently.  float64 in, float64 out.
    """
    img = np.asarray(img, dtype=np.float64)
    if img.ndim == 3:
        return np.stack([fourier_llf(ch, levels, a, T) for ch in img])
    lap_o, _ = fourier_llf_levels(img, levels, a, T)
    return collapse(lap_o)


def fourier_llf_adaptive(img, levels, c, T, gain):
    """Pixel-by-pixel enhancement with Fourier LLF (Sec. III-B), float64.

    The pyramids do not depend on the remap, so only the coefficients change
    per pixel: with the gain m replaced by m_p, every level below the top is

        L_l[O]_p = L_l[I]_p + (m_{l,p} - 1) sum_k c_k [ cos(omega_k g) L_l[sin(omega_k I)]_p
                                                     - sin(omega_k g) L_l[cos(omega_k I)]_p ],

    where c_k are the coefficients of the unit detail d exp(-d^2/(2 sigma_r^2))
    (the a_k of m - 1 = 1) and m_{l,p} = G_l[gain]_p (reading: the Gaussian
    pyramid of the level-0 gain map).  ``img``: (H, W) or (C, H, W); ``gain``:
    (H, W), shared by the channels.
    """
    img = np.asarray(img, dtype=np.float64)
    if img.ndim == 3:
        return np.stack([fourier_llf_adaptive(ch, levels, c, T, gain) for ch in img])
    gm = gaussian_pyramid(np.asarray(gain, dtype=np.float64), levels)
    g = gaussian_pyramid(img, levels)
    lap_i = laplacian_from_gaussian(g)
    out = [lap_i[l].copy() for l in range(levels - 1)]
    for ck, om in zip(c, omegas(T, len(c))):
        lap_c = laplacian_from_gaussian(gaussian_pyramid(np.cos(om * img), levels))
        lap_s = laplacian_from_gaussian(gaussian_pyramid(np.sin(om * img), levels))
        for l in range(levels - 1):
            cg, sg = np.cos(om * g[l]), np.sin(om * g[l])
            out[l] += (gm[l] - 1.0) * ck * (cg * lap_s[l] - sg * lap_c[l])
    out.append(g[-1])
    return collapse(out)


# BT.601 luma weights (reading: the paper's YUV is the BT.601 one).
LUMA_BT601 = (0.299, 0.587, 0.114)


def rgb_to_yuv(rgb):
    """BT.601 YUV of a planar (3, H, W) RGB image: Y = 0.299 R + 0.587 G +
    0.114 B, U = 0.492 (B - Y), V = 0.877 (R - Y)."""
    r, g, b = (np.asarray(c, dtype=np.float64) for c in rgb)
    y = LUMA_BT601[0] * r + LUMA_BT601[1] * g + LUMA_BT601[2] * b
    return np.stack([y, 0.492 * (b - y), 0.877 * (r - y)])


def yuv_to_rgb(yuv):
    """Inverse of ``rgb_to_yuv`` (solves its 3 x 3 matrix)."""
    m = np.array([[LUMA_BT601[0], LUMA_BT601[1], LUMA_BT601[2]],
                  [-0.492 * LUMA_BT601[0], -0.492 * LUMA_BT601[1], 0.492 * (1 - LUMA_BT601[2])],
                  [0.877 * (1 - LUMA_BT601[0]), -0.877 * LUMA_BT601[1], -0.877 * LUMA_BT601[2]]])
    flat = np.asarray(yuv, dtype=np.float64).reshape(3, -1)
    return np.linalg.solve(m, flat).reshape(np.shape(yuv))


def fourier_llf_luma(rgb, levels, a, T):
    """Colour processing of the paper's experiments (Sec. IV): LLF on the Y
    channel of YUV, the other components kept; float64, planar (3, H, W)."""
    yuv = rgb_to_yuv(rgb)
    yuv[0] = fourier_llf(yuv[0], levels, a, T)
    return yuv_to_rgb(yuv)
