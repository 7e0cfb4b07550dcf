"""FP64 CPU oracle for Fourier local Laplacian filtering.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
``libfllf.so`` and its Python binding) imports, calls or links this package.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.

It is a plain, slow, obviously-correct restatement of Sumiya et al.,
"Gaussian Fourier Pyramid for Local Laplacian Filter" (IEEE SPL, arXiv
2206.04681), in float64 numpy, following the paper's notation:

* ``pyramid``      Gaussian / Laplacian pyramids and collapse, Eqs. (1), (2), (4).
* ``remap``        the remap detail function, its Fourier sine coefficients
                   (quadrature and the closed form of Eqs. (9)-(11)) and the
                   period selection of Eq. (12).
* ``fourier_llf``  Fourier LLF, Eq. (13) expanded as Eq. (14).
* ``naive_llf``    naive LLF, the per-pixel per-level procedure of Sec. II-C,
                   on the whole image or on exact dependency windows.
* ``*_adaptive``   the pixel-by-pixel parameter of Sec. III-B (a gain map).
* ``fourier_llf_luma``  colour by LLF on the Y of YUV (Sec. IV).
* ``fast_llf``     fast LLF (Aubry et al.), the method the paper compares
                   against (Sec. II-D): S remapped pyramids interpolated by
                   the guide.

Every function is pinned by ``tests/test_oracle_*.py`` against facts the
paper or the mathematics fixes (library routines, closed forms, invariants,
brute force); see those tests for the pins.
"""

from .pyramid import (reflect101, reduce, expand, gaussian_pyramid,
                      laplacian_pyramid, collapse, level_shapes,
                      reduce_matrix, expand_matrix)
from .remap import (remap_detail, remap, omegas, coeffs_quadrature,
                    coeffs_closed_form, fourier_detail, period_error,
                    optimal_period, coeff_tail_bound)
from .fourier_llf import (fourier_llf, fourier_llf_levels, fourier_llf_adaptive, fourier_llf_luma,
                          rgb_to_yuv, yuv_to_rgb, LUMA_BT601)
from .naive_llf import naive_llf, naive_llf_adaptive
from .fast_llf import fast_llf, fast_samples, fast_bracket

__all__ = [
    "reflect101", "reduce", "expand", "gaussian_pyramid", "laplacian_pyramid",
    "collapse", "level_shapes", "reduce_matrix", "expand_matrix",
    "remap_detail", "remap", "omegas", "coeffs_quadrature",
    "coeffs_closed_form", "fourier_detail", "period_error", "optimal_period",
    "coeff_tail_bound", "fourier_llf", "fourier_llf_levels", "naive_llf",
    "fourier_llf_adaptive", "naive_llf_adaptive", "fourier_llf_luma", "rgb_to_yuv",
    "yuv_to_rgb", "LUMA_BT601", "fast_llf", "fast_samples", "fast_bracket",
]
