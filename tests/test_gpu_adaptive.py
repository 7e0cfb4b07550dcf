"""GPU parity of pixel-by-pixel enhancement (Sec. III-B, fllf_run_adaptive)
against the float64 oracle's adaptive Fourier LLF.

The gain map follows the paper's experiment (enhancement driven by the local
variance: flat regions get little).  FP32 storage must match the oracle to
max-abs <= 1e-4; FP16 storage must reach PSNR >= 60 dB.
"""

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image, variance_gain_map

from gpu_util import psnr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


def gpu_adaptive(img, gain, L, K, m_plan, sigma, T=2.0, precision="fp32"):
    C, H, W = img.shape
    p = pkg.make_params(H, W, C, L, K, m_plan, sigma, T, precision)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda()
        g = torch.from_numpy(np.ascontiguousarray(gain, np.float32)).cuda()
        y = torch.full_like(x, float("nan"))
        s = torch.cuda.current_stream()
        pkg.fllf_run_adaptive(plan, x.data_ptr(), g.data_ptr(), y.data_ptr(), s.cuda_stream)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.float64)
    finally:
        pkg.fllf_plan_destroy(plan)


def oracle_adaptive(img, gain, L, K, sigma, T=2.0):
    c = np.array(o.coeffs_quadrature(2.0, sigma, T, K))   # unit detail: m - 1 = 1
    return o.fourier_llf_adaptive(img.astype(np.float64), L, c, T, gain.astype(np.float64))


@pytest.mark.parametrize("H,W,C,L,K", [(96, 80, 1, 2, 4), (96, 80, 1, 3, 4), (120, 150, 3, 4, 8),
                                       (257, 300, 1, 6, 8), (200, 331, 2, 7, 6), (37, 53, 1, 5, 16)])
def test_adaptive_fp32_matches_oracle(H, W, C, L, K):
    img = synth_image(H, W, C, polygons=6, seed=H + W)
    gain = variance_gain_map(img, 0.5, 4.0)
    out = gpu_adaptive(img, gain, L, K, 3.0, 0.2)
    ref = oracle_adaptive(img, gain, L, K, 0.2)
    err = float(np.max(np.abs(out - ref)))
    assert np.all(np.isfinite(out))
    assert err <= FP32_TOL, f"max-abs {err:.3e}"


def test_adaptive_constant_map_is_the_fixed_filter_and_unit_map_is_identity():
    img = synth_image(140, 190, 3, polygons=6, seed=3)
    H, W = img.shape[1:]
    # a plan with gain 3 driven by a constant map of 1.7 equals the fixed filter at 1.7
    out = gpu_adaptive(img, np.full((H, W), 1.7, np.float32), 6, 8, 3.0, 0.2)
    a = np.array(o.coeffs_quadrature(1.7, 0.2, 2.0, 8))
    ref = o.fourier_llf(img.astype(np.float64), 6, a, 2.0)
    assert float(np.max(np.abs(out - ref))) <= FP32_TOL
    out1 = gpu_adaptive(img, np.ones((H, W), np.float32), 6, 8, 3.0, 0.2)
    assert float(np.max(np.abs(out1 - img))) <= 1e-6


def test_adaptive_fp16_psnr_and_rgb_many_tiles():
    img = synth_image(600, 1000, 3, polygons=12, seed=8)
    gain = variance_gain_map(img, 1.0, 3.5)
    ref = oracle_adaptive(img, gain, 7, 8, 0.2)
    out32 = gpu_adaptive(img, gain, 7, 8, 3.0, 0.2)
    assert float(np.max(np.abs(out32 - ref))) <= FP32_TOL
    out16 = gpu_adaptive(img, gain, 7, 8, 3.0, 0.2, precision="fp16")
    assert psnr(out16, ref) >= 60.0


def test_adaptive_rejects_unit_gain_plan_and_null_map():
    p = pkg.make_params(64, 64, 1, 4, 4, 1.0, 0.2, 2.0)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.zeros((1, 64, 64), device="cuda")
        y = torch.empty_like(x)
        g = torch.ones((64, 64), device="cuda")
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_run_adaptive(plan, x.data_ptr(), g.data_ptr(), y.data_ptr())
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_plan_destroy(plan)
    p = pkg.make_params(64, 64, 1, 4, 4, 3.0, 0.2, 2.0)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.zeros((1, 64, 64), device="cuda")
        y = torch.empty_like(x)
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_run_adaptive(plan, x.data_ptr(), 0, y.data_ptr())
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_plan_destroy(plan)


def test_adaptive_then_fixed_runs_in_one_process():
    # both variants of the fused level-0/1 kernel launch after each other
    # (each sets its own shared-memory limit)
    img = synth_image(150, 220, 1, polygons=5, seed=4)
    gain = variance_gain_map(img, 1.0, 3.0)
    p = pkg.make_params(150, 220, 1, 6, 8, 3.0, 0.2, 2.0)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.from_numpy(img).cuda()
        g = torch.from_numpy(gain).cuda()
        ya, yf = torch.empty_like(x), torch.empty_like(x)
        s = torch.cuda.current_stream().cuda_stream
        pkg.fllf_run_adaptive(plan, x.data_ptr(), g.data_ptr(), ya.data_ptr(), s)
        pkg.fllf_run(plan, x.data_ptr(), yf.data_ptr(), s)
        torch.cuda.synchronize()
        a = np.array(o.coeffs_quadrature(3.0, 0.2, 2.0, 8))
        ref = o.fourier_llf(img.astype(np.float64), 6, a, 2.0)
        assert float(np.max(np.abs(yf.cpu().numpy() - ref))) <= FP32_TOL
        assert float(np.max(np.abs(ya.cpu().numpy() - oracle_adaptive(img, gain, 6, 8, 0.2)))) <= FP32_TOL
    finally:
        pkg.fllf_plan_destroy(plan)
