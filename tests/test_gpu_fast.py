"""Fast LLF (Sec. II-D) on the GPU against the float64 fast LLF oracle.

FP32 storage must match the oracle to max-abs <= 1e-4 on [0, 1] images (the
Fourier path's bar); FP16 / BF16 storage of the sampled pyramids must reach
PSNR >= 60 dB.  Covers odd and even sample counts (the last plane half
empty), one to many chunks of planes, ragged sizes, 1 to 7 levels, RGB,
colour by luma, and the calls that reject fast plans (the no-allocation
entry point is checked in test_zz_no_alloc.py).
"""

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image

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


def _run(img, levels, S, m, sigma, precision="fp32"):
    C, H, W = img.shape
    plan = pkg.fllf_plan_create(pkg.make_fast_params(H, W, C, levels, S, m, sigma, precision), 0)
    try:
        assert pkg.fllf_plan_params(plan).K == (S + 1) // 2
        x = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()
        y = torch.full_like(x, float("nan"))
        pkg.run_tensor(plan, x, y)
        torch.cuda.synchronize()
        return y.cpu().numpy()
    finally:
        pkg.fllf_plan_destroy(plan)


@pytest.mark.parametrize("H,W,C,L,S,m,sigma", [
    (1, 1, 1, 1, 4, 3.0, 0.2),
    (2, 3, 1, 2, 2, 3.0, 0.2),
    (9, 14, 1, 3, 5, 2.0, 0.3),
    (37, 53, 3, 5, 16, 3.0, 0.2),
    (64, 64, 1, 6, 33, 4.0, 0.1),
    (129, 211, 2, 6, 9, 0.5, 0.3),
    (300, 517, 1, 7, 12, 3.0, 0.15),
    (31, 500, 1, 4, 3, 1.5, 0.4),
])
def test_fast_llf_fp32_matches_oracle(H, W, C, L, S, m, sigma):
    img = synth_image(H, W, C, polygons=5, seed=H * 7 + W)
    out = _run(img, L, S, m, sigma)
    ref = o.fast_llf(img.astype(np.float64), L, S, m, sigma)
    assert np.all(np.isfinite(out))
    err = float(np.max(np.abs(out - ref)))
    assert err <= FP32_TOL, f"max-abs {err:.3e}"


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_fast_llf_mixed_precision_psnr(precision):
    img = synth_image(256, 384, 1, polygons=8, seed=41)
    for S, sigma, m in ((16, 0.2, 3.0), (8, 0.1, 0.5)):
        out = _run(img, 6, S, m, sigma, precision)
        ref = o.fast_llf(img.astype(np.float64), 6, S, m, sigma)
        q = psnr(out, ref)
        assert q >= 60.0, f"{precision} S={S}: {q:.1f} dB"


def test_fast_llf_luma():
    H, W = 96, 130
    rgb = synth_image(H, W, 3, polygons=5, seed=44)
    plan = pkg.fllf_plan_create(pkg.make_fast_params(H, W, 1, 5, 10, 3.0, 0.2), 0)
    try:
        x = torch.from_numpy(rgb).cuda()
        y = torch.full_like(x, float("nan"))
        pkg.fllf_run_luma(plan, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        yuv = o.rgb_to_yuv(rgb.astype(np.float64))
        yuv[0] = o.fast_llf(yuv[0], 5, 10, 3.0, 0.2)
        ref = o.yuv_to_rgb(yuv)
        assert float(np.max(np.abs(y.cpu().numpy() - ref))) <= FP32_TOL
    finally:
        pkg.fllf_plan_destroy(plan)


def test_fast_plans_rejected_where_unsupported():
    img = synth_image(64, 80, 1, polygons=4, seed=46)
    plan = pkg.fllf_plan_create(pkg.make_fast_params(64, 80, 1, 4, 8, 3.0, 0.2), 0)
    try:
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        g = torch.ones(64, 80, device="cuda")
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_run_adaptive(plan, x.data_ptr(), g.data_ptr(), y.data_ptr())
        assert e.value.status == pkg.FLLF_EINVAL
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_batch_create([plan])
        assert e.value.status == pkg.FLLF_EINVAL
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_plan_coeffs(plan)
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_plan_destroy(plan)
    server = pkg.fllf_server_create(1 << 28, 4, 16, 1, 0)
    try:
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_server_submit(server, pkg.make_fast_params(64, 80, 1, 4, 8), x.data_ptr(), y.data_ptr())
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_server_destroy(server)


def test_fast_llf_approaches_naive_llf_with_more_samples():
    img = synth_image(48, 64, 1, polygons=4, seed=47)[0]
    L, m, sigma = 4, 3.0, 0.2
    naive = o.naive_llf(img.astype(np.float64), L, lambda d: o.remap_detail(d, m, sigma), window=False)
    errs = [float(np.max(np.abs(_run(img[None], L, S, m, sigma)[0] - naive))) for S in (4, 8, 16, 32)]
    assert errs[0] > errs[1] > errs[2] > errs[3]


def test_autotune_on_a_fast_plan_keeps_the_output():
    img = synth_image(300, 420, 3, polygons=6, seed=48)
    plan = pkg.fllf_plan_create(pkg.make_fast_params(300, 420, 3, 6, 12, 3.0, 0.2), 0)
    try:
        x = torch.from_numpy(img).cuda()
        ref = torch.empty_like(x)
        pkg.run_tensor(plan, x, ref)
        y = torch.empty_like(x)
        t, ms = pkg.fllf_plan_autotune(plan, x.data_ptr(), y.data_ptr(), reps=2,
                                       stream=torch.cuda.current_stream().cuda_stream)
        assert ms > 0
        z = torch.full_like(x, float("nan"))
        pkg.run_tensor(plan, x, z)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(z.cpu().numpy(), ref.cpu().numpy())
    finally:
        pkg.fllf_plan_destroy(plan)
