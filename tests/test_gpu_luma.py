"""GPU parity of colour by luma (fllf_run_luma: LLF on Y of BT.601 YUV, U and
V kept; Sec. IV) against the float64 oracle, FP32 max-abs <= 1e-4."""

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


@pytest.mark.parametrize("H,W,L,K,precision", [(90, 130, 5, 8, "fp32"), (257, 301, 6, 4, "fp32"),
                                               (512, 700, 7, 8, "fp16")])
def test_luma_mode_matches_oracle(H, W, L, K, precision):
    rgb = synth_image(H, W, 3, polygons=8, seed=H)
    p = pkg.make_params(H, W, 1, L, K, 3.0, 0.2, 2.0, precision)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.from_numpy(rgb).cuda()
        y = torch.full_like(x, float("nan"))
        for _ in range(2):   # the second call reuses the plan's luma buffers
            pkg.fllf_run_luma(plan, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        out = y.cpu().numpy().astype(np.float64)
    finally:
        pkg.fllf_plan_destroy(plan)
    a = np.array(o.coeffs_quadrature(3.0, 0.2, 2.0, K))
    ref = o.fourier_llf_luma(rgb.astype(np.float64), L, a, 2.0)
    err = float(np.max(np.abs(out - ref)))
    assert err <= (1e-4 if precision == "fp32" else 2e-3), f"max-abs {err:.3e}"


def test_luma_mode_needs_a_single_plane_plan():
    p = pkg.make_params(32, 32, 3, 3, 4, 3.0, 0.2, 2.0)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.zeros((3, 32, 32), device="cuda")
        y = torch.empty_like(x)
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_run_luma(plan, x.data_ptr(), y.data_ptr())
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_plan_destroy(plan)
