"""GPU parity: the CUDA path (through the C ABI) against the float64 oracle.

FP32 storage must match the oracle to max-abs <= 1e-4 on [0, 1] images.
FP16 / BF16 storage of the Fourier pyramids (float32 arithmetic) must reach
PSNR >= 60 dB against the oracle.
"""

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import SMALL_GRAY, UHD_RGB, synth_image, workload_image

from gpu_util import gpu_filter, psnr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


def _check_fp32(img, L, K, m, sigma, T=2.0):
    out, a = gpu_filter(img, L, K, m, sigma, T)
    ref = o.fourier_llf(img.astype(np.float64), L, a, T)
    err = float(np.max(np.abs(out - ref)))
    assert np.all(np.isfinite(out))
    assert err <= FP32_TOL, f"max-abs {err:.3e}"
    return out, ref, a


def test_small_gray_workload_fp32_and_naive_distance():
    cfg = SMALL_GRAY
    img = workload_image(cfg)
    out, ref, a = _check_fp32(img, cfg["levels"], cfg["K"], cfg["m"], cfg["sigma_r"], cfg["T"])
    # Distance to naive LLF with the exact remap is bounded by the series error (P8).
    f = lambda d: o.remap_detail(d, cfg["m"], cfg["sigma_r"])
    naive = o.naive_llf(img[0].astype(np.float64), cfg["levels"], f)
    d = np.linspace(-1, 1, 20001)
    sup = np.max(np.abs(o.fourier_detail(d, a, cfg["T"]) - f(d)))
    dist = float(np.max(np.abs(out[0] - naive)))
    assert dist <= 2 * (cfg["levels"] - 1) * sup + FP32_TOL
    print(f"small gray: max|GPU-oracle| {np.max(np.abs(out - ref)):.2e}, "
          f"max|GPU-naive| {dist:.2e}, PSNR vs naive {psnr(out[0], naive):.1f} dB")


@pytest.mark.parametrize("H,W,C,L,K", [
    (1, 1, 1, 1, 1), (1, 1, 1, 3, 4), (1, 7, 1, 3, 2), (2, 2, 1, 2, 3), (3, 3, 2, 2, 5),
    (5, 9, 1, 4, 4), (17, 33, 3, 5, 7), (37, 53, 1, 6, 8), (64, 64, 1, 7, 16),
    (129, 65, 2, 5, 9), (200, 301, 1, 6, 6), (31, 500, 1, 4, 3), (450, 29, 1, 5, 4),
])
def test_shapes_and_orders_fp32(H, W, C, L, K):
    img = synth_image(H, W, C, polygons=4, seed=H * 1000 + W)
    _check_fp32(img, L, K, 3.0, 0.2)


def test_many_tiles_ragged_fp32():
    img = synth_image(300, 517, 2, polygons=8, seed=7)
    _check_fp32(img, 6, 7, 2.5, 0.15)


@pytest.mark.parametrize("m,sigma,K", [(0.5, 0.4, 4), (4.0, 0.05, 16), (1.7, 0.3, 12)])
def test_parameter_range_fp32(m, sigma, K):
    img = synth_image(160, 224, 1, polygons=6, seed=11)
    _check_fp32(img, 6, K, m, sigma)


def test_identity_and_constant():
    img = synth_image(70, 90, 1, polygons=4, seed=3)
    out, _ = gpu_filter(img, 5, 8, 1.0, 0.2)
    assert np.max(np.abs(out - img)) <= 1e-6
    const = np.full((1, 45, 61), 0.3, np.float32)
    out, _ = gpu_filter(const, 5, 8, 3.0, 0.2)
    assert np.max(np.abs(out - 0.3)) <= 1e-6


def test_deterministic_runs():
    img = synth_image(130, 250, 3, polygons=6, seed=5)
    outs, _ = gpu_filter(img, 6, 8, 3.0, 0.2, runs=3)
    for x in outs[1:]:
        np.testing.assert_array_equal(x, outs[0])


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_mixed_precision_psnr(precision):
    img = synth_image(384, 512, 1, polygons=10, seed=21)
    for K, sigma, m in ((8, 0.2, 3.0), (16, 0.1, 0.5), (4, 0.4, 3.0)):
        out, a = gpu_filter(img, 7, K, m, sigma, precision=precision)
        ref = o.fourier_llf(img.astype(np.float64), 7, a, 2.0)
        q = psnr(out, ref)
        assert q >= 60.0, f"{precision} K={K} sigma={sigma} m={m}: {q:.1f} dB"


def test_run_host_submit_poll_and_errors():
    img = synth_image(100, 140, 3, polygons=5, seed=9)
    p = pkg.make_params(100, 140, 3, 5, 8, 3.0, 0.2, 2.0)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        pkg.run_tensor(plan, x, y)
        torch.cuda.synchronize()
        ref = y.cpu().numpy()
        # host-buffer end-to-end entry point
        hin = torch.from_numpy(img).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        pkg.fllf_run_host(plan, hin.data_ptr(), hout.data_ptr(), 0)
        np.testing.assert_array_equal(hout.numpy(), ref)
        # asynchronous submit / poll
        y2 = torch.empty_like(x)
        s = torch.cuda.current_stream()
        t = pkg.fllf_submit(plan, x.data_ptr(), y2.data_ptr(), s.cuda_stream)
        assert pkg.fllf_poll(t, -1) == pkg.FLLF_OK
        np.testing.assert_array_equal(y2.cpu().numpy(), ref)
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_poll(t, 0)
        assert e.value.status == pkg.FLLF_EINVAL
        # aliasing input and output is rejected
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_run(plan, x.data_ptr(), x.data_ptr(), s.cuda_stream)
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_plan_destroy(plan)


@pytest.mark.parametrize("H,W,C,precision", [(120, 136, 3, "fp32"), (97, 131, 1, "fp32"), (64, 203, 3, "fp16")])
def test_submit_host_stream_of_frames(H, W, C, precision):
    """Frames through the staging slots in turn (two in flight, more frames
    than slots): each result equals fllf_run's bit for bit, and the first is
    checked against the oracle (FP32 storage: max-abs; FP16: PSNR)."""
    L, K = 5, 8
    p = pkg.make_params(H, W, C, L, K, 3.0, 0.2, 2.0, precision)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        imgs = [synth_image(H, W, C, polygons=4 + i, seed=20 + i) for i in range(5)]
        refs = []
        for img in imgs:
            x = torch.from_numpy(img).cuda()
            y = torch.empty_like(x)
            pkg.run_tensor(plan, x, y)
            torch.cuda.synchronize()
            refs.append(y.cpu().numpy())
        hins = [torch.from_numpy(img).pin_memory() for img in imgs]
        houts = [torch.full_like(h, float("nan")).pin_memory() for h in hins]
        s = torch.cuda.Stream()
        pending = []
        for i in range(len(imgs)):
            if len(pending) == 2:
                assert pkg.fllf_poll(pending.pop(0), -1) == pkg.FLLF_OK
            pending.append(pkg.fllf_submit_host(plan, hins[i].data_ptr(), houts[i].data_ptr(), s.cuda_stream))
        for t in pending:
            assert pkg.fllf_poll(t, -1) == pkg.FLLF_OK
        for i in range(len(imgs)):
            np.testing.assert_array_equal(houts[i].numpy(), refs[i])
        a = np.array(o.coeffs_quadrature(3.0, 0.2, 2.0, K))
        ref0 = o.fourier_llf(imgs[0].astype(np.float64), L, a, 2.0)
        if precision == "fp32":
            assert float(np.max(np.abs(houts[0].numpy() - ref0))) <= FP32_TOL
        else:
            assert psnr(houts[0].numpy(), ref0) >= 60.0
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_submit_host(plan, 0, houts[0].data_ptr(), s.cuda_stream)
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_plan_destroy(plan)


def test_frames_in_flight_on_concurrent_plans():
    """Successive frames on three plans and three streams (each plan its own
    scratch), as a pipeline over a stream of frames runs them: every output
    equals the one-stream run of its frame, bit for bit."""
    H, W, C, L, K = 150, 212, 3, 6, 8
    imgs = [synth_image(H, W, C, polygons=5, seed=40 + i) for i in range(6)]
    p = pkg.make_params(H, W, C, L, K, 3.0, 0.2, 2.0)
    plans = [pkg.fllf_plan_create(p, 0) for _ in range(3)]
    try:
        xs = [torch.from_numpy(im).cuda() for im in imgs]
        refs = []
        for x in xs:
            y = torch.empty_like(x)
            pkg.run_tensor(plans[0], x, y)
            torch.cuda.synchronize()
            refs.append(y.cpu().numpy())
        streams = [torch.cuda.Stream() for _ in plans]
        outs = [torch.full_like(x, float("nan")) for x in xs]
        for rep in range(2):
            for i, (x, y) in enumerate(zip(xs, outs)):
                j = i % 3
                pkg.fllf_run(plans[j], x.data_ptr(), y.data_ptr(), streams[j].cuda_stream)
            torch.cuda.synchronize()
            for y, r in zip(outs, refs):
                np.testing.assert_array_equal(y.cpu().numpy(), r)
    finally:
        for q in plans:
            pkg.fllf_plan_destroy(q)


@pytest.fixture(scope="module")
def uhd():
    cfg = UHD_RGB
    img = workload_image(cfg)
    a = np.array(o.coeffs_quadrature(cfg["m"], cfg["sigma_r"], cfg["T"], cfg["K"]))
    ref = o.fourier_llf(img.astype(np.float64), cfg["levels"], a, cfg["T"])
    return cfg, img, ref


def test_uhd_rgb_fp32_full_frame(uhd):
    cfg, img, ref = uhd
    out, a = gpu_filter(img, cfg["levels"], cfg["K"], cfg["m"], cfg["sigma_r"], cfg["T"])
    err = float(np.max(np.abs(out - ref)))
    print(f"4K RGB fp32: max-abs {err:.2e}, PSNR {psnr(out, ref):.1f} dB")
    assert err <= FP32_TOL


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_uhd_rgb_mixed_full_frame(uhd, precision):
    cfg, img, ref = uhd
    out, _ = gpu_filter(img, cfg["levels"], cfg["K"], cfg["m"], cfg["sigma_r"], cfg["T"],
                        precision=precision)
    q = psnr(out, ref)
    print(f"4K RGB {precision}: max-abs {np.max(np.abs(out - ref)):.2e}, PSNR {q:.1f} dB")
    assert q >= 60.0


@pytest.mark.parametrize("W", [96, 95, 94, 93])
@pytest.mark.parametrize("fast", [False, True])
def test_input_load_routes_same_bits(W, fast):
    """The level-0 kernels read the input by TMA (rows on 16-byte
    boundaries), from the plan's staging copy (W % 4 != 0) or with plain
    loads (W % 4 == 0 at a misaligned address): every route gives the same
    bits, and the first matches the oracle."""
    H, C, L = 70, 3, 5
    img = synth_image(H, W, C, polygons=5, seed=W)
    p = (pkg.make_fast_params(H, W, C, L, 9, 3.0, 0.2) if fast
         else pkg.make_params(H, W, C, L, 8, 3.0, 0.2, 2.0))
    plan = pkg.fllf_plan_create(p, 0)
    try:
        n = img.size
        buf = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
        out = torch.empty(n + 4, dtype=torch.float32, device="cuda")
        s = torch.cuda.current_stream().cuda_stream
        res = []
        for off in (0, 1, 3):   # 16-byte aligned start, then 4 and 12 bytes past it
            buf.zero_()
            buf[off:off + n].copy_(torch.from_numpy(img.reshape(-1)))
            pkg.fllf_run(plan, buf.data_ptr() + 4 * off, out.data_ptr() + 4 * off, s)
            torch.cuda.synchronize()
            res.append(out[off:off + n].cpu().numpy().reshape(img.shape))
        for r in res[1:]:
            np.testing.assert_array_equal(r, res[0])
        if not fast:
            a = np.array(o.coeffs_quadrature(3.0, 0.2, 2.0, 8))
            ref = o.fourier_llf(img.astype(np.float64), L, a, 2.0)
            assert float(np.max(np.abs(res[0] - ref))) <= FP32_TOL
    finally:
        pkg.fllf_plan_destroy(plan)


@pytest.mark.parametrize("H,W,C,L,fast", [(37, 53, 3, 5, False), (130, 250, 2, 6, False), (64, 96, 3, 5, True)])
def test_run_host_plane_pipeline_same_bits(H, W, C, L, fast):
    # host buffers with C >= 2 run plane by plane with the copies overlapped;
    # H*W odd leaves the planes of the device copy unaligned (plain loads)
    img = synth_image(H, W, C, polygons=5, seed=H + W)
    p = (pkg.make_fast_params(H, W, C, L, 9, 3.0, 0.2) if fast
         else pkg.make_params(H, W, C, L, 8, 3.0, 0.2, 2.0))
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        pkg.run_tensor(plan, x, y)
        torch.cuda.synchronize()
        hin = torch.from_numpy(img).pin_memory()
        for _ in range(2):
            hout = torch.full_like(hin, float("nan")).pin_memory()
            pkg.fllf_run_host(plan, hin.data_ptr(), hout.data_ptr(), torch.cuda.current_stream().cuda_stream)
            np.testing.assert_array_equal(hout.numpy(), y.cpu().numpy())
    finally:
        pkg.fllf_plan_destroy(plan)
