"""The dataflow launch (every stage in one persistent grid, tasks claimed
from a queue with per-row-band completion counters) against the per-stage
launches: the same stage code on the same work items, so the same bits, for
every launch mode, task size and storage precision, run after run; and the
float64 oracle within the FP32 tolerance."""

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image, auto_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4
CASES = [  # H, W, C, levels, K, m, sigma_r
    (1, 1, 1, 1, 4, 3.0, 0.2),
    (7, 9, 1, 2, 4, 3.0, 0.2),
    (33, 47, 3, 3, 4, 2.0, 0.1),
    (64, 64, 1, 4, 16, 0.5, 0.4),
    (450, 29, 1, 4, 8, 3.0, 0.2),
    (257, 311, 3, None, 8, 3.0, 0.2),
    (1025, 769, 1, None, 5, 4.0, 0.05),
    (300, 517, 3, 7, 8, 2.5, 0.25),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


def _run(plan, x, mode=None, items=None, runs=1):
    if mode is not None or items is not None:
        t = pkg.fllf_plan_get_tuning(plan)
        if mode is not None:
            t.dataflow = mode
        if items is not None:
            for k, v in enumerate(items):
                t.task_items[k] = v
        pkg.fllf_plan_set_tuning(plan, t)
    outs = []
    for _ in range(runs):
        y = torch.full_like(x, float("nan"))
        pkg.run_tensor(plan, x, y)
        torch.cuda.synchronize()
        outs.append(y.cpu().numpy())
    return outs


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_modes_give_the_same_bits(precision):
    for i, (H, W, C, L, K, m, s) in enumerate(CASES):
        L = auto_levels(H, W) if L is None else L
        img = synth_image(H, W, C, polygons=5, seed=300 + i)
        plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, L, K, m, s, 2.0, precision), 0)
        try:
            x = torch.from_numpy(img).cuda()
            ref = _run(plan, x, mode=0)[0]
            for mode in (1, 2, 3):
                for out in _run(plan, x, mode=mode, runs=2):
                    np.testing.assert_array_equal(out, ref, err_msg=f"case {i} mode {mode}")
        finally:
            pkg.fllf_plan_destroy(plan)


@pytest.mark.parametrize("items", [[1, 1, 1, 1, 1], [16, 128, 8, 4, 8], [3, 7, 5, 3, 2]])
def test_task_sizes_give_the_same_bits(items):
    H, W, C, K = 517, 300, 3, 8
    img = synth_image(H, W, C, polygons=6, seed=350)
    plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, auto_levels(H, W), K, 3.0, 0.2, 2.0, "fp32"), 0)
    try:
        x = torch.from_numpy(img).cuda()
        ref = _run(plan, x, mode=0)[0]
        for mode in (1, 2, 3):
            np.testing.assert_array_equal(_run(plan, x, mode=mode, items=items)[0], ref)
    finally:
        pkg.fllf_plan_destroy(plan)


def test_dataflow_matches_oracle():
    for i in (2, 3, 5, 7):
        H, W, C, L, K, m, s = CASES[i]
        L = auto_levels(H, W) if L is None else L
        img = synth_image(H, W, C, polygons=5, seed=300 + i)
        plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, L, K, m, s, 2.0, "fp32"), 0)
        try:
            out = _run(plan, torch.from_numpy(img).cuda(), mode=1)[0]
        finally:
            pkg.fllf_plan_destroy(plan)
        a = np.array(o.coeffs_quadrature(m, s, 2.0, K))
        ref = o.fourier_llf(img.astype(np.float64), L, a, 2.0)
        assert float(np.max(np.abs(out - ref))) <= TOL


def test_uhd_frame_same_bits():
    H, W, C = 2160, 3840, 3
    img = synth_image(H, W, C, polygons=40, seed=2)
    plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, 8, 8, 3.0, 0.2, 2.0, "fp32"), 0)
    try:
        x = torch.from_numpy(img).cuda()
        ref = _run(plan, x, mode=0)[0]
        for mode in (1, 2, 3):
            outs = _run(plan, x, mode=mode, runs=3)
            for out in outs:
                np.testing.assert_array_equal(out, ref)
    finally:
        pkg.fllf_plan_destroy(plan)


def test_autotune_keeps_the_output():
    H, W, C = 700, 900, 3
    img = synth_image(H, W, C, polygons=8, seed=360)
    plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, auto_levels(H, W), 8, 3.0, 0.2, 2.0, "fp16"), 0)
    try:
        x = torch.from_numpy(img).cuda()
        ref = _run(plan, x, mode=0)[0]
        y = torch.empty_like(x)
        tun, ms = pkg.fllf_plan_autotune(plan, x.data_ptr(), y.data_ptr(), reps=2,
                                         stream=torch.cuda.current_stream().cuda_stream)
        assert ms > 0 and tun.dataflow in (0, 1, 2)
        np.testing.assert_array_equal(_run(plan, x)[0], ref)
    finally:
        pkg.fllf_plan_destroy(plan)
