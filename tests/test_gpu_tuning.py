"""Launch tuning and the autotuner: every launch setting (chain start,
small-tile threshold, CTAs per SM, REDUCE order) computes the same output
bit for bit, the autotuner keeps a valid setting, and the batch autotuner
keeps per-image results."""

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image, auto_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


NST = len(pkg.STAGES)
ALL = 1 << 40   # every combined level >= 2 on the small tiles


def _tuning(chain, cps, rev, small=ALL, dataflow=0, items=(0, 0, 0, 0, 0), bands=0):
    t = pkg.fllf_tuning()   # task sizes 0: the defaults
    t.reduce_bands = bands
    t.chain_pixels = chain
    for i, c in enumerate(cps):
        t.ctas_per_sm[i] = c
    t.reduce_reverse = rev
    t.small_pixels = small
    t.dataflow = dataflow
    for i, v in enumerate(items):
        t.task_items[i] = v
    return t


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_every_launch_setting_gives_the_same_bits(precision):
    img = synth_image(700, 1100, 2, polygons=8, seed=12)
    p = pkg.make_params(700, 1100, 2, 8, 8, 3.0, 0.2, 2.0, precision)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        d = pkg.fllf_plan_get_tuning(plan).as_dict()
        assert d["chain_pixels"] == 0 and d["reduce_reverse"] == 1 and d["small_pixels"] == ALL
        x = torch.from_numpy(img).cuda()
        outs = []
        for t in (_tuning(1 << 21, [0] * NST, 1), _tuning(0, [0] * NST, 0), _tuning(1 << 23, [1] * NST, 1),
                  _tuning(1 << 15, [2, 1, 1, 1, 1, 2], 0), _tuning(0, [0] * NST, 1, small=0),
                  _tuning(0, [0] * NST, 1, small=1 << 19), _tuning(1 << 17, [0, 0, 0, 0, 0, 1], 1, small=ALL),
                  _tuning(0, [0] * NST, 1, dataflow=1), _tuning(0, [0] * NST, 1, dataflow=2, items=(2, 16, 1, 1, 1)),
                  _tuning(0, [0] * NST, 1, bands=4), _tuning(1 << 21, [0] * NST, 0, bands=7),
                  _tuning(0, [0] * NST, 1, dataflow=3, bands=3)):
            pkg.fllf_plan_set_tuning(plan, t)
            y = torch.full_like(x, float("nan"))
            pkg.run_tensor(plan, x, y)
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy())
        for y in outs[1:]:
            np.testing.assert_array_equal(y, outs[0])
        if precision == "fp32":
            a = np.array(o.coeffs_quadrature(3.0, 0.2, 2.0, 8))
            ref = o.fourier_llf(img.astype(np.float64), 8, a, 2.0)
            assert float(np.max(np.abs(outs[0] - ref))) <= 1e-4
        with pytest.raises(pkg.FllfError):
            pkg.fllf_plan_set_tuning(plan, _tuning(-1, [0] * NST, 1))
        with pytest.raises(pkg.FllfError):
            pkg.fllf_plan_set_tuning(plan, _tuning(0, [0, 0, 99, 0, 0, 0], 1))
        with pytest.raises(pkg.FllfError):
            pkg.fllf_plan_set_tuning(plan, _tuning(0, [0] * NST, 1, small=-1))
    finally:
        pkg.fllf_plan_destroy(plan)


# The 32 x 16 small-level combine takes the same arithmetic steps as the
# 64 x 32 one: ragged sizes (partial tiles, odd widths and heights), orders
# padded in the top chunk (K = 5, 6) or several chunks (K = 12, 16), single
# planes and three, every storage precision, and the pixel-adaptive gain.
SMALL_CASES = [  # H, W, C, levels, K, m, sigma_r, precision
    (301, 517, 3, 7, 5, 3.0, 0.2, "fp32"),
    (200, 333, 1, 6, 12, 0.5, 0.3, "fp32"),
    (97, 1031, 2, 6, 16, 4.0, 0.05, "fp16"),
    (515, 131, 1, 7, 6, 2.0, 0.15, "bf16"),
    (64, 64, 3, 6, 8, 3.0, 0.2, "fp32"),
]


@pytest.mark.parametrize("case", SMALL_CASES)
def test_small_tile_combine_gives_the_same_bits(case):
    H, W, C, L, K, m, s, prec = case
    img = synth_image(H, W, C, polygons=6, seed=H + W)
    plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, L, K, m, s, 2.0, prec), 0)
    try:
        x = torch.from_numpy(img).cuda()
        outs = []
        for small in (0, ALL):
            pkg.fllf_plan_set_tuning(plan, _tuning(0, [0] * NST, 1, small=small))
            y = torch.full_like(x, float("nan"))
            pkg.run_tensor(plan, x, y)
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy())
        np.testing.assert_array_equal(outs[1], outs[0])
        assert np.all(np.isfinite(outs[0]))
    finally:
        pkg.fllf_plan_destroy(plan)


def test_small_tile_combine_adaptive_gain_same_bits():
    H, W, C = 260, 390, 1
    img = synth_image(H, W, C, polygons=6, seed=31)
    gain = np.linspace(0.5, 3.5, H * W, dtype=np.float32).reshape(H, W)
    plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, 7, 8, 2.5, 0.2, 2.0), 0)
    try:
        x = torch.from_numpy(img).cuda()
        g = torch.from_numpy(gain).cuda()
        outs = []
        for small in (0, ALL):
            pkg.fllf_plan_set_tuning(plan, _tuning(0, [0] * NST, 1, small=small))
            y = torch.full_like(x, float("nan"))
            pkg.fllf_run_adaptive(plan, x.data_ptr(), g.data_ptr(), y.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            outs.append(y.cpu().numpy())
        np.testing.assert_array_equal(outs[1], outs[0])
    finally:
        pkg.fllf_plan_destroy(plan)


def test_autotune_keeps_a_valid_setting_and_the_output():
    img = synth_image(540, 960, 3, polygons=10, seed=13)
    p = pkg.make_params(540, 960, 3, 7, 8, 3.0, 0.2, 2.0)
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.from_numpy(img).cuda()
        ref = torch.empty_like(x)
        pkg.run_tensor(plan, x, ref)
        y = torch.empty_like(x)
        t, ms = pkg.fllf_plan_autotune(plan, x.data_ptr(), y.data_ptr(), reps=3,
                                       stream=torch.cuda.current_stream().cuda_stream)
        assert ms > 0
        d = t.as_dict()
        assert d["chain_pixels"] in (0, 1 << 15, 1 << 17, 1 << 19, 1 << 21, 1 << 23)
        sizes = [h * w * 3 for h, w in o.level_shapes(540, 960, 7)[2:6]]
        assert d["small_pixels"] in [0, ALL] + sizes
        assert all(0 <= c <= 32 for c in d["ctas_per_sm"].values())
        z = torch.full_like(x, float("nan"))
        pkg.run_tensor(plan, x, z)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(z.cpu().numpy(), ref.cpu().numpy())
    finally:
        pkg.fllf_plan_destroy(plan)


def test_batch_autotune_keeps_per_image_results():
    cases = [(257, 311, 3, 8, 3.0, 0.2), (513, 200, 1, 8, 4.0, 0.05), (120, 800, 3, 4, 1.5, 0.3)]
    plans, ins, outs, refs = [], [], [], []
    try:
        for i, (H, W, C, K, m, s) in enumerate(cases):
            img = synth_image(H, W, C, polygons=5, seed=200 + i)
            plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, auto_levels(H, W), K, m, s, 2.0), 0)
            plans.append(plan)
            x = torch.from_numpy(img).cuda()
            r = torch.empty_like(x)
            pkg.run_tensor(plan, x, r)
            ins.append(x); outs.append(torch.empty_like(x)); refs.append(r)
        batch = pkg.fllf_batch_create(plans)
        try:
            st = torch.cuda.current_stream().cuda_stream
            caps, ms = pkg.fllf_batch_autotune(batch, [x.data_ptr() for x in ins],
                                               [y.data_ptr() for y in outs], reps=2, stream=st)
            assert ms > 0 and len(caps) == 4 and all(0 <= c <= 32 for c in caps)
            for y in outs:
                y.fill_(float("nan"))
            pkg.fllf_batch_run(batch, [x.data_ptr() for x in ins], [y.data_ptr() for y in outs], st)
            torch.cuda.synchronize()
            pkg.fllf_batch_check(batch)
            for y, r in zip(outs, refs):
                np.testing.assert_array_equal(y.cpu().numpy(), r.cpu().numpy())
        finally:
            pkg.fllf_batch_destroy(batch)
    finally:
        for p in plans:
            pkg.fllf_plan_destroy(p)
