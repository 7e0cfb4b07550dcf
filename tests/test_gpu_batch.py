"""Batched execution: one launch per stage kind over images of different
sizes, channel counts, levels, K and remap parameters must give exactly the
per-image results (same arithmetic), run after run (CUDA graph replay), and
match the float64 oracle."""

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image, auto_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [  # H, W, C, levels, K, m, sigma_r, precision-independent
    (257, 311, 3, None, 8, 3.0, 0.2),
    (64, 64, 1, None, 4, 0.5, 0.4),
    (513, 200, 1, None, 8, 4.0, 0.05),
    (33, 47, 3, 3, 4, 2.0, 0.1),
    (7, 9, 1, 1, 4, 3.0, 0.2),        # single level: output = input
    (120, 800, 3, 5, 8, 1.5, 0.3),
    (300, 300, 1, 2, 5, 3.0, 0.15),
    (1025, 769, 3, None, 8, 2.5, 0.25),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


def _setup(precision):
    plans, ins, outs, refs, imgs, params = [], [], [], [], [], []
    for i, (H, W, C, L, K, m, s) in enumerate(CASES):
        L = auto_levels(H, W) if L is None else L
        img = synth_image(H, W, C, polygons=5, seed=100 + i)
        p = pkg.make_params(H, W, C, L, K, m, s, 2.0, precision)
        plan = pkg.fllf_plan_create(p, 0)
        x = torch.from_numpy(img).cuda()
        y = torch.full_like(x, float("nan"))
        r = torch.full_like(x, float("nan"))
        pkg.run_tensor(plan, x, r)
        plans.append(plan); ins.append(x); outs.append(y); refs.append(r); imgs.append(img)
        params.append((L, K, m, s))
    torch.cuda.synchronize()
    return plans, ins, outs, refs, imgs, params


@pytest.mark.parametrize("precision,mode", [("fp32", 0), ("fp32", 1), ("fp32", 2), ("fp16", 1), ("bf16", 2)])
def test_batch_equals_per_image_runs(precision, mode):
    # every launch mode (per stage kind and level; one dataflow launch; the
    # dataflow launch and the batched fused combine): the per-image bits
    plans, ins, outs, refs, imgs, params = _setup(precision)
    batch = pkg.fllf_batch_create(plans)
    try:
        pkg.fllf_batch_set_mode(batch, mode, [3, 5, 2, 1, 3] if mode == 2 else None)
        assert pkg.fllf_batch_get_mode(batch)[0] == mode
        s = torch.cuda.current_stream().cuda_stream
        for rep in range(3):
            for y in outs:
                y.fill_(float("nan"))
            # the second run reads copies at other addresses (the level-0
            # maps and staging sources are set per run)
            cur = [x.clone() for x in ins] if rep == 1 else ins
            pkg.fllf_batch_run(batch, [x.data_ptr() for x in cur], [y.data_ptr() for y in outs], s)
            torch.cuda.synchronize()
            pkg.fllf_batch_check(batch)
            for y, r in zip(outs, refs):
                torch.testing.assert_close(y, r, rtol=0, atol=0)
    finally:
        pkg.fllf_batch_destroy(batch)
        for p in plans:
            pkg.fllf_plan_destroy(p)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_one_shot_batch_equals_per_image_runs(precision):
    plans, ins, outs, refs, imgs, params = _setup(precision)
    try:
        for y in outs:
            y.fill_(float("nan"))
        pkg.fllf_batch_run_plans(plans, [x.data_ptr() for x in ins], [y.data_ptr() for y in outs],
                                 torch.cuda.current_stream().cuda_stream)
        for y, r in zip(outs, refs):
            torch.testing.assert_close(y, r, rtol=0, atol=0)
    finally:
        for p in plans:
            pkg.fllf_plan_destroy(p)


def test_batch_matches_oracle():
    plans, ins, outs, refs, imgs, params = _setup("fp32")
    batch = pkg.fllf_batch_create(plans)
    try:
        pkg.fllf_batch_run(batch, [x.data_ptr() for x in ins], [y.data_ptr() for y in outs],
                           torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        for i in (1, 3, 4, 6):
            L, K, m, s = params[i]
            a = np.array(o.coeffs_quadrature(m, s, 2.0, K))
            ref = o.fourier_llf(imgs[i].astype(np.float64), L, a, 2.0)
            assert float(np.max(np.abs(outs[i].cpu().numpy() - ref))) <= 1e-4
    finally:
        pkg.fllf_batch_destroy(batch)
        for p in plans:
            pkg.fllf_plan_destroy(p)


def test_batch_rejects_mixed_precision():
    p1 = pkg.fllf_plan_create(pkg.make_params(32, 32, 1, 3, 4, precision="fp32"), 0)
    p2 = pkg.fllf_plan_create(pkg.make_params(32, 32, 1, 3, 4, precision="bf16"), 0)
    try:
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_batch_create([p1, p2])
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_plan_destroy(p1)
        pkg.fllf_plan_destroy(p2)
