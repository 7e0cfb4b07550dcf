"""fllf_run_noalloc: filtering with the library's fixed device scratch array.

Callers that cannot allocate device memory (code running inside an
allocator or memory pool it does not own, real-time loops that must not
block on an allocation, plugin hosts that only hand out the image buffers)
use this entry point.  It must give the same images as fllf_run with a plan
of the same parameters, call after call, since every call reuses the same
array.  This file is collected last on purpose.
"""

import numpy as np
import pytest

import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-4   # the FP32 parity tolerance of the GPU tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


def _with_plan(img, p):
    plan = pkg.fllf_plan_create(p, 0)
    try:
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        pkg.run_tensor(plan, x, y)
        torch.cuda.synchronize()
        return y.cpu().numpy()
    finally:
        pkg.fllf_plan_destroy(plan)


def _no_alloc(img, p, x=None, y=None):
    x = torch.from_numpy(img).cuda() if x is None else x
    y = torch.empty_like(x) if y is None else y
    s = torch.cuda.current_stream()
    pkg.fllf_run_noalloc(p, x.data_ptr(), y.data_ptr(), s.cuda_stream)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def test_matches_fllf_run_on_two_calls_in_a_row():
    # the same kernels on the same inputs: the same bits as fllf_run
    cases = [
        (synth_image(160, 224, 3, polygons=6, seed=31),
         pkg.make_params(160, 224, 3, 6, 8, 3.0, 0.2, 2.0, "fp32")),
        (synth_image(97, 131, 1, polygons=4, seed=32),
         pkg.make_params(97, 131, 1, 5, 5, 0.6, 0.3, 2.0, "fp16")),
    ]
    for img, p in cases:
        assert pkg.fllf_plan_scratch_bytes(p) + 512 <= pkg.NOALLOC_SCRATCH_BYTES
    refs = [_with_plan(img, p) for img, p in cases]
    outs = [_no_alloc(img, p) for img, p in cases]     # two calls in a row
    for out, ref in zip(outs, refs):
        assert np.all(np.isfinite(out))
        np.testing.assert_array_equal(out, ref)
        assert float(np.max(np.abs(out - ref))) <= TOL
    # and again after the array holds the second call's contents
    again = _no_alloc(*cases[0])
    np.testing.assert_array_equal(again, refs[0])


def test_allocates_no_device_memory_after_first_call():
    img = synth_image(120, 200, 1, polygons=5, seed=33)
    p = pkg.make_params(120, 200, 1, 5, 8, 3.0, 0.2, 2.0, "fp32")
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    _no_alloc(img, p, x, y)                       # first call: symbol lookup, module load

    def measure():
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        for _ in range(3):
            _no_alloc(img, p, x, y)
        free1, _ = torch.cuda.mem_get_info()
        stats1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        return free1 == free0, stats0 == stats1

    # the free-bytes figure is the whole device's: another process's
    # allocation in between would move it, so one retry is allowed
    ok_free, ok_torch = measure()
    if not ok_free:
        ok_free, ok_torch = measure()
    assert ok_torch and ok_free


def test_rejects_images_above_the_array_size():
    p = pkg.make_params(2160, 3840, 3, 8, 8, 3.0, 0.2, 2.0, "fp32")
    assert pkg.fllf_plan_scratch_bytes(p) > pkg.NOALLOC_SCRATCH_BYTES
    x = torch.zeros(3, 2160, 3840, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(pkg.FllfError) as e:
        pkg.fllf_run_noalloc(p, x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.status == pkg.FLLF_EINVAL
    assert "scratch" in e.value.detail


def test_fast_llf_same_as_plan():
    img = synth_image(70, 90, 2, polygons=4, seed=45)
    p = pkg.make_fast_params(70, 90, 2, 4, 7, 2.5, 0.25)
    np.testing.assert_array_equal(_no_alloc(img, p), _with_plan(img, p))
