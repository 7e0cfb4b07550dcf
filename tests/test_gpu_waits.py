"""Bounded device waits: a wait that runs out is reported to the host, and
the plan keeps working afterwards.

Every wait in the kernels (a TMA copy's mbarrier, a grid barrier of the
chained launch) gives up after a limit, sets the run's fault word and leaves
the kernel, and the host reports FLLF_ETIMEOUT.  To drive a wait to its
limit without faulting anything, the test hook raises the arrival count that
the chained launch's grid barriers wait for (no barrier can then complete;
no copy is in flight at a barrier) and shortens the limit to 10^5 SM cycles
(about 50 microseconds)."""

import numpy as np
import pytest

import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H, W, C, L, K = 300, 420, 1, 6, 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


def _chained_plan():
    plan = pkg.fllf_plan_create(pkg.make_params(H, W, C, L, K, 3.0, 0.2, 2.0, "fp32"), 0)
    t = pkg.fllf_plan_get_tuning(plan)
    t.chain_pixels = 1 << 40          # levels 2..5 in one chained cooperative launch
    pkg.fllf_plan_set_tuning(plan, t)
    return plan


def _host_run(plan, img):
    hin = torch.from_numpy(img).pin_memory()
    hout = torch.full_like(hin, float("nan")).pin_memory()
    pkg.fllf_run_host(plan, hin.data_ptr(), hout.data_ptr(), 0)
    return hout.numpy().copy()


def test_grid_barrier_timeout_is_reported_and_the_plan_recovers():
    img = synth_image(H, W, C, polygons=5, seed=71)
    fresh = _chained_plan()
    plan = _chained_plan()
    try:
        ref = _host_run(fresh, img)
        assert np.all(np.isfinite(ref))
        pkg.fllf_plan_set_wait_test(plan, 100_000, 1)
        with pytest.raises(pkg.FllfError) as e:
            _host_run(plan, img)
        assert e.value.status == pkg.FLLF_ETIMEOUT
        # the report clears the fault and the test settings: the next run is
        # a fresh plan's, bit for bit
        np.testing.assert_array_equal(_host_run(plan, img), ref)
        np.testing.assert_array_equal(_host_run(plan, img), ref)
    finally:
        pkg.fllf_plan_destroy(plan)
        pkg.fllf_plan_destroy(fresh)


def test_timeout_through_submit_and_poll():
    img = synth_image(H, W, C, polygons=5, seed=72)
    plan = _chained_plan()
    try:
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        s = torch.cuda.current_stream().cuda_stream
        pkg.fllf_run(plan, x.data_ptr(), y.data_ptr(), s)
        torch.cuda.synchronize()
        ref = y.cpu().numpy()
        pkg.fllf_plan_set_wait_test(plan, 100_000, 1)
        t = pkg.fllf_submit(plan, x.data_ptr(), y.data_ptr(), s)
        # the work finishes (every barrier gives up); the poll reports the
        # timeout and consumes the ticket
        assert pkg.fllf_poll(t, 10_000_000) == pkg.FLLF_ETIMEOUT
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_poll(t, 0)
        assert e.value.status == pkg.FLLF_EINVAL
        # two faulting runs polled newest first: each reports its timeout
        # (from its fault-word snapshot, though the first report clears the
        # device word)
        pkg.fllf_plan_set_wait_test(plan, 100_000, 1)
        t1 = pkg.fllf_submit(plan, x.data_ptr(), y.data_ptr(), s)
        t2 = pkg.fllf_submit(plan, x.data_ptr(), y.data_ptr(), s)
        assert pkg.fllf_poll(t2, 10_000_000) == pkg.FLLF_ETIMEOUT
        assert pkg.fllf_poll(t1, 10_000_000) == pkg.FLLF_ETIMEOUT
        t = pkg.fllf_submit(plan, x.data_ptr(), y.data_ptr(), s)
        assert pkg.fllf_poll(t, 10_000_000) == pkg.FLLF_OK
        np.testing.assert_array_equal(y.cpu().numpy(), ref)
    finally:
        pkg.fllf_plan_destroy(plan)


def test_timeout_through_submit_host():
    """Streamed host-buffer frames: the poll reads the fault word from its
    host-mapped snapshot, reports the timeout, and the next frame is clean."""
    img = synth_image(H, W, C, polygons=5, seed=73)
    plan = _chained_plan()
    try:
        ref = _host_run(plan, img)
        hin = torch.from_numpy(img).pin_memory()
        hout = torch.full_like(hin, float("nan")).pin_memory()
        pkg.fllf_plan_set_wait_test(plan, 100_000, 1)
        t = pkg.fllf_submit_host(plan, hin.data_ptr(), hout.data_ptr(), 0)
        assert pkg.fllf_poll(t, 10_000_000) == pkg.FLLF_ETIMEOUT
        # two faulting frames, polled newest first: the first report clears
        # the device word, and the older ticket still reports its own
        # timeout from its snapshot
        pkg.fllf_plan_set_wait_test(plan, 100_000, 1)
        hout2 = torch.full_like(hin, float("nan")).pin_memory()
        t1 = pkg.fllf_submit_host(plan, hin.data_ptr(), hout.data_ptr(), 0)
        t2 = pkg.fllf_submit_host(plan, hin.data_ptr(), hout2.data_ptr(), 0)
        assert pkg.fllf_poll(t2, 10_000_000) == pkg.FLLF_ETIMEOUT
        assert pkg.fllf_poll(t1, 10_000_000) == pkg.FLLF_ETIMEOUT
        t = pkg.fllf_submit_host(plan, hin.data_ptr(), hout.data_ptr(), 0)
        assert pkg.fllf_poll(t, 10_000_000) == pkg.FLLF_OK
        np.testing.assert_array_equal(hout.numpy(), ref)
    finally:
        pkg.fllf_plan_destroy(plan)


def test_submit_host_more_pending_tickets_than_snapshot_words():
    """70 frames submitted before any poll: the first 64 tickets take the
    plan's host-mapped snapshot words, the rest read the device word; every
    poll succeeds and every output is the synchronous run's."""
    h, w = 40, 56
    img = synth_image(h, w, 1, polygons=3, seed=74)
    plan = pkg.fllf_plan_create(pkg.make_params(h, w, 1, 4, 4, 3.0, 0.2, 2.0, "fp32"), 0)
    try:
        ref = _host_run(plan, img)
        hin = torch.from_numpy(img).pin_memory()
        outs = [torch.full_like(hin, float("nan")).pin_memory() for _ in range(70)]
        tickets = [pkg.fllf_submit_host(plan, hin.data_ptr(), o.data_ptr(), 0) for o in outs]
        for t in tickets:
            assert pkg.fllf_poll(t, 10_000_000) == pkg.FLLF_OK
        for o in outs:
            np.testing.assert_array_equal(o.numpy(), ref)
        # the words came back: another round takes them again
        tickets = [pkg.fllf_submit_host(plan, hin.data_ptr(), o.data_ptr(), 0) for o in outs[:8]]
        for t in tickets:
            assert pkg.fllf_poll(t, 10_000_000) == pkg.FLLF_OK
    finally:
        pkg.fllf_plan_destroy(plan)


def test_wait_hook_rejects_a_negative_limit():
    plan = _chained_plan()
    try:
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_plan_set_wait_test(plan, -1, 0)
        assert e.value.status == pkg.FLLF_EINVAL
    finally:
        pkg.fllf_plan_destroy(plan)
