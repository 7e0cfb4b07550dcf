"""The served loop: requests of mixed sizes and parameters queued on one
server, admitted into waves of batched launches while earlier waves run.

A request's result must not depend on what it was served with: the same
image gives bit-identical output alone and inside a mixed stream, equal to
the per-image plan's output and within the FP32 bound of the float64 oracle.
"""

import numpy as np
import pytest

import oracle as o
import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import synth_image, auto_levels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX = [  # H, W, C, levels (None: automatic), K, m, sigma_r
    (64, 64, 1, None, 4, 0.5, 0.4),
    (513, 200, 1, None, 8, 4.0, 0.05),
    (33, 47, 3, 3, 4, 2.0, 0.1),
    (7, 9, 1, 1, 4, 3.0, 0.2),
    (120, 800, 3, 5, 8, 1.5, 0.3),
    (300, 300, 1, 2, 5, 3.0, 0.15),
    (1025, 769, 3, None, 8, 2.5, 0.25),
    (96, 160, 3, None, 16, 3.0, 0.2),
]
TARGET = (257, 311, 3, None, 8, 3.0, 0.2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_04681_gb300 import build
    build.build_library()


def _request(case, seed, precision):
    H, W, C, L, K, m, s = case
    L = auto_levels(H, W) if L is None else L
    img = synth_image(H, W, C, polygons=5, seed=seed)
    p = pkg.make_params(H, W, C, L, K, m, s, 2.0, precision)
    x = torch.from_numpy(img).cuda()
    y = torch.full_like(x, float("nan"))
    return p, img, x, y


def _serve(server, reqs):
    torch.cuda.synchronize()  # inputs written on torch's stream before the server reads them
    tickets = [pkg.fllf_server_submit(server, p, x.data_ptr(), y.data_ptr()) for p, _, x, y in reqs]
    for t in tickets:
        assert pkg.fllf_server_poll(server, t, -1) == pkg.FLLF_OK


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_same_result_alone_and_in_a_mix(precision):
    server = pkg.fllf_server_create(4 << 30, max_slots=6, max_queue=256, max_waves=2)
    try:
        p, img, x, alone = _request(TARGET, 7, precision)
        _serve(server, [(p, img, x, alone)])
        # per-image plan on the same input
        plan = pkg.fllf_plan_create(p, 0)
        ref = torch.full_like(x, float("nan"))
        pkg.run_tensor(plan, x, ref)
        torch.cuda.synchronize()
        pkg.fllf_plan_destroy(plan)
        torch.testing.assert_close(alone, ref, rtol=0, atol=0)

        # the same image again, in the middle of a stream of other requests,
        # twice over so that it lands in a different wave position
        for rep in range(2):
            others = [_request(c, 200 + 10 * rep + i, precision) for i, c in enumerate(MIX)]
            mixed = torch.full_like(x, float("nan"))
            mid = len(others) // 2 + rep
            reqs = others[:mid] + [(p, img, x, mixed)] + others[mid:]
            _serve(server, reqs)
            torch.testing.assert_close(mixed, alone, rtol=0, atol=0)
            assert all(bool(torch.isfinite(y).all()) for _, _, _, y in reqs)
        st = pkg.fllf_server_stats_get(server)
        assert st["completed"] == st["submitted"] == 1 + 2 * (len(MIX) + 1)
        assert st["rejected"] == 0
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert st["mpixel_per_s"] > 0 and st["waves"] >= 2
        assert st["pool_peak_bytes"] <= st["pool_bytes"]
    finally:
        pkg.fllf_server_destroy(server)


def test_served_results_match_oracle():
    server = pkg.fllf_server_create(1 << 30, max_slots=4, max_queue=64, max_waves=3)
    try:
        reqs = [_request(c, 300 + i, "fp32") for i, c in enumerate(MIX[:6])]
        _serve(server, reqs)
        for (p, img, x, y) in reqs:
            a = np.array(o.coeffs_quadrature(p.m, p.sigma_r, p.T, p.K))
            ref = o.fourier_llf(img.astype(np.float64), p.levels, a, 2.0)
            assert float(np.max(np.abs(y.cpu().numpy() - ref))) <= 1e-4
    finally:
        pkg.fllf_server_destroy(server)


def test_mixed_precisions_and_memory_pressure():
    """A pool that holds about one large request at a time still serves a
    stream that alternates precisions; every result equals its plan's."""
    big = (1025, 769, 3, None, 8, 2.5, 0.25)
    need = pkg.fllf_plan_scratch_bytes(_request(big, 0, "fp32")[0])
    server = pkg.fllf_server_create(int(need * 1.5) + (1 << 20), max_slots=8, max_queue=64,
                                    max_waves=2)
    try:
        reqs = []
        for i in range(6):
            prec = ("fp32", "fp16", "bf16")[i % 3]
            reqs.append(_request(big if i % 2 == 0 else MIX[i], 400 + i, prec))
        _serve(server, reqs)
        for (p, img, x, y) in reqs:
            plan = pkg.fllf_plan_create(p, 0)
            ref = torch.full_like(x, float("nan"))
            pkg.run_tensor(plan, x, ref)
            torch.cuda.synchronize()
            pkg.fllf_plan_destroy(plan)
            torch.testing.assert_close(y, ref, rtol=0, atol=0)
        st = pkg.fllf_server_stats_get(server)
        assert st["pool_peak_bytes"] <= st["pool_bytes"]
        assert st["completed"] == 6
    finally:
        pkg.fllf_server_destroy(server)


def test_submit_and_poll_errors():
    server = pkg.fllf_server_create(64 << 20, max_slots=2, max_queue=8, max_waves=1)
    try:
        p, img, x, y = _request((2048, 2048, 3, None, 8, 3.0, 0.2), 1, "fp32")
        with pytest.raises(pkg.FllfError) as e:   # can never fit the 64 MiB pool
            pkg.fllf_server_submit(server, p, x.data_ptr(), y.data_ptr())
        assert e.value.status == pkg.FLLF_ENOMEM
        with pytest.raises(pkg.FllfError) as e:   # aliased input and output
            pkg.fllf_server_submit(server, p, x.data_ptr(), x.data_ptr())
        assert e.value.status == pkg.FLLF_EINVAL
        with pytest.raises(pkg.FllfError) as e:
            pkg.fllf_server_poll(server, 12345, 0)
        assert e.value.status == pkg.FLLF_EINVAL
        p, img, x, y = _request((64, 64, 1, None, 4, 3.0, 0.2), 2, "fp32")
        torch.cuda.synchronize()
        t = pkg.fllf_server_submit(server, p, x.data_ptr(), y.data_ptr())
        s = pkg.fllf_server_poll(server, t, 0)
        assert s in (pkg.FLLF_OK, pkg.FLLF_EAGAIN)
        if s != pkg.FLLF_OK:
            assert pkg.fllf_server_poll(server, t, 10_000_000) == pkg.FLLF_OK
        with pytest.raises(pkg.FllfError):        # a ticket is consumed by its successful poll
            pkg.fllf_server_poll(server, t, 0)
        pkg.fllf_server_stats_reset(server)
        assert pkg.fllf_server_stats_get(server)["completed"] == 0
    finally:
        pkg.fllf_server_destroy(server)


def test_plans_stay_resident():
    """Requests with a parameter set the server has seen reuse its resident
    coefficients: the quadrature runs once per set (in submit), never at
    admission, and the results stay those of the per-image plans."""
    server = pkg.fllf_server_create(2 << 30, max_slots=4, max_queue=64, max_waves=2)
    try:
        cases = [MIX[0], MIX[2], MIX[0], MIX[5], MIX[2], MIX[0]]   # 3 distinct parameter sets
        reqs = [_request(c, 80 + i, "fp32") for i, c in enumerate(cases)]
        _serve(server, reqs)
        st = pkg.fllf_server_stats_get(server)
        assert st["plan_cache_misses"] == 3 and st["plan_cache_hits"] == 3
        assert st["admission_quadratures"] == 0
        for p, img, x, y in reqs:
            plan = pkg.fllf_plan_create(p, 0)
            ref = torch.empty_like(x)
            pkg.run_tensor(plan, x, ref)
            torch.cuda.synchronize()
            pkg.fllf_plan_destroy(plan)
            torch.testing.assert_close(y, ref, rtol=0, atol=0)
        # a second round: every set is resident now
        _serve(server, [_request(c, 90 + i, "fp32") for i, c in enumerate(cases[:3])])
        st = pkg.fllf_server_stats_get(server)
        assert st["plan_cache_misses"] == 3 and st["plan_cache_hits"] == 6
    finally:
        pkg.fllf_server_destroy(server)
