"""The bench's replica path over ranks, on CPU with the gloo backend (world
size 2): each rank filters its own frames (its own seed, no collective on
the data path), the timed region's length is the slowest rank's (a max
all-reduce), and the reported value is the whole job's throughput (weak
scaling: every rank contributes one frame per step)."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.rank_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        seconds = [0.010, 0.025][r]                      # the second rank is slower
        slowest = bench.max_over_ranks(seconds, w, "cpu")
        dist.barrier()
        out[r] = (w, r, local, bench.rank_seed(bench.WORKLOAD, r), slowest,
                  bench.whole_job_mpixel_s(w, 8_294_400, slowest))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_report_the_whole_job():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    seeds = {res[r][3] for r in range(world)}
    assert len(seeds) == world                           # each rank its own frames
    for r in range(world):
        w, rr, local, _, slowest, value = res[r]
        assert (w, rr, local) == (world, r, r)
        assert slowest == pytest.approx(0.025)           # max over ranks, on every rank
        assert value == pytest.approx(2 * 8_294_400 / 0.025 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.5, 1, "cpu") == 0.5
    assert bench.whole_job_mpixel_s(1, 1_000_000, 0.001) == pytest.approx(1000.0)
