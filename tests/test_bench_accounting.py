"""The bench's per-stage accounting (host logic, no GPU): which levels each
stage kind covers under a launch tuning, the launches per step, and the
algorithmic bytes of the fused level-0/1 stage that the roofline divides
by the kernel's duration.  The level split mirrors the library's launch
sequence; the byte counts follow the path's definition (each input element
read once, each output written once)."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CFG = bench.WORKLOAD   # 3840 x 2160 x 3, 8 levels, K = 8


def _launches(split):
    up, chain_up, chain_down, down, small, fused = split
    return 1 + len(up) + (1 if chain_up or chain_down else 0) + len(down) + len(small) + 1


def test_default_tuning_splits_the_levels_like_the_library():
    up, chain_up, chain_down, down, small, fused = bench.stage_split(CFG)
    assert fused                                   # levels 1 and 0 in one stage
    assert up == [1, 2, 3, 4, 5, 6]                # REDUCE l -> l+1
    assert chain_up == [] and chain_down == []     # no chained launch by default
    assert down == [] and small == [6, 5, 4, 3, 2]
    assert _launches(bench.stage_split(CFG)) == 13


@pytest.mark.parametrize("chain,small,n_small,n_down,n_launch", [
    (0, 0, 0, 5, 13),                 # every combine on the 64 x 32 tiles
    (0, 1 << 19, 4, 1, 13),           # levels 3..6 small (level 2 holds 1.55 M pixels)
    (1 << 21, 1 << 40, 0, 0, 4),      # levels 2..7 chained: up0, REDUCE 1 -> 2, the chain, the fused stage
    (1 << 17, 1 << 40, 2, 0, 8),      # levels >= 4 chained (level 4 holds 97 k pixels)
])
def test_tuned_splits(chain, small, n_small, n_down, n_launch):
    split = bench.stage_split(CFG, chain, small)
    assert len(split[4]) == n_small and len(split[3]) == n_down
    assert _launches(split) == n_launch
    # every level 2..6 is combined exactly once, every REDUCE 1..6 runs once
    up, chain_up, chain_down, down, small_l, _ = split
    assert sorted(chain_down + down + small_l) == [2, 3, 4, 5, 6]
    assert sorted(up + chain_up) == [1, 2, 3, 4, 5, 6]


def test_fused_stage_bytes():
    # I and O (8 B per level-0 value), Z_1 (zb * K) + G_1 per level-1 value,
    # Z_2 (zb * K) + E_2 per level-2 value, for the 3 planes
    n0, n1, n2 = 3840 * 2160, 1920 * 1080, 960 * 540
    for zb in (8, 4):
        _, byt = bench.stage_work(CFG, zb)
        expect = 3 * (8 * n0 + (zb * 8 + 4) * n1 + (zb * 8 + 4) * n2)
        assert byt["down0"] == pytest.approx(expect)
    _, byt = bench.stage_work(CFG, 8)
    assert byt["down0"] / 1e6 == pytest.approx(727.8, abs=0.1)


def test_hbm_min_bytes_follow_the_definition():
    # input read + output write + guide pyramid (levels >= 1) written and read once
    got = bench.hbm_min_bytes(CFG)
    assert got / 1e6 == pytest.approx(265.4, abs=1.0)
