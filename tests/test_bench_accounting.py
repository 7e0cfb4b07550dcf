"""The bench's per-stage accounting (host logic, no GPU): which levels each
stage kind covers under a launch tuning, the launches per step, the
algorithmic op count per level that the ALU roofline divides by a kernel's
duration, the minimum HBM bytes, and the pyramid bytes kept apart from
them.  The level split mirrors the library's launch sequence."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CFG = bench.WORKLOAD   # 3840 x 2160 x 3, 8 levels, K = 8
N0, N1, N2 = 3840 * 2160, 1920 * 1080, 960 * 540


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


def test_op_count_per_value_is_the_methods():
    # summed over the levels, 24.67 K + 40.3 per value: the method's count of
    # about 25 K + 35 (139 at K = 4, 238 at K = 8, 435 at K = 16)
    for K, expect in ((4, 139.0), (8, 237.7), (16, 435.0)):
        cfg = dict(CFG, K=K)
        per_value = bench.step_ops(cfg) / (3 * N0)
        assert per_value == pytest.approx(expect, rel=0.01)


def test_op_count_is_the_same_under_every_launch_split():
    base, _, _ = bench.stage_accounts(CFG, 8)
    for chain, small in ((0, 0), (1 << 21, 1 << 40), (1 << 17, 1 << 19)):
        ops, _, _ = bench.stage_accounts(CFG, 8, chain, small)
        assert sum(ops.values()) == pytest.approx(sum(base.values()))


def test_fused_stage_ops_and_bytes():
    lo = bench.level_ops(CFG)
    ops, hbm, pyr = bench.stage_accounts(CFG, 8)
    # level 0: combine + residual; level 1: combine + coefficient pairs + residual
    expect = 3 * (N0 * (lo["combine"] + lo["resid"]) + N1 * (lo["combine"] + lo["gtrig"] + lo["resid"]))
    assert ops["down0"] == pytest.approx(expect)
    assert ops["down0"] / 1e9 == pytest.approx(2.76, abs=0.01)
    # algorithmic bytes: I read, O written, G_1 read (224 MB at 4K RGB)
    assert hbm["down0"] == pytest.approx(3 * (8 * N0 + 4 * N1))
    assert hbm["down0"] / 1e6 == pytest.approx(224.0, abs=0.1)
    # pyramid bytes, reported apart: Z_1 (zb K per level-1 pixel), Z_2 and E_2
    for zb in (8, 4):
        _, _, pyr = bench.stage_accounts(CFG, zb)
        assert pyr["down0"] == pytest.approx(3 * (zb * 8 * N1 + (zb * 8 + 4) * N2))


def test_stage_hbm_bytes_add_up_to_the_minimum():
    # the stages' image and guide bytes: I read twice (REDUCE and combine),
    # O once, each guide level written once and read by the REDUCE above it
    # and by its combine; the path's minimum counts I once and G read once
    _, hbm, _ = bench.stage_accounts(CFG, 8)
    assert sum(hbm.values()) >= bench.hbm_min_bytes(CFG)


def test_hbm_min_bytes_follow_the_definition():
    # input read + output write + guide pyramid (levels >= 1) written and read once
    got = bench.hbm_min_bytes(CFG)
    assert got / 1e6 == pytest.approx(265.4, abs=1.0)


@pytest.mark.parametrize("mode", [1, 2])
def test_dataflow_accounting_moves_the_work_into_one_kernel(mode):
    base = bench.stage_accounts(CFG, 8)
    flow = bench.stage_accounts(CFG, 8, dataflow=mode)
    for b, f in zip(base, flow):
        assert sum(f.values()) == pytest.approx(sum(b.values()))
    ops = flow[0]
    if mode == 1:
        assert ops["graph"] == pytest.approx(sum(base[0].values()))
    else:   # the fused level-1/level-0 combine stays its own kernel
        assert ops["down0"] == pytest.approx(base[0]["down0"])
        assert ops["graph"] == pytest.approx(sum(base[0].values()) - base[0]["down0"])
