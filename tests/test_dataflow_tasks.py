"""The dataflow launch's task list (host logic, no GPU).

The library cuts every stage of the path into tasks of a few tiles of one
row band and orders them so that a task comes after every task whose rows
it reads.  fllf_dataflow_check builds the list exactly as a run does and
executes it in order on one host worker: each task's producer bands must
be complete when its turn comes, every work item of every stage must be in
exactly one task, and every band must reach the count its readers wait for.
A task list that breaks this would make the device wait time out (or read
rows not yet written), so it is checked here for many shapes, level counts,
task sizes and batches."""

import pytest

import paper_2206_04681_gb300 as pkg
from paper_2206_04681_gb300.synth import batch_workload, auto_levels

SHAPES = [(1, 1), (3, 3), (2, 7), (7, 9), (33, 47), (64, 64), (450, 29), (29, 450), (257, 311),
          (1025, 769), (2160, 3840)]


def _params(H, W, C, L, K, precision="fp32"):
    return pkg.make_params(H, W, C, L, K, 3.0, 0.2, 2.0, precision)


@pytest.mark.parametrize("H,W", SHAPES)
def test_every_level_count(H, W):
    for L in range(1, 10):
        p = _params(H, W, 1, L, 4)
        if pkg.fllf_params_validate(p) != pkg.FLLF_OK:
            continue
        for with_d10 in (True, False):
            pkg.fllf_dataflow_check([p], with_d10=with_d10)
        # the small levels alone (dataflow mode 3)
        for lo in (2, 3, 4):
            if lo <= L - 2:
                nt, nb = pkg.fllf_dataflow_check([p], first_level=lo)
                assert nt >= nb > 0


@pytest.mark.parametrize("items", [[1, 1, 1, 1, 1], [4, 8, 4, 2, 4], [7, 13, 3, 5, 2], [64, 4096, 64, 64, 64]])
def test_task_sizes(items):
    for (H, W), C, K, prec in (((257, 311), 3, 8, "fp32"), ((1025, 769), 1, 5, "fp16"), ((64, 64), 3, 16, "bf16")):
        p = _params(H, W, C, auto_levels(H, W), K, prec)
        nt, nb = pkg.fllf_dataflow_check([p], items)
        assert nt >= nb > 0


def test_uhd_frame_list_size():
    p = _params(2160, 3840, 3, 8, 8)
    nt, nb = pkg.fllf_dataflow_check([p])
    # bands per plane: up0 1080 / 14 -> 78 tile rows; up(1..6) writes levels
    # 2..7 (540, 270, 135, 68, 34, 17 rows) in rows of 16: 34 + 17 + 9 + 5 + 3 + 2;
    # down_s(2..6): 34 + 17 + 9 + 5 + 3; down10: 2160 / 32 -> 68
    assert nb == 3 * (78 + (34 + 17 + 9 + 5 + 3 + 2) + (34 + 17 + 9 + 5 + 3) + 68)
    nt2, nb2 = pkg.fllf_dataflow_check([p], with_d10=False)
    assert nb2 == nb - 3 * 68 and nt2 < nt


def test_mixed_batch():
    items = batch_workload(64, seed=4)
    ps = [pkg.make_params(it["H"], it["W"], it["C"], it["levels"], it["K"], it["m"], it["sigma_r"], it["T"],
                          "fp32") for it in items]
    nt, nb = pkg.fllf_dataflow_check(ps)
    assert nt > 64 and nb > 64
    pkg.fllf_dataflow_check(ps, with_d10=False)


def test_rejects_fast_llf_and_mixed_precision():
    with pytest.raises(pkg.FllfError):
        pkg.fllf_dataflow_check([pkg.make_fast_params(64, 64, 1, 4, 8)])
    with pytest.raises(pkg.FllfError):
        pkg.fllf_dataflow_check([_params(64, 64, 1, 4, 4, "fp32"), _params(64, 64, 1, 4, 4, "fp16")])
    with pytest.raises(pkg.FllfError):
        pkg.fllf_dataflow_check([_params(64, 64, 1, 4, 4)], [0, 1, 1, 1, 1])
