"""The critical-path reader of per-task trace records, on hand-made records
whose critical path and hop times are known (no GPU)."""
import numpy as np
import pytest

from paper_2004_10908_b300.trace import FROM_NAMES, critical_path

HAND, RING, OWN, STEAL, INJ = range(5)


def rec(frm, blk):
    return (np.asarray(frm, np.uint32) << 16) | np.asarray(blk, np.uint32)


def test_chain_every_task_on_the_path():
    # 0 -> 1 -> 2 -> 3, each step 100 ns, each wait 30 ns
    src, dst = [0, 1, 2], [1, 2, 3]
    st = np.array([1000, 1130, 1260, 1390])
    en = st + 100
    wh = rec([INJ, HAND, RING, STEAL], [0, 0, 0, 5])
    cp = critical_path(src, dst, st, en, wh)
    assert cp["tasks"] == 4
    assert cp["span_ms"] == pytest.approx((1490 - 1000) / 1e6)
    assert cp["step_mean_us"] == pytest.approx(0.1)
    assert cp["wait_mean_us"] == pytest.approx(0.03)
    by = cp["hops_by_source"]
    assert set(by) == {"hand", "ring", "steal"}
    assert by["hand"]["hops"] == 1 and by["hand"]["same_block"] == 1
    assert by["steal"]["hops"] == 1 and by["steal"]["same_block"] == 0
    assert cp["all_tasks_by_source"] == {"hand": 1, "ring": 1, "own_deque": 0, "steal": 1, "injection": 1}


def test_the_later_predecessor_is_followed():
    # diamond 0 -> {1, 2} -> 3: task 2 ends after task 1, so the path is 0, 2, 3
    src, dst = [0, 0, 1, 2], [1, 2, 3, 3]
    st = np.array([100, 300, 310, 900])
    en = np.array([200, 400, 800, 1000])
    wh = rec([INJ, RING, RING, OWN], [1, 1, 2, 2])
    cp = critical_path(src, dst, st, en, wh)
    assert cp["tasks"] == 3
    # hops 0 -> 2 (wait 110 ns, ring, other block) and 2 -> 3 (wait 100 ns, own deque, same block)
    assert cp["wait_mean_us"] == pytest.approx(0.105)
    assert cp["hops_by_source"]["ring"] == {"hops": 1, "wait_p50_us": pytest.approx(0.11),
                                            "wait_p90_us": pytest.approx(0.11), "same_block": 0}
    assert cp["hops_by_source"]["own_deque"]["same_block"] == 1
    # steps on the path: 100, 490, 100 ns
    assert cp["step_mean_us"] == pytest.approx(0.23)


def test_a_late_sink_ends_the_path():
    # 0 -> 1 -> 2 and 0 -> 3 (a sink that ends last): the path is 0, 3
    src, dst = [0, 1, 0], [1, 2, 3]
    st = np.array([0, 150, 300, 160]) + 1
    en = np.array([100, 250, 400, 900]) + 1
    cp = critical_path(src, dst, st, en, rec([INJ, HAND, HAND, RING], [0, 0, 0, 0]))
    assert cp["tasks"] == 2 and set(cp["hops_by_source"]) == {"ring"}


def test_a_task_that_did_not_run_is_refused():
    with pytest.raises(ValueError):
        critical_path([0], [1], np.array([5, 0]), np.array([6, 0]), rec([INJ, RING], [0, 0]))
    assert FROM_NAMES[STEAL] == "steal"


def test_steps_are_grouped_and_their_overlaps_counted():
    from paper_2004_10908_b300.trace import step_summary
    # block 0: step A (tasks 0, 1: 100..300) and step B (task 2: 150..250) overlap;
    # block 1: step C (task 3: 0..1000) runs alone
    st = np.array([100, 100, 150, 1])
    en = np.array([300, 300, 250, 1001])
    s = step_summary(st, en, rec([RING, RING, RING, STEAL], [0, 0, 0, 1]))
    assert s["steps"] == 3 and s["tasks_per_step_mean"] == pytest.approx(4 / 3)
    assert s["by_tasks_in_step"]["1"]["steps"] == 2 and s["by_tasks_in_step"]["2-4"]["steps"] == 1
    assert s["by_tasks_in_step"]["2-4"]["dur_p50_us"] == pytest.approx(0.2)


def test_levels_gaps_blocks_and_waits():
    from paper_2004_10908_b300.trace import level_summary
    # two levels of two tasks: 0, 1 -> 2, 3 (every edge)
    src, dst = [0, 0, 1, 1], [2, 3, 2, 3]
    st = np.array([10, 20, 400, 700])
    en = np.array([110, 300, 500, 800])
    wh = rec([INJ, INJ, RING, STEAL], [0, 1, 0, 2])
    lv = level_summary(np.array([0, 0, 1, 1]), src, dst, st, en, wh)
    assert lv["levels"] == 2
    assert lv["level_gap_us"]["mean"] == pytest.approx(0.5)        # 300 -> 800 ns
    assert lv["blocks_per_level"]["mean"] == pytest.approx(2.0)
    assert lv["largest_block_share"]["mean"] == pytest.approx(1.0)
    assert lv["last_task_of_level_from"] == {"hand": 0, "ring": 0, "own_deque": 0, "steal": 1, "injection": 1}
    # ready at 300 (the later predecessor): task 2 waited 100 ns, task 3 400 ns; sources 0
    w_ = lv["wait_ready_to_taken_by_source"]
    assert w_["ring"]["p50_us"] == pytest.approx(0.1) and w_["steal"]["p50_us"] == pytest.approx(0.4)
    assert w_["injection"]["p50_us"] == pytest.approx(0.0)
