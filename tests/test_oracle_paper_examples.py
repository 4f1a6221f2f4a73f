"""The paper's worked examples, read from tests/golden/paper_examples.txt."""
import os

import numpy as np
import pytest

import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, *kv = line.split()
        rows[name] = dict(x.split("=") for x in kv)
    return rows


G = _golden()


def _check_counts(g, res, row):
    for task, want in row.items():
        if task == "status":
            continue
        assert int(res.cnt[g.meta[task]]) == int(want), (g.name, task)


def test_diamond(orc):
    g = w.diamond()
    r = orc.run(g)
    assert r.status == orc.OK
    _check_counts(g, r, G["diamond"])
    # D runs after B and C: its input is the sum of their outputs
    assert r.out[3] == orc.payload(3, 0, (int(r.out[1]) + int(r.out[2])) & 0xFFFFFFFF, 4)


@pytest.mark.parametrize("ret", [0, 1])
def test_if_else(orc, ret):
    g = w.if_else(ret)
    r = orc.run(g)
    assert r.status == orc.OK
    _check_counts(g, r, G[f"if_else_{ret}"])


def test_if_else_out_of_range_index_ends_path(orc):
    for ret in (2, -1, 100):
        r = orc.run(w.if_else(ret))
        assert r.status == orc.OK
        assert r.cnt.tolist() == [1, 1, 0, 0]


def test_do_while(orc):
    g = w.do_while()
    r = orc.run(g)
    assert r.status == orc.OK
    _check_counts(g, r, G["do_while"])
    assert r.execs == 202


def test_nested_loops_walkthrough(orc):
    """The graph stops only after F1, F2, F3 return 0 in a row (scheduling
    walk-through); replay each condition's decision from its hash."""
    for seed in range(200):
        g = w.nested_loops(seed)
        r = orc.run(g)
        assert r.status == orc.OK
        assert r.cnt[4] == 1 and r.cnt[0] == 1
        # last decisions of F3, F2, F1 were 0 ("go on")
        for f in (1, 2, 3):
            assert orc.cond_hash(seed, f, int(r.cnt[f]) - 1) % 2 == 0
        # F2 runs exactly as often as F1 chose 0; F3 as often as F2 chose 0
        f1_zero = sum(orc.cond_hash(seed, 1, i) % 2 == 0 for i in range(int(r.cnt[1])))
        f2_zero = sum(orc.cond_hash(seed, 2, i) % 2 == 0 for i in range(int(r.cnt[2])))
        assert r.cnt[2] == f1_zero and r.cnt[3] == f2_zero


def test_nested_loops_expectation(orc):
    row = G["nested_loops_mean"]
    N = 100_000
    f1 = np.zeros(N)
    conds = np.zeros(N)
    for seed in range(N):
        r = orc.run(w.nested_loops(seed, rounds=0))
        f1[seed] = r.cnt[1]
        conds[seed] = int(r.cnt[1]) + int(r.cnt[2]) + int(r.cnt[3])
    assert abs(f1.mean() / float(row["F1"]) - 1) < 0.01
    assert abs(conds.mean() / float(row["conditions"]) - 1) < 0.01


def test_pitfalls(orc):
    assert orc.run(w.pitfall_no_source()).status == orc.NO_SOURCE
    assert orc.run(w.pitfall_race()).status == orc.RACE
    g = w.pitfall_race(fixed=True)
    r = orc.run(g)
    assert r.status == orc.OK
    _check_counts(g, r, G["pitfall_race_fixed"])


def test_validation(orc):
    g = w.diamond()
    bad = w.from_lists("bad", [0, 0], [1, 1], [(0, 5)])
    assert orc.run(bad).status == orc.INVALID
    # explicit weak flags must match the kind of the edge's source task
    assert orc.run(g, weak=np.zeros(4, np.uint8)).status == orc.OK
    assert orc.run(g, weak=np.array([0, 1, 0, 0], np.uint8)).status == orc.EDGE_KIND
    # a condition with no successor, a loop with trip 0, an unknown kind
    assert orc.run(w.from_lists("c0", [0, 1], [1, 1], [(0, 1)])).status == orc.INVALID
    assert orc.run(w.from_lists("t0", [0, 2], [1, 1], [(0, 1), (1, 0)])).status == orc.INVALID
    assert orc.run(w.from_lists("k9", [9], [1], [])).status == orc.INVALID
    # a task with only a weak in-edge is not a source
    g2 = w.from_lists("weakonly", [3, 0], [w.pack_param(1, 0, 0), 1], [(0, 1), (1, 0)])
    assert orc.run(g2).status == orc.NO_SOURCE


def test_exec_cap(orc):
    g = w.do_while(iterations=100)
    assert orc.run(g, exec_cap=50).status == orc.EXEC_LIMIT
    assert orc.run(g, exec_cap=202).status == orc.OK
