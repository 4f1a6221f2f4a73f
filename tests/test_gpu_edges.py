"""Edge cases on the device, against the oracle bit for bit: the smallest
graph, a graph of sources only, the widest fan-out and fan-in a task may
have (65,535), duplicate edges, an execution cap of one, and the limits
validation enforces."""
import numpy as np
import pytest

import oracle
import workloads as w
from tests.gpu_util import assert_same, run_both
from workloads.graphs import COND_CONST, STATIC, from_lists, pack_param

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    from paper_2004_10908_b300 import Executor
    e = Executor(arena_bytes=1 << 30)
    yield e
    e.close()


def test_one_task(ex):
    for R in (0, 1, 300):
        g = from_lists(f"one_R{R}", [STATIC], [pack_param(R)], [])
        dev, ref = run_both(ex, g)
        assert_same(dev, ref, g.name)
        assert ref.execs == 1


def test_sources_only(ex):
    n = 10_000
    g = from_lists("sources", [STATIC] * n, pack_param(np.arange(n) % 37), [])
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, g.name)


@pytest.mark.parametrize("width", [1, 33, 4097, 65_535])
def test_widest_fan_out_and_fan_in(ex, width):
    """S -> width tasks -> J: one task releases `width` successors (many
    rounds of the flattened release) and J's join word counts `width`
    strong in-edges down to zero."""
    n = width + 2
    edges = [(0, 1 + k) for k in range(width)] + [(1 + k, n - 1) for k in range(width)]
    g = from_lists(f"fan{width}", [STATIC] * n, pack_param(np.full(n, 3)), edges)
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, g.name)


def test_degree_limits_are_validated(ex):
    from paper_2004_10908_b300 import binding as B
    width = 65_536
    n = width + 1
    kinds = np.zeros(n, np.uint8)
    params = np.ones(n, np.uint32)
    src = np.zeros(width, np.uint32)
    dst = np.arange(1, n, dtype=np.uint32)
    assert B.tg_graph_create(ex.ctx, kinds, params, src, dst)[0] == B.TG_ERR_INVALID     # out-degree
    assert B.tg_graph_create(ex.ctx, kinds, params, dst, src)[0] == B.TG_ERR_INVALID     # strong in-degree


def test_duplicate_edges_count_per_edge(ex):
    """u -> v three times: v waits for three releases and sums u's output
    three times; a condition's duplicate successors keep their indices."""
    g = from_lists("dups", [STATIC, STATIC, STATIC, COND_CONST, STATIC],
                   [pack_param(2), pack_param(2), pack_param(2), pack_param(2, 0, 2), pack_param(2)],
                   [(0, 1), (0, 1), (0, 1), (1, 2), (2, 3), (3, 4), (3, 4), (3, 4)])
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, g.name)
    assert ref.cnt[1] == 1 and ref.cnt[4] == 1


def test_exec_cap_of_one():
    from paper_2004_10908_b300 import Executor, binding as B
    with Executor(arena_bytes=1 << 26, exec_cap=1) as e:
        one = e.graph(from_lists("one", [STATIC], [pack_param(1)], []))
        assert e.run(one) == 0
        two = e.graph(from_lists("two", [STATIC, STATIC], pack_param([1, 1]), [(0, 1)]))
        assert e.run(two) == B.TG_ERR_EXEC_LIMIT
        assert oracle.run(from_lists("two", [STATIC, STATIC], pack_param([1, 1]), [(0, 1)]),
                          exec_cap=1).status == oracle.EXEC_LIMIT


def test_dot_dump_shows_the_packed_graph(ex):
    """The DOT text read back from the device lists every task with its kind
    and rounds, and every edge in insertion order: strong solid, weak dashed
    with its successor index."""
    import re
    from paper_2004_10908_b300 import binding as B
    from workloads.graphs import COND_BRANCH, COND_LOOP, MODULE, SUBFLOW
    inner = ex.graph(w.diamond())
    kinds = [STATIC, COND_BRANCH, STATIC, STATIC, COND_LOOP, MODULE, SUBFLOW, COND_CONST, STATIC]
    params = [pack_param(5), pack_param(6), pack_param(7), pack_param(8), pack_param(9, 3), pack_param(10),
              pack_param(11), pack_param(12, 0, -1 & 0xFF), pack_param(13)]
    edges = [(0, 1), (1, 2), (1, 3), (2, 4), (3, 4), (4, 2), (4, 5), (5, 6), (6, 7), (7, 8), (0, 8)]
    g = from_lists("all_kinds", kinds, params, edges)
    h = ex.graph(g, modules={5: inner, 6: inner})
    text = B.tg_graph_dot(ex.ctx, h.handle)
    nodes = dict(re.findall(r'n(\d+) \[label="\d+ (\w+) R=', text))
    names = {STATIC: "static", COND_BRANCH: "branch", COND_LOOP: "loop", COND_CONST: "const",
             MODULE: "module", SUBFLOW: "subflow"}
    assert {int(k): v for k, v in nodes.items()} == {v: names[k] for v, k in enumerate(kinds)}
    assert "T=3" in text and "r=-1" in text and "graph=" in text
    got = [(int(a), int(b), lab) for a, b, _, lab in re.findall(r'n(\d+) -> n(\d+)( \[style=dashed, label="(\d+)"\])?;', text)]
    want = []
    for s in range(len(kinds)):
        succ = [d for a, d in edges if a == s]
        cond = kinds[s] in (COND_BRANCH, COND_LOOP, COND_CONST)
        want += [(s, d, str(j) if cond else "") for j, d in enumerate(succ)]
    assert got == want
    h.destroy()
    inner.destroy()


def test_deadlocked_join_ends_without_running_it(ex):
    """A strong merge after a branch: only one arm runs, so the join's count
    never reaches zero; the run still ends (nothing queued or running) and
    the join has run zero times."""
    from workloads.graphs import COND_BRANCH
    g = from_lists("dead_join", [STATIC, COND_BRANCH, STATIC, STATIC, STATIC],
                   pack_param([3] * 5), [(0, 1), (1, 2), (1, 3), (2, 4), (3, 4)])
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, g.name)
    assert ref.status == oracle.OK and ref.cnt[4] == 0 and ref.cnt[2] + ref.cnt[3] == 1
