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
