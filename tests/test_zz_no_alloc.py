"""tg_run_noalloc: the entry point for callers that cannot allocate device
memory -- code running inside another framework's memory pool, or a plugin
handed fixed buffers -- so all of its scratch sits in one fixed array inside
the library.  Its per-task results must equal the regular entry point's (and
the oracle's), bit for bit, on two calls in a row; its limits, its
validation statuses and its promise to allocate nothing are checked too.
This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import workloads as w
from workloads.graphs import COND_BRANCH, COND_LOOP, from_lists, pack_param

pytestmark = pytest.mark.gpu

MAX_NODES, MAX_EDGES = 65536, 262144   # the limits include/tg.h states


def _csr(g):
    """Insertion-ordered successor lists (stable sort of the edges by source)."""
    order = np.argsort(g.src, kind="stable")
    succ = g.dst[order].astype(np.uint32)
    counts = np.bincount(g.src.astype(np.int64), minlength=g.n)
    off = np.zeros(g.n + 1, np.uint32)
    off[1:] = np.cumsum(counts)
    return off, succ


def _dev(a):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    if a.size == 0:
        a = np.zeros(1, a.dtype)
    return torch.from_numpy(a).cuda()


def _call(n, kinds, params, off, succ, m, seed, stream):
    """tg_run_noalloc on device copies of the given host arrays."""
    import torch
    from paper_2004_10908_b300 import binding as B
    dk, dp, do, ds = _dev(kinds), _dev(params), _dev(off), _dev(succ)
    out = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    cnt = torch.zeros_like(out)
    dig = torch.zeros_like(out)
    torch.cuda.synchronize()
    st = B.tg_run_noalloc(n, dk.data_ptr(), dp.data_ptr(), do.data_ptr(), ds.data_ptr(), m, seed,
                          out.data_ptr(), cnt.data_ptr(), dig.data_ptr(), stream)
    view = lambda t: t.cpu().numpy().view(np.uint32)[:n]
    return st, view(out), view(cnt), view(dig)


def _noalloc(g, stream):
    off, succ = _csr(g)
    return _call(g.n, g.kinds, g.params, off, succ, int(succ.size), g.seed, stream)


@pytest.fixture(scope="module")
def ex():
    from paper_2004_10908_b300 import Executor
    e = Executor(arena_bytes=512 << 20)
    yield e
    e.close()


GRAPHS = [w.config1(levels=6, width=40, trip=3, rounds=16),
          w.config3(seed=3, n_cond=60, body_levels=4, body_width=6, rounds=8, trip_max=6),
          w.config2a(seed=5, levels=40, width=300, rounds=8)]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_noalloc_matches_regular_entry_point_twice(ex, gi):
    import torch
    g = GRAPHS[gi]
    gh = ex.graph(g)
    assert ex.run(gh) == 0
    ref_out, ref_cnt, ref_dig, _ = ex.result(gh)
    gh.destroy()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        st, out, cnt, dig = _noalloc(g, stream)
        assert st == 0
        np.testing.assert_array_equal(cnt, ref_cnt)
        np.testing.assert_array_equal(out, ref_out)
        np.testing.assert_array_equal(dig, ref_dig)


def _at_the_limits():
    """Exactly 65,536 tasks and 262,144 edges: 16 levels of 4,096, every task
    past the first level with 4 distinct predecessors, duplicate edges into
    the second level to fill the count, and one loop condition (trip 1) whose
    two successors have no other in-edges, so that the regular kernel path
    (not the acyclic one) runs and exactly one of the two runs."""
    g = w.config2a(seed=77, levels=16, width=4096, d_lo=4, d_hi=4, rounds=8)
    a, b, c = MAX_NODES - 2, MAX_NODES - 1, MAX_NODES - 3
    keep = (g.dst != a) & (g.dst != b)
    src = list(g.src[keep].astype(np.int64))
    dst = list(g.dst[keep].astype(np.int64))
    for i in range(MAX_EDGES - len(src) - 2):
        src.append(i % 4096)
        dst.append(4096 + (i % 4096))
    kinds = g.kinds.copy()
    params = g.params.copy()
    kinds[c] = COND_LOOP
    params[c] = pack_param(8, 1)
    src += [c, c]
    dst += [a, b]
    out = from_lists("limits", kinds, params, list(zip(src, dst)), seed=77)
    assert out.n == MAX_NODES and out.m == MAX_EDGES
    return out


def test_noalloc_at_its_limits_equals_oracle_and_regular_entry_point(ex):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    # (a) the largest graph it takes; (b) as many tasks, no edges: every task
    # is a source, so the source list fills the edge region past m
    big = _at_the_limits()
    flat = from_lists("all_sources", np.zeros(MAX_NODES, np.uint8), pack_param(np.full(MAX_NODES, 4)), [], seed=3)
    for g in (big, flat):
        ref = oracle.run(g)
        assert ref.status == 0
        gh = ex.graph(g)
        assert ex.run(gh) == 0
        r_out, r_cnt, r_dig, _ = ex.result(gh)
        gh.destroy()
        for _ in range(2):
            st, out, cnt, dig = _noalloc(g, stream)
            assert st == 0
            for a, b, c in ((out, ref.out, r_out), (cnt, ref.cnt, r_cnt), (dig, ref.dig, r_dig)):
                np.testing.assert_array_equal(a, b)
                np.testing.assert_array_equal(a, c)


def test_noalloc_alternating_graphs():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    a, b = GRAPHS[1], GRAPHS[2]
    first = _noalloc(a, stream)
    _noalloc(b, stream)
    again = _noalloc(a, stream)
    for x, y in zip(first, again):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


def test_noalloc_refuses_sizes_beyond_its_array():
    import torch
    from paper_2004_10908_b300 import binding as B
    stream = torch.cuda.current_stream().cuda_stream
    # real device buffers, so that no check order could make a kernel read
    # a bad address
    k = torch.zeros(16, dtype=torch.uint8, device="cuda")
    buf = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    assert B.tg_run_noalloc(MAX_NODES + 1, k.data_ptr(), p, p, p, 4, 0, p, p, p, stream) == B.TG_ERR_BUDGET
    assert B.tg_run_noalloc(8, k.data_ptr(), p, p, p, MAX_EDGES + 1, 0, p, p, p, stream) == B.TG_ERR_BUDGET
    assert B.tg_run_noalloc(0, k.data_ptr(), p, p, p, 0, 0, p, p, p, stream) == B.TG_ERR_INVALID


def _small(kinds, params, off, succ):
    return (np.asarray(kinds, np.uint8), np.asarray(params, np.uint32), np.asarray(off, np.uint32),
            np.asarray(succ, np.uint32))


# every INVALID cause the device-side validation checks; none can make a
# kernel touch memory out of bounds (each check precedes its access)
INVALID_CASES = {
    "successor id >= n": _small([0, 0, 0, 0], pack_param([1] * 4), [0, 1, 2, 3, 3], [1, 2, 9]),
    "offsets decreasing": _small([0, 0, 0, 0], pack_param([1] * 4), [0, 2, 1, 3, 3], [1, 2, 3]),
    "offset past the edge count": _small([0, 0, 0, 0], pack_param([1] * 4), [0, 1, 5, 3, 3], [1, 2, 3]),
    "last offset != edge count": _small([0, 0, 0, 0], pack_param([1] * 4), [0, 1, 2, 2, 2], [1, 2, 3]),
    "condition without successors": _small([0, COND_BRANCH, 0, 0], pack_param([1] * 4), [0, 1, 1, 2, 2], [1, 3]),
    "loop trip 0": _small([0, COND_LOOP, 0, 0], pack_param([1] * 4, 0), [0, 1, 3, 3, 3], [1, 2, 3]),
    "unknown kind": _small([0, 7, 0, 0], pack_param([1] * 4), [0, 1, 2, 3, 3], [1, 2, 3]),
}


@pytest.mark.parametrize("case", sorted(INVALID_CASES))
def test_noalloc_validation_statuses(case):
    import torch
    from paper_2004_10908_b300 import binding as B
    stream = torch.cuda.current_stream().cuda_stream
    kinds, params, off, succ = INVALID_CASES[case]
    m = 3 if case != "condition without successors" else 2
    st, *_ = _call(4, kinds, params, off, succ, m, 0, stream)
    assert st == B.TG_ERR_INVALID, case
    # a graph whose every task has an in-edge has no source
    st, *_ = _noalloc(w.pitfall_no_source(), stream)
    assert st == B.TG_ERR_NO_SOURCE


def test_noalloc_allocates_no_device_memory():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    g = GRAPHS[2]
    off, succ = _csr(g)
    from paper_2004_10908_b300 import binding as B
    dk, dp, do, ds = _dev(g.kinds), _dev(g.params), _dev(off), _dev(succ)
    out = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros_like(out)
    dig = torch.zeros_like(out)

    def call():
        st = B.tg_run_noalloc(g.n, dk.data_ptr(), dp.data_ptr(), do.data_ptr(), ds.data_ptr(), int(succ.size),
                              g.seed, out.data_ptr(), cnt.data_ptr(), dig.data_ptr(), stream)
        assert st == 0

    for _ in range(2):   # first calls load the kernels
        call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(4):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
