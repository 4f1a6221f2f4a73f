"""tg_run_noalloc: the entry point for callers that cannot allocate device
memory (all of its scratch sits in a fixed array inside the library).  Its
per-task results must equal the regular entry point's, bit for bit, on two
calls in a row.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def _csr(g):
    """Insertion-ordered successor lists (stable sort of the edges by source)."""
    order = np.argsort(g.src, kind="stable")
    succ = g.dst[order].astype(np.uint32)
    counts = np.bincount(g.src.astype(np.int64), minlength=g.n)
    off = np.zeros(g.n + 1, np.uint32)
    off[1:] = np.cumsum(counts)
    return off, succ


def _noalloc(g, stream):
    import torch
    from paper_2004_10908_b300 import binding as B
    off, succ = _csr(g)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    kinds, params = dev(g.kinds), dev(g.params.view(np.int32))
    d_off, d_succ = dev(off.view(np.int32)), dev(succ.view(np.int32) if succ.size else np.zeros(1, np.int32))
    out = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros_like(out)
    dig = torch.zeros_like(out)
    torch.cuda.synchronize()
    st = B.tg_run_noalloc(g.n, kinds.data_ptr(), params.data_ptr(), d_off.data_ptr(), d_succ.data_ptr(),
                          int(succ.size), g.seed, out.data_ptr(), cnt.data_ptr(), dig.data_ptr(), stream)
    return st, out.cpu().numpy().view(np.uint32), cnt.cpu().numpy().view(np.uint32), dig.cpu().numpy().view(np.uint32)


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


def test_noalloc_alternating_graphs_and_limits():
    import torch
    from paper_2004_10908_b300 import binding as B
    stream = torch.cuda.current_stream().cuda_stream
    a, b = GRAPHS[1], GRAPHS[2]
    first = _noalloc(a, stream)
    _noalloc(b, stream)
    again = _noalloc(a, stream)
    for x, y in zip(first, again):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))
    # sizes beyond the fixed scratch array are refused before any GPU work
    assert B.tg_run_noalloc(70000, 1, 1, 1, 1, 10, 0, 0, 0, 0, stream) == B.TG_ERR_BUDGET
    assert B.tg_run_noalloc(10, 1, 1, 1, 1, 300000, 0, 0, 0, 0, stream) == B.TG_ERR_BUDGET
    # validation statuses: a task with no zero-dependency source
    st, *_ = _noalloc(w.pitfall_no_source(), stream)
    assert st == B.TG_ERR_NO_SOURCE
