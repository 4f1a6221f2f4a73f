"""Failure handling on the device without faulting the GPU: execution cap,
device time limit, host cancel; the context stays usable afterwards."""
import time

import numpy as np
import pytest

import oracle
import workloads as w
from tests.gpu_util import assert_same, run_both

pytestmark = pytest.mark.gpu


def _forever():
    # a condition that always jumps back to itself: never terminates by itself
    return w.from_lists("forever", [0, w.COND_CONST], [w.pack_param(4), w.pack_param(4, 0, 0)],
                        [(0, 1), (1, 1)])


def test_exec_cap():
    from paper_2004_10908_b300 import Executor, binding as B
    with Executor(arena_bytes=256 << 20, exec_cap=150) as ex:
        dev, ref = run_both(ex, w.do_while(), exec_cap=150)
        assert ref.status == oracle.EXEC_LIMIT and dev[0] == B.TG_ERR_EXEC_LIMIT
        dev, ref = run_both(ex, w.do_while(iterations=20), exec_cap=150)
        assert_same(dev, ref, "do_while within cap")


def test_time_limit_then_context_still_works():
    from paper_2004_10908_b300 import Executor, binding as B
    with Executor(arena_bytes=256 << 20, time_limit_ns=50_000_000) as ex:
        gh = ex.graph(_forever())
        t0 = time.time()
        assert ex.run(gh) == B.TG_ERR_TIMEOUT
        assert time.time() - t0 < 5
        gh.destroy()
        dev, ref = run_both(ex, w.config1(levels=3, width=10, trip=2, rounds=4))
        assert_same(dev, ref, "after timeout")


def test_cancel_then_context_still_works():
    from paper_2004_10908_b300 import Executor, binding as B
    with Executor(arena_bytes=256 << 20, time_limit_ns=20_000_000_000) as ex:
        gh = ex.graph(_forever())
        t = ex.submit(gh)
        time.sleep(0.05)
        assert ex.poll(t) == B.TG_PENDING
        ex.cancel()
        assert ex.wait(t) == B.TG_ERR_CANCELLED
        gh.destroy()
        dev, ref = run_both(ex, w.do_while())
        assert_same(dev, ref, "after cancel")


def test_context_destroy_frees_what_the_caller_left():
    """Graphs, instances, composed graphs and batches left alive are freed
    with their context; a new context on the same device works."""
    from paper_2004_10908_b300 import Executor
    from workloads.graphs import MODULE, STATIC, from_lists, pack_param
    for _ in range(3):
        e = Executor(arena_bytes=1 << 28)
        g = e.graph(w.config1(levels=3, width=20, trip=2, rounds=4))
        e.instance(g)
        inner = e.graph(w.diamond())
        top = e.graph(from_lists("t", [STATIC, MODULE], pack_param([2, 2]), [(0, 1)]), modules={1: inner})
        b = e.batch([g, top])
        b.launch()
        assert b.wait()[0] == 0
        e.capture_run(inner, 2)
        e.close()           # nothing destroyed by hand
    with Executor(arena_bytes=1 << 28) as e:
        h = e.graph(w.diamond())
        assert e.run(h) == 0
