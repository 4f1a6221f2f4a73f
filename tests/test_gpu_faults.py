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


def _wide_forever(width=3000):
    # source -> head -> `width` tasks -> a condition that always jumps back
    # to the head: at any moment many activations sit in the queues
    n = width + 3
    kinds = [0] * (width + 2) + [w.COND_CONST]
    params = [w.pack_param(32)] * (width + 2) + [w.pack_param(4, 0, 0)]
    edges = [(0, 1)] + [(1, 2 + i) for i in range(width)] + [(2 + i, n - 1) for i in range(width)] + [(n - 1, 1)]
    return w.from_lists("wide_forever", kinds, params, edges)


def test_aborted_launch_leaves_clean_queues_for_the_next_submission():
    """A launch that hits its time limit with activations still queued, and
    another graph submitted behind it before the host has read the first
    status: the second run must match the oracle (the aborted launch's
    queues are emptied on the device before the next launch starts)."""
    from paper_2004_10908_b300 import Executor, binding as B
    g_ok = w.config2a(seed=4, levels=40, width=400, rounds=8)
    ref = oracle.run(g_ok)
    with Executor(arena_bytes=512 << 20, time_limit_ns=50_000_000) as ex:
        ga = ex.graph(_wide_forever())
        gb = ex.graph(g_ok)
        for _ in range(3):
            ta = ex.submit(ga)
            tb = ex.submit(gb)
            assert ex.wait(ta) == B.TG_ERR_TIMEOUT
            st = ex.wait(tb)
            assert_same((st,) + tuple(ex.result(gb)), ref, "behind an aborted launch")
        ga.destroy()
        gb.destroy()


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
