"""Capturer baseline (Algorithm 1): a static DAG run as a CUDA graph of one
kernel per task over round-robin streams must produce the oracle's outputs,
counts and digests bit for bit, for any stream count and on every replay."""
import pytest

import oracle
import workloads as w
from tests.gpu_util import assert_same
from workloads.graphs import from_lists

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    from paper_2004_10908_b300 import Executor
    e = Executor(arena_bytes=1 << 30)
    yield e
    e.close()


def test_captured_dags_equal_oracle(ex):
    graphs = [w.diamond(), w.config2a(seed=9, levels=20, width=60, rounds=8),
              w.config2b(seed=2, side=24, rounds=16),
              from_lists("fan", [0] * 40, [3] * 40, [(0, t) for t in range(1, 39)] + [(t, 39) for t in range(1, 39)])]
    for g in graphs:
        ref = oracle.run(g)
        gh = ex.graph(g)
        for k in (1, 2, 4, 32):
            for _ in range(2):
                st, ns = ex.capture_run(gh, k)
                assert st == 0 and ns > 0
                out, cnt, dig, execs = ex.result(gh)
                assert_same((st, out, cnt, dig, execs), ref, f"{g.name} streams={k}")
        # the persistent scheduler still runs the same graph afterwards
        assert ex.run(gh) == 0
        assert_same((0,) + tuple(ex.result(gh)), ref, g.name)
        gh.destroy()


def test_capture_refuses_conditions_and_bad_stream_counts(ex):
    from paper_2004_10908_b300 import binding as B
    gh = ex.graph(w.do_while(5, 2))
    assert ex.capture_run(gh, 2)[0] == B.TG_ERR_INVALID
    gh.destroy()
    gh = ex.graph(w.diamond())
    assert ex.capture_run(gh, 0)[0] == B.TG_ERR_INVALID
    assert ex.capture_run(gh, 33)[0] == B.TG_ERR_INVALID
    gh.destroy()


def test_instances_do_not_share_the_templates_capture(ex):
    """An instance made after its template was captured has its own capture;
    destroying the instance leaves the template's intact."""
    from paper_2004_10908_b300 import binding as B
    g = w.diamond()
    ref = oracle.run(g)
    gh = ex.graph(g)
    assert ex.capture_run(gh, 2)[0] == 0
    inst = ex.instance(gh)
    assert ex.capture_run(inst, 2)[0] == 0
    inst.destroy()
    st, _ = ex.capture_run(gh, 2)
    assert st == 0
    assert_same((st,) + tuple(ex.result(gh)), ref, "template after instance")
    gh.destroy()
