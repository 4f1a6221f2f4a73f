"""Serving: a resident scheduler admits graph executions as they arrive
(memory budget, free graph slots), runs them overlapped on the device, and
each request's result equals the same graph run alone."""
import numpy as np
import pytest

import oracle
import workloads as w
from workloads.rng import Stream

pytestmark = pytest.mark.gpu


def _templates(count, seed=21, n_hi=20_000):
    out = []
    for i in range(count):
        st = Stream(seed * 7919 + i, 9)
        n = int(st.integers(1, 64, n_hi)[0])
        out.append(w.motif_graph(st, n, seed=seed * 1000 + i, rounds=16, name=f"req{i}"))
    return out


def _same(res, ref, name):
    out, cnt, dig, execs = res
    assert ref.status == 0
    np.testing.assert_array_equal(cnt, ref.cnt, err_msg=name)
    np.testing.assert_array_equal(out, ref.out, err_msg=name)
    np.testing.assert_array_equal(dig, ref.dig, err_msg=name)


@pytest.fixture(scope="module")
def ex():
    from paper_2004_10908_b300 import Executor
    e = Executor(arena_bytes=1 << 30, exec_cap=100_000)
    yield e
    e.close()


def test_instances_equal_oracle(ex):
    g = _templates(1, seed=3, n_hi=5000)[0]
    t = ex.graph(g)
    insts = [ex.instance(t) for _ in range(3)]
    ref = oracle.run(g, exec_cap=100_000)
    for h in [t] + insts:
        assert ex.run(h) == 0
        _same(ex.result(h), ref, g.name)
    b = ex.batch(insts)                      # instances of one graph run together
    b.launch()
    st, sts = b.wait()
    assert st == 0
    for h in insts:
        _same(ex.result(h), ref, g.name)
    b.destroy()
    from paper_2004_10908_b300 import binding as B
    assert B.tg_graph_destroy(ex.ctx, t.handle) == B.TG_ERR_BUSY    # instances alive
    for h in insts:
        h.destroy()
    t.destroy()


def test_mix_equals_alone(ex):
    gs = _templates(16)
    ts = [ex.graph(g) for g in gs]
    refs = [oracle.run(g, exec_cap=100_000) for g in gs]
    n_req = 240
    rng = np.random.default_rng(5)
    which = rng.integers(0, len(gs), n_req).astype(np.uint32)
    arrival = np.cumsum(rng.exponential(20e3, n_req)).astype(np.uint64)   # ~50k requests/s
    ex.serve_start(time_limit_ns=30_000_000_000)
    try:
        st, lat, sts, peak, kept = ex.serve_replay(ts, which, arrival, keep=True)
    finally:
        assert ex.serve_stop() == 0
    assert st == 0 and (sts == 0).all()
    assert peak > 1                          # requests overlapped on the device
    assert (lat > 0).all()
    for r in range(n_req):
        _same(ex.result(kept[r]), refs[which[r]], gs[which[r]].name)
        kept[r].destroy()
    for t in ts:
        t.destroy()


def test_budget_limits_admission():
    from paper_2004_10908_b300 import Executor
    from paper_2004_10908_b300 import binding as B
    gs = _templates(4, seed=31, n_hi=20_000)
    with Executor(arena_bytes=1 << 30) as ex2:
        ts = [ex2.graph(g) for g in gs]
        tmpl_bytes = sum(B.tg_graph_get_info(t.handle)["device_bytes"] for t in ts)
    # a budget that holds the templates plus two instances of the largest
    inst = [((g.n + 255) // 256) * 256 * 36 for g in gs]
    per_inst, min_inst = max(inst), min(inst)
    with Executor(arena_bytes=1 << 30, mem_budget_bytes=tmpl_bytes + 2 * per_inst + 1) as ex3:
        ts = [ex3.graph(g) for g in gs]
        n_req = 40
        which = (np.arange(n_req) % len(gs)).astype(np.uint32)
        arrival = np.zeros(n_req, np.uint64)          # all at once: admission must wait
        ex3.serve_start(time_limit_ns=30_000_000_000)
        try:
            st, lat, sts, peak, _ = ex3.serve_replay(ts, which, arrival)
        finally:
            assert ex3.serve_stop() == 0
        assert st == 0 and (sts == 0).all()
        assert 1 <= peak <= (2 * per_inst) // min_inst


def test_errors_stay_inside_their_request(ex):
    from paper_2004_10908_b300 import binding as B
    good = _templates(3, seed=41, n_hi=3000)
    forever = w.from_lists("forever", [0, w.COND_CONST], [w.pack_param(2), w.pack_param(2, 0, 0)],
                           [(0, 1), (1, 1)])
    gs = good + [forever]
    ts = [ex.graph(g) for g in gs]
    which = np.array([0, 3, 1, 2, 3, 0], np.uint32)
    arrival = np.arange(6, dtype=np.uint64) * 1000
    ex.serve_start(time_limit_ns=30_000_000_000)
    try:
        st, lat, sts, peak, kept = ex.serve_replay(ts, which, arrival, keep=True)
    finally:
        assert ex.serve_stop() == 0
    assert st == B.TG_ERR_EXEC_LIMIT
    for r, wi in enumerate(which):
        if wi == 3:
            assert sts[r] == B.TG_ERR_EXEC_LIMIT
        else:
            assert sts[r] == 0
            _same(ex.result(kept[r]), oracle.run(gs[wi], exec_cap=100_000), gs[wi].name)
        kept[r].destroy()
    for t in ts:
        t.destroy()


def test_submit_and_poll_while_serving(ex):
    from paper_2004_10908_b300 import binding as B
    gs = _templates(3, seed=51, n_hi=4000)
    ts = [ex.graph(g) for g in gs]
    ex.serve_start(time_limit_ns=30_000_000_000)
    try:
        assert ex.run(ts[0]) == B.TG_ERR_BUSY           # one-shot launches wait for the server
        tickets = [ex.submit(t) for t in ts]
        st2, _ = B.tg_submit(ex.ctx, ts[0].handle)
        assert st2 in (B.TG_ERR_BUSY, B.TG_OK)
        for t in tickets:
            assert ex.wait(t) == 0
        if st2 == B.TG_OK:
            pass
    finally:
        assert ex.serve_stop() == 0
    for g, t in zip(gs, ts):
        _same(ex.result(t), oracle.run(g, exec_cap=100_000), g.name)
        t.destroy()


def test_plain_runs_after_serving_and_beside_other_block_shapes(orc):
    """A server (narrower blocks) or a second context with another block
    shape checked in between must leave a context's own launch shape valid."""
    from paper_2004_10908_b300 import Executor
    g = _templates(1, seed=8, n_hi=3000)[0]
    ref = orc.run(g, exec_cap=100_000)
    with Executor(arena_bytes=256 << 20, warps_per_block=16) as wide, \
            Executor(arena_bytes=256 << 20, warps_per_block=4) as narrow:
        hw, hn = wide.graph(g), narrow.graph(g)
        for _ in range(2):
            assert wide.run(hw) == 0
            _same(wide.result(hw), ref, "wide")
            assert narrow.run(hn) == 0
            _same(narrow.result(hn), ref, "narrow")
        wide.serve_start()
        assert wide.wait(wide.submit(hw)) == 0
        assert wide.serve_stop() == 0
        _same(wide.result(hw), ref, "served")
        assert wide.run(hw) == 0
        _same(wide.result(hw), ref, "after serving")


def _request(i, n):
    """The serving workload's request graph i (64 rounds, graph seed i), at a
    chosen task count instead of the log-uniform draw."""
    from workloads.graphs import _logu
    st = Stream(i, 5)
    _logu(st, 64, 262144)
    return w.motif_graph(st, n, seed=i, rounds=64, name=f"request{i}")


def test_full_size_requests_served_together_equal_oracle():
    """Requests of the serving recipe up to its largest size (262,144 tasks,
    64 rounds, 5 % loop conditions), admitted while the others run, each
    equal to the oracle element by element; only the masked requests'
    instances are kept."""
    from paper_2004_10908_b300 import Executor
    sizes = [262144, 64, 180000, 4096, 262144, 1000]
    gs = [_request(100 + i, n) for i, n in enumerate(sizes)]
    with Executor(arena_bytes=2 << 30) as ex2:
        ts = [ex2.graph(g) for g in gs]
        which = np.array([0, 1, 2, 3, 4, 5, 0, 2], np.uint32)
        arrival = (np.arange(which.shape[0], dtype=np.uint64) * 20_000)   # 50k requests/s
        mask = np.array([1, 1, 1, 1, 1, 1, 0, 1], bool)
        ex2.serve_start(time_limit_ns=60_000_000_000)
        try:
            st, lat, sts, peak, kept = ex2.serve_replay(ts, which, arrival, keep=mask)
        finally:
            assert ex2.serve_stop() == 0
        assert st == 0 and (sts == 0).all()
        assert peak > 1
        assert kept[6] is None
        refs = {}
        for r, wi in enumerate(which):
            if not mask[r]:
                continue
            if wi not in refs:
                refs[wi] = oracle.run(gs[wi])
            _same(ex2.result(kept[r]), refs[wi], gs[wi].name)
            kept[r].destroy()
        for t in ts:
            t.destroy()


def test_serving_first_thing_in_a_fresh_process():
    """A process whose first launches are the server's: the kernels the host
    launches while the resident scheduler runs are loaded before it starts
    (with lazy module loading a first launch would wait for the running
    server, which waits for that launch -- until its time limit).  The run
    is bounded by a 20 s server limit and a 180 s process timeout."""
    import os
    import subprocess
    import sys
    code = r'''
import numpy as np, sys
sys.path.insert(0, sys.argv[1])
import workloads as w, oracle
from workloads.rng import Stream
from paper_2004_10908_b300 import Executor
st = Stream(7, 9)
gs = [w.motif_graph(st, 3000 + 500 * i, seed=70 + i, rounds=16) for i in range(3)]
with Executor(arena_bytes=1 << 29) as ex:
    ts = [ex.graph(g) for g in gs]
    ex.serve_start(time_limit_ns=20_000_000_000)
    try:
        rc, lat, sts, peak, kept = ex.serve_replay(ts, np.array([0, 1, 2, 1], np.uint32),
                                                   np.arange(4, dtype=np.uint64) * 1000, keep=True)
    finally:
        stop = ex.serve_stop()
    assert rc == 0 and stop == 0 and (sts == 0).all(), (rc, stop, list(sts))
    for r, wi in enumerate([0, 1, 2, 1]):
        out, cnt, dig, _ = ex.result(kept[r])
        ref = oracle.run(gs[wi])
        assert (out == ref.out).all() and (cnt == ref.cnt).all() and (dig == ref.dig).all()
        kept[r].destroy()
print("served")
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", code, root], capture_output=True, text=True, timeout=180)
    assert res.returncode == 0 and "served" in res.stdout, res.stdout[-2000:] + res.stderr[-2000:]
