"""Batches: many graphs in one CUDA-graph-captured persistent launch.  Every
graph's result must equal the oracle and the same graph run alone; errors
stay inside the graph that caused them; autotuning keeps results exact."""
import numpy as np
import pytest

import oracle
import workloads as w
from paper_2004_10908_b300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    from paper_2004_10908_b300 import Executor
    e = Executor(arena_bytes=1 << 30, exec_cap=200_000)
    yield e
    e.close()


def _check_against_oracle(ex, gs, hs, exec_cap=200_000):
    for g, h in zip(gs, hs):
        out, cnt, dig, execs = ex.result(h)
        r = oracle.run(g, exec_cap=exec_cap)
        assert r.status == 0
        np.testing.assert_array_equal(cnt, r.cnt, err_msg=g.name)
        np.testing.assert_array_equal(out, r.out, err_msg=g.name)
        np.testing.assert_array_equal(dig, r.dig, err_msg=g.name)


def test_batch_equals_oracle_and_alone(ex):
    gs = w.config4(seed=11, n_graphs=96, n_lo=16, n_hi=4000)
    hs = [ex.graph(g) for g in gs]
    b = ex.batch(hs)
    b.launch()
    st, sts = b.wait()
    assert st == 0 and (sts == 0).all()
    _check_against_oracle(ex, gs, hs)
    batched = [ex.result(h) for h in hs]
    for h, bres in zip(hs[:24], batched[:24]):        # the same graph alone
        assert ex.run(h) == 0
        for x, y in zip(ex.result(h)[:3], bres[:3]):
            np.testing.assert_array_equal(x, y)
    for _ in range(2):                                 # replays of the captured graph
        b.launch()
        st, sts = b.wait()
        assert st == 0
    for h, bres in zip(hs, batched):
        for x, y in zip(ex.result(h)[:3], bres[:3]):
            np.testing.assert_array_equal(x, y)
    b.destroy()
    for h in hs:
        h.destroy()


def test_errors_stay_inside_their_graph(ex):
    from paper_2004_10908_b300 import binding as B
    good = w.config4(seed=12, n_graphs=20, n_lo=16, n_hi=2000)
    forever = w.from_lists("forever", [0, w.COND_CONST], [w.pack_param(2), w.pack_param(2, 0, 0)],
                           [(0, 1), (1, 1)])
    racy = w.nested_loops(5, extra_init_to_f2=True)
    gs = good[:10] + [forever] + good[10:] + [racy]
    hs = [ex.graph(g) for g in gs]
    b = ex.batch(hs)
    b.launch()
    st, sts = b.wait()
    assert sts[10] == B.TG_ERR_EXEC_LIMIT
    assert sts[-1] in (B.TG_ERR_RACE, B.TG_OK)
    ok_idx = [i for i in range(len(gs)) if i not in (10, len(gs) - 1)]
    assert all(sts[i] == 0 for i in ok_idx)
    _check_against_oracle(ex, [gs[i] for i in ok_idx], [hs[i] for i in ok_idx])
    b.destroy()
    for h in hs:
        h.destroy()


def test_graph_in_flight_is_busy(ex):
    from paper_2004_10908_b300 import binding as B
    gs = w.config4(seed=13, n_graphs=8, n_lo=2000, n_hi=4000)
    hs = [ex.graph(g) for g in gs]
    b = ex.batch(hs)
    b.launch()
    st2, _ = B.tg_submit(ex.ctx, hs[0].handle)
    assert st2 in (B.TG_ERR_BUSY, B.TG_OK)
    st, sts = b.wait()
    assert st == 0
    if st2 == B.TG_OK:
        ex.stream.synchronize()
    b.destroy()
    for h in hs:
        h.destroy()


def test_autotune_keeps_results_exact(ex, tmp_path):
    gs = w.config4(seed=14, n_graphs=64, n_lo=16, n_hi=3000)
    hs = [ex.graph(g) for g in gs]
    b = ex.batch(hs)
    cache = str(tmp_path / "tune.txt")
    chosen, ns = b.autotune(trials=1, cache_path=cache)
    assert ns > 0 and chosen["warps_per_block"] in (4, 8, 16)
    assert open(cache).read().count("\n") == 1
    chosen2, ns2 = b.autotune(trials=1, cache_path=cache)     # served from the cache
    assert chosen2["warps_per_block"] == chosen["warps_per_block"]
    assert chosen2["worker_blocks"] == chosen["worker_blocks"]
    b.launch()
    st, sts = b.wait()
    assert st == 0
    _check_against_oracle(ex, gs, hs)
    b.destroy()
    for h in hs:
        h.destroy()


def test_launch_geometry_variants_are_exact(ex):
    gs = w.config4(seed=15, n_graphs=32, n_lo=16, n_hi=3000)
    hs = [ex.graph(g) for g in gs]
    try:
        for geo in (dict(warps_per_block=4, worker_blocks=148, steal_policy=1, max_steal=2, max_thieves=4),
                    dict(warps_per_block=16, deque_depth=256, max_thieves=64),
                    dict(steal_backoff_ns=4096, idle_sleep_ns=1024),
                    dict(steal_backoff_ns=32, worker_blocks=296, warps_per_block=8, hand_batch=1),
                    dict(worker_blocks=1, warps_per_block=1)):
            ex.set_launch(**geo)
            b = ex.batch(hs)
            b.launch()
            st, sts = b.wait()
            assert st == 0, geo
            _check_against_oracle(ex, gs, hs)
            b.destroy()
        with pytest.raises(B.TgError):
            ex.set_launch(steal_backoff_ns=1_000_001)   # above the documented limit
    finally:
        ex.set_launch()
        for h in hs:
            h.destroy()


@pytest.mark.slow
def test_full_size_batch_sampled():
    """4,096 graphs, 33M tasks, one launch; 64 sampled graphs vs the oracle."""
    from paper_2004_10908_b300 import Executor
    gs = w.config4()
    with Executor(arena_bytes=8 << 30, max_nodes=40_000_000, max_edges=450_000_000) as ex2:
        hs = [ex2.graph(g) for g in gs]
        b = ex2.batch(hs)
        b.launch()
        st, sts = b.wait()
        assert st == 0 and (sts == 0).all()
        idx = np.random.default_rng(1).choice(len(gs), 64, replace=False)
        _check_against_oracle(ex2, [gs[i] for i in idx], [hs[i] for i in idx], exec_cap=1 << 31)
        b.destroy()


def test_graph_autotune_keeps_results_and_caches(tmp_path):
    """Per-graph autotuning: the chosen geometry is valid, later runs still
    equal the oracle, and a second call is answered from the cache."""
    import oracle as orc_mod
    from paper_2004_10908_b300 import Executor
    g = w.config1(levels=6, width=60, trip=3, rounds=16)
    ref = orc_mod.run(g)
    cache = str(tmp_path / "tune.txt")
    with Executor(arena_bytes=1 << 30) as e:
        h = e.graph(g)
        chosen, ns = e.autotune(h, trials=1, cache_path=cache)
        assert ns > 0 and 1 <= chosen["warps_per_block"] <= 32 and chosen["worker_blocks"] > 0
        assert e.run(h) == 0
        out, cnt, dig, execs = e.result(h)
        np.testing.assert_array_equal(cnt, ref.cnt)
        np.testing.assert_array_equal(out, ref.out)
        np.testing.assert_array_equal(dig, ref.dig)
        assert e.stats()["warps_per_block"] == chosen["warps_per_block"]
        lines = open(cache).read().splitlines()
        assert len(lines) == 1 and "|graph|" in lines[0]
        chosen2, ns2 = e.autotune(h, trials=1, cache_path=cache)
        assert chosen2 == chosen and ns2 == ns
        assert len(open(cache).read().splitlines()) == 1


def test_graph_in_a_live_batch_cannot_be_destroyed(ex):
    from paper_2004_10908_b300 import binding as B
    gs = [w.diamond(), w.do_while(3, 2)]
    hs = [ex.graph(g) for g in gs]
    b = ex.batch(hs)
    assert B.tg_graph_destroy(ex.ctx, hs[0].handle) == B.TG_ERR_BUSY
    b.launch()
    st, sts = b.wait()
    assert st == 0
    b.destroy()
    for h in hs:
        assert B.tg_graph_destroy(ex.ctx, h.handle) == 0
        h.handle = None
