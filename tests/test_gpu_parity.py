"""CUDA path against the oracle, element by element, bit-exact (integer
work: every task's output, execution count and digest)."""
import random

import numpy as np
import pytest

import oracle
import workloads as w
from tests import pins
from tests.gpu_util import assert_same, run_both

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    from paper_2004_10908_b300 import Executor
    e = Executor(arena_bytes=2 << 30)
    yield e
    e.close()


def test_paper_examples(ex):
    gs = [w.diamond(), w.if_else(0), w.if_else(1), w.if_else(2), w.if_else(-1), w.do_while(),
          w.pitfall_race(fixed=True)] + [w.nested_loops(s) for s in range(20)]
    for g in gs:
        dev, ref = run_both(ex, g)
        assert_same(dev, ref, g.name)


def test_racy_graphs_report_race_or_match_a_schedule(ex):
    """Pitfall 2 and the walk-through's init -> F2 edge are non-confluent: a
    run must end with RACE or equal one of the brute-force schedules."""
    from paper_2004_10908_b300 import STATUS_NAMES
    graphs = [w.pitfall_race()] + [w.nested_loops(s, extra_init_to_f2=True) for s in range(8)]
    seen = set()
    for g in graphs:
        outs = pins.brute_force(g, exec_cap=1 << 31, max_states=300000)
        assert ("RACE",) in outs
        for _ in range(20):
            gh = ex.graph(g)
            st = ex.run(gh)
            out, cnt, dig, execs = ex.result(gh)
            gh.destroy()
            name = STATUS_NAMES[st]
            mine = ("OK", tuple(int(x) for x in out), tuple(int(x) for x in cnt), tuple(int(x) for x in dig))
            assert name == "RACE" or (name == "OK" and mine in outs), (g.name, name)
            seen.add(name)
    assert oracle.run(w.pitfall_race()).status == oracle.RACE


def test_validation_statuses_match_oracle(ex):
    from paper_2004_10908_b300 import binding as B
    cases = [w.from_lists("bad_idx", [0, 0], [1, 1], [(0, 5)]),
             w.from_lists("cond_no_succ", [0, 1], [1, 1], [(0, 1)]),
             w.from_lists("trip0", [0, 2], [1, 1], [(0, 1), (1, 0)]),
             w.from_lists("kind9", [9], [1], []),
             w.pitfall_no_source(),
             w.from_lists("weakonly", [3, 0], [w.pack_param(1, 0, 0), 1], [(0, 1), (1, 0)])]
    for g in cases:
        st, h = B.tg_graph_create(ex.ctx, g.kinds, g.params, g.src, g.dst, g.seed)
        assert h is None
        assert B.STATUS_NAMES[st] == oracle.STATUS_NAMES[oracle.run(g).status], g.name
    g = w.diamond()
    st, h = B.tg_graph_create(ex.ctx, g.kinds, g.params, g.src, g.dst, 0, np.array([0, 1, 0, 0], np.uint8))
    assert st == B.TG_ERR_EDGE_KIND and oracle.run(g, weak=np.array([0, 1, 0, 0], np.uint8)).status == oracle.EDGE_KIND


def test_tiny_graphs_against_all_schedules(ex):
    rng = random.Random(11)
    checked = 0
    for _ in range(400):
        n = rng.randint(1, 5)
        kinds = [rng.choice([0, 0, 0, 1, 2]) for _ in range(n)]
        params = [rng.randint(0, 3) | (rng.randint(1, 3) << 16) for _ in range(n)]
        edges = [(v, rng.randrange(n)) for v in range(n) for _ in range(rng.randint(1 if kinds[v] else 0, 3))]
        g = w.from_lists("tiny", kinds, params, edges, seed=rng.getrandbits(32))
        ref = oracle.run(g, exec_cap=10_000)
        if ref.status in (oracle.INVALID, oracle.NO_SOURCE, oracle.EXEC_LIMIT):
            continue   # invalid, or loops past any cap worth enumerating
        try:
            outs = pins.brute_force(g, exec_cap=40, max_states=4000)
        except RuntimeError:
            continue
        if any(o[0] == "EXEC_LIMIT" for o in outs):
            continue   # loops too long to enumerate every schedule
        gh = ex.graph(g)
        st = ex.run(gh)
        out, cnt, dig, execs = ex.result(gh)
        gh.destroy()
        from paper_2004_10908_b300 import STATUS_NAMES
        if len(outs) == 1:
            assert_same((st, out, cnt, dig, execs), ref, "tiny")
        else:   # racy graph: report the race or equal some schedule
            mine = ("OK", tuple(int(x) for x in out), tuple(int(x) for x in cnt), tuple(int(x) for x in dig))
            assert STATUS_NAMES[st] == "RACE" or (st == 0 and mine in outs)
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("levels,width", [(3, 1), (5, 33), (37, 333), (100, 100)])
def test_layered_dag(ex, levels, width):
    g = w.config2a(seed=levels * width, levels=levels, width=width)
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, g.name)


@pytest.mark.parametrize("side,rounds", [(1, 3), (17, 9), (100, 16)])
def test_wavefront(ex, side, rounds):
    g = w.config2b(side=side, rounds=rounds)
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, g.name)


def test_config1_full(ex):
    g = w.config1()
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, "config1")
    assert dev[4] == 5012


def test_config2a_full(ex):
    g = w.config2a()
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, "config2a")


def test_config2b_full(ex):
    g = w.config2b()
    dev, ref = run_both(ex, g)
    assert_same(dev, ref, "config2b")


def test_config3_small_and_full(ex):
    for g in (w.config3(seed=7, n_cond=200, body_levels=4, body_width=7, rounds=5),
              w.config3()):
        dev, ref = run_both(ex, g)
        assert_same(dev, ref, g.name)


def test_motif_graphs(ex):
    for g in w.config4(seed=9, n_graphs=16, n_lo=16, n_hi=5000):
        dev, ref = run_both(ex, g)
        assert_same(dev, ref, g.name)


def test_repeated_runs_are_identical(ex):
    g = w.config3(seed=5, n_cond=100, body_levels=3, body_width=6, rounds=4)
    gh = ex.graph(g)
    first = None
    for _ in range(5):
        assert ex.run(gh) == 0
        r = ex.result(gh)
        if first is None:
            first = r
        for a, b in zip(first[:3], r[:3]):
            np.testing.assert_array_equal(a, b)
    gh.destroy()


def test_submit_poll_wait_and_busy(ex):
    from paper_2004_10908_b300 import binding as B
    g = w.config2a(levels=200, width=200, rounds=64)
    gh = ex.graph(g)
    t = ex.submit(gh)
    st = ex.poll(t)
    assert st in (B.TG_PENDING, B.TG_OK)
    st2, _ = B.tg_submit(ex.ctx, gh.handle)
    assert st2 in (B.TG_ERR_BUSY, B.TG_OK)
    if st2 == B.TG_OK:
        pytest.skip("the first run finished before the second submit")
    assert ex.wait(t) == B.TG_OK
    assert ex.poll(t) == B.TG_OK
    out, cnt, dig, execs = ex.result(gh)
    ref = oracle.run(g)
    np.testing.assert_array_equal(out, ref.out)
    gh.destroy()


def test_stats_count_every_execution(ex):
    g = w.config1(levels=5, width=50, trip=4, rounds=8)
    gh = ex.graph(g)
    assert ex.run(gh) == 0
    s = ex.stats()
    _, _, _, execs = ex.result(gh)
    assert s["tasks"] == execs
    assert s["kernel_ns"] > 0
    gh.destroy()


def test_payload_kernel_matches_oracle_payload(ex):
    for R in (0, 1, 16, 64):
        n = 100_003
        ns, cs = ex.bench_payload(n, R)
        ref = oracle.payload_many(np.arange(n), np.zeros(n), np.zeros(n), np.full(n, R))
        assert cs == int(np.bitwise_xor.reduce(ref)), R


def test_chain_floor_kernel_matches_oracle_payload_chain(ex):
    """The dependency-floor kernel computes the payloads of a path: output
    of hop h feeds the input sum of hop h + 1."""
    for hops, R in ((1, 0), (37, 5), (300, 16)):
        ns, last = ex.bench_chain(hops, R)
        x = 0
        for h in range(hops):
            x = oracle.payload(h, 0, x, R)
        assert last == x, (hops, R)


def test_adaptive_thieves_parity_and_fewer_wasted_steals():
    """Adaptive thief mode (Alg. 3/6): same results as the oracle on DAGs,
    loops, branches and racy-free tiny graphs; on a chain (one task ready at
    a time) it wastes far fewer steal rounds than a fixed cap of 16 thieves,
    because all but the last failed thief park."""
    from paper_2004_10908_b300 import Executor
    from workloads.graphs import STATIC, from_lists, pack_param
    graphs = [w.config1(levels=6, width=40, trip=3, rounds=16), w.do_while(200, 4),
              w.config2a(seed=5, levels=30, width=300, rounds=8),
              w.config3(seed=3, n_cond=60, body_levels=4, body_width=6, rounds=8, trip_max=6)] + \
             [w.nested_loops(s) for s in range(6)]
    with Executor(arena_bytes=1 << 30, thief_mode=1) as ex:
        assert ex.opts()["thief_mode"] == 1
        for g in graphs:
            dev, ref = run_both(ex, g)
            assert_same(dev, ref, g.name)
    n = 3000
    chain = from_lists("chain", [STATIC] * n, [pack_param(0)] * n, [(i, i + 1) for i in range(n - 1)])
    wasted = {}
    for mode in (0, 1):
        with Executor(arena_bytes=1 << 28, thief_mode=mode) as ex:
            h = ex.graph(chain)
            assert ex.run(h) == 0
            s = ex.stats()
            wasted[mode] = s["failed_rounds"]
            if mode == 1:
                assert s["parks"] > 0
                assert 1 <= s["peak_thieves"] <= s["worker_blocks"]
    assert wasted[1] * 4 < wasted[0], wasted


def test_wasteful_steals_within_the_papers_bound():
    """The paper's bound on wasteful steals (Analysis, third theorem): at any
    moment at most MAX_STEALS x (|W| + |D| E / e_s) of them, W the workers
    (here worker blocks), one domain, E the longest task, e_s one steal
    round.  Counted in rounds over windows of length E, a run of length T
    wastes at most (|W| + E / e_s) x ceil(T / E) rounds.  E is measured as
    one payload of the chain's tasks, e_s from the device's own count of the
    cycles its failed rounds took.  Checked for both thief modes on the worst
    case the proof names (one task ready at a time: a chain) and on a wide
    layered DAG."""
    import math

    import torch
    from paper_2004_10908_b300 import Executor
    from workloads.graphs import STATIC, from_lists, pack_param
    try:
        mhz = float(torch.cuda.clock_rate(0)) or 2032.0
    except Exception:   # noqa: BLE001 -- no clock query available: the maximum clock
        mhz = 2032.0
    R = 64
    chain = from_lists("chain", [STATIC] * 2000, [pack_param(R)] * 2000, [(i, i + 1) for i in range(1999)])
    wide = w.config2a(seed=5, levels=60, width=500, rounds=R)
    for mode in (0, 1):
        with Executor(arena_bytes=1 << 29, thief_mode=mode) as ex:
            E_ns = ex.bench_chain(200, R)[0] / 200.0
            for g in (chain, wide):
                h = ex.graph(g)
                assert ex.run(h) == 0
                s = ex.stats()
                h.destroy()
                failed, cyc = s["failed_rounds"], s["round_cycles"]
                assert failed > 0 and cyc > 0
                e_s_ns = cyc / failed / (mhz * 1e-3)
                bound = (s["worker_blocks"] + E_ns / e_s_ns) * math.ceil(s["kernel_ns"] / E_ns)
                assert failed <= bound, (mode, g.name, failed, bound, E_ns, e_s_ns)


def test_adaptive_thieves_finish_a_wide_wavefront():
    """Adaptive thieves with a short local backlog on a wide wavefront: busy
    warps spill to their block's deque while other blocks park; the run must
    finish (well inside its time limit) with the oracle's results."""
    from paper_2004_10908_b300 import Executor
    g = w.config2b(seed=2, side=192, rounds=64)
    ref = oracle.run(g)
    for geo in (dict(thief_mode=1, local_keep=16, max_thieves=8), dict(thief_mode=1, local_keep=16, batch_max=8),
                dict(hand_batch=1), dict(hand_batch=1, warps_per_block=4, worker_blocks=148)):
        with Executor(arena_bytes=1 << 29, time_limit_ns=5_000_000_000, **geo) as e:
            for _ in range(3):
                gh = e.graph(g)
                st = e.run(gh)
                res = (st,) + tuple(e.result(gh))
                gh.destroy()
                assert_same(res, ref, f"wavefront {geo}")


def test_tracing_keeps_results_and_records_times():
    """TG_OPT_TRACE (the extended scheduler variant): same results; every
    executed task has a start no later than its publish time, and the phase
    cycle counters are filled."""
    from paper_2004_10908_b300 import Executor, binding as B
    g = w.config1(levels=4, width=50, trip=2, rounds=16)
    ref = oracle.run(g)
    with Executor(arena_bytes=1 << 28, flags=B.TG_OPT_TRACE) as e:
        gh = e.graph(g)
        st = e.run(gh)
        assert_same((st,) + tuple(e.result(gh)), ref, "traced")
        s = e.stats()
        assert all(c > 0 for c in s["phase_cycles"])
        t0, t1, wh = B.tg_trace_copy(e.ctx, gh.handle, g.n)
        ran = ref.cnt > 0
        assert (t0[ran] > 0).all() and (t1[ran] >= t0[ran]).all()
        assert ((wh[ran] >> 16) <= B.TG_TRACE_FROM_INJECTION).all()
        gh.destroy()


def test_task_trace_in_the_lean_variant_reads_the_critical_path():
    """TG_OPT_TRACE_TASKS keeps the lean scheduler variant: results equal the
    oracle, every task carries a take time, a later step end and where it
    came from, the sources came from the injection queue, and on a layered
    DAG (every task has a predecessor one level up) the chain of
    last-finishing predecessors crosses every level exactly once."""
    from paper_2004_10908_b300 import Executor, binding as B
    from paper_2004_10908_b300.trace import critical_path
    levels, width = 40, 300
    g = w.config2a(seed=5, levels=levels, width=width, d_lo=1, d_hi=6, rounds=8)
    ref = oracle.run(g)
    with Executor(arena_bytes=1 << 28, flags=B.TG_OPT_TRACE_TASKS) as e:
        for geo in (dict(), dict(warps_per_block=4, worker_blocks=296, batch_max=8)):
            e.set_launch(**geo)
            gh = e.graph(g)
            st = e.run(gh)
            assert_same((st,) + tuple(e.result(gh)), ref, f"task trace {geo}")
            assert all(c == 0 for c in e.stats()["phase_cycles"])   # no phase counters: lean variant
            t0, t1, wh = B.tg_trace_copy(e.ctx, gh.handle, g.n)
            assert (t0 > 0).all() and (t1 >= t0).all()
            frm = wh >> 16
            assert (frm <= B.TG_TRACE_FROM_INJECTION).all()
            assert ((wh & 0xFFFF) < e.stats()["worker_blocks"]).all()
            assert (frm[:width] == B.TG_TRACE_FROM_INJECTION).all()   # level 0: the sources
            cp = critical_path(g.src, g.dst, t0, t1, wh)
            last_level = int(np.argmax(t1)) // width
            assert cp["tasks"] == last_level + 1 and last_level >= levels - 2
            assert sum(v["hops"] for v in cp["hops_by_source"].values()) == last_level
            assert sum(cp["all_tasks_by_source"].values()) == g.n
            gh.destroy()
        e.set_launch()


def test_looping_graphs_never_report_a_false_race():
    """Graphs whose conditions loop back (a task re-activated soon after its
    own step, often by a sibling warp of the same block) run many times at
    several launch shapes: every run must be OK and equal the oracle -- the
    in-flight flag a task clears must be visible to the flag test of its
    next activation."""
    from paper_2004_10908_b300 import Executor
    graphs = [w.config1(levels=6, width=60, trip=3, rounds=16), w.do_while(300, 2),
              w.config3(seed=4, n_cond=80, body_levels=3, body_width=5, rounds=4, trip_max=6)] + \
             [w.nested_loops(s) for s in range(3)]
    refs = [oracle.run(g) for g in graphs]
    for geo in (dict(), dict(warps_per_block=4, worker_blocks=592), dict(warps_per_block=8, batch_max=8),
                dict(keep_idle=1), dict(keep_idle=1, warps_per_block=4, worker_blocks=296, local_keep=16),
                dict(hand_batch=1), dict(hand_batch=1, keep_idle=1, batch_max=8)):
        with Executor(arena_bytes=1 << 29, **geo) as ex:
            hs = [ex.graph(g) for g in graphs]
            for _ in range(8):
                for g, h, ref in zip(graphs, hs, refs):
                    st = ex.run(h)
                    assert_same((st,) + tuple(ex.result(h)), ref, f"{g.name} {geo}")


def test_graphs_created_while_another_runs(ex):
    """Ingest uploads on its own stream: graphs created while a long graph
    runs on the context stream, then run themselves, all equal the oracle."""
    long_g = w.config2b(side=256, rounds=128)
    others = [w.config2a(seed=31 + i, levels=30, width=300, rounds=8) for i in range(3)] + [w.config1(levels=5, width=40)]
    h_long = ex.graph(long_g)
    t_long = ex.submit(h_long)
    hs = [ex.graph(g) for g in others]          # created while the long graph runs
    assert ex.wait(t_long) == 0
    assert_same((0,) + tuple(ex.result(h_long)), oracle.run(long_g), "long graph")
    for g, h in zip(others, hs):
        st = ex.run(h)
        assert_same((st,) + tuple(ex.result(h)), oracle.run(g), g.name)
        h.destroy()
    h_long.destroy()


def test_results_read_while_the_next_graph_runs(ex):
    """tg_result_copy waits for its graph's own launch only: a graph's results
    are read (and are the oracle's) while a graph submitted after it runs."""
    g1 = w.config2a(seed=21, levels=60, width=300)
    g2 = w.config2b(side=300, rounds=64)
    h1, h2 = ex.graph(g1), ex.graph(g2, device_pack=True)
    try:
        t1 = ex.submit(h1)
        t2 = ex.submit(h2)
        assert ex.wait(t1) == 0
        r1 = ex.result(h1)
        assert_same((0,) + tuple(r1), oracle.run(g1), g1.name)
        assert ex.wait(t2) == 0
        assert_same((0,) + tuple(ex.result(h2)), oracle.run(g2), g2.name)
        # a resubmitted graph: the read waits for its new launch
        t1 = ex.submit(h1)
        r1b = ex.result(h1)
        assert ex.wait(t1) == 0
        assert_same((0,) + tuple(r1b), oracle.run(g1), g1.name)
    finally:
        h1.destroy()
        h2.destroy()


def test_heavy_stealing_keeps_looping_results_exact():
    """The condition-heavy graph (10,000 conditions, nested loops) with up to
    128 blocks stealing at once: every run that reports OK equals the oracle
    element by element (a looping task's final output was once left stale
    here), a run may report the race check's known false positive, and with
    the check off every run is OK and exact."""
    from paper_2004_10908_b300 import Executor, binding as B
    g = w.config3()
    ref = oracle.run(g)
    for flags in (0, B.TG_OPT_NO_RACE_CHECK):
        with Executor(arena_bytes=1 << 30, flags=flags) as e:
            h = e.graph(g)
            ok = 0
            for thieves in (64, 128):
                e.set_launch(max_thieves=thieves)
                for _ in range(6):
                    st = e.run(h)
                    assert st == B.TG_OK or (flags == 0 and st == B.TG_ERR_RACE), B.STATUS_NAMES[st]
                    if st == B.TG_OK:
                        ok += 1
                        assert_same((st,) + tuple(e.result(h)), ref, f"config3 thieves {thieves}")
            assert ok >= 6
            h.destroy()
