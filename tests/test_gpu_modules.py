"""Module tasks (Composable Tasking) and joined subflows (Dynamic Tasking) on
the device: every graph of a composition ends with the composed oracle's
outputs, counts and digests, bit for bit; misuse is refused."""
import numpy as np
import pytest

import oracle
import workloads as w
from oracle import composed as oc
from workloads.graphs import COND_LOOP, MODULE, STATIC, SUBFLOW, from_lists, pack_param

pytestmark = pytest.mark.gpu
R = 4


@pytest.fixture(scope="module")
def ex():
    from paper_2004_10908_b300 import Executor
    e = Executor(arena_bytes=1 << 30)
    yield e
    e.close()


def _run_composed(ex, graphs, modules, root, order):
    """Create the graphs bottom-up (`order`), run the root, compare all."""
    handles = {}
    for key in order:
        mods = {v: handles[k] for v, k in modules.get(key, {}).items()}
        handles[key] = ex.graph(graphs[key], modules=mods if mods else None)
    st = ex.run(handles[root])
    ref = oc.run(graphs, modules, root)
    for key in order:
        if key not in ref:
            continue        # a subflow template: its copies are internal to their tasks
        out, cnt, dig, execs = ex.result(handles[key])
        rst, rout, rcnt, rdig, rexecs = ref[key]
        if key == root:
            assert st == rst, (key, st, rst)
        if rst == oracle.OK:
            np.testing.assert_array_equal(cnt, rcnt, err_msg=f"{key}: cnt")
            np.testing.assert_array_equal(out, rout, err_msg=f"{key}: out")
            np.testing.assert_array_equal(dig, rdig, err_msg=f"{key}: dig")
            assert execs == rexecs, key
    return st, handles


def _destroy(handles, order):
    for key in reversed(order):
        handles[key].destroy()


def test_paper_composition_example(ex):
    tf1 = from_lists("taskflow1", [STATIC, STATIC], pack_param([R, R]), [(0, 1)])
    tf2 = from_lists("taskflow2", [STATIC, STATIC, MODULE], pack_param([R, R, R]), [(0, 1), (1, 2)])
    st, h = _run_composed(ex, {"tf1": tf1, "tf2": tf2}, {"tf2": {2: "tf1"}}, "tf2", ["tf1", "tf2"])
    assert st == 0
    _destroy(h, ["tf1", "tf2"])


@pytest.mark.parametrize("T", [1, 2, 5, 9])
def test_module_in_a_loop(ex, T):
    body = w.config2a(seed=7, levels=5, width=70, rounds=6)       # 70 sources: several warp rounds
    top = from_lists("loop", [STATIC, MODULE, COND_LOOP, STATIC],
                     [pack_param(R), pack_param(R), pack_param(R, T), pack_param(R)],
                     [(0, 1), (1, 2), (2, 1), (2, 3)])
    st, h = _run_composed(ex, {"b": body, "t": top}, {"t": {1: "b"}}, "t", ["b", "t"])
    assert st == 0
    _destroy(h, ["b", "t"])


def test_nested_repeated_and_conditional_modules(ex):
    g1 = w.nested_loops(3)
    g2 = from_lists("g2", [STATIC, MODULE, STATIC], pack_param([R] * 3), [(0, 1), (1, 2)])
    g3 = from_lists("g3", [STATIC, MODULE, MODULE, STATIC, STATIC], pack_param([R] * 5),
                    [(0, 1), (1, 2), (2, 3), (0, 4), (4, 3)])
    graphs = {"g1": g1, "g2": g2, "g3": g3}
    mods = {"g3": {1: "g2", 2: "g2"}, "g2": {1: "g1"}}
    for _ in range(3):          # repeated launches start every graph afresh
        st, h = _run_composed(ex, graphs, mods, "g3", ["g1", "g2", "g3"])
        assert st == 0
        _destroy(h, ["g1", "g2", "g3"])


def test_concurrent_use_is_a_race_or_a_schedule(ex):
    """Two module tasks with no order between them compose one graph: the
    run ends RACE, or (if they did not overlap) with the oracle's result."""
    g1 = w.do_while(40, 16)
    top = from_lists("par", [STATIC, MODULE, MODULE, STATIC], pack_param([R] * 4),
                     [(0, 1), (0, 2), (1, 3), (2, 3)])
    from paper_2004_10908_b300 import binding as B
    seen = set()
    for _ in range(10):
        h1 = ex.graph(g1)
        ht = ex.graph(top, modules={1: h1, 2: h1})
        st = ex.run(ht)
        seen.add(st)
        if st == 0:
            ref = oc.run({"g": g1, "t": top}, {"t": {1: "g", 2: "g"}}, "t")
            np.testing.assert_array_equal(ex.result(ht)[1], ref["t"][2])
        else:
            assert st == B.TG_ERR_RACE
        ht.destroy()
        h1.destroy()
    assert seen <= {0, B.TG_ERR_RACE}


def test_errors_inside_a_module_reach_the_caller():
    from paper_2004_10908_b300 import Executor, binding as B
    with Executor(arena_bytes=1 << 28, exec_cap=40) as e:
        loop = w.do_while(50, 1)
        top = from_lists("top", [STATIC, MODULE, STATIC], pack_param([R] * 3), [(0, 1), (1, 2)])
        hl = e.graph(loop)
        ht = e.graph(top, modules={1: hl})
        assert e.run(ht) == B.TG_ERR_EXEC_LIMIT
        assert oc.run({"l": loop, "t": top}, {"t": {1: "l"}}, "t", exec_cap=40)["t"][0] == oracle.EXEC_LIMIT
        # the context stays usable: the composed graph alone, then the composition again
        assert e.run(hl) == B.TG_ERR_EXEC_LIMIT
        ht.destroy()
        hl.destroy()


def test_refusals_and_standalone_use(ex):
    from paper_2004_10908_b300 import binding as B
    g1 = w.diamond()
    top = from_lists("top", [STATIC, MODULE], pack_param([R, R]), [(0, 1)])
    h1 = ex.graph(g1)
    ht = ex.graph(top, modules={1: h1})
    assert B.tg_instance_create(ex.ctx, ht.handle)[0] == B.TG_ERR_INVALID
    assert ex.capture_run(ht, 2)[0] == B.TG_ERR_INVALID
    assert B.tg_graph_destroy(ex.ctx, h1.handle) == B.TG_ERR_BUSY        # still composed
    # module task without a graph, a graph for a static task
    assert B.tg_graph_create_composed(ex.ctx, top.kinds, top.params, top.src, top.dst, {})[0] == B.TG_ERR_INVALID
    assert B.tg_graph_create_composed(ex.ctx, top.kinds, top.params, top.src, top.dst,
                                      {0: h1.handle, 1: h1.handle})[0] == B.TG_ERR_INVALID
    assert B.tg_graph_create(ex.ctx, top.kinds, top.params, top.src, top.dst)[0] == B.TG_ERR_INVALID
    # the composed graph runs alone like any graph
    assert ex.run(ht) == 0
    assert ex.run(h1) == 0
    ref = oracle.run(g1)
    np.testing.assert_array_equal(ex.result(h1)[0], ref.out)
    ht.destroy()
    assert B.tg_graph_destroy(ex.ctx, h1.handle) == 0
    h1.handle = None


def test_paper_subflow_example(ex):
    sub = from_lists("B_subflow", [STATIC] * 3, pack_param([R] * 3), [(0, 2), (1, 2)])
    top = from_lists("fig", [STATIC, SUBFLOW, STATIC, STATIC], pack_param([R] * 4),
                     [(0, 1), (0, 2), (1, 3), (2, 3)])
    st, h = _run_composed(ex, {"s": sub, "t": top}, {"t": {1: "s"}}, "t", ["s", "t"])
    assert st == 0
    _destroy(h, ["s", "t"])


@pytest.mark.parametrize("T", [1, 3, 7])
def test_subflow_in_a_loop(ex, T):
    tmpl = w.config2a(seed=11, levels=4, width=50, rounds=5)       # 50 sources, many sinks
    top = from_lists("loop", [STATIC, SUBFLOW, COND_LOOP, STATIC],
                     [pack_param(R), pack_param(R), pack_param(R, T), pack_param(R)],
                     [(0, 1), (1, 2), (2, 1), (2, 3)])
    st, h = _run_composed(ex, {"s": tmpl, "t": top}, {"t": {1: "s"}}, "t", ["s", "t"])
    assert st == 0
    _destroy(h, ["s", "t"])


def test_parallel_subflows_modules_and_conditional_templates(ex):
    """Four subflow tasks (two templates, one with nested loops) run side by
    side with a module task; repeated launches start afresh."""
    loops = w.nested_loops(4)
    dag = w.config2a(seed=12, levels=3, width=40, rounds=3)
    modg = w.diamond(R)
    top = from_lists("mix", [STATIC, SUBFLOW, SUBFLOW, SUBFLOW, SUBFLOW, MODULE, STATIC],
                     pack_param([R] * 7),
                     [(0, 1), (0, 2), (0, 3), (0, 4), (0, 5), (1, 6), (2, 6), (3, 6), (4, 6), (5, 6)])
    graphs = {"loops": loops, "dag": dag, "mod": modg, "t": top}
    mods = {"t": {1: "loops", 2: "loops", 3: "dag", 4: "dag", 5: "mod"}}
    for _ in range(3):
        st, h = _run_composed(ex, graphs, mods, "t", ["loops", "dag", "mod", "t"])
        assert st == 0
        _destroy(h, ["loops", "dag", "mod", "t"])


def test_subflow_refusals(ex):
    from paper_2004_10908_b300 import binding as B
    inner = w.diamond()
    hi = ex.graph(inner)
    comp = ex.graph(from_lists("c", [STATIC, MODULE], pack_param([R, R]), [(0, 1)]), modules={1: hi})
    top = from_lists("t", [STATIC, SUBFLOW], pack_param([R, R]), [(0, 1)])
    # a template holds no module or subflow tasks
    assert B.tg_graph_create_composed(ex.ctx, top.kinds, top.params, top.src, top.dst,
                                      {1: comp.handle})[0] == B.TG_ERR_INVALID
    ht = ex.graph(top, modules={1: hi})
    assert B.tg_graph_destroy(ex.ctx, hi.handle) == B.TG_ERR_BUSY      # its copy exists
    assert ex.run(ht) == 0
    ht.destroy()
    comp.destroy()
    assert B.tg_graph_destroy(ex.ctx, hi.handle) == 0
    hi.handle = None


def test_composed_graphs_in_a_batch(ex):
    """A batch of composed graphs -- module loops, parallel subflows, plain
    members -- in one captured launch, replayed: every member and every
    composed graph ends with the composed oracle's results."""
    mods = [w.diamond(R), w.nested_loops(5)]
    tmpl = w.config2a(seed=13, levels=3, width=20, rounds=4)
    hm = [ex.graph(g) for g in mods]
    ht = ex.graph(tmpl)
    members, refs = [], []
    for i in range(6):
        T = 2 + i
        loop = from_lists(f"loop{i}", [STATIC, MODULE, COND_LOOP, STATIC],
                          [pack_param(R), pack_param(R), pack_param(R, T), pack_param(R)],
                          [(0, 1), (1, 2), (2, 1), (2, 3)])
        fan = from_lists(f"fan{i}", [STATIC, SUBFLOW, SUBFLOW, STATIC], pack_param([R] * 4),
                         [(0, 1), (0, 2), (1, 3), (2, 3)])
        # each loop member composes its own graph (no two members share one)
        mg = ex.graph(mods[i % 2]) if i >= 2 else hm[i]
        members.append((ex.graph(loop, modules={1: mg}), loop, {"m": mods[i % 2], "t": loop}, {"t": {1: "m"}}, mg))
        members.append((ex.graph(fan, modules={1: ht, 2: ht}), fan, {"s": tmpl, "t": fan}, {"t": {1: "s", 2: "s"}}, None))
    plain = w.config1(levels=3, width=20, trip=2, rounds=8)
    hp = ex.graph(plain)
    b = ex.batch([m[0] for m in members] + [hp])
    for _ in range(2):
        b.launch()
        st, sts = b.wait()
        assert st == 0 and (sts == 0).all()
        for h, top, graphs, mmap, mg in members:
            ref = oc.run(graphs, mmap, "t")
            out, cnt, dig, execs = ex.result(h)
            np.testing.assert_array_equal(cnt, ref["t"][2], err_msg=top.name)
            np.testing.assert_array_equal(out, ref["t"][1], err_msg=top.name)
            np.testing.assert_array_equal(dig, ref["t"][3], err_msg=top.name)
            if mg is not None:
                mout, mcnt, mdig, _ = ex.result(mg)
                np.testing.assert_array_equal(mcnt, ref["m"][2], err_msg=top.name + " module")
                np.testing.assert_array_equal(mout, ref["m"][1], err_msg=top.name + " module")
        pref = oracle.run(plain)
        np.testing.assert_array_equal(ex.result(hp)[1], pref.cnt)
    b.destroy()
    for h, _, _, _, mg in members:
        h.destroy()
    for h, _, _, _, mg in members:
        if mg is not None and mg not in hm:
            mg.destroy()
    hp.destroy()
    ht.destroy()
    for h in hm:
        h.destroy()


def test_detached_subflows(ex):
    """Detached subflows: successors released at once with the task's output;
    the launch still waits for every copy (the execution counter includes
    them); inside a composed graph the module task resumes only after the
    detached copies of that graph ended; in a batch too."""
    sub = from_lists("B_subflow", [STATIC] * 3, pack_param([R] * 3), [(0, 2), (1, 2)])
    big = w.config2a(seed=17, levels=6, width=80, rounds=40)
    det = from_lists("fig_det", [STATIC, SUBFLOW, SUBFLOW, STATIC],
                     [pack_param(R), pack_param(R, 0, 1), pack_param(R, 0, 1), pack_param(R)],
                     [(0, 1), (0, 2), (1, 3), (2, 3)])
    hs, hb = ex.graph(sub), ex.graph(big)
    ht = ex.graph(det, modules={1: hs, 2: hb})
    for _ in range(3):
        st = ex.run(ht)
        ref = oc.run({"s": sub, "b": big, "t": det}, {"t": {1: "s", 2: "b"}}, "t")
        assert st == 0 == ref["t"][0]
        out, cnt, dig, execs = ex.result(ht)
        np.testing.assert_array_equal(out, ref["t"][1])
        np.testing.assert_array_equal(cnt, ref["t"][2])
        assert ex.stats()["tasks"] == ref["*"]
    # a module whose graph holds a detached subflow: the module task resumes
    # only once that copy is done too
    top = from_lists("outer", [STATIC, MODULE, STATIC], pack_param([R] * 3), [(0, 1), (1, 2)])
    ho = ex.graph(top, modules={1: ht})
    assert ex.run(ho) == 0
    ref = oc.run({"s": sub, "b": big, "t": det, "o": top}, {"o": {1: "t"}, "t": {1: "s", 2: "b"}}, "o")
    np.testing.assert_array_equal(ex.result(ho)[0], ref["o"][1])
    assert ex.stats()["tasks"] == ref["*"]
    # in a batch, beside a plain graph
    plain = w.config1(levels=3, width=20, trip=2, rounds=8)
    hp = ex.graph(plain)
    b = ex.batch([ho, hp])
    b.launch()
    st, sts = b.wait()
    assert st == 0
    np.testing.assert_array_equal(ex.result(ho)[0], ref["o"][1])
    assert ex.stats()["tasks"] == ref["*"] + oracle.run(plain).execs
    b.destroy()
    hp.destroy()
    ho.destroy()
    ht.destroy()
    hs.destroy()
    hb.destroy()
