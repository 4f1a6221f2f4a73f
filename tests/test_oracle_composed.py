"""Composed graphs (module tasks) in the oracle, pinned: the paper's
composition example with its outputs recomputed from the pinned payload,
closed-form counts for modules in loops and nested modules, agreement with
the C oracle when no module task is present, and error propagation."""
import random

import numpy as np

import oracle
import workloads as w
from oracle import composed as oc
from workloads.graphs import COND_LOOP, MODULE, STATIC, from_lists, pack_param

R = 4


def test_paper_composition_example():
    """Composable Tasking example: taskflow1 = A -> B; taskflow2 = C -> D ->
    E, E composed of taskflow1 (D is a static task here: subflows are not
    part of this build)."""
    tf1 = from_lists("taskflow1", [STATIC, STATIC], pack_param([R, R]), [(0, 1)])
    tf2 = from_lists("taskflow2", [STATIC, STATIC, MODULE], pack_param([R, R, R]), [(0, 1), (1, 2)])
    res = oc.run({"tf1": tf1, "tf2": tf2}, {"tf2": {2: "tf1"}}, "tf2")
    st2, out2, cnt2, dig2, ex2 = res["tf2"]
    st1, out1, cnt1, dig1, ex1 = res["tf1"]
    assert st2 == oracle.OK and list(cnt2) == [1, 1, 1] and list(cnt1) == [1, 1]
    c = oracle.payload(0, 0, 0, R)
    d = oracle.payload(1, 0, c, R)
    e = oracle.payload(2, 0, d, R)
    a = oracle.payload(0, 0, e, R)      # the module's source receives E's output
    b = oracle.payload(1, 0, a, R)
    assert list(out2) == [c, d, e] and list(out1) == [a, b]
    assert list(dig1) == [oracle.mix32(a), oracle.mix32(b)]


def test_module_in_a_loop_runs_its_graph_each_time():
    """I -> E (module of a 3-chain) -> C (loop, trip T) -> weak [E, X]."""
    for T in (1, 2, 5, 9):
        body = from_lists("chain3", [STATIC] * 3, pack_param([R] * 3), [(0, 1), (1, 2)])
        top = from_lists("loop", [STATIC, MODULE, COND_LOOP, STATIC],
                         [pack_param(R), pack_param(R), pack_param(R, T), pack_param(R)],
                         [(0, 1), (1, 2), (2, 1), (2, 3)])
        res = oc.run({"b": body, "t": top}, {"t": {1: "b"}}, "t")
        st, out, cnt, dig, execs = res["t"]
        assert st == oracle.OK and list(cnt) == [1, T, T, 1]
        _, bout, bcnt, bdig, bexecs = res["b"]
        assert list(bcnt) == [T, T, T] and bexecs == 3 * T
        # last entry: the chain's input is E's output of its last execution
        e_last = out[1]
        x0 = oracle.payload(0, T - 1, e_last, R)
        x1 = oracle.payload(1, T - 1, x0, R)
        x2 = oracle.payload(2, T - 1, x1, R)
        assert list(bout) == [x0, x1, x2]


def test_nested_and_repeated_modules():
    """g3: S -> M1 (composes g2) -> M2 (composes g2 again) -> Z;
    g2: P -> N (composes g1) -> Q; g1: a diamond."""
    g1 = w.diamond(R)
    g2 = from_lists("g2", [STATIC, MODULE, STATIC], pack_param([R] * 3), [(0, 1), (1, 2)])
    g3 = from_lists("g3", [STATIC, MODULE, MODULE, STATIC], pack_param([R] * 4), [(0, 1), (1, 2), (2, 3)])
    res = oc.run({"g1": g1, "g2": g2, "g3": g3}, {"g3": {1: "g2", 2: "g2"}, "g2": {1: "g1"}}, "g3")
    assert res["g3"][0] == oracle.OK
    assert list(res["g3"][2]) == [1, 1, 1, 1]
    assert list(res["g2"][2]) == [2, 2, 2]
    assert list(res["g1"][2]) == [2, 2, 2, 2]
    assert res["g1"][4] == 8


def test_without_modules_equals_the_c_oracle():
    rnd = random.Random(3)
    graphs = [w.config1(levels=4, width=10, trip=3, rounds=8), w.do_while(7, 3)] + \
             [w.nested_loops(s) for s in range(10)] + \
             [w.config3(seed=3, n_cond=30, body_levels=3, body_width=4, rounds=4, trip_max=4)]
    for g in graphs:
        ref = oracle.run(g)
        st, out, cnt, dig, execs = oc.run({"g": g}, {}, "g")["g"]
        assert st == ref.status, g.name
        if st == oracle.OK:
            np.testing.assert_array_equal(cnt, ref.cnt, err_msg=g.name)
            np.testing.assert_array_equal(out, ref.out, err_msg=g.name)
            np.testing.assert_array_equal(dig, ref.dig, err_msg=g.name)
            assert execs == ref.execs


def test_errors_inside_a_module_end_the_run():
    racy = w.pitfall_race()
    top = from_lists("top", [STATIC, MODULE], pack_param([R, R]), [(0, 1)])
    assert oracle.run(racy).status == oracle.RACE
    assert oc.run({"r": racy, "t": top}, {"t": {1: "r"}}, "t")["t"][0] == oracle.RACE
    loop = w.do_while(50, 1)
    assert oc.run({"l": loop, "t": top}, {"t": {1: "l"}}, "t", exec_cap=40)["t"][0] == oracle.EXEC_LIMIT


def test_paper_subflow_example():
    """Dynamic Tasking example: A precedes B and C, D succeeds B and C; B
    spawns B1, B2 -> B3 (joined).  B's successors receive B's output plus
    the outputs of the subflow's sinks (here B3)."""
    from workloads.graphs import SUBFLOW
    sub = from_lists("B_subflow", [STATIC] * 3, pack_param([R] * 3), [(0, 2), (1, 2)])
    top = from_lists("fig", [STATIC, SUBFLOW, STATIC, STATIC], pack_param([R] * 4),
                     [(0, 1), (0, 2), (1, 3), (2, 3)])
    res = oc.run({"s": sub, "t": top}, {"t": {1: "s"}}, "t")
    st, out, cnt, dig, execs = res["t"]
    assert st == oracle.OK and list(cnt) == [1, 1, 1, 1]
    a = oracle.payload(0, 0, 0, R)
    b = oracle.payload(1, 0, a, R)
    b1 = oracle.payload(0, 0, b, R)
    b2 = oracle.payload(1, 0, b, R)
    b3 = oracle.payload(2, 0, (b1 + b2) & 0xFFFFFFFF, R)
    c = oracle.payload(2, 0, a, R)
    d = oracle.payload(3, 0, (b + b3 + c) & 0xFFFFFFFF, R)
    assert list(out) == [a, b, c, d]
    assert "s" not in res          # a subflow's copies are internal to their spawning task


def test_subflow_in_a_loop_is_fresh_each_time():
    """I -> S (subflow of a 2-chain) -> C (loop, trip T) -> weak [S, X]: every
    spawn starts the chain from iteration 0."""
    from workloads.graphs import SUBFLOW
    T = 4
    chain = from_lists("c2", [STATIC, STATIC], pack_param([R, R]), [(0, 1)])
    top = from_lists("loop", [STATIC, SUBFLOW, COND_LOOP, STATIC],
                     [pack_param(R), pack_param(R), pack_param(R, T), pack_param(R)],
                     [(0, 1), (1, 2), (2, 1), (2, 3)])
    res = oc.run({"c": chain, "t": top}, {"t": {1: "c"}}, "t")
    st, out, cnt, dig, execs = res["t"]
    assert st == oracle.OK and list(cnt) == [1, T, T, 1]
    i_out = oracle.payload(0, 0, 0, R)
    insum = i_out
    for k in range(T):
        s = oracle.payload(1, k, insum, R)
        c0 = oracle.payload(0, 0, s, R)          # fresh copy: iteration 0 every spawn
        c1 = oracle.payload(1, 0, c0, R)
        join = (s + c1) & 0xFFFFFFFF
        cond = oracle.payload(2, k, join, R)
        insum = cond                             # weak jump back to S carries C's output
    x = oracle.payload(3, 0, cond, R)
    assert out[1] == s and out[2] == cond and out[3] == x


def test_parallel_subflows_of_one_template_are_independent():
    """Two subflow tasks spawning one template get independent fresh copies:
    the same results as two identical but separate templates, and different
    from a module (whose one graph keeps its state between entries)."""
    from workloads.graphs import SUBFLOW
    tmpl = w.nested_loops(2)
    twin = w.nested_loops(2)
    par = from_lists("par", [STATIC, SUBFLOW, SUBFLOW, STATIC], pack_param([R] * 4),
                     [(0, 1), (0, 2), (1, 3), (2, 3)])
    shared = oc.run({"n": tmpl, "t": par}, {"t": {1: "n", 2: "n"}}, "t")["t"]
    separate = oc.run({"n": tmpl, "m": twin, "t": par}, {"t": {1: "n", 2: "m"}}, "t")["t"]
    assert shared[0] == oracle.OK
    for a, b in zip(shared[1:4], separate[1:4]):
        np.testing.assert_array_equal(a, b)
    seq = from_lists("seq", [STATIC, SUBFLOW, SUBFLOW, STATIC], pack_param([R] * 4),
                     [(0, 1), (1, 2), (2, 3)])
    as_sub = oc.run({"n": tmpl, "t": seq}, {"t": {1: "n", 2: "n"}}, "t")["t"]
    seq_mod = from_lists("seqm", [STATIC, MODULE, MODULE, STATIC], pack_param([R] * 4),
                         [(0, 1), (1, 2), (2, 3)])
    as_mod = oc.run({"n": tmpl, "t": seq_mod}, {"t": {1: "n", 2: "n"}}, "t")["t"]
    assert as_sub[0] == as_mod[0] == oracle.OK
    assert as_sub[1][3] != as_mod[1][3]    # join values differ from the module's plain output


def test_detached_subflow_releases_at_once_and_still_runs():
    """A detached subflow (Dynamic Tasking's detach): B's successors get B's
    own output, and the copy's executions still count in the run."""
    from workloads.graphs import SUBFLOW
    sub = from_lists("B_subflow", [STATIC] * 3, pack_param([R] * 3), [(0, 2), (1, 2)])
    det = from_lists("fig_det", [STATIC, SUBFLOW, STATIC, STATIC],
                     [pack_param(R), pack_param(R, 0, 1), pack_param(R), pack_param(R)],
                     [(0, 1), (0, 2), (1, 3), (2, 3)])
    res = oc.run({"s": sub, "t": det}, {"t": {1: "s"}}, "t")
    st, out, cnt, dig, execs = res["t"]
    assert st == oracle.OK and list(cnt) == [1, 1, 1, 1]
    a = oracle.payload(0, 0, 0, R)
    b = oracle.payload(1, 0, a, R)
    c = oracle.payload(2, 0, a, R)
    d = oracle.payload(3, 0, (b + c) & 0xFFFFFFFF, R)    # no join value
    assert list(out) == [a, b, c, d]
    assert res["*"] == 4 + 3
    joined = from_lists("fig", [STATIC, SUBFLOW, STATIC, STATIC], pack_param([R] * 4),
                        [(0, 1), (0, 2), (1, 3), (2, 3)])
    rj = oc.run({"s": sub, "t": joined}, {"t": {1: "s"}}, "t")
    assert rj["t"][1][3] != d and rj["*"] == 7
