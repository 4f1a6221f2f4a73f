"""Algorithm 1 (capturer -> CUDA graph): the levelizer and round-robin
stream plan.  The oracle is pinned to the paper's worked example and to
brute-force longest paths; the library's host-only entry points
(tg_levelize, tg_stream_plan) must equal it exactly."""
import os
import random


from oracle import capturer as cap

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "capturer_example.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, val = line.split(":", 1)
        out[key] = val.strip()
    pairs = lambda s: [tuple(int(x) for x in p.split()) for p in s.split(",")]
    return (pairs(out["edges"]), int(out["max_streams"]), [int(x) for x in out["index"].split()],
            set(pairs(out["cross"])))


def _random_dag(rnd, n, p_edge, dup=False):
    perm = list(range(n))
    rnd.shuffle(perm)
    edges = [(perm[a], perm[b]) for a in range(n) for b in range(a + 1, n) if rnd.random() < p_edge]
    if dup and edges:
        edges += rnd.sample(edges, min(3, len(edges)))
    rnd.shuffle(edges)
    return edges


def _longest_paths(n, edges):
    """Brute force: the most edges on any path ending at v, by walking every path."""
    succ = [[] for _ in range(n)]
    for p, t in edges:
        succ[p].append(t)
    best = [0] * n
    has_pred = {t for _, t in edges}

    def walk(v, depth):
        best[v] = max(best[v], depth)
        for t in succ[v]:
            walk(t, depth + 1)
    for v in range(n):
        if v not in has_pred:
            walk(v, 0)
    return best


def test_oracle_paper_example():
    edges, k, index, cross = _golden()
    level, idx, nl = cap.levels(5, edges)
    assert level == [0, 0, 1, 1, 1] and nl == 2
    assert idx == index
    stream, n_events, n_waits, got = cap.stream_plan(5, edges, k)
    assert got == cross and n_waits == 2 and n_events == 2
    assert stream == [0, 1, 0, 1, 0]


def test_oracle_levels_are_longest_paths():
    rnd = random.Random(11)
    for trial in range(400):
        n = rnd.randint(1, 8)
        edges = _random_dag(rnd, n, rnd.random() * 0.6)
        level, index, nl = cap.levels(n, edges)
        assert level == _longest_paths(n, edges)
        # ids: a bijection onto 0..size-1 per level, ascending with the task id
        for lv in range(nl):
            members = [v for v in range(n) if level[v] == lv]
            assert [index[v] for v in members] == list(range(len(members)))


def test_oracle_rejects_cycles():
    assert cap.levels(3, [(0, 1), (1, 2), (2, 0)]) is None
    assert cap.levels(2, [(0, 0), (0, 1)]) is None
    assert cap.stream_plan(2, [(1, 0), (0, 1)], 2) is None


def test_one_stream_needs_no_events_and_wide_levels_need_many():
    edges = [(0, t) for t in range(1, 9)] + [(t, 9) for t in range(1, 9)]
    _, n_events, n_waits, _ = cap.stream_plan(10, edges, 1)
    assert n_events == 0 and n_waits == 0
    stream, n_events, n_waits, cross = cap.stream_plan(10, edges, 4)
    # level 1 holds tasks 1..8 with ids 0..7: streams 0,1,2,3,0,1,2,3
    assert [stream[t] for t in range(1, 9)] == [0, 1, 2, 3, 0, 1, 2, 3]
    assert cross == {(0, t) for t in range(1, 9) if stream[t] != 0} | {(t, 9) for t in range(1, 9) if stream[t] != 0}
    assert n_waits == len(cross)


def test_library_levelize_and_stream_plan_equal_oracle():
    import numpy as np
    from paper_2004_10908_b300 import binding as B
    rnd = random.Random(5)
    for trial in range(300):
        n = rnd.randint(1, 120)
        edges = _random_dag(rnd, n, rnd.random() * 0.1, dup=trial % 3 == 0)
        src = np.array([p for p, _ in edges], np.uint32)
        dst = np.array([t for _, t in edges], np.uint32)
        st, level, index, nl = B.tg_levelize(n, src, dst)
        ref = cap.levels(n, edges)
        assert st == 0
        assert list(level) == ref[0] and list(index) == ref[1] and nl == ref[2]
        for k in (1, 2, 3, 32):
            st, stream, ne, nw = B.tg_stream_plan(n, src, dst, k)
            rs, rne, rnw, _ = cap.stream_plan(n, edges, k)
            assert st == 0 and list(stream) == rs and (ne, nw) == (rne, rnw)
    cyc = np.array([0, 1, 2], np.uint32), np.array([1, 2, 0], np.uint32)
    assert B.tg_levelize(3, *cyc)[0] == B.TG_ERR_INVALID
    assert B.tg_stream_plan(3, *cyc, 2)[0] == B.TG_ERR_INVALID
    assert B.tg_stream_plan(3, np.array([0], np.uint32), np.array([1], np.uint32), 33)[0] == B.TG_ERR_INVALID
    assert B.tg_levelize(2, np.array([0], np.uint32), np.array([5], np.uint32))[0] == B.TG_ERR_INVALID
