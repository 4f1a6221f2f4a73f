"""ORACLE (test infrastructure): Algorithm 1 of the paper (transforming a
capturer graph into a CUDA graph over round-robin streams), written out
plainly in Python.  Only tests, the smoke check and the benchmark's
CPU-baseline leg use it; it shares nothing with the CUDA path.

levels(n, edges)
    Levelize by a topological traversal: a task without predecessors is on
    level 0, any other task one level below its deepest predecessor; each
    task's id is its position on its level (Algorithm 1, "levelize"; the
    text's example numbers A, B as 0, 1 and C, D, E as 0, 1, 2, i.e. in
    order on the level, taken here as ascending task id).
stream_plan(n, edges, max_streams)
    stream = id mod max_streams (Algorithm 1, the modulo line); a task
    records an event when one of its successors is on another stream, and a
    task waits once on each predecessor that is on another stream.
"""
from __future__ import annotations


def levels(n, edges):
    """Returns (level, index, n_levels), or None when the graph has a cycle."""
    preds = [[] for _ in range(n)]
    succs = [[] for _ in range(n)]
    for p, t in edges:
        preds[t].append(p)
        succs[p].append(t)
    # topological order by repeatedly taking tasks whose predecessors are all placed
    remaining = [len(preds[v]) for v in range(n)]
    order = [v for v in range(n) if remaining[v] == 0]
    i = 0
    while i < len(order):
        v = order[i]
        i += 1
        for t in succs[v]:
            remaining[t] -= 1
            if remaining[t] == 0:
                order.append(t)
    if len(order) != n:
        return None
    level = [0] * n
    for v in order:
        if preds[v]:
            level[v] = 1 + max(level[p] for p in preds[v])
    n_levels = max(level) + 1 if n else 0
    index = [0] * n
    for lv in range(n_levels):
        on_level = sorted(v for v in range(n) if level[v] == lv)
        for k, v in enumerate(on_level):
            index[v] = k
    return level, index, n_levels


def stream_plan(n, edges, max_streams):
    """Returns (stream, n_events, n_waits, cross) with cross the set of
    (predecessor, task) pairs on different streams, or None on a cycle."""
    lv = levels(n, edges)
    if lv is None:
        return None
    _, index, _ = lv
    stream = [index[v] % max_streams for v in range(n)]
    cross = {(p, t) for p, t in edges if stream[p] != stream[t]}
    n_events = len({p for p, _ in cross})
    return stream, n_events, len(cross), cross
