"""Reading per-task trace records (TG_OPT_TRACE_TASKS) along a graph's
critical path.

tg_trace_copy gives, for each task's last execution, when a warp took it
from a queue, when that warp's step ended (before the step's new
activations were published), and where it was taken from.  In an acyclic
graph every task runs once, so these records describe the whole run.
Following, back from the task whose step ended last, each task's
predecessor whose step ended last gives the chain of hand-offs that set the
run's length.  Each hop of it splits into a wait (the predecessor's step end
to this task being taken: publication, time in a queue, the taking) and a
step (taken to step end: record read, payload, release).
"""
from __future__ import annotations

import numpy as np

FROM_NAMES = ("hand", "ring", "own_deque", "steal", "injection")


def _pct(a, p):
    return float(np.percentile(a, p)) / 1e3 if len(a) else None


def critical_path(src, dst, start_ns, end_ns, where) -> dict:
    """Critical-path summary of one traced run of an acyclic graph.

    src, dst    its strong edges (task indices)
    start_ns, end_ns, where   tg_trace_copy's three arrays
    Times are reported in microseconds."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    st = np.asarray(start_ns, np.int64)
    en = np.asarray(end_ns, np.int64)
    wh = np.asarray(where, np.uint32)
    n = len(st)
    if n == 0 or (st == 0).any() or (en < st).any():
        raise ValueError("every task must have run once, with its step ending after it was taken")
    frm = (wh >> 16).astype(np.int64)
    blk = (wh & 0xFFFF).astype(np.int64)
    # each task's predecessor whose step ended last (ties: the later edge)
    last = np.full(n, -1, np.int64)
    order = np.argsort(en[src], kind="stable")
    last[dst[order]] = src[order]
    path = []
    t = int(np.argmax(en))
    while t >= 0 and len(path) <= n:
        path.append(t)
        t = int(last[t])
    path = np.array(path[::-1], np.int64)
    a, b = path[:-1], path[1:]
    wait = (st[b] - en[a]).astype(np.float64)
    step = (en[path] - st[path]).astype(np.float64)
    by = {}
    for c, name in enumerate(FROM_NAMES):
        m = frm[b] == c
        if m.any():
            by[name] = {"hops": int(m.sum()), "wait_p50_us": _pct(wait[m], 50), "wait_p90_us": _pct(wait[m], 90),
                        "same_block": int((m & (blk[b] == blk[a])).sum())}
    return {
        "tasks": int(len(path)),
        "span_ms": float(en[path[-1]] - st[path[0]]) / 1e6,
        "step_mean_us": float(step.mean()) / 1e3,
        "wait_mean_us": float(wait.mean()) / 1e3 if len(wait) else 0.0,
        "hops_by_source": by,
        "all_tasks_by_source": {name: int((frm == c).sum()) for c, name in enumerate(FROM_NAMES)},
    }
