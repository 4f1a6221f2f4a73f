"""Reading per-task trace records (TG_OPT_TRACE_TASKS) along a graph's
critical path, step by step, and level by level.

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


def _steps(start_ns, end_ns, where):
    """The warp steps of a traced run: tasks sharing a block, a take time and
    a step end.  Returns (block, take, end, tasks) per step and, per step,
    how many steps of its block ran at its midpoint (itself included)."""
    st = np.asarray(start_ns, np.int64)
    en = np.asarray(end_ns, np.int64)
    blk = (np.asarray(where, np.uint32) & 0xFFFF).astype(np.int64)
    key = np.stack([blk, st, en], 1)
    uk, cnt = np.unique(key, axis=0, return_counts=True)
    sb, ss, se = uk[:, 0], uk[:, 1], uk[:, 2]
    conc = np.zeros(len(uk), np.int64)
    for b in np.unique(sb):
        i = np.nonzero(sb == b)[0]
        mid = (ss[i] + se[i]) // 2
        conc[i] = np.searchsorted(np.sort(ss[i]), mid, "right") - np.searchsorted(np.sort(se[i]), mid, "right")
    return sb, ss, se, cnt, conc


def step_summary(start_ns, end_ns, where) -> dict:
    """Step durations (microseconds) by the number of tasks in the step and
    by the number of steps of the same block running at once."""
    sb, ss, se, cnt, conc = _steps(start_ns, end_ns, where)
    dur = (se - ss).astype(np.float64)
    by_size = {}
    for lo, hi in ((1, 1), (2, 4), (5, 9), (10, 16), (17, 24), (25, 32)):
        m = (cnt >= lo) & (cnt <= hi)
        if m.any():
            by_size[f"{lo}-{hi}" if hi > lo else f"{lo}"] = {"steps": int(m.sum()), "dur_p50_us": _pct(dur[m], 50)}
    by_conc = {}
    for c in np.unique(conc):
        m = conc == c
        if m.sum() >= 50:
            by_conc[int(c)] = {"steps": int(m.sum()), "dur_p50_us": _pct(dur[m], 50),
                               "tasks_mean": float(cnt[m].mean())}
    return {"steps": int(len(cnt)), "tasks_per_step_mean": float(cnt.mean()), "dur_p50_us": _pct(dur, 50),
            "by_tasks_in_step": by_size, "by_block_steps_at_once": by_conc}


def level_summary(level, src, dst, start_ns, end_ns, where) -> dict:
    """A levelled graph (level[task], levels numbered from 0) read level by
    level: when each level completed, how many blocks ran it, the largest
    share one block took, where each level's last-ending task came from, and
    the wait from ready (the last predecessor's step end; a source: taken at
    once) to taken, by source.  Times in microseconds."""
    level = np.asarray(level, np.int64)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    st = np.asarray(start_ns, np.int64)
    en = np.asarray(end_ns, np.int64)
    wh = np.asarray(where, np.uint32)
    frm = (wh >> 16).astype(np.int64)
    blk = (wh & 0xFFFF).astype(np.int64)
    n = len(st)
    ready = st.copy()
    has_pred = np.zeros(n, bool)
    has_pred[dst] = True
    ready[has_pred] = 0
    np.maximum.at(ready, dst, en[src])
    wait = (st - ready).astype(np.float64)
    nl = int(level.max()) + 1
    order = np.argsort(level, kind="stable")
    bounds = np.searchsorted(level[order], np.arange(nl + 1))
    lend = np.empty(nl, np.int64)
    nblk = np.empty(nl, np.int64)
    top = np.empty(nl, np.int64)
    last_src = np.empty(nl, np.int64)
    for l in range(nl):
        i = order[bounds[l]:bounds[l + 1]]
        lend[l] = en[i].max()
        nblk[l] = len(np.unique(blk[i]))
        top[l] = np.bincount(blk[i]).max()
        last_src[l] = frm[i[np.argmax(en[i])]]
    gap = np.diff(lend).astype(np.float64)
    return {
        "levels": nl,
        "level_gap_us": {"mean": float(gap.mean()) / 1e3 if len(gap) else 0.0, "p50": _pct(gap, 50),
                         "p90": _pct(gap, 90)},
        "blocks_per_level": {"mean": float(nblk.mean()), "p10": float(np.percentile(nblk, 10)),
                             "p90": float(np.percentile(nblk, 90))},
        "largest_block_share": {"mean": float(top.mean()), "p90": float(np.percentile(top, 90))},
        "last_task_of_level_from": {name: int((last_src == c).sum()) for c, name in enumerate(FROM_NAMES)},
        "wait_ready_to_taken_by_source": {name: {"tasks": int((frm == c).sum()), "p50_us": _pct(wait[frm == c], 50),
                                                 "p90_us": _pct(wait[frm == c], 90)}
                                          for c, name in enumerate(FROM_NAMES) if (frm == c).any()},
    }
