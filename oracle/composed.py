"""ORACLE (test infrastructure): composed task graphs ("Composable Tasking":
a module task runs another task graph by reference), executed sequentially
in plain Python.  Only tests, the smoke check and the benchmark's
CPU-baseline leg use it; it shares nothing with the CUDA path.  The task
arithmetic (payload, mix, condition rule) is the oracle's, from tg_oracle.c.

Semantics, written out (the paper's module task, with the reading this
project takes where the paper is silent -- the paper's module runs the
composed taskflow to completion and only then lets the module's successors
proceed; it says nothing about data, so the module task's own output is what
flows).  Subflow tasks ("Dynamic Tasking", joined -- the default) follow
after the module rules:
  - a module task computes its payload like a static task (count, digest,
    output), then runs its composed graph to completion: that graph's
    sources are activated with the module task's output as their input sum,
    and the composed graph's tasks keep their counts, digests and outputs
    across entries within one run;
  - when the composed graph has nothing queued or running, the module task
    releases its own successors (strong edges) with its output;
  - an error inside a composed graph (race, execution cap) ends the whole
    run with that status;
  - every graph of the composition starts a run from its initial state;
  - a subflow task (kind 5) computes its payload, then spawns a fresh copy of
    its template graph (initial state, every time) whose sources take the
    task's output as their input sum, runs it to completion, and releases its
    own successors with its output plus the sum of the outputs of every
    execution of a static task without successors in that copy (the join
    value, mod 2^32); copies spawned by different tasks are independent;
  - a detached subflow task (bit 0 of its parameter word's top byte set)
    releases its successors at once with its own output; its copy runs on
    its own and the run ends only when the copy has ended too.  Nothing of
    the copy flows back, so running it to completion at the spawn gives the
    same results as any interleaving.

run() also reports, under the key "*", the executions of every graph of the
run, spawned copies included.

graphs: dict key -> workloads.Graph; modules: dict key -> {task: key of the
graph it composes, or of the template it spawns}; kinds use 4 for a module
task and 5 for a subflow task.
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import condition_index, mix32, payload, OK, RACE, EXEC_LIMIT, DEFAULT_EXEC_CAP

STATIC, COND_BRANCH, COND_LOOP, COND_CONST, MODULE, SUBFLOW = 0, 1, 2, 3, 4, 5


class _Failed(Exception):
    def __init__(self, status):
        self.status = status


class _State:
    def __init__(self, g):
        self.g = g
        n = g.n
        self.kinds = [int(k) for k in g.kinds]
        self.params = [int(p) for p in g.params]
        self.succ = [[] for _ in range(n)]
        self.sin = [0] * n
        win = [0] * n
        for s, d in zip(g.src.tolist(), g.dst.tolist()):   # insertion order
            self.succ[s].append(d)
            if self.kinds[s] in (STATIC, MODULE, SUBFLOW):
                self.sin[d] += 1
            else:
                win[d] += 1
        self.sources = [v for v in range(n) if self.sin[v] == 0 and win[v] == 0]
        self.w_cnt = list(self.sin)
        self.w_sum = [0] * n
        self.cnt = [0] * n
        self.out = [0] * n
        self.dig = [0] * n
        self.queued = [False] * n
        self.execs = 0


def run(graphs, modules, root, exec_cap=DEFAULT_EXEC_CAP):
    """Returns {key: (status, out, cnt, dig, execs)} for every graph of the
    composition reachable from `root` (status is the run's status)."""
    states = {}
    copies = []

    def state(key):
        if key not in states:
            states[key] = _State(graphs[key])
        return states[key]

    def run_graph(key, source_insum, st=None):
        """Run a graph to completion; returns the sum of its sink outputs."""
        st = st or state(key)
        sink_sum = 0
        q = deque()

        def push(v, s):
            if st.queued[v]:
                raise _Failed(RACE)
            st.queued[v] = True
            q.append((v, s))

        for v in st.sources:
            push(v, source_insum)
        while q:
            v, s = q.popleft()
            st.queued[v] = False
            it = st.cnt[v]
            x = payload(v, it, s, st.params[v] & 0xFFFF)
            st.out[v] = x
            st.cnt[v] += 1
            st.dig[v] = mix32(st.dig[v] ^ x)
            st.execs += 1
            if st.execs > exec_cap:
                raise _Failed(EXEC_LIMIT)
            kind = st.kinds[v]
            if kind == STATIC and not st.succ[v]:
                sink_sum = (sink_sum + x) & 0xFFFFFFFF
            if kind in (COND_BRANCH, COND_LOOP, COND_CONST):
                r = condition_index(kind, st.params[v], int(st.g.seed), v, it, len(st.succ[v]))
                if 0 <= r < len(st.succ[v]):
                    push(st.succ[v][r], x)
                continue
            if kind == MODULE:
                run_graph(modules[key][v], x)   # the composed graph runs to completion first
            elif kind == SUBFLOW:
                tmpl = modules[key][v]         # a fresh copy of the template
                copy = _State(graphs[tmpl])
                copies.append(copy)
                copy_sum = run_graph(tmpl, x, copy)
                if not (st.params[v] >> 24) & 1:   # joined: the join value flows on
                    x = (x + copy_sum) & 0xFFFFFFFF
            for u in st.succ[v]:
                st.w_sum[u] = (st.w_sum[u] + x) & 0xFFFFFFFF
                st.w_cnt[u] -= 1
                if st.w_cnt[u] == 0:
                    s2 = st.w_sum[u]
                    st.w_cnt[u] = st.sin[u]
                    st.w_sum[u] = 0
                    push(u, s2)
        return sink_sum

    status = OK
    try:
        run_graph(root, 0)
    except _Failed as f:
        status = f.status
    res = {}
    for key, st in states.items():
        res[key] = (status, np.array(st.out, np.uint32), np.array(st.cnt, np.uint32),
                    np.array(st.dig, np.uint32), st.execs)
    res["*"] = sum(st.execs for st in states.values()) + sum(c.execs for c in copies)
    return res
