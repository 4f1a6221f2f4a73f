"""Independent evaluators that pin the oracle to something other than itself.

None of these walks the oracle's FIFO/join-counter machinery.  Each is a
different route to the result the paper's rules fix:

  * definitional_dag     -- for a DAG of static tasks every task runs once and
                            out(v) = P(v, 0, sum of strong predecessors' outputs);
                            evaluated by memoised recursion over predecessors.
  * unrolled_config1     -- the loop of the config-1 graph written as a plain
                            `for t in range(T)` program over the body.
  * structured_lane      -- one config-3 lane written as three nested loops with
                            an explicit arm choice (the control flow the lane's
                            condition tasks encode).
  * motif_counts         -- closed-form execution counts of a motif graph.
  * brute_force          -- every interleaving of the ready activations of a tiny
                            graph (a nondeterministic reading of the rules).

The payload and condition hash enter as library primitives from the oracle.
"""
from __future__ import annotations

import sys
from collections import defaultdict

import numpy as np

import oracle
from workloads import STATIC, COND_LOOP


def mix32_inverse(y: int) -> int:
    """Inverse of the lowbias32 mixer, derived from its published shifts and
    multipliers: undo x ^= x >> k by fixed-point iteration and the odd
    multiplications by their inverses modulo 2^32."""
    M = 0xFFFFFFFF

    def unxorshift(v, k):
        x = v
        for _ in range(32 // k + 1):
            x = v ^ (x >> k)
        return x & M

    y &= M
    y = unxorshift(y, 16)
    y = (y * pow(0x846CA68B, -1, 1 << 32)) & M
    y = unxorshift(y, 15)
    y = (y * pow(0x7FEB352D, -1, 1 << 32)) & M
    y = unxorshift(y, 16)
    return y


def _rounds(g, v):
    return int(g.params[v]) & 0xFFFF


def strong_preds(g):
    preds = defaultdict(list)
    for s, d in zip(g.src.tolist(), g.dst.tolist()):
        if g.kinds[s] == STATIC:
            preds[d].append(s)
    return preds


def definitional_dag(g):
    """out(v) = P(v, 0, sum_{p strong pred of v} out(p)) by memoised recursion;
    cnt = 1 and dig = mix32(out) for every task (one execution each)."""
    preds = strong_preds(g)
    memo = {}
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10 * g.n + 1000))

    def out(v):
        if v in memo:
            return memo[v]
        s = 0
        for p in preds.get(v, ()):
            s = (s + out(p)) & 0xFFFFFFFF
        memo[v] = oracle.payload(v, 0, s, _rounds(g, v))
        return memo[v]

    try:
        o = np.array([out(v) for v in range(g.n)], dtype=np.uint32)
    finally:
        sys.setrecursionlimit(old)
    return o, np.ones(g.n, np.uint32), oracle.mix32_many(o)


def wavefront_dp(side, rounds):
    """The 2D wavefront as a dynamic programme over (i, j)."""
    out = np.zeros((side, side), np.uint64)
    for i in range(side):
        for j in range(side):
            s = 0
            if i > 0:
                s += int(out[i - 1, j])
            if j > 0:
                s += int(out[i, j - 1])
            out[i, j] = oracle.payload(i * side + j, 0, s & 0xFFFFFFFF, rounds)
    return out.reshape(-1).astype(np.uint32)


def unrolled_config1(g):
    """Config-1 graph as a program: run I once; then for t in 0..T-1 run H
    (fed by I at t=0, by C's previous output afterwards), the body with
    iteration t, and C; finally D fed by C's last output."""
    I, H, C, D = g.meta["I"], g.meta["H"], g.meta["C"], g.meta["D"]
    b0, b1 = g.meta["body"]
    T = g.meta["trip"]
    preds = strong_preds(g)
    n = g.n
    out = np.zeros(n, np.uint64)
    cnt = np.zeros(n, np.uint64)
    dig = np.zeros(n, np.uint64)

    def run(v, t, s):
        x = oracle.payload(v, t, s & 0xFFFFFFFF, _rounds(g, v))
        out[v] = x
        cnt[v] += 1
        dig[v] = oracle.mix32(int(dig[v]) ^ x)
        return x

    xi = run(I, 0, 0)
    feed = xi
    for t in range(T):
        run(H, t, feed)
        for v in range(b0, b1):   # body ids are in level order
            run(v, t, sum(int(out[p]) for p in preds[v]))
        feed = run(C, t, sum(int(out[p]) for p in preds[C]))
    run(D, 0, feed)
    return out.astype(np.uint32), cnt.astype(np.uint32), dig.astype(np.uint32)


def structured_lane(g, lane, seed, out, cnt, dig, s_out):
    """One config-3 lane as nested loops: for i1 < T1 { h1; for i2 < T2 { h2;
    cb; j = arm chosen by cb; for i3 < T3_j { h3_j; body_j; c3_j }; M; c2 };
    c1 }; X.  Data follow the graph's edges: a strong edge feeds the
    producer's output, a condition feeds its output to the task it selects."""
    preds = lane["_preds"]

    def run(v, s):
        t = int(cnt[v])
        x = oracle.payload(v, t, s & 0xFFFFFFFF, _rounds(g, v))
        out[v] = x
        cnt[v] = t + 1
        dig[v] = oracle.mix32(int(dig[v]) ^ x)
        return x, t

    h1, h2, cb, M, c2, c1, X = (lane[k] for k in ("h1", "h2", "cb", "M", "c2", "c1", "X"))
    k = lane["k"]
    feed_h1 = s_out
    for _i1 in range(lane["T1"]):
        x_h1, _ = run(h1, feed_h1)
        feed_h2 = x_h1
        for _i2 in range(lane["T2"]):
            x_h2, _ = run(h2, feed_h2)
            x_cb, t_cb = run(cb, x_h2)
            j = oracle.cond_hash(seed, cb, t_cb) % k
            h3, b0, c3, T3 = lane["arms"][j]
            feed_h3 = x_cb
            for _i3 in range(T3):
                run(h3, feed_h3)
                for v in range(b0, c3):
                    run(v, sum(int(out[p]) for p in preds[v]))
                x_c3, _ = run(c3, sum(int(out[p]) for p in preds[c3]))
                feed_h3 = x_c3
            x_m, _ = run(M, x_c3)
            x_c2, _ = run(c2, x_m)
            feed_h2 = x_c2
        x_c1, _ = run(c1, x_c2)
        feed_h1 = x_c1
    run(X, x_c1)


def structured_config3(g):
    n = g.n
    out = np.zeros(n, np.uint64)
    cnt = np.zeros(n, np.uint64)
    dig = np.zeros(n, np.uint64)
    preds = strong_preds(g)
    S = g.meta["S"]
    x_s = oracle.payload(S, 0, 0, _rounds(g, S))
    out[S], cnt[S], dig[S] = x_s, 1, oracle.mix32(x_s)
    for lane in g.meta["lanes"]:
        lane = dict(lane, _preds=preds)
        structured_lane(g, lane, g.seed, out, cnt, dig, x_s)
    return out.astype(np.uint32), cnt.astype(np.uint32), dig.astype(np.uint32)


def motif_counts(g):
    """Closed-form counts of a motif graph: DAG tasks once; each motif's h and
    c run T times; c then exits to arm 1 + (hash mod (k-1)) (k > 2) or arm 1."""
    cnt = np.zeros(g.n, np.int64)
    cnt[: g.meta["n_d"]] = 1
    for h, c, k, T in zip(g.meta["h"], g.meta["c"], g.meta["k"], g.meta["trips"]):
        cnt[h] = T
        cnt[c] = T
        if k <= 2:
            r = 1
        else:
            r = 1 + oracle.cond_hash(g.seed, int(c), int(T) - 1) % (int(k) - 1)
        cnt[c + r] = 1   # arm r sits at c + r (ids: h, c, arm_1, ...)
    return cnt


def brute_force(g, exec_cap=64, max_states=200_000):
    """Explore every order in which ready activations can run.

    Returns the set of distinct terminal outcomes (status, out, cnt, dig).
    An activation of a task that is already queued ends that schedule with
    RACE; exceeding exec_cap ends it with EXEC_LIMIT."""
    n = g.n
    kinds = [int(k) for k in g.kinds]
    params = [int(p) for p in g.params]
    succ = [[] for _ in range(n)]
    sin = [0] * n
    win = [0] * n
    for s, d in zip(g.src.tolist(), g.dst.tolist()):
        succ[s].append(d)
        if kinds[s] == STATIC:
            sin[d] += 1
        else:
            win[d] += 1
    sources = [v for v in range(n) if sin[v] == 0 and win[v] == 0]
    if not sources:
        return {("NO_SOURCE",)}
    M = 0xFFFFFFFF
    start = (tuple(sorted((v, 0) for v in sources)), tuple(sin), tuple([0] * n),
             tuple([0] * n), tuple([0] * n), tuple([0] * n), 0)
    outcomes = set()
    seen = set()
    stack = [start]
    while stack:
        st = stack.pop()
        if st in seen:
            continue
        seen.add(st)
        if len(seen) > max_states:
            raise RuntimeError("state space too large")
        q, wc, ws, out, cnt, dig, ex = st
        if not q:
            outcomes.add(("OK", out, cnt, dig))
            continue
        for qi, (v, s) in enumerate(q):
            rest = list(q[:qi] + q[qi + 1:])
            wc2, ws2 = list(wc), list(ws)
            out2, cnt2, dig2 = list(out), list(cnt), list(dig)
            it = cnt2[v]
            x = oracle.payload(v, it, s, params[v] & 0xFFFF)
            out2[v] = x
            cnt2[v] = it + 1
            dig2[v] = oracle.mix32(dig2[v] ^ x)
            ex2 = ex + 1
            if ex2 > exec_cap:
                outcomes.add(("EXEC_LIMIT",))
                continue
            pushes = []
            if kinds[v] != STATIC:
                r = oracle.condition_index(kinds[v], params[v], g.seed, v, it, len(succ[v]))
                if 0 <= r < len(succ[v]):
                    pushes.append((succ[v][r], x))
            else:
                for u in succ[v]:
                    ws2[u] = (ws2[u] + x) & M
                    wc2[u] -= 1
                    if wc2[u] == 0:
                        pushes.append((u, ws2[u]))
                        wc2[u] = sin[u]
                        ws2[u] = 0
            race = False
            for u, su in pushes:
                if any(w == u for w, _ in rest):
                    race = True
                    break
                rest.append((u, su))
            if race:
                outcomes.add(("RACE",))
                continue
            stack.append((tuple(sorted(rest)), tuple(wc2), tuple(ws2), tuple(out2), tuple(cnt2),
                          tuple(dig2), ex2))
    return outcomes
