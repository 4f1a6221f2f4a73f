"""Seeded synthetic task graphs shaped like the paper's workloads.

A graph is given the way a Taskflow user builds one: a node list (kind +
parameters) and an edge list in insertion ("precede") order.  The order
matters only for the out-edges of a condition task, whose return value
indexes its successors in that order (Conditional Tasking section).

Kinds and the parameter word are the input encoding shared by every consumer:

    kind   0 static, 1 condition "branch", 2 condition "loop", 3 condition "constant"
    param  rounds (bits 0-15) | trip (bits 16-23) | const index, int8 (bits 24-31)

Everything random comes from workloads.rng (splitmix64).  This module holds
no payload, hash or digest arithmetic of the method itself.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .rng import Stream

STATIC, COND_BRANCH, COND_LOOP, COND_CONST, MODULE, SUBFLOW = 0, 1, 2, 3, 4, 5


def pack_param(rounds, trip=0, const_index=0):
    rounds = np.asarray(rounds, dtype=np.int64)
    trip = np.asarray(trip, dtype=np.int64)
    ci = np.asarray(const_index, dtype=np.int64)
    return ((rounds & 0xFFFF) | ((trip & 0xFF) << 16) | ((ci & 0xFF) << 24)).astype(np.uint32)


@dataclass
class Graph:
    name: str
    kinds: np.ndarray      # uint8 [n]
    params: np.ndarray     # uint32 [n]
    src: np.ndarray        # uint32 [m], insertion order
    dst: np.ndarray        # uint32 [m]
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.kinds.shape[0])

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def from_lists(name, kinds, params, edges, seed=0, meta=None) -> Graph:
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2) if len(edges) else np.zeros((0, 2), np.int64)
    return Graph(name, np.asarray(kinds, dtype=np.uint8), np.asarray(params, dtype=np.uint32),
                 e[:, 0].astype(np.uint32), e[:, 1].astype(np.uint32), int(seed), dict(meta or {}))


# ---------------------------------------------------------------------------
# distinct predecessor sampling (uniform, without replacement)
# ---------------------------------------------------------------------------
_K = 12          # candidates drawn per row before the per-row fallback
_CHUNK = 1 << 20


def sample_distinct(stream: Stream, width: np.ndarray, d: np.ndarray) -> np.ndarray:
    """For row i pick d[i] distinct integers uniformly from [0, width[i]).

    Returns an int64 array [N, max(d)] padded with -1, picks in draw order.
    Rows whose first _K draws hold fewer than d[i] distinct values take the
    first d[i] entries of a random permutation instead (drawn from the same
    stream, in row order), so the result is deterministic for a given seed.
    """
    width = np.asarray(width, dtype=np.int64)
    d = np.asarray(d, dtype=np.int64)
    N = width.shape[0]
    dmax = int(d.max()) if N else 0
    out = np.full((N, max(dmax, 1)), -1, dtype=np.int64)
    if N == 0 or dmax == 0:
        return out[:, :dmax]
    ar = np.arange(_K, dtype=np.int64)
    for c0 in range(0, N, _CHUNK):
        c1 = min(N, c0 + _CHUNK)
        w = width[c0:c1]
        dd = d[c0:c1]
        n = c1 - c0
        cand = stream.below(n * _K, np.repeat(w, _K)).reshape(n, _K)
        key = np.sort(cand * _K + ar, axis=1)
        val = key // _K
        pos = key % _K
        first = np.ones_like(key, dtype=bool)
        first[:, 1:] = val[:, 1:] != val[:, :-1]
        kept = np.where(first, pos, _K)
        kept.sort(axis=1)
        kept = kept[:, :dmax]
        ok = first.sum(axis=1) >= dd
        picks = np.take_along_axis(cand, np.minimum(kept, _K - 1), axis=1)
        mask = np.arange(dmax)[None, :] < dd[:, None]
        blk = np.where(mask, picks, -1)
        for r in np.nonzero(~ok)[0]:
            keys = stream.u64(int(w[r]))
            perm = np.argsort(keys, kind="stable")[: dd[r]]
            blk[r, :] = -1
            blk[r, : dd[r]] = perm
        out[c0:c1] = blk
    return out


def _layered_edges(stream: Stream, first_id: int, widths, d_lo: int, d_hi: int):
    """Edges of a layered DAG whose levels have the given widths; level 0 has no
    predecessors, every node of level L>0 draws d ~ U{d_lo..d_hi} (capped at
    the width of level L-1) distinct predecessors from level L-1.
    Edges come out ordered by destination, predecessors in draw order."""
    widths = np.asarray(widths, dtype=np.int64)
    starts = first_id + np.concatenate([[0], np.cumsum(widths)[:-1]])
    if widths.shape[0] < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    lvl = np.repeat(np.arange(1, widths.shape[0]), widths[1:])
    node = np.arange(starts[1], starts[-1] + widths[-1], dtype=np.int64)
    wprev = widths[lvl - 1]
    d = np.minimum(stream.integers(node.shape[0], d_lo, d_hi), wprev)
    rel = sample_distinct(stream, wprev, d)
    valid = rel >= 0
    src = (starts[lvl - 1][:, None] + rel)[valid]
    dst = np.broadcast_to(node[:, None], rel.shape)[valid]
    return src, dst


# ---------------------------------------------------------------------------
# worked examples of the paper (Static Tasking / Conditional Tasking sections)
# ---------------------------------------------------------------------------
def diamond(rounds=4) -> Graph:
    """Four static tasks: A precedes B and C, D succeeds B and C (Listing 1)."""
    return from_lists("diamond", [STATIC] * 4, pack_param([rounds] * 4),
                      [(0, 1), (0, 2), (1, 3), (2, 3)],
                      meta={"A": 0, "B": 1, "C": 2, "D": 3})


def if_else(ret: int, rounds=4) -> Graph:
    """init -> cond -> {yes (index 0), no (index 1)}; cond returns `ret`."""
    return from_lists("if_else", [STATIC, COND_CONST, STATIC, STATIC],
                      [pack_param(rounds), pack_param(rounds, 0, ret), pack_param(rounds), pack_param(rounds)],
                      [(0, 1), (1, 2), (1, 3)],
                      meta={"init": 0, "cond": 1, "yes": 2, "no": 3})


def do_while(iterations=100, rounds=4) -> Graph:
    """init -> body -> cond -> {body (0), done (1)}; cond loops `iterations` times."""
    return from_lists("do_while", [STATIC, STATIC, COND_LOOP, STATIC],
                      [pack_param(rounds), pack_param(rounds), pack_param(rounds, iterations), pack_param(rounds)],
                      [(0, 1), (1, 2), (2, 1), (2, 3)],
                      meta={"init": 0, "body": 1, "cond": 2, "done": 3, "iterations": iterations})


def nested_loops(seed: int, rounds=2, extra_init_to_f2=False) -> Graph:
    """init -> F1; F1 -> {F2, F1}; F2 -> {F3, F1}; F3 -> {stop, F1}: three
    condition tasks that each go on with probability 1/2 (Conditional
    Tasking section).  With extra_init_to_f2 the strong edge init -> F2 of
    the scheduling walk-through is added, which makes F2 racy."""
    edges = [(0, 1), (1, 2), (1, 1), (2, 3), (2, 1), (3, 4), (3, 1)]
    if extra_init_to_f2:
        edges.append((0, 2))
    return from_lists("nested_loops", [STATIC, COND_BRANCH, COND_BRANCH, COND_BRANCH, STATIC],
                      pack_param([rounds] * 5), edges, seed=seed,
                      meta={"init": 0, "F1": 1, "F2": 2, "F3": 3, "stop": 4})


def pitfall_no_source() -> Graph:
    """Every task has an in-edge, so the scheduler has nowhere to start."""
    return from_lists("pitfall_no_source", [COND_CONST, STATIC], [pack_param(1, 0, 0), pack_param(1)],
                      [(0, 1), (1, 0)])


def pitfall_race(fixed=False) -> Graph:
    """S -> {C, E}; C (condition, returns 0) jumps to D while E strongly
    precedes D, so D can be activated twice.  With fixed=True the control
    flow is partitioned through an auxiliary task X: C -> X, X -> D, E -> D."""
    if not fixed:
        return from_lists("pitfall_race", [STATIC, COND_CONST, STATIC, STATIC],
                          [pack_param(1), pack_param(1, 0, 0), pack_param(1), pack_param(1)],
                          [(0, 1), (0, 2), (1, 3), (2, 3)], meta={"S": 0, "C": 1, "E": 2, "D": 3})
    return from_lists("pitfall_race_fixed", [STATIC, COND_CONST, STATIC, STATIC, STATIC],
                      [pack_param(1), pack_param(1, 0, 0), pack_param(1), pack_param(1), pack_param(1)],
                      [(0, 1), (0, 2), (1, 4), (4, 3), (2, 3)], meta={"S": 0, "C": 1, "E": 2, "D": 3, "X": 4})


# ---------------------------------------------------------------------------
# the five workloads (seeded; sizes are parameters so tests can shrink them)
# ---------------------------------------------------------------------------
def config1(seed=0, levels=10, width=100, d_lo=1, d_hi=4, rounds=64, trip=5) -> Graph:
    """Plain single graph: I -> H -> layered body (levels x width) -> C, with
    C a loop condition of `trip` passes whose successors are [H, D].
    I and H are helper tasks (H is the loop entry the condition jumps to; I
    is the zero-dependency source H needs besides its weak in-edge)."""
    st = Stream(seed, 1)
    nb = levels * width
    I, H, b0 = 0, 1, 2
    C, D = b0 + nb, b0 + nb + 1
    n = nb + 4
    bs, bd = _layered_edges(st, b0, [width] * levels, d_lo, d_hi)
    has_succ = np.zeros(n, bool)
    has_succ[bs] = True
    sinks = np.nonzero(~has_succ[b0:b0 + nb])[0] + b0
    src = np.concatenate([[I], np.full(width, H), bs, sinks, [C, C]])
    dst = np.concatenate([[H], np.arange(b0, b0 + width), bd, np.full(sinks.shape[0], C), [H, D]])
    kinds = np.zeros(n, np.uint8)
    kinds[C] = COND_LOOP
    params = pack_param(np.full(n, rounds))
    params[C] = pack_param(rounds, trip)
    return Graph("config1", kinds, params, src.astype(np.uint32), dst.astype(np.uint32), seed,
                 {"I": I, "H": H, "C": C, "D": D, "body": (b0, b0 + nb), "trip": trip})


def config2a(seed=1, levels=1000, width=1000, d_lo=1, d_hi=8, rounds=16) -> Graph:
    """Large layered random DAG: levels x width static tasks, in-degree U{1..8}."""
    st = Stream(seed, 2)
    n = levels * width
    src, dst = _layered_edges(st, 0, [width] * levels, d_lo, d_hi)
    return Graph("config2a", np.zeros(n, np.uint8), pack_param(np.full(n, rounds)),
                 src.astype(np.uint32), dst.astype(np.uint32), seed, {"levels": levels, "width": width})


def config2b(seed=2, side=1024, rounds=256) -> Graph:
    """2D wavefront: cell (i, j) depends on (i-1, j) and (i, j-1)."""
    n = side * side
    ids = np.arange(n, dtype=np.int64).reshape(side, side)
    down_s, down_d = ids[:-1, :], ids[1:, :]
    right_s, right_d = ids[:, :-1], ids[:, 1:]
    # insertion order: for each cell in row-major order, [down, right]
    s = np.full((side, side, 2), -1, np.int64)
    d = np.full((side, side, 2), -1, np.int64)
    s[:-1, :, 0], d[:-1, :, 0] = down_s, down_d
    s[:, :-1, 1], d[:, :-1, 1] = right_s, right_d
    ok = s.reshape(-1) >= 0
    return Graph("config2b", np.zeros(n, np.uint8), pack_param(np.full(n, rounds)),
                 s.reshape(-1)[ok].astype(np.uint32), d.reshape(-1)[ok].astype(np.uint32), seed,
                 {"side": side})


def _lane_ks(st: Stream, n_cond: int):
    """Arm counts k in {2,3,4} of the lanes of config 3; a lane holds 3 + k
    condition tasks and the lanes together hold exactly n_cond of them."""
    ks, total = [], 0
    while n_cond - total > 21:
        k = int(st.integers(1, 2, 4)[0])
        ks.append(k)
        total += 3 + k
    rem = n_cond - total
    if ks or rem >= 15:
        extra = rem - 9
        base, r = divmod(extra, 3)
        ks += [base + (1 if i < r else 0) for i in range(3)]
    else:  # small test sizes: one lane per 3 + k conditions, as far as possible
        while rem >= 5:
            k = min(4, rem - 3)
            ks.append(k)
            rem -= 3 + k
    return ks


def config3(seed=3, n_cond=10_000, body_levels=10, body_width=10, d_lo=1, d_hi=4, rounds=32,
            trip_max=16) -> Graph:
    """Condition-heavy graph: lanes of loops nested to depth 3 fanning out of
    one source S.  Lane: h1 -> h2 -> cb; cb (branch over k arms) -> h3_j;
    h3_j -> body_j -> c3_j (loop) -> [h3_j, M]; M -> c2 (loop) -> [h2, c1];
    c1 (loop) -> [h1, X].  Trip counts are U{1..trip_max}."""
    st = Stream(seed, 3)
    ks = _lane_ks(st, n_cond)
    n_arms = sum(ks)
    bsz = body_levels * body_width
    # bodies, generated together: relative edges inside one body
    lvl = np.repeat(np.arange(1, body_levels), body_width)
    rel_node = np.arange(body_width, bsz, dtype=np.int64)
    nper = rel_node.shape[0]
    d = np.minimum(st.integers(n_arms * nper, d_lo, d_hi), body_width)
    rel = sample_distinct(st, np.full(n_arms * nper, body_width), d).reshape(n_arms, nper, -1)
    trips = st.integers(n_arms + 2 * len(ks), 1, trip_max)
    kinds, params, src, dst = [], [], [], []
    meta_lanes = []
    nid = 1  # node 0 is S
    kinds.append(np.array([STATIC], np.uint8))
    params.append(pack_param([rounds]))
    arm = 0
    ti = 0
    R = int(rounds)
    for li, k in enumerate(ks):
        h1, h2, cb = nid, nid + 1, nid + 2
        nid += 3
        lane_k = [STATIC, STATIC, COND_BRANCH]
        lane_p = [R, R, R]
        lane_t = [0, 0, 0]
        e = [(0, h1), (h1, h2), (h2, cb)]
        arms = []
        for j in range(k):
            h3 = nid
            b0 = nid + 1
            c3 = b0 + bsz
            nid = c3 + 1
            e.append((cb, h3))
            arms.append((h3, b0, c3))
        M, c2, c1, X = nid, nid + 1, nid + 2, nid + 3
        nid += 4
        ek = []
        for j, (h3, b0, c3) in enumerate(arms):
            r = rel[arm]
            valid = r >= 0
            ps = (b0 + (lvl - 1)[:, None] * body_width + r)[valid]
            pd = np.broadcast_to((b0 + rel_node)[:, None], r.shape)[valid]
            has = np.zeros(bsz, bool)
            has[ps - b0] = True
            sinks = np.nonzero(~has)[0] + b0
            T3 = int(trips[ti]); ti += 1
            lane_k += [STATIC] + [STATIC] * bsz + [COND_LOOP]
            lane_p += [R] * (bsz + 2)
            lane_t += [0] * (bsz + 1) + [T3]
            ek.append(np.stack([np.full(body_width, h3), b0 + np.arange(body_width)], 1))
            ek.append(np.stack([ps, pd], 1))
            ek.append(np.stack([sinks, np.full(sinks.shape[0], c3)], 1))
            ek.append(np.array([[c3, h3], [c3, M]]))
            arms[j] = (h3, b0, c3, T3)
            arm += 1
        T2 = int(trips[ti]); T1 = int(trips[ti + 1]); ti += 2
        lane_k += [STATIC, COND_LOOP, COND_LOOP, STATIC]
        lane_p += [R, R, R, R]
        lane_t += [0, T2, T1, 0]
        tail = np.array([[M, c2], [c2, h2], [c2, c1], [c1, h1], [c1, X]])
        kinds.append(np.array(lane_k, np.uint8))
        params.append(pack_param(np.array(lane_p), np.array(lane_t)))
        src.append(np.array(e, np.int64).reshape(-1, 2))
        src.extend(ek)
        src.append(tail)
        meta_lanes.append({"h1": h1, "h2": h2, "cb": cb, "M": M, "c2": c2, "c1": c1, "X": X,
                           "T1": T1, "T2": T2, "arms": arms, "k": k})
    E = np.concatenate(src, 0)
    kinds = np.concatenate(kinds)
    params = np.concatenate(params)
    return Graph("config3", kinds, params, E[:, 0].astype(np.uint32), E[:, 1].astype(np.uint32), seed,
                 {"lanes": meta_lanes, "S": 0, "n_cond": n_cond, "body": (body_levels, body_width)})


def motif_graph_py(st: Stream, n: int, seed: int, rounds=None, r_lo=8, r_hi=512, d_lo=1, d_hi=8,
                   cond_frac=0.05, trip_max=16, name="motif") -> Graph:
    """Layered random DAG of width round(sqrt(n_d)) plus loop motifs: about
    cond_frac * n loop conditions c, each anchored on a distinct DAG task s:
    s -> h -> c, c -> [h, arm_1 .. arm_{k-1}], k ~ U{2..4}, arms static leaves.

    This is the readable definition; motif_graph() draws the same graph with
    the native twin in motif.c (a test checks that they agree)."""
    n_c = max(1, int(round(cond_frac * n)))
    ks = st.integers(n_c, 2, 4)
    n_d = n - int((ks + 1).sum())
    if n_d < n_c:
        raise ValueError("graph too small for its motifs")
    w = max(1, int(round(np.sqrt(n_d))))
    widths = [w] * (n_d // w) + ([n_d % w] if n_d % w else [])
    ds, dd = _layered_edges(st, 0, widths, d_lo, d_hi)
    anchors = np.argsort(st.u64(n_d), kind="stable")[:n_c]
    trips = st.integers(n_c, 1, trip_max)
    kinds = np.zeros(n, np.uint8)
    # motif node ids: after the DAG, motif i takes [h, c, arms...]
    sizes = ks + 1
    base = n_d + np.concatenate([[0], np.cumsum(sizes)[:-1]])
    h = base
    c = base + 1
    kinds[c] = COND_LOOP
    if rounds is None:
        R = st.integers(n, r_lo, r_hi)
    else:
        R = np.full(n, rounds)
    trip_arr = np.zeros(n, np.int64)
    trip_arr[c] = trips
    params = pack_param(R, trip_arr)
    # motif edges: s -> h, h -> c, then each condition's out-edges in the
    # order [h, arm_1, arm_2, ...] (its successor indices)
    maxk = int(ks.max())
    es = np.concatenate([ds, anchors])
    ed = np.concatenate([dd, h])
    cs = [c[:, None]]
    cd = [h[:, None]]
    for j in range(1, maxk):
        col_s = np.where(ks > j, c, -1)
        col_d = np.where(ks > j, base + 1 + j, -1)
        cs.append(col_s[:, None]); cd.append(col_d[:, None])
    cs = np.concatenate(cs, 1).reshape(-1)
    cd = np.concatenate(cd, 1).reshape(-1)
    ok = cs >= 0
    src = np.concatenate([es, h, cs[ok]])
    dst = np.concatenate([ed, c, cd[ok]])
    return Graph(name, kinds, params, src.astype(np.uint32), dst.astype(np.uint32), seed,
                 {"n_d": n_d, "anchors": anchors, "h": h, "c": c, "k": ks, "trips": trips})


_motif_lib = None


def _motif():
    """libmotif.so, compiled from motif.c on first use (plain C, gcc)."""
    global _motif_lib
    if _motif_lib is None:
        import ctypes
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        src, lib = os.path.join(here, "motif.c"), os.path.join(here, "libmotif.so")
        if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
            os.replace(tmp, lib)
        L = ctypes.CDLL(lib)
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        L.wl_motif_graph.restype = ctypes.c_int
        L.wl_motif_graph.argtypes = [u64, u64, u32, u32, ctypes.c_int32, u32, u32, u32, u32, u32,
                                     vp, vp, vp, vp, u64, ctypes.POINTER(u64), vp, vp, vp,
                                     ctypes.POINTER(u32), ctypes.POINTER(u64)]
        _motif_lib = L
    return _motif_lib


def motif_graph(st: Stream, n: int, seed: int, rounds=None, r_lo=8, r_hi=512, d_lo=1, d_hi=8,
                cond_frac=0.05, trip_max=16, name="motif") -> Graph:
    """The motif graph of motif_graph_py, drawn by the native twin (about 50x
    faster; the ctypes call releases the GIL, so threads generate in
    parallel).  Advances `st` exactly as motif_graph_py does."""
    import ctypes
    n_c = max(1, int(round(cond_frac * n)))
    if d_hi > 8:
        return motif_graph_py(st, n, seed, rounds, r_lo, r_hi, d_lo, d_hi, cond_frac, trip_max, name)
    cap = n * d_hi + 4 * n_c + 8
    kinds = np.zeros(n, np.uint8)
    params = np.zeros(n, np.uint32)
    src = np.empty(cap, np.uint32)
    dst = np.empty(cap, np.uint32)
    ks = np.zeros(n_c, np.uint32)
    anchors = np.zeros(n_c, np.uint32)
    trips = np.zeros(n_c, np.uint32)
    m = ctypes.c_uint64(0)
    n_d = ctypes.c_uint32(0)
    pos = ctypes.c_uint64(0)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = _motif().wl_motif_graph(st.state, st.pos, n, n_c, -1 if rounds is None else int(rounds), r_lo, r_hi,
                                 d_lo, d_hi, trip_max, ptr(kinds), ptr(params), ptr(src), ptr(dst), cap,
                                 ctypes.byref(m), ptr(ks), ptr(anchors), ptr(trips), ctypes.byref(n_d),
                                 ctypes.byref(pos))
    if rc == -1:
        raise ValueError("graph too small for its motifs")
    if rc != 0:
        raise RuntimeError(f"wl_motif_graph failed ({rc})")
    st.pos = pos.value
    nd = int(n_d.value)
    sizes = ks.astype(np.int64) + 1
    base = nd + np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    mm = int(m.value)
    return Graph(name, kinds, params, src[:mm].copy(), dst[:mm].copy(), seed,
                 {"n_d": nd, "anchors": anchors.astype(np.int64), "h": base, "c": base + 1,
                  "k": ks.astype(np.int64), "trips": trips.astype(np.int64)})


def _logu(st: Stream, lo: int, hi: int) -> int:
    u = float(st.uniform(1)[0])
    return int(round(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))))


def config4(seed=4, n_graphs=4096, n_lo=16, n_hi=65536, r_lo=8, r_hi=512):
    """Batched: n_graphs independent motif graphs, node counts log-uniform in
    [n_lo, n_hi], per-task rounds U{r_lo..r_hi}."""
    out = []
    for g in range(n_graphs):
        st = Stream(seed * 1_000_003 + g, 4)
        n = _logu(st, n_lo, n_hi)
        out.append(motif_graph(st, n, seed=(seed << 16) ^ g, r_lo=r_lo, r_hi=r_hi, name=f"config4[{g}]"))
    return out


def config5_request(i: int, n_lo=64, n_hi=262144, rounds=64) -> Graph:
    """Serving request i: a motif graph with n log-uniform in [n_lo, n_hi],
    every task 64 rounds, graph seed = i."""
    st = Stream(i, 5)
    n = _logu(st, n_lo, n_hi)
    return motif_graph(st, n, seed=i, rounds=rounds, name=f"config5[{i}]")


def config5_arrivals(lam: float, count: int, seed=5) -> np.ndarray:
    """Poisson arrival times (seconds) of `count` requests at rate lam."""
    u = Stream(seed, 6).uniform(count)
    gaps = -np.log1p(-u) / float(lam)
    return np.cumsum(gaps)
