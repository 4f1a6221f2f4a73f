"""Thin ctypes binding of libtg.so: the same names as the C-ABI in
include/tg.h, argument marshalling only.  Every step of graph execution runs
in the library's CUDA kernels; PyTorch supplies the device arena and the
stream.  There is no CPU fallback: if libtg.so is missing or no CUDA device
is present, the calls raise."""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtg.so")

TG_STATIC, TG_COND_BRANCH, TG_COND_LOOP, TG_COND_CONST, TG_MODULE, TG_SUBFLOW = 0, 1, 2, 3, 4, 5
TG_OK, TG_PENDING = 0, 1
TG_ERR_INVALID, TG_ERR_NO_SOURCE, TG_ERR_EDGE_KIND, TG_ERR_BUDGET = -1, -2, -3, -4
TG_ERR_RACE, TG_ERR_EXEC_LIMIT, TG_ERR_TIMEOUT, TG_ERR_CANCELLED = -5, -6, -7, -8
TG_ERR_CUDA, TG_ERR_INTERNAL, TG_ERR_BUSY = -9, -10, -11
TG_OPT_NO_RACE_CHECK = 0x1
TG_OPT_TRACE = 0x2
TG_OPT_TRACE_TASKS = 0x4
# where a traced task was taken from (tg_trace_copy: where >> 16)
TG_TRACE_FROM_HAND, TG_TRACE_FROM_RING, TG_TRACE_FROM_OWN_DEQUE, TG_TRACE_FROM_STEAL, TG_TRACE_FROM_INJECTION = 0, 1, 2, 3, 4

STATUS_NAMES = {TG_OK: "OK", TG_PENDING: "PENDING", TG_ERR_INVALID: "INVALID",
                TG_ERR_NO_SOURCE: "NO_SOURCE", TG_ERR_EDGE_KIND: "EDGE_KIND", TG_ERR_BUDGET: "BUDGET",
                TG_ERR_RACE: "RACE", TG_ERR_EXEC_LIMIT: "EXEC_LIMIT", TG_ERR_TIMEOUT: "TIMEOUT",
                TG_ERR_CANCELLED: "CANCELLED", TG_ERR_CUDA: "CUDA", TG_ERR_INTERNAL: "INTERNAL",
                TG_ERR_BUSY: "BUSY"}


class TgError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)} ({tg_strerror(status)})")


class tg_ctx_opts(ctypes.Structure):
    _fields_ = [("worker_blocks", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("deque_depth", ctypes.c_int32), ("steal_policy", ctypes.c_int32),
                ("max_steal", ctypes.c_int32), ("smem_ring", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("idle_sleep_ns", ctypes.c_uint32),
                ("max_thieves", ctypes.c_int32), ("batch_max", ctypes.c_int32),
                ("local_keep", ctypes.c_int32), ("thief_mode", ctypes.c_int32),
                ("time_limit_ns", ctypes.c_uint64), ("exec_cap", ctypes.c_uint64),
                ("mem_budget_bytes", ctypes.c_uint64), ("max_nodes", ctypes.c_uint64),
                ("max_edges", ctypes.c_uint64), ("steal_backoff_ns", ctypes.c_uint32), ("keep_idle", ctypes.c_int32),
                ("hand_batch", ctypes.c_int32)]


class tg_graph_info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_uint32), ("n_edges", ctypes.c_uint32),
                ("n_sources", ctypes.c_uint32), ("n_conditions", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64), ("pack_ns", ctypes.c_uint64),
                ("upload_ns", ctypes.c_uint64)]


class tg_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("tasks", "pops_local", "pops_own", "steal_attempts", "steal_hits", "inject_pops",
                 "spills", "idle_loops", "warp_iters", "pops_hand", "kernel_ns")] + \
               [("worker_blocks", ctypes.c_uint32), ("warps_per_block", ctypes.c_uint32),
                ("phase_cycles", ctypes.c_uint64 * 5), ("parks", ctypes.c_uint64),
                ("peak_thieves", ctypes.c_uint64), ("failed_rounds", ctypes.c_uint64),
                ("round_cycles", ctypes.c_uint64)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k == "phase_cycles" else getattr(self, k)) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_lib = None

# exported symbol -> (restype, argtypes); every symbol declared in include/tg.h
SIGNATURES = {
    "tg_ctx_create": (ctypes.c_int, [_vp, ctypes.c_size_t, _vp, ctypes.POINTER(tg_ctx_opts),
                                     ctypes.POINTER(_vp)]),
    "tg_ctx_destroy": (ctypes.c_int, [_vp]),
    "tg_graph_create": (ctypes.c_int, [_vp, _u32, _vp, _vp, _u32, _vp, _vp, _vp, _u32, ctypes.POINTER(_vp)]),
    "tg_graph_create_dev": (ctypes.c_int, [_vp, _u32, _vp, _vp, _u32, _vp, _vp, _vp, _u32, ctypes.POINTER(_vp)]),
    "tg_graph_packed_copy": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(_u64)]),
    "tg_graph_autotune": (ctypes.c_int, [_vp, _vp, _u32, ctypes.c_char_p, ctypes.POINTER(tg_ctx_opts),
                                         ctypes.POINTER(_u64)]),
    "tg_graph_create_composed": (ctypes.c_int, [_vp, _u32, _vp, _vp, _u32, _vp, _vp, _vp, _u32, _vp,
                                                ctypes.POINTER(_vp)]),
    "tg_graph_destroy": (ctypes.c_int, [_vp, _vp]),
    "tg_graph_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(tg_graph_info)]),
    "tg_run": (ctypes.c_int, [_vp, _vp]),
    "tg_submit": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_u64)]),
    "tg_poll": (ctypes.c_int, [_vp, _u64]),
    "tg_wait": (ctypes.c_int, [_vp, _u64]),
    "tg_cancel": (ctypes.c_int, [_vp]),
    "tg_result_copy": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_u64)]),
    "tg_batch_create": (ctypes.c_int, [_vp, _vp, _u32, ctypes.POINTER(_vp)]),
    "tg_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "tg_batch_wait": (ctypes.c_int, [_vp, _vp, _vp]),
    "tg_batch_destroy": (ctypes.c_int, [_vp, _vp]),
    "tg_run_batch": (ctypes.c_int, [_vp, _vp, _u32, _vp]),
    "tg_ctx_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(tg_stats)]),
    "tg_ctx_get_opts": (ctypes.c_int, [_vp, ctypes.POINTER(tg_ctx_opts)]),
    "tg_ctx_set_launch": (ctypes.c_int, [_vp, ctypes.POINTER(tg_ctx_opts)]),
    "tg_instance_create": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "tg_serve_start": (ctypes.c_int, [_vp, _u64]),
    "tg_serve_stop": (ctypes.c_int, [_vp]),
    "tg_serve_replay": (ctypes.c_int, [_vp, _vp, _u32, _vp, _vp, _u32, _vp, _vp, ctypes.POINTER(_u32), _vp, _vp]),
    "tg_batch_autotune": (ctypes.c_int, [_vp, _vp, _u32, ctypes.c_char_p, ctypes.POINTER(tg_ctx_opts),
                                         ctypes.POINTER(_u64)]),
    "tg_bench_payload": (ctypes.c_int, [_vp, _u64, _u32, ctypes.POINTER(_u64), ctypes.POINTER(_u32)]),
    "tg_bench_atomics": (ctypes.c_int, [_vp, _u64, _u64, ctypes.POINTER(_u64)]),
    "tg_bench_payload_tasks": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, ctypes.POINTER(_u64), ctypes.POINTER(_u32)]),
    "tg_bench_chain": (ctypes.c_int, [_vp, _u32, _u32, ctypes.POINTER(_u64), ctypes.POINTER(_u32)]),
    "tg_levelize": (ctypes.c_int, [_u32, _u32, _vp, _vp, _vp, _vp, ctypes.POINTER(_u32)]),
    "tg_stream_plan": (ctypes.c_int, [_u32, _u32, _vp, _vp, _u32, _vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "tg_capture_run": (ctypes.c_int, [_vp, _vp, _u32, ctypes.POINTER(_u64)]),
    "tg_graph_dot": (ctypes.c_int, [_vp, _vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "tg_run_noalloc": (ctypes.c_int, [_u32, _vp, _vp, _vp, _vp, _u32, _u32, _vp, _vp, _vp, _vp]),
    "tg_trace_copy": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "tg_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}


def load(path: str = LIB_PATH):
    """Load libtg.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"libtg.so not built at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_vp)


def _check(st, what):
    if st != TG_OK:
        raise TgError(st, what)


def tg_strerror(status: int) -> str:
    return load().tg_strerror(status).decode()


def tg_ctx_create(dev_arena_ptr: int, arena_bytes: int, cuda_stream: int, opts: tg_ctx_opts | None = None):
    out = _vp()
    st = load().tg_ctx_create(_vp(dev_arena_ptr), arena_bytes, _vp(cuda_stream),
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(out))
    _check(st, "tg_ctx_create")
    return out.value


def tg_ctx_destroy(ctx):
    return load().tg_ctx_destroy(_vp(ctx))


def tg_graph_create(ctx, kinds, params, src, dst, seed=0, weak=None):
    """Returns (status, handle); handle is None unless status == TG_OK."""
    k, kp = _arr(kinds, np.uint8)
    p, pp = _arr(params, np.uint32)
    s, sp = _arr(src, np.uint32)
    d, dp = _arr(dst, np.uint32)
    wp = None
    if weak is not None:
        w, wp = _arr(weak, np.uint8)
    out = _vp()
    st = load().tg_graph_create(_vp(ctx), k.shape[0], kp, pp, s.shape[0], sp, dp, wp, seed & 0xFFFFFFFF,
                                ctypes.byref(out))
    return st, (out.value if st == TG_OK else None)


def tg_graph_create_dev(ctx, kinds, params, src, dst, seed=0, weak=None):
    """As tg_graph_create, packed on the device.  Returns (status, handle)."""
    k, kp = _arr(kinds, np.uint8)
    p, pp = _arr(params, np.uint32)
    s, sp = _arr(src, np.uint32)
    d, dp = _arr(dst, np.uint32)
    wp = None
    if weak is not None:
        w, wp = _arr(weak, np.uint8)
    out = _vp()
    st = load().tg_graph_create_dev(_vp(ctx), k.shape[0], kp, pp, s.shape[0], sp, dp, wp, seed & 0xFFFFFFFF,
                                    ctypes.byref(out))
    return st, (out.value if st == TG_OK else None)


def tg_graph_create_composed(ctx, kinds, params, src, dst, modules, seed=0, weak=None):
    """modules: {task: graph handle} for the TG_MODULE tasks.  Returns (status, handle)."""
    k, kp = _arr(kinds, np.uint8)
    p, pp = _arr(params, np.uint32)
    s, sp = _arr(src, np.uint32)
    d, dp = _arr(dst, np.uint32)
    wp = None
    if weak is not None:
        w, wp = _arr(weak, np.uint8)
    table = (_vp * max(1, k.shape[0]))()
    for v, h in modules.items():
        table[int(v)] = h
    out = _vp()
    st = load().tg_graph_create_composed(_vp(ctx), k.shape[0], kp, pp, s.shape[0], sp, dp, wp, seed & 0xFFFFFFFF,
                                         ctypes.cast(table, _vp), ctypes.byref(out))
    return st, (out.value if st == TG_OK else None)


def tg_graph_destroy(ctx, g):
    return load().tg_graph_destroy(_vp(ctx), _vp(g))


def tg_graph_get_info(g) -> dict:
    info = tg_graph_info()
    _check(load().tg_graph_get_info(_vp(g), ctypes.byref(info)), "tg_graph_get_info")
    return {k: getattr(info, k) for k, _ in info._fields_}


def tg_run(ctx, g) -> int:
    return load().tg_run(_vp(ctx), _vp(g))


def tg_submit(ctx, g):
    t = _u64(0)
    st = load().tg_submit(_vp(ctx), _vp(g), ctypes.byref(t))
    return st, t.value


def tg_poll(ctx, ticket) -> int:
    return load().tg_poll(_vp(ctx), ticket)


def tg_wait(ctx, ticket) -> int:
    return load().tg_wait(_vp(ctx), ticket)


def tg_cancel(ctx) -> int:
    return load().tg_cancel(_vp(ctx))


def tg_result_copy(ctx, g, n):
    out = np.empty(n, np.uint32)
    cnt = np.empty(n, np.uint32)
    dig = np.empty(n, np.uint32)
    tot = _u64(0)
    _check(load().tg_result_copy(_vp(ctx), _vp(g), out.ctypes.data_as(_vp), cnt.ctypes.data_as(_vp),
                                 dig.ctypes.data_as(_vp), ctypes.byref(tot)), "tg_result_copy")
    return out, cnt, dig, tot.value


def _handles(gs):
    arr = (_vp * len(gs))(*[_vp(g) for g in gs])
    return arr


def tg_batch_create(ctx, gs):
    out = _vp()
    st = load().tg_batch_create(_vp(ctx), ctypes.cast(_handles(gs), _vp), len(gs), ctypes.byref(out))
    return st, (out.value if st == TG_OK else None)


def tg_batch_launch(ctx, b) -> int:
    return load().tg_batch_launch(_vp(ctx), _vp(b))


def tg_batch_wait(ctx, b, n):
    sts = np.zeros(n, np.int32)
    st = load().tg_batch_wait(_vp(ctx), _vp(b), sts.ctypes.data_as(_vp))
    return st, sts


def tg_batch_destroy(ctx, b) -> int:
    return load().tg_batch_destroy(_vp(ctx), _vp(b))


def tg_run_batch(ctx, gs):
    sts = np.zeros(len(gs), np.int32)
    st = load().tg_run_batch(_vp(ctx), ctypes.cast(_handles(gs), _vp), len(gs), sts.ctypes.data_as(_vp))
    return st, sts


def tg_ctx_get_stats(ctx) -> dict:
    s = tg_stats()
    _check(load().tg_ctx_get_stats(_vp(ctx), ctypes.byref(s)), "tg_ctx_get_stats")
    return s.as_dict()


def tg_ctx_get_opts(ctx) -> dict:
    o = tg_ctx_opts()
    _check(load().tg_ctx_get_opts(_vp(ctx), ctypes.byref(o)), "tg_ctx_get_opts")
    return {k: getattr(o, k) for k, _ in o._fields_}


def tg_instance_create(ctx, g):
    out = _vp()
    st = load().tg_instance_create(_vp(ctx), _vp(g), ctypes.byref(out))
    return st, (out.value if st == TG_OK else None)


def tg_serve_start(ctx, time_limit_ns=0) -> int:
    return load().tg_serve_start(_vp(ctx), time_limit_ns)


def tg_serve_stop(ctx) -> int:
    return load().tg_serve_stop(_vp(ctx))


def tg_serve_replay(ctx, templates, which, arrival_ns, keep=False):
    """Returns (status, latency_ns[], status[], max_in_flight, kept instance
    handles or None).  keep: False, True (every request) or a boolean mask of
    the requests whose instances are kept."""
    which = np.ascontiguousarray(which, dtype=np.uint32)
    arrival = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
    n = which.shape[0]
    lat = np.zeros(n, np.uint64)
    sts = np.zeros(n, np.int32)
    peak = _u32(0)
    want = keep is not False and keep is not None
    kept = (_vp * n)() if want else None
    mask = None
    if want and keep is not True:
        mask = np.ascontiguousarray(np.asarray(keep, dtype=bool).astype(np.uint8))
        assert mask.shape[0] == n
    st = load().tg_serve_replay(_vp(ctx), ctypes.cast(_handles(templates), _vp), len(templates),
                                which.ctypes.data_as(_vp), arrival.ctypes.data_as(_vp), n,
                                lat.ctypes.data_as(_vp), sts.ctypes.data_as(_vp), ctypes.byref(peak),
                                ctypes.cast(kept, _vp) if want else None,
                                mask.ctypes.data_as(_vp) if mask is not None else None)
    return st, lat, sts, peak.value, ([kept[i] for i in range(n)] if want else None)


def tg_ctx_set_launch(ctx, **fields) -> int:
    o = tg_ctx_opts()
    for k, v in fields.items():
        setattr(o, k, v)
    return load().tg_ctx_set_launch(_vp(ctx), ctypes.byref(o))


def tg_batch_autotune(ctx, b, trials=2, cache_path=None):
    """Returns (status, chosen options dict, best device ns)."""
    o = tg_ctx_opts()
    t = _u64(0)
    st = load().tg_batch_autotune(_vp(ctx), _vp(b), trials, cache_path.encode() if cache_path else None,
                                  ctypes.byref(o), ctypes.byref(t))
    return st, {k: getattr(o, k) for k, _ in o._fields_}, t.value


def tg_graph_autotune(ctx, g, trials=2, cache_path=None):
    """Returns (status, chosen options dict, best device ns)."""
    o = tg_ctx_opts()
    t = _u64(0)
    st = load().tg_graph_autotune(_vp(ctx), _vp(g), trials, cache_path.encode() if cache_path else None,
                                  ctypes.byref(o), ctypes.byref(t))
    return st, {k: getattr(o, k) for k, _ in o._fields_}, t.value


def tg_bench_payload(ctx, count, rounds):
    ns = _u64(0)
    cs = _u32(0)
    _check(load().tg_bench_payload(_vp(ctx), count, rounds, ctypes.byref(ns), ctypes.byref(cs)), "tg_bench_payload")
    return ns.value, cs.value


def tg_levelize(n, src, dst):
    """Returns (status, level[n], index[n], n_levels) of the DAG (src[e] -> dst[e])."""
    s, sp = _arr(src, np.uint32)
    d, dp = _arr(dst, np.uint32)
    level = np.zeros(n, np.uint32)
    index = np.zeros(n, np.uint32)
    nl = _u32(0)
    st = load().tg_levelize(n, len(s), sp, dp, level.ctypes.data_as(_vp), index.ctypes.data_as(_vp),
                            ctypes.byref(nl))
    return st, level, index, nl.value


def tg_stream_plan(n, src, dst, max_streams):
    """Returns (status, stream[n], n_events, n_waits) of Algorithm 1's round-robin layout."""
    s, sp = _arr(src, np.uint32)
    d, dp = _arr(dst, np.uint32)
    stream = np.zeros(n, np.uint32)
    ne = _u32(0)
    nw = _u32(0)
    st = load().tg_stream_plan(n, len(s), sp, dp, max_streams, stream.ctypes.data_as(_vp), ctypes.byref(ne),
                               ctypes.byref(nw))
    return st, stream, ne.value, nw.value


def tg_graph_packed_copy(ctx, g, n):
    """The packed graph word for word: (records as an (n, 8) uint32 array,
    successor entries followed by the source list)."""
    words = _u64(0)
    _check(load().tg_graph_packed_copy(_vp(ctx), _vp(g), None, None, ctypes.byref(words)), "tg_graph_packed_copy")
    rec = np.empty((n, 8), np.uint32)
    edges = np.empty(words.value, np.uint32)
    _check(load().tg_graph_packed_copy(_vp(ctx), _vp(g), rec.ctypes.data_as(_vp), edges.ctypes.data_as(_vp), None),
           "tg_graph_packed_copy")
    return rec, edges


def tg_graph_dot(ctx, g) -> str:
    """The packed graph as Graphviz DOT text."""
    n = ctypes.c_size_t(0)
    st = load().tg_graph_dot(_vp(ctx), _vp(g), None, 0, ctypes.byref(n))
    if st not in (TG_OK, TG_ERR_BUDGET):
        raise TgError(st, "tg_graph_dot")
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(load().tg_graph_dot(_vp(ctx), _vp(g), buf, n.value + 1, ctypes.byref(n)), "tg_graph_dot")
    return buf.value.decode()


def tg_capture_run(ctx, g, max_streams):
    """Returns (status, device ns of the replay)."""
    ns = _u64(0)
    st = load().tg_capture_run(_vp(ctx), _vp(g), max_streams, ctypes.byref(ns))
    return st, ns.value


def tg_bench_chain(ctx, hops, rounds):
    """Returns (device ns, final output) of `hops` dependent payloads."""
    ns = _u64(0)
    last = _u32(0)
    _check(load().tg_bench_chain(_vp(ctx), hops, rounds, ctypes.byref(ns), ctypes.byref(last)), "tg_bench_chain")
    return ns.value, last.value


def tg_bench_payload_tasks(ctx, n, ids_ptr, rounds_ptr, cnt_ptr):
    """Returns (device ns, checksum) of the payloads of a given execution
    multiset (device arrays of n uint32 each; see include/tg.h)."""
    ns = _u64(0)
    cs = _u32(0)
    _check(load().tg_bench_payload_tasks(_vp(ctx), n, _vp(ids_ptr), _vp(rounds_ptr), _vp(cnt_ptr), ctypes.byref(ns),
                                         ctypes.byref(cs)), "tg_bench_payload_tasks")
    return ns.value, cs.value


def tg_bench_atomics(ctx, count, footprint_words):
    ns = _u64(0)
    _check(load().tg_bench_atomics(_vp(ctx), count, footprint_words, ctypes.byref(ns)), "tg_bench_atomics")
    return ns.value


def tg_run_noalloc(n_nodes, kinds_ptr, params_ptr, succ_off_ptr, succ_ptr, n_edges, seed,
                   out_ptr, cnt_ptr, dig_ptr, cuda_stream) -> int:
    """Device pointers in, device pointers out; see include/tg.h."""
    return load().tg_run_noalloc(n_nodes, _vp(kinds_ptr), _vp(params_ptr), _vp(succ_off_ptr), _vp(succ_ptr),
                                 n_edges, seed & 0xFFFFFFFF, _vp(out_ptr), _vp(cnt_ptr), _vp(dig_ptr),
                                 _vp(cuda_stream))


def tg_trace_copy(ctx, g, n):
    """(start_ns[n], end_ns[n], where[n]) of each task's last execution
    (TG_OPT_TRACE_TASKS or TG_OPT_TRACE): when a warp took it from a queue,
    when that step ended, and TG_TRACE_FROM_* << 16 | worker block."""
    a = np.zeros(n, np.uint64)
    b = np.zeros(n, np.uint64)
    c = np.zeros(n, np.uint32)
    _check(load().tg_trace_copy(_vp(ctx), _vp(g), a.ctypes.data_as(_vp), b.ctypes.data_as(_vp),
                                c.ctypes.data_as(_vp)), "tg_trace_copy")
    return a, b, c
