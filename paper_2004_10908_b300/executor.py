"""Executor: a context on one CUDA device whose arena and stream come from
PyTorch, with graph handles that own their device pools.  A thin layer over
the C-ABI names in binding.py."""
from __future__ import annotations

import numpy as np

from . import binding as B


class GraphHandle:
    def __init__(self, ex: "Executor", handle: int, n: int, m: int, name: str = ""):
        self.ex, self.handle, self.n, self.m, self.name = ex, handle, n, m, name

    def info(self) -> dict:
        return B.tg_graph_get_info(self.handle)

    def destroy(self):
        if self.handle:
            B.tg_graph_destroy(self.ex.ctx, self.handle)
            self.handle = None


class Batch:
    def __init__(self, ex: "Executor", handle: int, graphs):
        self.ex, self.handle, self.graphs = ex, handle, list(graphs)

    def launch(self):
        st = B.tg_batch_launch(self.ex.ctx, self.handle)
        if st != B.TG_OK:
            raise B.TgError(st, "tg_batch_launch")

    def wait(self):
        return B.tg_batch_wait(self.ex.ctx, self.handle, len(self.graphs))

    def autotune(self, trials=2, cache_path=None):
        """Pick and apply the fastest launch geometry (see tg_batch_autotune)."""
        st, chosen, ns = B.tg_batch_autotune(self.ex.ctx, self.handle, trials, cache_path)
        if st != B.TG_OK:
            raise B.TgError(st, "tg_batch_autotune")
        return chosen, ns

    def destroy(self):
        if self.handle:
            B.tg_batch_destroy(self.ex.ctx, self.handle)
            self.handle = None


class Executor:
    """Device-resident task-graph executor on the current CUDA device.

    arena_bytes: size of the torch-allocated device arena the library
    sub-allocates; stream: a torch.cuda.Stream (default: a new one);
    opts: any tg_ctx_opts field (worker_blocks, warps_per_block, deque_depth,
    steal_policy, max_steal, smem_ring, flags, idle_sleep_ns, max_thieves,
    batch_max, local_keep, thief_mode, time_limit_ns, exec_cap,
    mem_budget_bytes, max_nodes, max_edges, steal_backoff_ns, keep_idle, hand_batch)."""

    def __init__(self, arena_bytes: int = 1 << 30, stream=None, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        B.load()
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device="cuda")
        o = B.tg_ctx_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        self.ctx = B.tg_ctx_create(self.arena.data_ptr(), int(arena_bytes), self.stream.cuda_stream, o)

    # -- graphs -----------------------------------------------------------
    def create(self, kinds, params, src, dst, seed=0, weak=None, name="", device_pack=False):
        """device_pack: ingest, validate and pack on the device (tg_graph_create_dev)."""
        fn = B.tg_graph_create_dev if device_pack else B.tg_graph_create
        st, h = fn(self.ctx, kinds, params, src, dst, seed, weak)
        if st != B.TG_OK:
            raise B.TgError(st, f"{fn.__name__} {name}")
        return GraphHandle(self, h, len(kinds), len(src), name)

    def graph(self, g, weak=None, modules=None, device_pack=False):
        """Upload a workloads.Graph-like object (kinds, params, src, dst, seed).
        modules: {task: GraphHandle} naming the graph each TG_MODULE task composes.
        device_pack: ingest, validate and pack on the device (no modules)."""
        if modules is None:
            return self.create(g.kinds, g.params, g.src, g.dst, g.seed, weak, getattr(g, "name", ""), device_pack)
        st, h = B.tg_graph_create_composed(self.ctx, g.kinds, g.params, g.src, g.dst,
                                           {v: gh.handle for v, gh in modules.items()}, g.seed, weak)
        if st != B.TG_OK:
            raise B.TgError(st, f"tg_graph_create_composed {getattr(g, 'name', '')}")
        return GraphHandle(self, h, len(g.kinds), len(g.src), getattr(g, "name", ""))

    def autotune(self, gh: GraphHandle, trials=2, cache_path=None):
        """Pick and keep the fastest launch geometry for gh (tg_graph_autotune)."""
        st, chosen, ns = B.tg_graph_autotune(self.ctx, gh.handle, trials, cache_path)
        if st != B.TG_OK:
            raise B.TgError(st, "tg_graph_autotune")
        return chosen, ns

    def instance(self, gh: GraphHandle) -> GraphHandle:
        """Another execution instance of gh (own state, shared packed form)."""
        st, h = B.tg_instance_create(self.ctx, gh.handle)
        if st != B.TG_OK:
            raise B.TgError(st, "tg_instance_create")
        return GraphHandle(self, h, gh.n, gh.m, gh.name)

    # -- serving ------------------------------------------------------------
    def serve_start(self, time_limit_ns=0):
        st = B.tg_serve_start(self.ctx, time_limit_ns)
        if st != B.TG_OK:
            raise B.TgError(st, "tg_serve_start")

    def serve_stop(self) -> int:
        return B.tg_serve_stop(self.ctx)

    def serve_replay(self, templates, which, arrival_ns, keep=False):
        """Run a request trace through the server; see tg_serve_replay."""
        st, lat, sts, peak, kept = B.tg_serve_replay(self.ctx, [t.handle for t in templates], which,
                                                     arrival_ns, keep)
        if kept is not None:
            kept = [GraphHandle(self, h, templates[wi].n, templates[wi].m, templates[wi].name) if h else None
                    for h, wi in zip(kept, which)]
        return st, lat, sts, peak, kept

    def run(self, gh: GraphHandle) -> int:
        return B.tg_run(self.ctx, gh.handle)

    def submit(self, gh: GraphHandle) -> int:
        st, t = B.tg_submit(self.ctx, gh.handle)
        if st != B.TG_OK:
            raise B.TgError(st, "tg_submit")
        return t

    def poll(self, ticket) -> int:
        return B.tg_poll(self.ctx, ticket)

    def wait(self, ticket) -> int:
        return B.tg_wait(self.ctx, ticket)

    def cancel(self):
        return B.tg_cancel(self.ctx)

    def result(self, gh: GraphHandle):
        return B.tg_result_copy(self.ctx, gh.handle, gh.n)

    def batch(self, graphs) -> Batch:
        st, h = B.tg_batch_create(self.ctx, [g.handle for g in graphs])
        if st != B.TG_OK:
            raise B.TgError(st, "tg_batch_create")
        return Batch(self, h, graphs)

    def run_batch(self, graphs):
        return B.tg_run_batch(self.ctx, [g.handle for g in graphs])

    # -- measurement --------------------------------------------------------
    def stats(self) -> dict:
        return B.tg_ctx_get_stats(self.ctx)

    def opts(self) -> dict:
        return B.tg_ctx_get_opts(self.ctx)

    def set_launch(self, **fields):
        st = B.tg_ctx_set_launch(self.ctx, **fields)
        if st != B.TG_OK:
            raise B.TgError(st, "tg_ctx_set_launch")

    def bench_payload(self, count, rounds):
        return B.tg_bench_payload(self.ctx, count, rounds)

    def bench_payload_tasks(self, ids, rounds, cnt):
        """Payload-only time of an execution multiset given as host arrays
        (task ids, rounds, execution counts), in the arrays' order."""
        t = self.torch
        dev = [t.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda() for a in (ids, rounds, cnt)]
        out = B.tg_bench_payload_tasks(self.ctx, len(ids), *(d.data_ptr() for d in dev))
        del dev
        return out

    def bench_atomics(self, count, footprint_words):
        return B.tg_bench_atomics(self.ctx, count, footprint_words)

    def bench_chain(self, hops, rounds):
        return B.tg_bench_chain(self.ctx, hops, rounds)

    def capture_run(self, gh: GraphHandle, max_streams: int):
        """Run a static DAG as the CUDA graph of Algorithm 1 (one kernel per
        task on round-robin streams); returns (status, device ns)."""
        return B.tg_capture_run(self.ctx, gh.handle, max_streams)

    def close(self):
        if self.ctx:
            B.tg_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
