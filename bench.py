"""Benchmark: device-resident task-graph execution on one B300.

Headline (`value`): the large static DAGs in plain form -- the 1,000 x 1,000
layered random DAG (in-degree U{1..8}, 16 rounds) and the 1024 x 1024
wavefront (256 rounds), 2,048,576 task executions per step.  One step = for
each graph: re-arm its state (join words, counts, digests, queues, sources),
run the persistent scheduler until every task ran, finalise the status.
Each graph runs at the launch geometry its own autotuning picked (before
timing).  Graph inputs are resident in HBM when the timed region starts; L2
(126 MB) is flushed between timed steps by writing a 512 MB buffer.

Measured in the same run and reported beside it:
  roofline  the scheduler kernel against what bounds it, the dependency
            floor of its graphs (their longest paths' payloads run back to
            back by one thread); the HBM (with DRAM traffic from an ncu
            capture), atomic and integer-ALU views beside it
  critical_path   each graph's floor against its scheduler time
  plain_single_graph  the 1,004-task looping graph: microseconds per run,
            ns/task, beside an empty launch; checked against the oracle
  condition_heavy   the 10,000-condition graph: tasks/s, the ALU and atomic
            fractions, the oracle on one core; checked against the oracle
  thief_policies  capped vs adaptive thieves (Alg. 3/6): time, failed rounds,
            and the paper's bound on wasteful steals with measured E and e_s
  critical_path_trace  per-task trace records of each headline graph read
            along its critical path: step vs wait per hop, by where each task
            was taken from
  capturer_baseline  Algorithm 1's CUDA graph of per-task kernels vs the
            persistent scheduler on static DAGs
  composition   module tasks in a loop and parallel joined subflows in one
            launch vs the host re-running the composed graph
  batched   4,096 motif graphs (33M tasks) in one CUDA-graph-captured
            persistent launch, autotuned, versus one launch + sync per graph
            and the oracle on every host core
  serving   Poisson request streams at 1k / 10k / 50k / 100k requests/s
            through the resident scheduler, request i its own graph (seed i),
            (p50 / p99 latency, tasks/s), served results checked against the
            oracle (all at 1k, 1 in 50 above), the plain form (one launch per
            request) beside it at rates it sustains, graph creation cost
  e2e       the headline workload through the C-ABI with host buffers:
            inputs copied from pinned host memory, validated and packed on
            the device (tg_graph_create_dev), submit, wait, download every
            result; each graph is ingested while the previous one runs; the
            same with the host packer (tg_graph_create) beside it

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]
                  [--small] [--batched-graphs N] [--skip-batched] [--skip-serving] [--skip-extras]

--impl reference times the oracle (the sequential CPU executor) on the
headline workload, as the comparison arm.  Prints ONE JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402

METRIC = "tasks/s and ns/task overhead, batched vs plain per-graph; serving p50/p99"
UNIT = "tasks/s"
WORKLOAD = "large static DAGs, plain form: layered 1000x1000 (d~U{1..8}, R=16) + wavefront 1024x1024 (R=256)"
SMALL = False   # --small: every section at reduced size (profiler captures; not a bench line)
BATCHED_GRAPHS = 0   # --batched-graphs: the first N graphs of the batched generator (profiler captures)
# launch geometries the headline graphs' autotuning picked, for this process only
TUNE_CACHE = os.path.join(__import__("tempfile").gettempdir(), f"tg_tune_{os.getpid()}.txt")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def _graphs():
    if SMALL:
        return [w.config2a(levels=100, width=1000), w.config2b(side=256)]
    return [w.config2a(), w.config2b()]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"),
                                          f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_baseline(graphs):
    """The oracle as it stands, one host core, over the whole headline workload."""
    import oracle
    t0 = time.perf_counter()
    execs = 0
    for g in graphs:
        r = oracle.run(g)
        assert r.status == 0
        execs += r.execs
    dt = time.perf_counter() - t0
    return {"value": execs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"full headline workload ({execs} executions) on 1 host core, {dt:.2f} s"}


def run_reference(args):
    graphs = _graphs()
    times = []
    cb = None
    for _ in range(args.steps):
        cb = _cpu_baseline(graphs)
        times.append(sum(g.n for g in graphs) / cb["value"])
    execs = sum(g.n for g in graphs)
    ms = 1000 * statistics.mean(times)
    val = execs / (ms / 1000)
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 0,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                      "data": "synthetic", "config": {"workload": WORKLOAD},
                      "cpu_baseline": cb,
                      "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------
# DRAM bytes per scheduler launch on the headline graphs, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass, full size).  They
# describe the kernel source they were taken on, so they are reported only
# while tg_kernels.cu still has that hash.
MEASURED_TRAFFIC = {
    "kernels_sha256": "1bd7644b9a978660a5343dc97203a125abf6be992341d14913111b1f4ebd5178",
    "bytes_per_launch": {"config2a": 51_790_000, "config2b": 44_320_000},
}


def measured_traffic(graphs):
    import hashlib
    src = os.path.join(ROOT, "paper_2004_10908_b300", "csrc", "tg_kernels.cu")
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    per = MEASURED_TRAFFIC["bytes_per_launch"]
    if digest != MEASURED_TRAFFIC["kernels_sha256"] or any(g.name not in per for g in graphs):
        return None
    return sum(per[g.name] for g in graphs) / len(graphs)


def algorithmic_bytes(g):
    """Graph metadata a task execution must touch: its 32-byte record read,
    8 bytes of count/digest and 4 bytes of output written, and per successor
    the 4-byte id read plus the 8-byte join word read and written."""
    return 44 * g.n + 20 * g.m


def critical_path_tasks(g):
    """Tasks on the longest path of the layered or wavefront DAG."""
    if "levels" in g.meta:
        return int(g.meta["levels"])
    return 2 * int(g.meta["side"]) - 1


def headline(ex, graphs, args, torch, B, world=1):
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = ex.stream
    handles = [ex.graph(g) for g in graphs]
    # each graph keeps the launch geometry its own autotuning picks (untimed)
    tuned = {}
    t0 = time.perf_counter()
    for h, g in zip(handles, graphs):
        chosen, _ = ex.autotune(h, trials=2, cache_path=TUNE_CACHE)
        tuned[g.name] = {k: chosen[k] for k in ("worker_blocks", "warps_per_block", "batch_max", "local_keep",
                                                "max_thieves", "thief_mode", "steal_policy", "max_steal",
                                                "steal_backoff_ns", "idle_sleep_ns", "hand_batch")}
    tuned["autotune_s"] = time.perf_counter() - t0

    def step():
        for h in handles:
            st = B.tg_submit(ex.ctx, h.handle)[0]
            if st != 0:
                raise B.TgError(st, "tg_submit")

    for _ in range(args.warmup):
        step()
        torch.cuda.synchronize()
    step_ms = []
    with ClockSampler() as clk:
        torch.cuda.synchronize()
        barrier(world)
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier(world)
    # scheduler-kernel time per graph (events around the kernel, same stream)
    per_graph = {}
    for h, g in zip(handles, graphs):
        ts = []
        for _ in range(3):
            with torch.cuda.stream(stream):
                flush.zero_()
            assert ex.run(h) == 0
            ts.append(ex.stats()["kernel_ns"])
        per_graph[g.name] = statistics.median(ts)
        out, cnt, dig, execs = ex.result(h)
        assert execs == g.n and (cnt == 1).all()
    stats = ex.stats()
    for h in handles:
        h.destroy()
    return step_ms, per_graph, clk.summary(), stats, tuned


def e2e(ex, graphs, reps, device_pack=True):
    """The user's path, as a stream of graphs through the public API: create
    (ingest, validate, pack, upload), take the tuned geometry from the tuning
    cache (no runs), submit, wait, read every result back, destroy.  As a
    user pipelines the asynchronous API, each graph is ingested while the
    previous one runs, step after step.  A step is every headline graph once
    -- ingested, uploaded, run and read back -- and its time is the stream's
    wall time over its steps.  device_pack: tg_graph_create_dev, which copies
    the inputs (held in pinned host memory, as such a user holds them) to
    the device and validates and packs them there; else tg_graph_create,
    which packs on one host core and uploads the packed graph."""
    import torch
    h2d = d2h = 0
    parts = {"create_pack": 0.0, "create_upload": 0.0, "create_other": 0.0, "wait": 0.0, "read_back": 0.0,
             "other": 0.0}
    keep = []
    inputs = []
    for g in graphs:
        if not device_pack:
            inputs.append(g)
            continue
        class _Pinned:
            pass
        p = _Pinned()
        for k in ("kinds", "params", "src", "dst"):
            t = torch.from_numpy(np.ascontiguousarray(getattr(g, k))).pin_memory()
            keep.append(t)
            setattr(p, k, t.numpy())
        p.seed, p.name = g.seed, g.name
        inputs.append(p)

    def finish(gh, ticket):
        t1 = time.perf_counter()
        assert ex.wait(ticket) == 0
        t2 = time.perf_counter()
        ex.result(gh)
        t3 = time.perf_counter()
        gh.destroy()
        parts["wait"] += (t2 - t1) * 1e3
        parts["read_back"] += (t3 - t2) * 1e3

    # one untimed step first: the context's first creation and read-back
    # allocate their scratch
    for gin in inputs:
        gh = ex.graph(gin, device_pack=device_pack)
        ex.autotune(gh, cache_path=TUNE_CACHE)
        assert ex.wait(ex.submit(gh)) == 0
        ex.result(gh)
        gh.destroy()
    pending = None
    t0 = time.perf_counter()
    for _ in range(reps):
        for g, gin in zip(graphs, inputs):
            t1 = time.perf_counter()
            gh = ex.graph(gin, device_pack=device_pack)
            inf = gh.info()
            dt = (time.perf_counter() - t1) * 1e3
            parts["create_pack"] += inf["pack_ns"] / 1e6
            parts["create_upload"] += inf["upload_ns"] / 1e6
            parts["create_other"] += dt - (inf["pack_ns"] + inf["upload_ns"]) / 1e6
            ex.autotune(gh, cache_path=TUNE_CACHE)
            # queued behind the previous graph's run, whose results are then
            # read while this one runs
            ticket = ex.submit(gh)
            if pending is not None:
                finish(*pending)
            pending = (gh, ticket)
            if device_pack:
                # copied per graph: kinds, parameters, sources and targets of
                # the edges; back: the validation words, then the outputs and
                # the packed count/digest words
                h2d += g.n * 5 + g.m * 8
                d2h += 16 + g.n * 4 + g.n * 8
            else:
                # copied per graph: successor lists and sources, task records,
                # chunk table, descriptor; back: outputs and the packed
                # count/digest words
                h2d += g.m * 4 + g.n * 4 + 32 * g.n + 64 + ((g.n + 255) // 256) * 4
                d2h += g.n * 4 + g.n * 8
    finish(*pending)
    total = (time.perf_counter() - t0) * 1e3 / reps
    parts = {k: v / reps for k, v in parts.items()}
    parts["other"] = total - sum(parts.values())
    return total, h2d // reps, d2h // reps, parts


def _same_as_oracle(res, ref):
    out, cnt, dig, execs = res
    return bool(ref.status == 0 and (out == ref.out).all() and (cnt == ref.cnt).all() and (dig == ref.dig).all()
                and execs == ref.execs)


def plain_single_graph(Executor, torch, B):
    """The plain single graph (1,004 tasks: a 10 x 100 layered body, 64
    rounds, looped 5 times by one loop condition; 5,012 executions): device
    time of one whole run (re-arm, scheduler, finalise) and the host's
    submit-to-result wall time, per task, beside the cost of an empty kernel
    launch + synchronisation; results checked against the oracle."""
    import oracle
    g = w.config1()
    t0 = time.perf_counter()
    ref = oracle.run(g)
    oracle_s = time.perf_counter() - t0
    with Executor(arena_bytes=256 << 20) as ex:
        h = ex.graph(g)
        chosen, _ = ex.autotune(h, trials=3)
        dev, wall, kern = [], [], []
        for _ in range(25):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t1 = time.perf_counter()
            e0.record(ex.stream)
            st, tk = B.tg_submit(ex.ctx, h.handle)
            e1.record(ex.stream)
            assert st == 0 and ex.wait(tk) == 0
            wall.append((time.perf_counter() - t1) * 1e6)
            # the ticket completes when the run's status reaches the host,
            # which can be before the stream has passed the end event
            e1.synchronize()
            dev.append(e0.elapsed_time(e1) * 1e3)
            kern.append(ex.stats()["kernel_ns"] / 1e3)
        ok = _same_as_oracle(ex.result(h), ref)
        # an empty kernel launch + synchronisation on the same stream
        empty = []
        for _ in range(25):
            t1 = time.perf_counter()
            ex.bench_chain(0, 0)
            empty.append((time.perf_counter() - t1) * 1e6)
        floor_ns = min(ex.bench_chain(5 * 12 + 1, 64)[0] for _ in range(3))
        h.destroy()
    d, wl, k = statistics.median(dev[3:]), statistics.median(wall[3:]), statistics.median(kern[3:])
    return {"workload": "plain single graph: I -> H -> 10 x 100 layered body (d~U{1..4}, 64 rounds) -> loop "
                        "condition (5 passes) -> [H, D]; seed 0",
            "tasks": g.n, "executions": ref.execs, "device_us": d, "scheduler_us": k, "wall_us": wl,
            "ns_per_task_device": d * 1e3 / ref.execs, "ns_per_task_wall": wl * 1e3 / ref.execs,
            "tasks_s_device": ref.execs / (d * 1e-6),
            "empty_launch_sync_us": statistics.median(empty[3:]),
            "dependency_floor_us": floor_ns / 1e3, "critical_path_tasks": 61,
            "floor_frac": floor_ns / 1e3 / k,
            "launch_geometry": {kk: chosen[kk] for kk in ("worker_blocks", "warps_per_block", "batch_max", "local_keep",
                                                         "keep_idle", "hand_batch", "thief_mode")},
            "oracle_match": ok, "oracle_1core_us": oracle_s * 1e6}


def condition_heavy(Executor, torch, peaks, atom_ceiling):
    """The condition-heavy graph: exactly 10,000 condition tasks in lanes of
    loops nested 3 deep, branch conditions over 2-4 arms, 100-task bodies,
    32 rounds (522,764 tasks, 106.5 M executions), at its autotuned launch
    geometry.  Device time, tasks/s,
    the payload-only ALU ceiling on the same execution count at 32 rounds,
    the release atomics per second against the measured atomic ceiling, the
    oracle on one host core, and an element-by-element check."""
    import oracle
    g = w.config3()
    t0 = time.perf_counter()
    ref = oracle.run(g)
    oracle_s = time.perf_counter() - t0
    with Executor(arena_bytes=1 << 30) as ex:
        h = ex.graph(g)
        # its own launch geometry, as the headline graphs get theirs
        t_tune = time.perf_counter()
        tuned, _ = ex.autotune(h, trials=1)
        tune_s = time.perf_counter() - t_tune
        ts = []
        for _ in range(3):
            assert ex.run(h) == 0
            ts.append(ex.stats()["kernel_ns"])
        ok = _same_as_oracle(ex.result(h), ref)
        sched_ns = statistics.median(ts)
        pay_ns, _ = ex.bench_payload(int(ref.execs), 32)
        h.destroy()
    # atomics per execution: one join-word atomic per strong edge whose target
    # has another strong in-edge, one in-flight-flag atomic per activation,
    # one join-word re-arm per activation of a task with strong in-degree > 1
    cond = (g.kinds >= 1) & (g.kinds <= 3)
    sin = np.bincount(g.dst[~cond[g.src]].astype(np.int64), minlength=g.n)
    joins = np.zeros(g.n, np.int64)
    strong_e = ~cond[g.src]
    np.add.at(joins, g.src[strong_e].astype(np.int64), (sin[g.dst[strong_e]] > 1).astype(np.int64))
    cnt = ref.cnt.astype(np.int64)
    atomics = int((cnt * joins).sum() + cnt.sum() + (cnt * (sin > 1)).sum())
    alu_peak = 148 * 64 * peaks.get("sm_max_mhz", 2032.0) * 1e6
    return {"workload": "condition-heavy: 10,000 condition tasks, loops nested 3 deep, branch over k in {2,3,4} "
                        "arms, 10 x 10 bodies (d~U{1..4}), 32 rounds; seed 3",
            "tasks": g.n, "edges": g.m, "executions": ref.execs, "sched_ms": sched_ns / 1e6,
            "launch_geometry": {k: tuned[k] for k in ("worker_blocks", "warps_per_block", "batch_max", "local_keep",
                                                      "max_thieves", "steal_policy", "max_steal", "keep_idle",
                                                      "hand_batch", "steal_backoff_ns", "idle_sleep_ns")},
            "autotune_s": tune_s,
            "tasks_s": ref.execs / (sched_ns * 1e-9), "ns_per_task": sched_ns / ref.execs,
            "payload_only_ms": pay_ns / 1e6, "alu_frac_of_payload_ceiling": pay_ns / sched_ns,
            "alu_frac_of_int_peak": 9 * 32 * ref.execs / (sched_ns * 1e-9) / alu_peak,
            "atomics": atomics, "atomics_per_s": atomics / (sched_ns * 1e-9), "atomic_ceiling_per_s": atom_ceiling,
            "atomic_frac": atomics / (sched_ns * 1e-9) / atom_ceiling,
            "oracle_match": ok, "oracle_1core_s": oracle_s, "oracle_1core_tasks_s": ref.execs / oracle_s}


def creation_cost(Executor):
    """Cost of graph creation the way the paper's Table 3 reports it
    (time per task and per edge, amortised over many): validation + packing
    of 1,000,000 tasks without edges, then of the same tasks with 8,000,000
    edges (each task 8 successors in the next 1,000-task level); the
    difference over the edge count is the cost per edge.  The upload to the
    device is reported apart.  Host packer (tg_graph_create), then the
    device path (tg_graph_create_dev)."""
    n, width, deg = 1_000_000, 1000, 8
    rng = np.random.default_rng(7)
    v = np.arange(n - width, dtype=np.int64)
    src = np.repeat(v, deg)
    dst = ((v // width + 1) * width)[:, None] + rng.integers(0, width, (v.shape[0], deg))
    kinds = np.zeros(n, np.uint8)
    params = np.full(n, 16, np.uint32)
    import torch

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()

    rows = {}
    with Executor(arena_bytes=2 << 30) as ex:
        for dev in (False, True):
            for name, s_, d_ in (("tasks", np.zeros(0, np.uint32), np.zeros(0, np.uint32)),
                                 ("tasks_edges", src.astype(np.uint32), dst.reshape(-1).astype(np.uint32))):
                ins = [kinds, params, s_, d_]
                if dev:
                    ins = [pinned(a) for a in ins]
                    keep, ins = ins, [t.numpy() for t in ins]
                best = None
                for _ in range(3):
                    h = ex.create(*ins, 0, name=name, device_pack=dev)
                    inf = h.info()
                    h.destroy()
                    if best is None or inf["pack_ns"] < best["pack_ns"]:
                        best = inf
                rows[(dev, name)] = (best, int(s_.shape[0]))

    def per(dev):
        t, te = rows[(dev, "tasks")][0], rows[(dev, "tasks_edges")][0]
        m = rows[(dev, "tasks_edges")][1]
        return {"pack_ns_per_task": t["pack_ns"] / n, "pack_ns_per_edge": (te["pack_ns"] - t["pack_ns"]) / m,
                "upload_ns_per_task": t["upload_ns"] / n,
                "upload_ns_per_edge": (te["upload_ns"] - t["upload_ns"]) / m}

    out = {"tasks": n, "edges": rows[(False, "tasks_edges")][1], **per(False),
           "paper": "61 ns/task, 14 ns/edge (Table 3, one host thread of a 40-core machine)"}
    # tg_graph_create_dev: device time of validation + pack, and of the
    # input copies from pinned host memory
    out["device_pack"] = per(True)
    return out


def thief_policies(Executor):
    """Fixed cap of 16 thieves vs the adaptive invariant (Alg. 3/6) on the
    plain single graph (config 1) and the two large DAGs: scheduler time and
    the polling each wastes (steal rounds that found nothing)."""
    graphs = [w.config1(), w.config2a(), w.config2b()]
    out = {}
    for mode in (0, 1):
        with Executor(arena_bytes=4 << 30, thief_mode=mode) as ex:
            for g in graphs:
                h = ex.graph(g)
                rows = []
                for _ in range(3):
                    assert ex.run(h) == 0
                    s = ex.stats()
                    rows.append((s["kernel_ns"], s["failed_rounds"], s["parks"], s["peak_thieves"],
                                 s["round_cycles"], s["worker_blocks"]))
                # the longest task's execution time: one payload of the
                # graph's largest round count (a chain of 200, per hop)
                R = int(g.params.max() & 0xFFFF)
                E_ns = ex.bench_chain(200, R)[0] / 200.0
                h.destroy()
                rows.sort()
                ns, failed, parks, peak, rcyc, W = rows[1]
                out.setdefault(g.name, {})["adaptive" if mode else "capped16"] = {
                    "sched_ms": ns / 1e6, "failed_rounds": failed, "failed_rounds_per_ms": failed / (ns / 1e6),
                    "parks": parks, "peak_thieves": peak,
                    "theorem3": theorem3_bound(ns, failed, rcyc, W, E_ns)}
    return out


def theorem3_bound(run_ns, failed_rounds, round_cycles, workers, E_ns, clock_mhz=2032.0):
    """The paper's bound on wasteful steals (Analysis, third theorem): at any
    moment at most MAX_STEALS x (|W| + |D| E / e_s) of them, with W the
    workers (here the worker blocks), one domain, E the longest task and e_s
    one steal round.  Counted in steal rounds (each round holds up to
    MAX_STEALS attempts) and summed over the run's windows of length E: at
    most (|W| + E / e_s) x ceil(T / E) failed rounds.  e_s is measured: the
    SM cycles the failed rounds took over their number."""
    e_s_ns = (round_cycles / max(1, failed_rounds)) / (clock_mhz * 1e-3)
    windows = int(np.ceil(run_ns / max(1.0, E_ns)))
    bound = (workers + E_ns / max(1e-9, e_s_ns)) * windows
    return {"E_ns": E_ns, "e_s_ns": e_s_ns, "workers": workers, "windows": windows,
            "bound_rounds": bound, "failed_rounds": failed_rounds, "holds": failed_rounds <= bound,
            "failed_over_bound": failed_rounds / bound}


def critical_path_trace(Executor, B, graphs, tuned):
    """One run of each headline graph at its tuned geometry with per-task
    trace records (TG_OPT_TRACE_TASKS: the lean scheduler variant still
    runs), read along the graph's critical path: how much of each hand-off
    is the step and how much is waiting, by where the task was taken from;
    then step by step (duration by tasks in the step and by the steps of
    the same block running at once) and level by level (layers of the
    layered DAG, anti-diagonals of the wavefront)."""
    from paper_2004_10908_b300.trace import critical_path, level_summary, step_summary
    out = {}
    with Executor(arena_bytes=4 << 30, flags=B.TG_OPT_TRACE_TASKS) as ex:
        for g in graphs:
            ex.set_launch(**tuned.get(g.name, {}))
            h = ex.graph(g)
            ts = []
            for _ in range(3):
                assert ex.run(h) == 0
                ts.append(ex.stats()["kernel_ns"] / 1e6)
            st, en, wh = B.tg_trace_copy(ex.ctx, h.handle, g.n)
            r = critical_path(g.src, g.dst, st, en, wh)
            r["traced_sched_ms"] = statistics.median(ts)
            r["steps"] = step_summary(st, en, wh)
            ids = np.arange(g.n, dtype=np.int64)
            if "width" in g.meta:
                r["levels"] = level_summary(ids // g.meta["width"], g.src, g.dst, st, en, wh)
            elif "side" in g.meta:
                r["levels"] = level_summary(ids // g.meta["side"] + ids % g.meta["side"], g.src, g.dst, st, en, wh)
            out[g.name] = r
            h.destroy()
            ex.set_launch()
    return out


def capturer_baseline(Executor, torch, B):
    """Algorithm 1's form (one kernel per task in a CUDA graph over
    round-robin streams) against the persistent scheduler on static DAGs:
    the plain single graph's body (10 x 100, in-degree 1-4, 64 rounds) and a
    wider one (20 x 1,000, in-degree 1-8, 16 rounds).  Whole runs (re-arm
    included) on the device clock."""
    out = []
    for g in (w.config2a(seed=0, levels=10, width=100, d_lo=1, d_hi=4, rounds=64),
              w.config2a(seed=1, levels=20, width=1000, d_lo=1, d_hi=8, rounds=16)):
        with Executor(arena_bytes=1 << 30) as ex:
            h = ex.graph(g)
            ref = None
            ts = []
            for _ in range(6):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(ex.stream)
                st, t = B.tg_submit(ex.ctx, h.handle)
                e1.record(ex.stream)
                assert st == 0 and ex.wait(t) == 0
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ref = ex.result(h)
            row = {"graph": f"layered {g.meta['levels']} x {g.meta['width']}, R={int(g.params[0] & 0xFFFF)}",
                   "tasks": g.n, "persistent_ms": statistics.median(ts[1:]), "cuda_graph_ms": {}}
            for k in (1, 4, 32):
                t0 = time.perf_counter()
                st, _ = ex.capture_run(h, k)
                build_s = time.perf_counter() - t0
                assert st == 0
                ns = sorted(ex.capture_run(h, k)[1] for _ in range(5))[2]
                got = ex.result(h)
                assert all((np.asarray(a) == np.asarray(b)).all() for a, b in zip(got[:3], ref[:3]))
                row["cuda_graph_ms"][str(k)] = {"replay_ms": ns / 1e6, "build_s": build_s}
            h.destroy()
        out.append(row)
    return out


def oracle_all_cores(graphs, what):
    """The oracle as it stands, one instance per graph over every host core
    (threads: the foreign call releases the GIL), on a bounded sample."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    res = oracle.run_many(graphs, threads=cores)
    dt = time.perf_counter() - t0
    execs = sum(int(r.execs) for r in res)
    return {"value": execs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what}: {len(graphs)} graphs, {execs} executions, {dt:.2f} s"}


def composition(Executor, torch):
    """Module tasks and joined subflows in one launch, against the host
    re-launching the same graphs: a module task entered 50 times in a loop
    (composed graph: layered 10 x 100, in-degree 1-4, 16 rounds), and 64
    subflow tasks side by side, each spawning a copy of that graph.  Root
    results are checked against the composed oracle."""
    from oracle import composed as oc
    from workloads.graphs import COND_LOOP, MODULE, STATIC, SUBFLOW, from_lists, pack_param
    body = w.config2a(seed=21, levels=10, width=100, d_lo=1, d_hi=4, rounds=16)
    T, K, R = 50, 64, 16
    loop = from_lists("module_loop", [STATIC, MODULE, COND_LOOP, STATIC],
                      [pack_param(R), pack_param(R), pack_param(R, T), pack_param(R)],
                      [(0, 1), (1, 2), (2, 1), (2, 3)])
    fan = from_lists("subflow_fan", [STATIC] + [SUBFLOW] * K + [STATIC], pack_param([R] * (K + 2)),
                     [(0, 1 + k) for k in range(K)] + [(1 + k, K + 1) for k in range(K)])
    out = {"composed_graph": "layered 10 x 100, in-degree 1-4, 16 rounds (1,000 tasks)"}
    with Executor(arena_bytes=2 << 30) as ex:
        hb = ex.graph(body)

        def dev_ms(fn):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(ex.stream)
            fn()
            e1.record(ex.stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        def run_on_stream(h):
            st, t = B_submit(ex, h)
            assert st == 0
            return t

        for name, top, mods, n_exec in (("module_loop", loop, {1: hb}, T * body.n + 2 * T + 2),
                                        ("subflow_fan", fan, {k + 1: hb for k in range(K)}, K * body.n + K + 2)):
            ht = ex.graph(top, modules=mods)
            ts = []
            for _ in range(4):
                tickets = []
                ts.append(dev_ms(lambda: tickets.append(run_on_stream(ht))))
                assert ex.wait(tickets[0]) == 0
            ref = oc.run({"b": body, "t": top}, {"t": {v: "b" for v in mods}}, "t")["t"]
            got = ex.result(ht)
            assert ref[0] == 0 and (np.asarray(got[0]) == ref[1]).all() and (np.asarray(got[1]) == ref[2]).all()
            reps = T if name == "module_loop" else K
            # wall clock, both ways: one composed run vs the host running the
            # composed graph `reps` times (launch + wait each)
            wall = []
            for _ in range(3):
                t0 = time.perf_counter()
                assert ex.run(ht) == 0
                wall.append((time.perf_counter() - t0) * 1e3)
            plain = []
            for _ in range(2):
                t0 = time.perf_counter()
                for _ in range(reps):
                    assert ex.run(hb) == 0
                plain.append((time.perf_counter() - t0) * 1e3)
            ms = statistics.median(ts[1:])
            out[name] = {"entries": reps, "executions": n_exec, "composed_device_ms": ms,
                         "tasks_s": n_exec / (ms / 1000.0), "composed_wall_ms": min(wall),
                         "host_relaunch_wall_ms": min(plain), "relaunch_over_composed": min(plain) / min(wall)}
            ht.destroy()
        hb.destroy()
    return out


def B_submit(ex, h):
    from paper_2004_10908_b300 import binding as B
    return B.tg_submit(ex.ctx, h.handle)


def batched(Executor, torch):
    """4,096 graphs in one autotuned, CUDA-graph-captured launch vs one launch each."""
    t0 = time.time()
    if BATCHED_GRAPHS:
        gs = w.config4(n_graphs=BATCHED_GRAPHS)
    else:
        gs = w.config4(n_graphs=256, n_hi=8192) if SMALL else w.config4()
    gen_s = time.time() - t0
    with Executor(arena_bytes=8 << 30, max_nodes=40_000_000, max_edges=450_000_000) as ex:
        hs = [ex.graph(g, device_pack=True) for g in gs]   # (validated and packed on the device)
        b = ex.batch(hs)
        b.launch()
        st, sts = b.wait()
        assert st == 0 and (sts == 0).all()
        execs = ex.stats()["tasks"]
        t1 = time.time()
        chosen, tuned_ns = b.autotune(trials=2)
        tune_s = time.time() - t1
        ms = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(ex.stream)
            b.launch()
            e1.record(ex.stream)
            st, sts = b.wait()
            assert st == 0
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        # the payload-only ceiling on the identical multiset of (id, iter,
        # rounds) the launch executed: in task order (lanes mixing rounds
        # U{8..512}), and sorted by work per task (a warp's lanes do equal
        # work: the ALU ceiling of this multiset)
        import oracle
        ids, rnd, cnt_all, checked, ok = [], [], [], 0, True
        for gi, (g, h) in enumerate(zip(gs, hs)):
            res = ex.result(h)
            c = res[1]
            keep = c > 0
            ids.append(np.nonzero(keep)[0].astype(np.uint32))
            rnd.append((g.params & 0xFFFF)[keep].astype(np.uint32))
            cnt_all.append(c[keep].astype(np.uint32))
            if gi % 64 == 0:   # a fixed sample checked element by element
                ok = ok and _same_as_oracle(res, oracle.run(g))
                checked += 1
        ids, rnd, cnt_all = np.concatenate(ids), np.concatenate(rnd), np.concatenate(cnt_all)
        work = rnd.astype(np.int64) * cnt_all.astype(np.int64)
        pay_task = min(ex.bench_payload_tasks(ids, rnd, cnt_all)[0] for _ in range(3))
        order = np.argsort(-work, kind="stable")
        pay_ns = min(ex.bench_payload_tasks(ids[order], rnd[order], cnt_all[order])[0] for _ in range(3))
        rounds = int(work.sum())
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for h in hs:
            assert ex.run(h) == 0
        plain_s = time.perf_counter() - t1
        b.destroy()
    best_ms = min(ms)
    n_hi = 8192 if SMALL and not BATCHED_GRAPHS else 65536
    return {"workload": f"{len(gs)} motif graphs, n log-uniform [16, {n_hi}], 5% loop conditions, rounds U{{8..512}}",
            "graphs": len(gs), "tasks": int(sum(g.n for g in gs)), "executions": int(execs),
            "batched_ms": best_ms, "batched_tasks_s": execs / (best_ms / 1000),
            "plain_s": plain_s, "plain_tasks_s": execs / plain_s,
            "batched_over_plain": (execs / (best_ms / 1000)) / (execs / plain_s),
            "ns_per_task_overhead": (best_ms * 1e6 - pay_ns) / execs,
            "payload_only_ms": pay_ns / 1e6, "payload_only_frac": (pay_ns / 1e6) / best_ms,
            "payload_only_task_order_ms": pay_task / 1e6,
            "payload_only_task_order_frac": (pay_task / 1e6) / best_ms,
            "payload_ceiling": "the executed (id, iter, rounds) multiset, one thread per task, sorted by work",
            "mean_rounds": rounds / execs,
            "oracle_checked_graphs": checked, "oracle_match": ok,
            "autotuned": {k: chosen[k] for k in ("worker_blocks", "warps_per_block", "deque_depth",
                                                 "steal_policy", "max_steal", "max_thieves", "batch_max",
                                                 "local_keep", "steal_backoff_ns", "idle_sleep_ns", "hand_batch")},
            "autotune_s": tune_s, "generate_s": gen_s,
            "cpu_all_cores": oracle_all_cores(gs[::8], "every 8th graph of the batch")}


SERVE_REQUESTS = 20_000   # request i is the serving generator's graph with seed i


def _gen_requests(ids, threads):
    """Request graphs by id, generated on host threads (the native generator
    releases the GIL), yielded in id order in chunks."""
    from concurrent.futures import ThreadPoolExecutor
    chunk = 256
    with ThreadPoolExecutor(max_workers=threads) as pool:
        nxt = None
        for c0 in range(0, len(ids), chunk):
            cur = nxt if nxt is not None else [pool.submit(w.config5_request, int(i)) for i in ids[c0:c0 + chunk]]
            c1 = c0 + chunk
            nxt = [pool.submit(w.config5_request, int(i)) for i in ids[c1:c1 + chunk]] if c1 < len(ids) else None
            for f in cur:
                yield f.result()


def _check_requests(ex, kept, ids, threads):
    """Every kept request's per-task outputs, counts and digests against the
    oracle on its own graph (regenerated from its seed).  Returns (checked,
    mismatching request ids)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    def one(i, res):
        g = w.config5_request(int(i))
        r = oracle.run(g)
        out, cnt, dig, _ = res
        ok = r.status == 0 and (out == r.out).all() and (cnt == r.cnt).all() and (dig == r.dig).all()
        return int(i), bool(ok)

    bad, checked = [], 0
    with ThreadPoolExecutor(max_workers=threads) as pool:
        for c0 in range(0, len(ids), 512):
            futs = []
            for i in ids[c0:c0 + 512]:
                futs.append(pool.submit(one, i, ex.result(kept[i])))
                kept[i].destroy()
                kept[i] = None
            for f in futs:
                i, ok = f.result()
                checked += 1
                if not ok:
                    bad.append(i)
    return checked, bad


def serving(Executor, torch):
    """Poisson request streams through the resident scheduler: request i is
    its own graph (the serving generator with seed i: n log-uniform [64,
    262,144], 5 % loop conditions, 64 rounds), registered in advance; every
    served result of the 1k req/s stream and a fixed 1-in-50 sample at 10k and
    50k req/s is compared with the oracle after the run.  Beside it: the
    plain form (one launch + sync per request) and the served form at rates
    the plain form can sustain, and the cost of creating the request graphs
    (validated and packed on the device)."""
    threads = os.cpu_count() or 1
    n_req = 400 if SMALL else SERVE_REQUESTS
    ids = np.arange(n_req)
    out = {"workload": f"{n_req} request graphs, request i = serving generator with seed i "
                       f"(n log-uniform [64, 262144], 5% loop conditions, 64 rounds)", "lambdas": []}
    # pools sized for every request graph resident at once (about 637 M task
    # slots) plus the instances kept for checking (5,000 at 1k req/s, about
    # 160 M) and those in flight; the 64 GB budget covers all of them
    with Executor(arena_bytes=(8 << 30) if SMALL else (58 << 30), max_nodes=0 if SMALL else 850_000_000,
                  max_edges=0 if SMALL else 2_600_000_000, mem_budget_bytes=64 << 30) as ex:
        t0 = time.perf_counter()
        ts, n_tasks, n_edges, n_exec, pack_ns, up_ns = [], [], [], [], [], []
        # validated and packed on the device (tg_graph_create_dev): the checks
        # of served results below then also check that path on every size
        for g in _gen_requests(ids, threads):
            h = ex.graph(g, device_pack=True)
            ts.append(h)
            inf = h.info()
            n_tasks.append(g.n)
            n_edges.append(g.m)
            # executions: every layered task once; a loop motif's head and
            # condition T times each, then one exit arm (the checked results
            # confirm the counts)
            n_exec.append(g.meta["n_d"] + int((2 * np.asarray(g.meta["trips"]) + 1).sum()))
            pack_ns.append(inf["pack_ns"])
            up_ns.append(inf["upload_ns"])
        n_tasks = np.array(n_tasks, np.float64)
        n_edges = np.array(n_edges, np.float64)
        n_exec = np.array(n_exec, np.float64)
        out["register_s"] = time.perf_counter() - t0
        out["mean_tasks"] = float(n_tasks.mean())
        out["mean_executions"] = float(n_exec.mean())
        used = sum(B_info(h)["device_bytes"] for h in ts)
        out["creation_request_graphs"] = {"path": "tg_graph_create_dev (inputs from pageable host memory)",
                                          "pack_ns_per_task_all_in": float(np.sum(pack_ns) / n_tasks.sum()),
                                          "upload_ns_per_task": float(np.sum(up_ns) / n_tasks.sum())}
        rng = w.Stream(5, 7)

        def stream(lam, count, check_every, label):
            gaps = -np.log1p(-rng.uniform(count)) / lam
            arr = (np.cumsum(gaps) * 1e9).astype(np.uint64)
            which = ids[:count].astype(np.uint32)
            mask = (np.arange(count) % check_every) == 0
            ex.serve_start(time_limit_ns=180_000_000_000)
            try:
                t1 = time.perf_counter()
                st, lat, sts, peak, kept = ex.serve_replay(ts, which, arr, keep=mask)
                wall = time.perf_counter() - t1
            finally:
                stop = ex.serve_stop()
            assert stop == 0 and st == 0 and (sts == 0).all(), (label, st, stop)
            t2 = time.perf_counter()
            checked, bad = _check_requests(ex, kept, list(np.nonzero(mask)[0]), threads)
            row = {"req_per_s": lam, "requests": count, "p50_ms": float(np.percentile(lat, 50) / 1e6),
                   "p99_ms": float(np.percentile(lat, 99) / 1e6), "mean_ms": float(lat.mean() / 1e6),
                   "tasks_s": float(n_exec[:count].sum() / wall), "max_in_flight": int(peak),
                   "completed_per_s": count / wall,
                   "checked": checked, "check": "every request" if check_every == 1 else f"1 in {check_every}",
                   "mismatches": len(bad), "mismatching_requests": bad[:10], "check_s": time.perf_counter() - t2}
            return row

        plan = ((50000, n_req, 1),) if SMALL else ((1000, 5000, 1), (10000, n_req, 50), (50000, n_req, 50),
                                                   (100000, n_req, 50))
        for lam, count, every in plan:
            out["lambdas"].append(stream(lam, count, every, f"{lam}/s"))
        # plain vs served at rates the plain form can sustain: the same
        # requests, one launch + wait each in arrival order (host clock)
        cmp = []
        for lam in (() if SMALL else (300, 500, 1000)):
            count = 1000
            gaps = -np.log1p(-rng.uniform(count)) / lam
            arr = np.cumsum(gaps) * 1e9
            lat, svc = [], []
            t1 = time.perf_counter()
            for r in range(count):
                now = (time.perf_counter() - t1) * 1e9
                if now < arr[r]:
                    time.sleep((arr[r] - now) / 1e9)
                s0 = time.perf_counter()
                assert ex.run(ts[r]) == 0
                s1 = time.perf_counter()
                svc.append(s1 - s0)
                lat.append((s1 - t1) * 1e9 - arr[r])
            lat = np.array(lat)
            served = stream(lam, count, 10, f"served {lam}/s")
            cmp.append({"req_per_s": lam, "requests": count,
                        "plain_p50_ms": float(np.percentile(lat, 50) / 1e6),
                        "plain_p99_ms": float(np.percentile(lat, 99) / 1e6),
                        "plain_mean_service_ms": 1e3 * float(np.mean(svc)),
                        "served_p50_ms": served["p50_ms"], "served_p99_ms": served["p99_ms"],
                        "served_mismatches": served["mismatches"], "served_checked": served["checked"]})
        out["plain_vs_served"] = cmp
        if cmp:
            svc_ms = float(np.mean([c["plain_mean_service_ms"] for c in cmp]))
            out["plain_capacity_req_s"] = 1e3 / svc_ms
        out["budget"] = {"bytes": 64 << 30, "templates_bytes": int(used),
                         "binds": False,
                         "note": "the requests in flight (at most max_in_flight instances of about 36 B per "
                                 "task) never approach the budget left after the registered graphs; "
                                 "admission is limited by arrivals, and by the budget only in the "
                                 "budget test"}
        for h in ts:
            h.destroy()
    if not SMALL:
        out["cpu_all_cores"] = oracle_all_cores([w.config5_request(i) for i in range(256)],
                                                "request graphs 0..255, once each")
    return out


def B_info(h):
    from paper_2004_10908_b300 import binding as B
    return B.tg_graph_get_info(h.handle)


# ---------------------------------------------------------------------------
# ranks: N independent replicas (one per GPU), no data-path collective; the
# timed region is bracketed by barriers and its time is the max over ranks
# ---------------------------------------------------------------------------
def rank_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def init_ranks(world, backend="nccl"):
    """One process group over the replicas (NCCL on GPUs, gloo on CPU)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank_step, world, ms_per_step):
    """Units all ranks processed per second, with the slowest rank's time."""
    return units_per_rank_step * world / (ms_per_step / 1000.0)


def run_b300(args):
    import torch

    from paper_2004_10908_b300 import Executor
    from paper_2004_10908_b300 import binding as B

    rank, world = rank_world()
    init_ranks(world)
    graphs = _graphs()
    execs_per_step = sum(g.n for g in graphs)   # static DAGs: every task runs once
    peaks, peak_kind = _peaks()

    ex = Executor(arena_bytes=(512 << 20) if SMALL else (4 << 30))
    step_ms, per_graph, clocks, stats, tuned = headline(ex, graphs, args, torch, B, world)
    tot_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = tot_ms / args.steps
    value = whole_job_value(execs_per_step, world, ms_per_step)

    # roofline of the dominant kernel (the scheduler): graph-metadata bytes
    # per launch over its average launch time, against the measured HBM copy
    # bandwidth; beside it the integer-ALU view and the atomic ceiling
    sched_ns = sum(per_graph.values())
    n_launch = len(graphs)
    alg_bytes = sum(algorithmic_bytes(g) for g in graphs)
    achieved_gbs = (alg_bytes / n_launch) / (sched_ns / n_launch * 1e-9) / 1e9
    rounds_total = sum(int((g.params & 0xFFFF).astype(np.int64).sum()) for g in graphs)
    alu_peak = 148 * 64 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    alu_achieved = 9 * rounds_total / (sched_ns * 1e-9) / 1e12
    pay_ns = 0
    for g in graphs:
        ns, _ = ex.bench_payload(g.n, int(g.params[0] & 0xFFFF))
        pay_ns += ns
    # the dependency floor: the payloads along each graph's longest path run
    # back to back by one thread, with no scheduling at all
    crit = {}
    for g in graphs:
        hops = critical_path_tasks(g)
        floor_ns = min(ex.bench_chain(hops, int(g.params[0] & 0xFFFF))[0] for _ in range(3))
        crit[g.name] = {"path_tasks": hops, "floor_ms": floor_ns / 1e6, "sched_ms": per_graph[g.name] / 1e6,
                        "frac": floor_ns / per_graph[g.name],
                        "overhead_us_per_hop": (per_graph[g.name] - floor_ns) / 1e3 / hops}
    # random returning atomics over a footprint the arena's scratch holds
    atom_count, atom_words = (1 << 24, 1 << 20) if SMALL else (1 << 26, 1 << 24)
    atom_ns = ex.bench_atomics(atom_count, atom_words)
    atom_ceiling = atom_count / (atom_ns * 1e-9)
    # join-word atomics: one per edge into a task with another strong
    # in-edge (a sole in-edge needs none; launches without condition tasks
    # set no in-flight flags and re-arm nothing), plus two pending-count
    # updates per warp step
    joins = 0
    for g in graphs:
        sin = np.bincount(g.dst.astype(np.int64), minlength=g.n)
        joins += int((sin[g.dst.astype(np.int64)] > 1).sum())
    atomics_per_launch = joins + 2 * stats["warp_iters"]
    e2e_ms, h2d, d2h, e2e_parts = e2e(ex, graphs, max(3, min(args.steps, 6)))
    e2e_host_ms, _, _, e2e_host_parts = e2e(ex, graphs, 3, device_pack=False)
    ex.close()
    floor_ns = sum(c["floor_ms"] for c in crit.values()) * 1e6
    hbm_peak = peaks.get("hbm_gbs", 6400.0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "graphs": [g.name for g in graphs], "tasks_per_step": execs_per_step,
                   "l2": "flushed between steps (512 MB write)", "launch_geometry": tuned},
        "e2e": {"value": execs_per_step / (e2e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "host_ms_per_step": e2e_parts,
                "create": "tg_graph_create_dev (ingest, validation and pack on the device, inputs in pinned "
                          "host memory)",
                "host_pack": {"value": execs_per_step / (e2e_host_ms / 1000.0), "ms_per_step": e2e_host_ms,
                              "host_ms_per_step": e2e_host_parts,
                              "create": "tg_graph_create (packed on one host core, then uploaded)"}},
        # the scheduler kernel is bound by its graphs' dependency chains: the
        # ceiling is every graph at its dependency floor (its longest path's
        # payloads back to back, measured in the same run); the bandwidth,
        # atomic and integer-ALU views stay far from theirs
        "roofline": {"bound": "dependency", "unit": "tasks/s",
                     "achieved": execs_per_step / (sched_ns * 1e-9),
                     "peak": execs_per_step / (floor_ns * 1e-9), "frac": floor_ns / sched_ns,
                     "per_graph_frac": {k: v["frac"] for k, v in crit.items()},
                     "peak_kind": "measured dependency floor (same run)",
                     "traffic": None if SMALL else measured_traffic(graphs),
                     "views": {
                         "hbm": {"achieved_gbs": achieved_gbs, "peak_gbs": hbm_peak, "frac": achieved_gbs / hbm_peak,
                                 "peak_kind": peak_kind,
                                 "bytes": "44 B/task + 20 B/edge of graph metadata per launch"},
                         "atomics": {"achieved_per_s": atomics_per_launch / (sched_ns * 1e-9),
                                     "ceiling_per_s": atom_ceiling,
                                     "frac": atomics_per_launch / (sched_ns * 1e-9) / atom_ceiling},
                         "alu": {"achieved_tops": alu_achieved, "peak_tops": alu_peak,
                                 "frac": alu_achieved / alu_peak, "payload_only_ms": pay_ns / 1e6,
                                 "payload_only_frac": pay_ns / sched_ns}},
                     "note": "traffic = DRAM bytes per launch (ncu, mean of the two graphs) for the kernel source "
                             "it was taken on, else null"},
        "ns_per_task_overhead": (sched_ns - pay_ns) / execs_per_step,
        "per_graph_sched_ms": {k: v / 1e6 for k, v in per_graph.items()},
        "critical_path": crit,
        "scheduler_stats": {k: stats[k] for k in ("steal_attempts", "steal_hits", "spills", "warp_iters",
                                                  "pops_hand", "pops_local")},
        "gpu_launches": 3 * len(graphs) * args.steps,
        "clocks": clocks,
    }
    # the single-GPU comparisons and the CPU baseline: rank 0 only.  A
    # section that fails is reported as such in the line (its assertion or
    # error text); the headline above does not depend on it.
    def section(name, fn, *a):
        try:
            line[name] = fn(*a)
        except Exception as ex_:   # noqa: BLE001 -- recorded, not hidden
            log(f"section {name} failed: {ex_!r}")
            line[name] = {"error": repr(ex_)[:400]}

    if rank == 0 and not SMALL and not args.skip_extras:
        section("plain_single_graph", plain_single_graph, Executor, torch, B)
        section("creation", creation_cost, Executor)
        section("condition_heavy", condition_heavy, Executor, torch, peaks, atom_ceiling)
        section("thief_policies", thief_policies, Executor)
        section("critical_path_trace", critical_path_trace, Executor, B, graphs, tuned)
        section("capturer_baseline", capturer_baseline, Executor, torch, B)
        section("composition", composition, Executor, torch)
    if rank == 0 and not args.skip_batched:
        section("batched", batched, Executor, torch)
    if rank == 0 and not args.skip_serving:
        section("serving", serving, Executor, torch)
    if rank == 0:
        line["cpu_baseline"] = _cpu_baseline(graphs)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--small", action="store_true",
                    help="every section small: layered 100x1000 + wavefront 256x256, 256 batched graphs, "
                         "400 served requests (profiler captures; not a bench line)")
    ap.add_argument("--batched-graphs", type=int, default=0,
                    help="batched section over the first N graphs of the full-size generator "
                         "(profiler captures of a mid-size batch; not a bench line)")
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--skip-serving", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="leave out the thief-policy and capturer-baseline comparisons")
    args = ap.parse_args()
    global SMALL, BATCHED_GRAPHS
    SMALL = args.small
    BATCHED_GRAPHS = max(0, args.batched_graphs)
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args)
    else:
        run_b300(args)


if __name__ == "__main__":
    main()
