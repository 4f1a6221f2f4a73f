"""ORACLE (test infrastructure): ctypes access to the sequential CPU executor
in tg_oracle.c.  Only tests, the smoke check and the benchmark's CPU-baseline
leg use this package; it imports nothing from the CUDA path.

Status codes mirror the meaning of the library's codes by name (OK, INVALID,
NO_SOURCE, EDGE_KIND, RACE, EXEC_LIMIT) without sharing any header with it.
"""
from __future__ import annotations

import ctypes
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from .build import build

OK, INVALID, NO_SOURCE, EDGE_KIND, RACE, EXEC_LIMIT, NOMEM = 0, -1, -2, -3, -5, -6, -10
STATUS_NAMES = {OK: "OK", INVALID: "INVALID", NO_SOURCE: "NO_SOURCE", EDGE_KIND: "EDGE_KIND",
                RACE: "RACE", EXEC_LIMIT: "EXEC_LIMIT", NOMEM: "NOMEM"}
DEFAULT_EXEC_CAP = 1 << 31

_lib = None
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_mix32.restype = ctypes.c_uint32
        L.orc_mix32.argtypes = [ctypes.c_uint32]
        L.orc_payload.restype = ctypes.c_uint32
        L.orc_payload.argtypes = [ctypes.c_uint32] * 4
        L.orc_cond_hash.restype = ctypes.c_uint32
        L.orc_cond_hash.argtypes = [ctypes.c_uint32] * 3
        L.orc_condition_index.restype = ctypes.c_int32
        L.orc_condition_index.argtypes = [ctypes.c_uint32] * 6
        L.orc_run.restype = ctypes.c_int
        L.orc_run.argtypes = [ctypes.c_uint32, _u8p, _u32p, ctypes.c_uint32, _u32p, _u32p, _u8p,
                              ctypes.c_uint32, ctypes.c_uint64, _u32p, _u32p, _u32p,
                              ctypes.POINTER(ctypes.c_uint64)]
        L.orc_payload_many.restype = None
        L.orc_payload_many.argtypes = [ctypes.c_uint64, _u32p, _u32p, _u32p, _u32p, _u32p]
        L.orc_mix32_many.restype = None
        L.orc_mix32_many.argtypes = [ctypes.c_uint64, _u32p, _u32p]
        _lib = L
    return _lib


def _p32(a):
    return a.ctypes.data_as(_u32p)


def _p8(a):
    return a.ctypes.data_as(_u8p)


def mix32(x: int) -> int:
    return lib().orc_mix32(x & 0xFFFFFFFF)


def payload(task_id: int, it: int, insum: int, rounds: int) -> int:
    return lib().orc_payload(task_id & 0xFFFFFFFF, it & 0xFFFFFFFF, insum & 0xFFFFFFFF, rounds)


def cond_hash(seed: int, task_id: int, it: int) -> int:
    return lib().orc_cond_hash(seed & 0xFFFFFFFF, task_id & 0xFFFFFFFF, it & 0xFFFFFFFF)


def condition_index(kind: int, param: int, seed: int, task_id: int, it: int, nsucc: int) -> int:
    return lib().orc_condition_index(kind, param & 0xFFFFFFFF, seed & 0xFFFFFFFF, task_id, it, nsucc)


def payload_many(ids, iters, insums, rounds) -> np.ndarray:
    ids, iters, insums, rounds = (np.ascontiguousarray(a, dtype=np.uint32) for a in (ids, iters, insums, rounds))
    out = np.empty(ids.shape[0], np.uint32)
    lib().orc_payload_many(ids.shape[0], _p32(ids), _p32(iters), _p32(insums), _p32(rounds), _p32(out))
    return out


def mix32_many(xs) -> np.ndarray:
    xs = np.ascontiguousarray(xs, dtype=np.uint32)
    out = np.empty(xs.shape[0], np.uint32)
    lib().orc_mix32_many(xs.shape[0], _p32(xs), _p32(out))
    return out


@dataclass
class Result:
    status: int
    out: np.ndarray
    cnt: np.ndarray
    dig: np.ndarray
    execs: int


def run_arrays(kinds, params, src, dst, seed, weak=None, exec_cap=DEFAULT_EXEC_CAP) -> Result:
    kinds = np.ascontiguousarray(kinds, dtype=np.uint8)
    params = np.ascontiguousarray(params, dtype=np.uint32)
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    n, m = kinds.shape[0], src.shape[0]
    out = np.zeros(n, np.uint32)
    cnt = np.zeros(n, np.uint32)
    dig = np.zeros(n, np.uint32)
    ex = ctypes.c_uint64(0)
    wp = None
    if weak is not None:
        weak = np.ascontiguousarray(weak, dtype=np.uint8)
        wp = _p8(weak)
    st = lib().orc_run(n, _p8(kinds), _p32(params), m, _p32(src), _p32(dst), wp, seed & 0xFFFFFFFF,
                       exec_cap, _p32(out), _p32(cnt), _p32(dig), ctypes.byref(ex))
    return Result(st, out, cnt, dig, ex.value)


def run(g, exec_cap=DEFAULT_EXEC_CAP, weak=None) -> Result:
    """Run a workloads.Graph (any object with kinds/params/src/dst/seed)."""
    return run_arrays(g.kinds, g.params, g.src, g.dst, g.seed, weak=weak, exec_cap=exec_cap)


def run_many(graphs, threads=None, exec_cap=DEFAULT_EXEC_CAP):
    """Run independent graphs on `threads` host threads (ctypes releases the
    GIL during the foreign call, so the runs proceed in parallel)."""
    threads = threads or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda g: run(g, exec_cap), graphs))
