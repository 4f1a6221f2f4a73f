"""The C-ABI library loads and exports every entry point include/tg.h
declares; the binding declares a signature for each (no GPU needed)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tg_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2004_10908_b300 import _build, binding
    lib = _build.build()
    declared = _declared()
    assert len(declared) >= 20
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib], text=True)
    exported = set(re.findall(r"\bT (tg_\w+)", out))
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    L = binding.load(lib)
    for d in declared:
        assert hasattr(L, d)
        assert d in binding.SIGNATURES, d


def test_strerror_without_gpu():
    from paper_2004_10908_b300 import binding
    assert binding.tg_strerror(0) == "ok"
    assert "race" in binding.tg_strerror(binding.TG_ERR_RACE)
    assert binding.tg_strerror(12345) == "unknown status"


def test_ctx_create_rejects_bad_arguments_without_touching_a_gpu():
    from paper_2004_10908_b300 import binding
    L = binding.load()
    import ctypes
    out = ctypes.c_void_p()
    # NULL arena and a misaligned arena are rejected before any CUDA call
    assert L.tg_ctx_create(None, 1 << 20, None, None, ctypes.byref(out)) == binding.TG_ERR_INVALID
    assert L.tg_ctx_create(ctypes.c_void_p(0x1001), 1 << 20, None, None, ctypes.byref(out)) == binding.TG_ERR_INVALID
    assert L.tg_graph_create(None, 0, None, None, 0, None, None, None, 0, ctypes.byref(out)) == binding.TG_ERR_INVALID


def test_null_arguments_are_refused_without_touching_the_device():
    """Every entry point that takes a context, graph or batch handle refuses
    a null one with TG_ERR_INVALID before any CUDA call (runs without a GPU)."""
    import ctypes
    from paper_2004_10908_b300 import binding as B
    L = B.load()
    u64 = ctypes.c_uint64(0)
    out = ctypes.c_void_p()
    INV = B.TG_ERR_INVALID
    assert L.tg_ctx_create(None, 1 << 20, None, None, ctypes.byref(out)) == INV
    assert L.tg_ctx_create(ctypes.c_void_p(0x1001), 1 << 20, None, None, ctypes.byref(out)) == INV   # unaligned arena
    assert L.tg_ctx_destroy(None) == INV
    assert L.tg_graph_destroy(None, None) == INV
    assert L.tg_run(None, None) == INV
    assert L.tg_submit(None, None, ctypes.byref(u64)) == INV
    assert L.tg_poll(None, 1) == INV
    assert L.tg_wait(None, 1) == INV
    assert L.tg_cancel(None) == INV
    assert L.tg_result_copy(None, None, None, None, None, None) == INV
    assert L.tg_batch_launch(None, None) == INV
    assert L.tg_batch_destroy(None, None) == INV
    assert L.tg_instance_create(None, None, ctypes.byref(out)) == INV
    assert L.tg_serve_start(None, 0) == INV
    assert L.tg_serve_stop(None) == INV
    assert L.tg_graph_get_info(None, None) == INV
    assert L.tg_ctx_get_stats(None, None) == INV
    assert L.tg_ctx_get_opts(None, None) == INV
    assert L.tg_ctx_set_launch(None, None) == INV
