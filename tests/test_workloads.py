"""The input generators: the native motif-graph twin (workloads/motif.c)
draws exactly the graph of the readable definition (motif_graph_py), and
the serving workload's request graphs are reproducible from their seed."""
import numpy as np

import workloads as w
from workloads.graphs import _logu, motif_graph, motif_graph_py
from workloads.rng import Stream


def _same(a, b):
    assert np.array_equal(a.kinds, b.kinds)
    assert np.array_equal(a.params, b.params)
    assert np.array_equal(a.src, b.src)
    assert np.array_equal(a.dst, b.dst)
    assert a.meta["n_d"] == b.meta["n_d"]
    for k in ("anchors", "h", "c", "k", "trips"):
        assert np.array_equal(np.asarray(a.meta[k]), np.asarray(b.meta[k])), k


def test_native_motif_graph_equals_the_definition():
    checked = 0
    for i in range(120):
        for kw in ({}, {"rounds": 64}, {"d_lo": 1, "d_hi": 4}, {"cond_frac": 0.2, "trip_max": 3}):
            s1, s2 = Stream(7000 + i, 5), Stream(7000 + i, 5)
            n = _logu(s1, 16, 9000)
            _logu(s2, 16, 9000)
            try:
                a = motif_graph_py(s1, n, seed=i, **kw)
            except ValueError:
                try:
                    motif_graph(s2, n, seed=i, **kw)
                except ValueError:
                    continue
                raise AssertionError("the native twin accepted a graph too small for its motifs")
            b = motif_graph(s2, n, seed=i, **kw)
            _same(a, b)
            assert s1.pos == s2.pos   # both leave the stream at the same place
            checked += 1
    assert checked > 400


def test_native_twin_takes_the_permutation_fallback():
    # width-4 levels with in-degree up to 4: twelve candidates often hold
    # fewer than d distinct predecessors, so rows fall back to a permutation
    for i in range(40):
        s1, s2 = Stream(90 + i, 5), Stream(90 + i, 5)
        a = motif_graph_py(s1, 40, seed=i, d_lo=3, d_hi=8)
        b = motif_graph(s2, 40, seed=i, d_lo=3, d_hi=8)
        _same(a, b)


def test_request_graphs_are_reproducible_and_well_formed():
    for i in (0, 1, 17, 4999):
        a, b = w.config5_request(i), w.config5_request(i)
        _same(a, b)
        assert a.seed == i
        assert 64 <= a.n <= 262144
        assert (a.params & 0xFFFF == 64).all()
        assert a.src.max() < a.n and a.dst.max() < a.n
        # every loop condition's successors: [h, arms...], h first
        c = np.asarray(a.meta["c"])
        for cc, hh in zip(c[:5], np.asarray(a.meta["h"])[:5]):
            out = a.dst[a.src == cc]
            assert out[0] == hh
