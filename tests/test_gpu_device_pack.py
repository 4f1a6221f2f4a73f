"""tg_graph_create_dev: ingest, validation and CSR pack on the device give
the host packer's statuses and packed graph, and the oracle's results."""
import numpy as np
import pytest

import oracle
import workloads as w
from paper_2004_10908_b300 import binding as B
from tests.gpu_util import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    from paper_2004_10908_b300 import Executor
    e = Executor(arena_bytes=2 << 30)
    yield e
    e.close()


def shuffled_edges(g, seed):
    """The same graph with its edges given in another order.  A condition's
    returned index refers to its successors' insertion order, so each
    condition's own edges keep their relative order (the graph means the
    same); every other edge moves anywhere."""
    rng = np.random.default_rng(seed)
    key = rng.random(len(g.src))
    cond = (g.kinds[g.src] >= 1) & (g.kinds[g.src] <= 3)
    for s_ in np.unique(g.src[cond]):
        idx = np.nonzero(cond & (g.src == s_))[0]
        key[idx] = np.sort(key[idx])
    p = np.argsort(key, kind="stable")
    return w.Graph(g.name + "_shuffled", g.kinds, g.params, g.src[p], g.dst[p], g.seed, g.meta)


def small_graphs():
    return [w.diamond(), w.if_else(1), w.do_while(7), w.nested_loops(3),
            w.from_lists("single", [0], [w.pack_param(3)], []),
            w.from_lists("duplicates", [0, 0, 0], [1, 2, 3], [(0, 1), (0, 1), (1, 2), (0, 2), (0, 1)]),
            w.config1(), w.config2a(seed=5, levels=37, width=333), w.config2b(side=100, rounds=16),
            w.config3(seed=7, n_cond=200, body_levels=4, body_width=7, rounds=5),
            shuffled_edges(w.config3(seed=8, n_cond=150, body_levels=3, body_width=6, rounds=4), 1),
            shuffled_edges(w.config2a(seed=6, levels=20, width=400), 2)] + \
        list(w.config4(seed=9, n_graphs=6, n_lo=16, n_hi=5000))


def test_same_packed_graph_and_oracle_results(ex):
    for g in small_graphs():
        gh = ex.graph(g)
        gd = ex.graph(g, device_pack=True)
        try:
            assert B.tg_graph_dot(ex.ctx, gd.handle) == B.tg_graph_dot(ex.ctx, gh.handle), g.name
            # word for word: records (successor offsets relative to the graph's
            # lists), successor entries with their flags, source list
            rh, eh = B.tg_graph_packed_copy(ex.ctx, gh.handle, g.n)
            rd, ed = B.tg_graph_packed_copy(ex.ctx, gd.handle, g.n)
            np.testing.assert_array_equal(rd, rh, err_msg=f"{g.name}: records")
            np.testing.assert_array_equal(ed, eh, err_msg=f"{g.name}: successor and source lists")
            ih, idv = gh.info(), gd.info()
            for k in ("n_nodes", "n_edges", "n_sources", "n_conditions", "device_bytes"):
                assert ih[k] == idv[k], (g.name, k)
            st = ex.run(gd)
            dev = (st,) + tuple(ex.result(gd))
        finally:
            gh.destroy()
            gd.destroy()
        assert_same(dev, oracle.run(g), g.name)


def test_full_size_headline_graphs(ex):
    for g in (w.config2a(), w.config2b()):
        gd = ex.graph(g, device_pack=True)
        try:
            info = gd.info()
            assert info["n_nodes"] == len(g.kinds) and info["n_edges"] == len(g.src)
            st = ex.run(gd)
            dev = (st,) + tuple(ex.result(gd))
        finally:
            gd.destroy()
        assert_same(dev, oracle.run(g), g.name)


def test_statuses_match_the_host_packer(ex):
    big = 65536
    cases = [
        (w.from_lists("bad_idx", [0, 0], [1, 1], [(0, 5)]), None),
        (w.from_lists("bad_src", [0, 0], [1, 1], [(7, 1)]), None),
        (w.from_lists("cond_no_succ", [0, 1], [1, 1], [(0, 1)]), None),
        (w.from_lists("trip0", [0, 2], [1, 1], [(0, 1), (1, 0)]), None),
        (w.from_lists("kind9", [9], [1], []), None),
        (w.from_lists("module_kind", [0, 4], [1, 1], [(0, 1)]), None),
        (w.pitfall_no_source(), None),
        (w.from_lists("weakonly", [3, 0], [w.pack_param(1, 0, 0), 1], [(0, 1), (1, 0)]), None),
        (w.diamond(), np.array([0, 1, 0, 0], np.uint8)),   # a strong edge given as weak
        (w.diamond(), np.array([0, 0, 0, 0], np.uint8)),   # right: every edge strong
        (w.if_else(1), None),
        # out-degree above 65535
        (w.Graph("fan_out", np.zeros(big + 1, np.uint8), np.ones(big + 1, np.uint32),
                 np.zeros(big, np.uint32), np.arange(1, big + 1, dtype=np.uint32), 0, {}), None),
        # strong in-degree above 65535
        (w.Graph("fan_in", np.zeros(big + 1, np.uint8), np.ones(big + 1, np.uint32),
                 np.arange(big, dtype=np.uint32), np.full(big, big, np.uint32), 0, {}), None),
        # both an index out of range and an edge-kind mismatch: INVALID comes first
        (w.from_lists("two_causes", [0, 0], [1, 1], [(0, 1), (0, 9)]), np.array([1, 0], np.uint8)),
    ]
    for g, weak in cases:
        st_h, h = B.tg_graph_create(ex.ctx, g.kinds, g.params, g.src, g.dst, g.seed, weak)
        st_d, d = B.tg_graph_create_dev(ex.ctx, g.kinds, g.params, g.src, g.dst, g.seed, weak)
        for x in (h, d):
            if x is not None:
                B.tg_graph_destroy(ex.ctx, x)
        assert st_d == st_h, (g.name, B.STATUS_NAMES[st_d], B.STATUS_NAMES[st_h])
        assert (h is None) == (st_h != B.TG_OK) and (d is None) == (st_d != B.TG_OK)


def test_budget_is_checked_after_validation():
    from paper_2004_10908_b300 import Executor
    g = w.config2a(seed=3, levels=40, width=500)
    with Executor(arena_bytes=256 << 20, mem_budget_bytes=1 << 20) as e:
        st_h, h = B.tg_graph_create(e.ctx, g.kinds, g.params, g.src, g.dst, g.seed)
        st_d, d = B.tg_graph_create_dev(e.ctx, g.kinds, g.params, g.src, g.dst, g.seed)
        assert h is None and d is None and st_h == st_d == B.TG_ERR_BUDGET
        bad = w.from_lists("bad_idx", [0, 0], [1, 1], [(0, 5)])
        st_d, d = B.tg_graph_create_dev(e.ctx, bad.kinds, bad.params, bad.src, bad.dst, 0)
        assert st_d == B.TG_ERR_INVALID


def test_random_graphs_valid_and_invalid(ex):
    """Random graphs, some with an error planted: the device path returns the
    host packer's status, and for every graph created its packed graph."""
    rng = np.random.default_rng(2024)
    created = 0
    for t in range(120):
        n = int(rng.integers(1, 3000))
        m = int(rng.integers(0, 4 * n + 1))
        kinds = rng.choice([0, 0, 0, 1, 2, 3], size=n).astype(np.uint8)
        params = (rng.integers(1, 40, n) | (rng.integers(1, 6, n) << 16) |
                  (rng.integers(0, 4, n) << 24)).astype(np.uint32)
        src = rng.integers(0, n, m).astype(np.uint32)
        dst = rng.integers(0, n, m).astype(np.uint32)
        # forward edges, so that sources exist; every condition gets a successor
        lo, hi = np.minimum(src, dst), np.maximum(src, dst)
        cv = np.nonzero((kinds >= 1) & (kinds <= 3))[0].astype(np.uint32)
        src = np.concatenate([lo, cv]).astype(np.uint32)
        dst = np.concatenate([hi, np.minimum(cv + 1, n - 1)]).astype(np.uint32)
        m = len(src)
        weak = None
        fault = t % 6
        if fault == 1 and m:
            dst[rng.integers(0, m)] = n + int(rng.integers(0, 5))       # index out of range
        elif fault == 2:
            kinds[rng.integers(0, n)] = 9                                # unknown kind
        elif fault == 3 and m:
            weak = ((kinds[src] >= 1) & (kinds[src] <= 3)).astype(np.uint8)
            if t % 12 == 3:
                weak[rng.integers(0, m)] ^= 1                            # one edge kind flipped
        elif fault == 4:
            loops = np.nonzero(kinds == 2)[0]
            if loops.size:
                params[loops[0]] &= ~np.uint32(0xFF << 16)               # loop trip 0
        elif fault == 5:
            every = np.arange(n, dtype=np.uint32)                        # a self-edge on every task: no source
            src, dst = np.concatenate([src, every]), np.concatenate([dst, every])
        st_h, h = B.tg_graph_create(ex.ctx, kinds, params, src, dst, t, weak)
        st_d, d = B.tg_graph_create_dev(ex.ctx, kinds, params, src, dst, t, weak)
        try:
            assert st_d == st_h, (t, B.STATUS_NAMES[st_d], B.STATUS_NAMES[st_h])
            if st_h == B.TG_OK:
                n = len(kinds)
                rh, eh = B.tg_graph_packed_copy(ex.ctx, h, n)
                rd, ed = B.tg_graph_packed_copy(ex.ctx, d, n)
                np.testing.assert_array_equal(rd, rh, err_msg=f"graph {t}: records")
                np.testing.assert_array_equal(ed, eh, err_msg=f"graph {t}: lists")
                created += 1
        finally:
            for x in (h, d):
                if x is not None:
                    B.tg_graph_destroy(ex.ctx, x)
    assert created > 20
