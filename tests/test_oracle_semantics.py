"""The oracle against evaluators that do not use its queue/counter machinery
(tests/pins.py): definitional DAG recursion, unrolled and structured loop
programs, closed-form counts and brute force over all schedules."""
import random

import numpy as np
import pytest

import workloads as w
from tests import pins


def _same(res, ref):
    out, cnt, dig = ref
    np.testing.assert_array_equal(res.cnt, cnt)
    np.testing.assert_array_equal(res.out, out)
    np.testing.assert_array_equal(res.dig, dig)


@pytest.mark.parametrize("levels,width,seed", [(6, 7, 11), (30, 40, 1), (60, 25, 9)])
def test_layered_dag_matches_definition(orc, levels, width, seed):
    g = w.config2a(seed=seed, levels=levels, width=width)
    r = orc.run(g)
    assert r.status == orc.OK and r.execs == g.n
    _same(r, pins.definitional_dag(g))


def test_wavefront_matches_dp(orc):
    side = 40
    g = w.config2b(side=side, rounds=5)
    r = orc.run(g)
    assert r.status == orc.OK
    np.testing.assert_array_equal(r.out, pins.wavefront_dp(side, 5))
    assert (r.cnt == 1).all()


def test_motif_graph_dag_part_and_counts(orc):
    for gi, g in enumerate(w.config4(seed=4, n_graphs=12, n_lo=16, n_hi=3000)):
        r = orc.run(g)
        assert r.status == orc.OK, gi
        np.testing.assert_array_equal(r.cnt, pins.motif_counts(g))
        # the DAG tasks see no condition output: their outputs follow the definition
        nd = g.meta["n_d"]
        dag = w.Graph("dag", g.kinds[:nd], g.params[:nd],
                      g.src[(g.src < nd) & (g.dst < nd)], g.dst[(g.src < nd) & (g.dst < nd)], g.seed)
        out, _, _ = pins.definitional_dag(dag)
        np.testing.assert_array_equal(r.out[:nd], out)


@pytest.mark.parametrize("trip", [1, 2, 5])
def test_config1_matches_unrolled_loop(orc, trip):
    g = w.config1(levels=4, width=9, trip=trip, rounds=7)
    r = orc.run(g)
    assert r.status == orc.OK
    _same(r, pins.unrolled_config1(g))
    m = g.meta
    assert r.cnt[m["H"]] == trip and r.cnt[m["C"]] == trip and r.cnt[m["D"]] == 1
    b0, b1 = m["body"]
    assert (r.cnt[b0:b1] == trip).all()


def test_config1_full_size_counts(orc):
    g = w.config1()
    r = orc.run(g)
    assert r.status == orc.OK
    assert r.execs == 5012            # I + 5*(H + 1000 body + C) + D
    _same(r, pins.unrolled_config1(g))


def test_config3_matches_structured_program(orc):
    g = w.config3(seed=3, n_cond=40, body_levels=3, body_width=4, rounds=3, trip_max=4)
    r = orc.run(g)
    assert r.status == orc.OK
    _same(r, pins.structured_config3(g))
    # closed-form counts per lane
    for lane in g.meta["lanes"]:
        T1, T2 = lane["T1"], lane["T2"]
        assert r.cnt[lane["h1"]] == T1 and r.cnt[lane["c1"]] == T1 and r.cnt[lane["X"]] == 1
        for k in ("h2", "c2", "cb", "M"):
            assert r.cnt[lane[k]] == T1 * T2
        sel = [0] * lane["k"]
        for it in range(T1 * T2):
            sel[orc.cond_hash(g.seed, lane["cb"], it) % lane["k"]] += 1
        for j, (h3, b0, c3, T3) in enumerate(lane["arms"]):
            assert r.cnt[h3] == sel[j] * T3 and r.cnt[c3] == sel[j] * T3
            assert (r.cnt[b0:c3] == sel[j] * T3).all()


def test_config3_full_size_counts(orc):
    g = w.config3()
    assert int((g.kinds != 0).sum()) == 10_000
    r = orc.run(g)
    assert r.status == orc.OK
    total = 1
    for lane in g.meta["lanes"]:
        T1, T2 = lane["T1"], lane["T2"]
        sel = [0] * lane["k"]
        for it in range(T1 * T2):
            sel[orc.cond_hash(g.seed, lane["cb"], it) % lane["k"]] += 1
        total += 2 * T1 + 4 * T1 * T2 + 1
        for j, (h3, b0, c3, T3) in enumerate(lane["arms"]):
            total += sel[j] * T3 * (c3 - h3 + 1)
    assert r.execs == total


def _tiny_graphs(count, seed):
    rng = random.Random(seed)
    for _ in range(count):
        n = rng.randint(1, 5)
        kinds = [rng.choice([0, 0, 0, 1, 2]) for _ in range(n)]
        params = [rng.randint(0, 3) | (rng.randint(1, 3) << 16) for _ in range(n)]
        edges = []
        for v in range(n):
            deg = rng.randint(1 if kinds[v] else 0, 3)
            for _ in range(deg):
                edges.append((v, rng.randrange(n)))
        yield w.from_lists("tiny", kinds, params, edges, seed=rng.getrandbits(32))


def test_brute_force_all_schedules(orc):
    confluent = racy = 0
    for g in _tiny_graphs(3000, 1):
        try:
            outs = pins.brute_force(g, exec_cap=40, max_states=20000)
        except RuntimeError:
            continue
        r = orc.run(g, exec_cap=40)
        name = orc.STATUS_NAMES[r.status]
        if name == "INVALID":
            continue
        mine = (name,) if name != "OK" else ("OK", tuple(int(x) for x in r.out),
                                              tuple(int(x) for x in r.cnt), tuple(int(x) for x in r.dig))
        if len(outs) == 1:
            confluent += 1
            assert mine in outs, g
        else:
            racy += 1
            assert name == "RACE" or mine in outs
    assert confluent > 500 and racy > 20


def test_brute_force_init_f2_race(orc):
    """Scheduling walk-through: adding init -> F2 may race on F2."""
    g = w.nested_loops(3, extra_init_to_f2=True)
    outs = pins.brute_force(g, exec_cap=60, max_states=200000)
    assert ("RACE",) in outs
    g0 = w.nested_loops(3)
    assert len(pins.brute_force(g0, exec_cap=200, max_states=200000)) == 1


@pytest.mark.parametrize("seed", range(6))
def test_random_general_dag_matches_definition(orc, seed):
    """Random DAGs beyond the layered shape: edges between any earlier and
    later task (a random permutation hides the order), duplicate edges,
    isolated tasks, wide fan-in and fan-out, mixed rounds per task."""
    rng = random.Random(seed)
    n = rng.randint(2, 300)
    perm = list(range(n))
    rng.shuffle(perm)
    edges = []
    for _ in range(rng.randint(0, 4 * n)):
        a, b = sorted(rng.sample(range(n), 2))
        edges.append((perm[a], perm[b]))
        if rng.random() < 0.05:
            edges.append((perm[a], perm[b]))       # a duplicate counts per edge
    hub = perm[0]
    edges += [(hub, perm[k]) for k in range(1, n) if rng.random() < 0.2]   # wide fan-out
    kinds = [w.STATIC] * n
    params = [w.pack_param(rng.randint(0, 40)) for _ in range(n)]
    g = w.from_lists(f"random_dag_{seed}", kinds, params, edges, seed=rng.getrandbits(32))
    r = orc.run(g)
    assert r.status == orc.OK and r.execs == g.n
    _same(r, pins.definitional_dag(g))
