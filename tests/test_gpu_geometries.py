"""Parity across launch geometries: the same graphs, run alone and in one
batch launch, at seeded random settings of every launch knob, equal the
oracle element by element (or, at most, report the race check's known false
positive).  Geometry changes which warp, block and queue each activation
takes, so this is where ordering mistakes show."""
import random

import numpy as np
import pytest

import oracle
import workloads as w
from paper_2004_10908_b300 import binding as B
from tests.gpu_util import assert_same

pytestmark = pytest.mark.gpu

SPACE = dict(warps_per_block=[4, 8, 16], worker_blocks=[148, 296], batch_max=[1, 8, 24, 32],
             local_keep=[16, 64, 512], max_thieves=[8, 16, 64], keep_idle=[0, 1], hand_batch=[0, 1],
             steal_policy=[0, 1], max_steal=[2, 8, 32], steal_backoff_ns=[128, 512, 4096],
             idle_sleep_ns=[128, 256, 1024], deque_depth=[256, 4096])


def test_random_geometries_single_and_batched():
    from paper_2004_10908_b300 import Executor
    graphs = [w.config1(), w.config3(seed=7, n_cond=200, body_levels=4, body_width=7, rounds=5),
              w.config2a(seed=5, levels=37, width=333), w.config2b(side=100, rounds=16), w.nested_loops(3),
              w.do_while(50)] + list(w.config4(seed=21, n_graphs=6, n_lo=16, n_hi=4000))
    refs = [oracle.run(g) for g in graphs]
    rng = random.Random(17)
    geos = [{k: rng.choice(v) for k, v in SPACE.items()} for _ in range(10)]
    exact = 0
    with Executor(arena_bytes=2 << 30) as ex:
        for gi, geo in enumerate(geos):
            ex.set_launch(**geo)
            hs = [ex.graph(g, device_pack=(gi % 2 == 1)) for g in graphs]
            try:
                for g, h, r in zip(graphs, hs, refs):
                    st = ex.run(h)
                    assert st in (B.TG_OK, B.TG_ERR_RACE), (g.name, geo, B.STATUS_NAMES[st])
                    if st == B.TG_OK:
                        assert_same((st,) + tuple(ex.result(h)), r, f"{g.name} {geo}")
                        exact += 1
                _, sts = ex.run_batch(hs)
                for g, h, r, st in zip(graphs, hs, refs, sts):
                    assert st in (B.TG_OK, B.TG_ERR_RACE), (g.name, geo, B.STATUS_NAMES[st])
                    if st == B.TG_OK:
                        assert_same((int(st),) + tuple(ex.result(h)), r, f"batched {g.name} {geo}")
                        exact += 1
            finally:
                for h in hs:
                    h.destroy()
    assert exact >= 0.95 * 2 * len(geos) * len(graphs)
