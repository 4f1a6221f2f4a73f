"""The dependency floor the bench divides by: the number of tasks on the
longest path of each headline graph, checked against the longest path found
by dynamic programming over the graph itself (no GPU)."""
import numpy as np

import bench
import workloads as w


def longest_path_tasks(g):
    # every edge of these generators goes from a lower task id to a higher
    # one, so task-id order is a topological order
    src = g.src.astype(np.int64)
    dst = g.dst.astype(np.int64)
    assert (src < dst).all()
    depth = np.ones(g.n, np.int64)
    order = np.argsort(dst, kind="stable")
    s, d = src[order], dst[order]
    for i in range(len(s)):
        if depth[s[i]] + 1 > depth[d[i]]:
            depth[d[i]] = depth[s[i]] + 1
    return int(depth.max())


def test_layered_and_wavefront_floors():
    for g in (w.config2a(seed=3, levels=20, width=50), w.config2a(seed=4, levels=7, width=300, d_lo=1, d_hi=2),
              w.config2b(side=30, rounds=4), w.config2b(side=1, rounds=4)):
        assert bench.critical_path_tasks(g) == longest_path_tasks(g), g.name
