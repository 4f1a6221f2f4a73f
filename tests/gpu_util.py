"""Helpers shared by the GPU tests."""
import numpy as np

import oracle
from paper_2004_10908_b300 import STATUS_NAMES

ORACLE_TO_NAME = oracle.STATUS_NAMES


def run_both(ex, g, exec_cap=None):
    """Run g on the device and in the oracle; return (device, oracle) results."""
    gh = ex.graph(g)
    try:
        st = ex.run(gh)
        out, cnt, dig, execs = ex.result(gh)
    finally:
        gh.destroy()
    ref = oracle.run(g, exec_cap=exec_cap) if exec_cap is not None else oracle.run(g)
    return (st, out, cnt, dig, execs), ref


def assert_same(dev, ref, name=""):
    st, out, cnt, dig, execs = dev
    assert STATUS_NAMES[st] == ORACLE_TO_NAME[ref.status], (name, STATUS_NAMES[st], ORACLE_TO_NAME[ref.status])
    if ref.status == 0:
        np.testing.assert_array_equal(cnt, ref.cnt, err_msg=f"{name}: cnt")
        np.testing.assert_array_equal(out, ref.out, err_msg=f"{name}: out")
        np.testing.assert_array_equal(dig, ref.dig, err_msg=f"{name}: dig")
        assert execs == ref.execs, name
