"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and
the benchmark.  Random numbers only (splitmix64): no arithmetic of the method."""
from .rng import Stream, mix64_scalar
from .graphs import (STATIC, COND_BRANCH, COND_LOOP, COND_CONST, Graph, pack_param, from_lists,
                     diamond, if_else, do_while, nested_loops, pitfall_no_source, pitfall_race,
                     config1, config2a, config2b, config3, config4, config5_request,
                     config5_arrivals, motif_graph, motif_graph_py, sample_distinct)
