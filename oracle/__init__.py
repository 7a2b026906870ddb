"""CPU oracle (test infrastructure only; never imported by the library).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg use
it.  See ``mapsq_oracle`` for what each function computes and which passage of
the paper it follows.
"""
from .mapsq_oracle import (  # noqa: F401
    LEFT, RIGHT, VAR_S, VAR_P, VAR_O,
    as_rows, canonical, join_nested_loop, join_mapreduce, distinct_triples,
    scan_pattern, evaluate_bgp, brute_force_bgp, join_batch, split_by_predicate,
    project, distinct, decode, join_star,
)
